"""Pins the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against what the paper and the mathematics fix:
printed textbook LJ values (the paper, Sec. 4.1, names the potential without
printing it), FCC lattice sums, exact rational arithmetic, Newton's third law
(Sec. 2.1), F = -grad U, symmetry invariances, and brute-force enumeration of
the pair sets that linked cells and Verlet lists must reproduce (Sec. 2.1.1).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2512_03565_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lj_textbook.json")))
TWO32 = 2 ** 32


def two_particles(L, d_fp, axis=0, base=0):
    pos = np.zeros((3, 2), dtype=np.uint32)
    pos[:, 0] = base
    pos[:, 1] = base
    pos[axis, 1] = (base + d_fp) % TWO32
    return pos


# --- exact integer cutoff threshold (reading R2) ------------------------------

@pytest.mark.parametrize("L,r", [(10.7722, 2.5), (111.81788, 2.8), (8.0, 2.5), (673.6, 2.5),
                                 (7.94, 2.8), (5.0, 1.0), (3.3, 1.0), (1e4, 3.0)])
def test_cut2_int_is_exact(orc, L, r):
    q = Fraction(r) * TWO32 / Fraction(L)
    expect = math.floor(q * q)
    assert orc.cut2_int(L, r) == expect


def test_r2_int_minimum_image(orc):
    # wrap-around difference: 2^32 - 5 and 7 are 12 units apart
    assert orc.r2_int((TWO32 - 5, 0, 0), (7, 0, 0)) == 144
    assert orc.r2_int((0, TWO32 - 1, 3), (0, 1, 0)) == 4 + 9
    # the L/2 tie maps to -2^31 (int32 wrap), squared 2^62
    assert orc.r2_int((0, 0, 0), (2 ** 31, 0, 0)) == 2 ** 62


def test_quantize(orc):
    L = 10.0
    assert orc.quantize(0.0, L) == 0
    assert orc.quantize(5.0, L) == 2 ** 31
    assert orc.quantize(-2.5, L) == 3 * 2 ** 30
    assert orc.quantize(12.5, L) == 2 ** 30
    assert orc.quantize(L * (1 - 2 ** -40), L) == TWO32 - 1


# --- two-particle closed forms -------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("base", [0, TWO32 - 2 ** 29, 12345])
def test_two_particle_textbook_values(orc, axis, base):
    L = 8.0                      # u = 2^-29: sigma, 2 and 2.5 are exact fixed-point distances
    u = L / TWO32
    for r, Uref, Fref in [(1.0, GOLD["U_at_sigma"], GOLD["F_at_sigma"]),
                          (2.0, GOLD["U_at_2"], GOLD["F_at_2"]),
                          (2.5, GOLD["U_at_2p5"], GOLD["F_at_2p5"])]:
        d = int(round(r / u))
        assert d * u == r
        F, U, Wv, n = orc.forces_bruteforce(two_particles(L, d, axis, base), L, 2.5)
        assert n == 1
        assert U == pytest.approx(Uref, rel=1e-11, abs=1e-14)
        # F_ij along the axis: the radial force F(r) (positive = repulsive)
        # pushes particle 0 (at lower coordinate) towards -axis
        assert -F[axis, 0] == pytest.approx(Fref, rel=1e-11, abs=1e-14)
        assert F[axis, 1] == -F[axis, 0]
        assert np.all(F[[a for a in range(3) if a != axis]] == 0.0)
        assert Wv == pytest.approx(Fref * r, rel=1e-11, abs=1e-14)


def test_two_particle_minimum(orc):
    L = 8.0
    u = L / TWO32
    d = int(round(GOLD["r_min"] / u))
    F, U, _, _ = orc.forces_bruteforce(two_particles(L, d), L, 2.5)
    # within one fixed-point unit of the minimum: |F| <= k * u, U = -1 to 2nd order
    assert abs(F[0, 0]) <= GOLD["k_at_r_min"] * u * 1.01
    assert U == pytest.approx(GOLD["U_at_r_min"], abs=1e-12)


def test_cutoff_is_inclusive_in_integer_units(orc):
    L = 8.0
    u = L / TWO32
    d = int(round(2.5 / u))
    assert orc.forces_bruteforce(two_particles(L, d), L, 2.5)[3] == 1
    assert orc.forces_bruteforce(two_particles(L, d + 1), L, 2.5)[3] == 0
    # diagonal pair: R^2 = 3 d^2 decides exactly
    Rc2 = orc.cut2_int(L, 2.5)
    k = math.isqrt(Rc2 // 3)
    pos = np.array([[0, k], [0, k], [0, k]], dtype=np.uint32)
    assert orc.forces_bruteforce(pos, L, 2.5)[3] == (1 if 3 * k * k <= Rc2 else 0)
    pos = np.array([[0, k + 1], [0, k + 1], [0, k + 1]], dtype=np.uint32)
    assert orc.forces_bruteforce(pos, L, 2.5)[3] == (1 if 3 * (k + 1) ** 2 <= Rc2 else 0)


def test_periodic_image_across_each_face(orc):
    L = 8.0
    u = L / TWO32
    d = int(round(1.5 / u))
    for axis in range(3):
        pos = np.zeros((3, 2), dtype=np.uint32)
        pos[axis, 0] = int(round(0.5 / u))
        pos[axis, 1] = TWO32 - int(round(1.0 / u))       # at L - 1: distance 1.5 through the face
        F, U, _, n = orc.forces_bruteforce(pos, L, 2.5)
        ref, _, _, _ = orc.forces_bruteforce(two_particles(L, d, axis), L, 2.5)
        assert n == 1
        # particle 1 sits "below" particle 0 through the face
        np.testing.assert_allclose(F[:, 0], -ref[:, 0], rtol=1e-14)


def test_zero_separation_is_excluded(orc):
    pos = np.array([[5, 5, 1000], [7, 7, 9], [9, 9, 3]], dtype=np.uint32)
    F, U, _, n = orc.forces_bruteforce(pos, 8.0, 2.5)
    assert np.isfinite(F).all() and n == 2


# --- lattice sums ------------------------------------------------------------

def U_lj(r):
    return 4.0 * (r ** -12 - r ** -6)


def test_fcc_energy_equals_shell_sum_and_forces_vanish(orc):
    rho, rc = 0.8, 2.5
    sysm = W.perfect_fcc(8, rho)                # 2048 sites, exact fixed-point positions
    a = (4.0 / rho) ** (1.0 / 3.0)
    F, U, _, npairs = orc.forces_bruteforce(sysm.pos, sysm.L, rc)
    shells = [(k, m) for k, m in GOLD["fcc_shells_k_multiplicity"] if a * math.sqrt(k / 2) <= rc]
    assert [m for _, m in shells] == [12, 6, 24, 12]
    e_shell = 0.5 * sum(m * U_lj(a * math.sqrt(k / 2)) for k, m in shells)
    assert U / sysm.n == pytest.approx(e_shell, rel=1e-12)
    assert npairs == sysm.n * sum(m for _, m in shells) // 2
    assert np.abs(F).max() < 1e-10


def test_fcc_large_cutoff_matches_lattice_sums(orc):
    rho, rc = 0.8, 10.0
    sysm = W.perfect_fcc(16, rho)               # L = 27.4 > 2 rc
    a = (4.0 / rho) ** (1.0 / 3.0)
    _, U, _, _ = orc.forces_bruteforce(sysm.pos, sysm.L, rc)
    s = 1.0 / (a / math.sqrt(2.0))
    e_inf = 2.0 * (GOLD["fcc_A12"] * s ** 12 - GOLD["fcc_A6"] * s ** 6)
    tail = 8.0 * math.pi * rho * (rc ** -9 / 9.0 - rc ** -3 / 3.0)   # continuum tail beyond rc
    assert U / sysm.n + tail == pytest.approx(e_inf, rel=2e-4)


# --- invariants ---------------------------------------------------------------

def test_newton3_zero_net_force(orc):
    s = W.stratified(3000, 0.75, 11)
    F, _, _, _ = orc.forces_bruteforce(s.pos, s.L, 2.5)
    scale = np.sqrt((F ** 2).sum(0).mean())
    assert np.abs(F.sum(axis=1)).max() < 1e-11 * scale * s.n


def test_force_is_minus_gradient_of_energy(orc):
    s = W.stratified(64, 0.6, 3)
    L = s.L
    u = L / TWO32
    h_fp = int(round(1e-6 / u))
    h = h_fp * u
    F, _, _, _ = orc.forces_bruteforce(s.pos, L, 2.5)
    rng = np.random.default_rng(5)
    for i in rng.choice(s.n, 6, replace=False):
        for axis in range(3):
            p, m = s.pos.copy(), s.pos.copy()
            p[axis, i] = (int(p[axis, i]) + h_fp) % TWO32
            m[axis, i] = (int(m[axis, i]) - h_fp) % TWO32
            Up = orc.forces_bruteforce(p, L, 2.5)[1]
            Um = orc.forces_bruteforce(m, L, 2.5)[1]
            fd = -(Up - Um) / (2 * h)
            assert fd == pytest.approx(F[axis, i], rel=1e-6, abs=1e-6)


def test_permutation_and_translation_invariance(orc):
    s = W.stratified(2000, 0.75, 17)
    F, U, Wv, n = orc.forces_bruteforce(s.pos, s.L, 2.5)
    perm = np.random.default_rng(1).permutation(s.n)
    Fp, Up, Wp, n_p = orc.forces_bruteforce(s.pos[:, perm], s.L, 2.5)
    np.testing.assert_allclose(Fp, F[:, perm], rtol=1e-12, atol=1e-12 * np.abs(F).max())
    assert n_p == n and Up == pytest.approx(U, rel=1e-13)
    shift = np.array([[123456789], [2 ** 31 + 7], [4000000000]], dtype=np.uint64)
    Ft, Ut, Wt, nt = orc.forces_bruteforce(((s.pos.astype(np.uint64) + shift) % TWO32).astype(np.uint32), s.L, 2.5)
    assert np.array_equal(Ft, F) and nt == n          # per-particle sums run in the same order
    assert Ut == pytest.approx(U, rel=1e-13) and Wt == pytest.approx(Wv, rel=1e-13)   # OpenMP reduction order


def test_linked_cells_equals_bruteforce_forces(orc):
    s = W.stratified(5000, 0.8, 23)
    F, U, Wv, n = orc.forces_bruteforce(s.pos, s.L, 2.5)
    Fc, Uc, Wc, nc_ = orc.forces_cells(s.pos, s.L, 2.5)
    assert nc_ == n
    np.testing.assert_allclose(Fc, F, rtol=0, atol=1e-12 * np.abs(F).max())
    assert Uc == pytest.approx(U, rel=1e-12)


# --- pair sets: cells and Verlet lists against brute force (Sec. 2.1.1) -------

def tiny_cases():
    rng = np.random.default_rng(99)
    out = []
    for L, n in [(3.3, 20), (4.0, 60), (5.0, 120), (3.0, 90)]:
        out.append(("uniform", L, rng.integers(0, TWO32, size=(3, n), dtype=np.uint64).astype(np.uint32)))
    # every particle in one cell
    out.append(("one_cell", 4.0, rng.integers(0, 2 ** 30, size=(3, 50), dtype=np.uint64).astype(np.uint32)))
    # particles exactly on cell faces and at 0 (nc = 4: faces at multiples of 2^30)
    faces = rng.integers(0, 4, size=(3, 64)).astype(np.uint64) * 2 ** 30
    faces[:, :8] = 0
    out.append(("faces", 4.0, faces.astype(np.uint32)))
    # empty cells: everything in one octant
    out.append(("octant", 5.0, rng.integers(0, 2 ** 31, size=(3, 80), dtype=np.uint64).astype(np.uint32)))
    return out


@pytest.mark.parametrize("name,L,pos", tiny_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_cell_pairs_equal_bruteforce(orc, name, L, pos):
    r = 1.0
    nc = orc.ncells(L, r)
    assert nc >= 3
    bf = orc.pairs_bruteforce(pos, L, r)
    lc = orc.pairs_cells(pos, L, r, nc)
    assert np.array_equal(bf, lc)


def test_pairs_exactly_at_cutoff(orc):
    L, r = 4.0, 1.0
    u = L / TWO32
    d = int(round(r / u))
    assert d * u == r
    pos = np.array([[0, d, 0, 2 ** 31], [0, 0, d + 1, 2 ** 31], [0, 0, 0, 0]], dtype=np.uint32)
    bf = orc.pairs_bruteforce(pos, L, r)
    assert [tuple(p) for p in bf] == [(0, 1)]
    assert np.array_equal(orc.pairs_cells(pos, L, r, orc.ncells(L, r)), bf)


def test_minimum_image_half_box_tie(orc):
    # exactly L/2 apart: int32 wrap gives -2^31 either way; with r_c < L/2 never a pair
    pos = np.array([[0, 2 ** 31], [0, 0], [0, 0]], dtype=np.uint32)
    assert orc.pairs_bruteforce(pos, 4.0, 1.9).shape[0] == 0


@pytest.mark.parametrize("half", [0, 1])
def test_verlet_lists_equal_bruteforce(orc, half):
    for name, L, pos in tiny_cases():
        rl = 1.0
        nc = orc.ncells(L, rl)
        perm, cs, nbr, nnbr, over = orc.verlet(pos, L, rl, nc, half, 128)
        assert not over
        n = pos.shape[1]
        inv = np.empty(n, dtype=np.int64)
        inv[perm] = np.arange(n)
        bf = orc.pairs_bruteforce(pos, L, rl)
        want = [set() for _ in range(n)]
        for i, j in bf:
            a, b = inv[i], inv[j]
            if not half or b > a:
                want[a].add(int(b))
            if not half or a > b:
                want[b].add(int(a))
        got = [set(int(v) for v in nbr[a, :nnbr[a]]) for a in range(n)]
        assert got == want, name
        assert all(len(set(nbr[a, :nnbr[a]])) == nnbr[a] for a in range(n))


def test_bin_cells_is_stable_counting_sort(orc):
    s = W.uniform(5000, 0.8, 4)
    nc = orc.ncells(s.L, 2.5)
    perm, cs = orc.bin_cells(s.pos, nc)
    cell = np.array([orc.cell_of(s.pos[:, i], nc) for i in range(s.n)])
    # stable sort by cell id == numpy's stable argsort of the cell ids
    assert np.array_equal(perm, np.argsort(cell, kind="stable"))
    assert np.array_equal(cs, np.searchsorted(np.sort(cell), np.arange(nc ** 3 + 1), side="left"))
    # cell coordinate of a fixed-point value: floor(x * nc / 2^32)
    for xv in [0, 1, 2 ** 31, TWO32 - 1, 123456789]:
        assert orc.cell_of((xv, 0, 0), nc) == (xv * nc) // TWO32


# --- Verlet cluster lists (Sec. 2.1.1; cluster sizes of Sec. 5.1; reading R19) --

@pytest.mark.parametrize("n,M,k", [(1, 4, 1), (3, 4, 1), (1000, 4, 6), (1048576, 4, 64), (1048576, 8, 50),
                                   (1048576, 6, 55), (2000000, 8, 62)])
def test_vcl_tower_count(orc, n, M, k):
    assert orc.vcl_ntower(n, M) == k
    assert k ** 3 * M <= n or k == 1
    assert (k + 1) ** 3 * M > n


def vcl_cases():
    rng = np.random.default_rng(7)
    out = [(name, L, pos) for name, L, pos in tiny_cases()]
    s = W.stratified(3000, 0.75, 11)
    out.append(("fluid", s.L, s.pos))
    s = W.slab(2500, 0.8, 0.02, 0.4, 12)
    out.append(("slab", s.L, s.pos))
    out.append(("dup_z", 6.0, np.vstack([rng.integers(0, TWO32, size=(2, 200), dtype=np.uint64),
                                         np.repeat(rng.integers(0, TWO32, size=(1, 20), dtype=np.uint64), 10, axis=1)]
                                        ).astype(np.uint32)))
    return out


@pytest.mark.parametrize("M", [1, 4, 6, 8])
def test_vcl_order_is_tower_z_sort(orc, M):
    for name, L, pos in vcl_cases():
        n = pos.shape[1]
        perm, cls = orc.vcl_order(pos, M)
        nt = orc.vcl_ntower(n, M)
        assert np.array_equal(np.sort(perm), np.arange(n)), name
        col = (pos[0].astype(np.int64) * nt >> 32) * nt + (pos[1].astype(np.int64) * nt >> 32)
        # a lexicographic sort by (column, z, original index), written with numpy
        assert np.array_equal(perm, np.lexsort((np.arange(n), pos[2], col))), name
        sizes = np.diff(cls)
        assert cls[0] == 0 and cls[-1] == n and sizes.min() >= 1 and sizes.max() <= M, name
        ccol = col[perm]
        for c in range(len(sizes)):
            members = ccol[cls[c]:cls[c + 1]]
            assert (members == members[0]).all(), name               # one tower per cluster
            last_of_tower = cls[c + 1] == n or ccol[cls[c + 1]] != members[0]
            assert sizes[c] == M or last_of_tower, name               # only a tower's last cluster is short
            if cls[c] > 0 and ccol[cls[c] - 1] == members[0]:
                assert sizes[c - 1] == M, name


def _clusters_of(perm, cls, n):
    cl = np.empty(n, dtype=np.int64)
    for c in range(len(cls) - 1):
        cl[perm[cls[c]:cls[c + 1]]] = c
    return cl


def test_vcl_lists_with_singleton_clusters_are_verlet_lists(orc):
    """M = 1: a cluster is one particle and its only member pair with J is
    the particle pair, so the cluster lists are the particle Verlet lists
    (pairs at zero separation excluded, no particle lists itself)."""
    for name, L, pos in vcl_cases()[:6]:
        n, rl = pos.shape[1], 1.0
        perm, cls, lists, masks = orc.vcl_lists(pos, L, rl, 1, 0, masks=True)
        cl = _clusters_of(perm, cls, n)
        want = [set() for _ in range(n)]
        for i, j in orc.pairs_bruteforce(pos, L, rl):
            want[cl[i]].add(int(cl[j]))
            want[cl[j]].add(int(cl[i]))
        got = [set(int(v) for v in lists[c]) for c in range(n)]
        assert got == [want[c] for c in range(n)], name
        assert all(np.all(m == 1) for m in masks), name


@pytest.mark.parametrize("M", [4, 6, 8])
def test_vcl_lists_and_masks_are_the_member_pairs_within_rl(orc, M):
    """Against the brute-force r_l pair set, independently of the cluster
    search: the listed cluster pairs of the full lists are exactly the
    cluster pairs of the brute-force pairs (both directions), and the mask
    bits of the listed pairs, mapped back to particles, are exactly those
    pairs; half lists hold each pair once (J > I, or J = I with b > a) and
    are the full lists' entries with J >= I."""
    for name, L, pos in vcl_cases():
        n = pos.shape[1]
        rl = 1.0 if L < 7 else 2.8
        perm, cls, full, fmask = orc.vcl_lists(pos, L, rl, M, 0, masks=True)
        _, _, half, hmask = orc.vcl_lists(pos, L, rl, M, 1, masks=True)
        ncl = len(cls) - 1
        cl = _clusters_of(perm, cls, n)
        rank = np.empty(n, dtype=np.int64)
        for c in range(ncl):
            rank[perm[cls[c]:cls[c + 1]]] = np.arange(cls[c + 1] - cls[c])
        bf = {(int(i), int(j)) for i, j in orc.pairs_bruteforce(pos, L, rl)}
        want_full = {(int(cl[i]), int(cl[j])) for i, j in bf} | {(int(cl[j]), int(cl[i])) for i, j in bf}
        got_full = {(I, int(J)) for I in range(ncl) for J in full[I]}
        assert got_full == want_full, name
        assert all(list(full[I]) == sorted(full[I]) for I in range(ncl)), name
        pairs_full, pairs_half = set(), []
        for I in range(ncl):
            mi = perm[cls[I]:cls[I + 1]]
            for J, m in zip(full[I], fmask[I]):
                mj = perm[cls[J]:cls[J + 1]]
                for a in range(len(mi)):
                    for b in range(len(mj)):
                        if (int(m) >> (a * M + b)) & 1:
                            pairs_full.add((min(mi[a], mj[b]), max(mi[a], mj[b])))
            for J, m in zip(half[I], hmask[I]):
                assert J >= I and m != 0, name
                mj = perm[cls[J]:cls[J + 1]]
                for a in range(len(mi)):
                    for b in range(len(mj)):
                        if (int(m) >> (a * M + b)) & 1:
                            assert J > I or b > a, name
                            pairs_half.append((min(mi[a], mj[b]), max(mi[a], mj[b])))
            assert [int(J) for J in half[I]] == [int(J) for J in full[I] if J >= I], name
        assert pairs_full == bf, name
        assert len(pairs_half) == len(bf) and set(pairs_half) == bf, name


# --- integrator ----------------------------------------------------------------

def test_velocity_verlet_two_body_harmonic_period(orc):
    """Small oscillations of a bound pair about r_min have the textbook period
    2 pi sqrt(mu / U''(r_min)), mu = m/2."""
    L = 16.0
    u = L / TWO32
    amp = 1e-3
    r0 = GOLD["r_min"] + amp
    pos = np.zeros((3, 2), dtype=np.uint32)
    pos[0, 1] = int(round(r0 / u))
    vel = np.zeros((3, 2))
    dt, steps = 0.001, 2000
    xs = []
    p, v = pos, vel
    F = None
    for _ in range(steps):
        p, v, F, _, _ = orc.vv_run(p, v, L, 2.5, 1.0, dt, 1, use_cells=False, forces=F)
        xs.append(int(p[0, 1]) - int(p[0, 0]))
    sep = np.array(xs) * u - GOLD["r_min"]
    cross = np.where((sep[:-1] > 0) & (sep[1:] <= 0))[0]
    period = np.diff(cross).mean() * dt
    expect = 2 * math.pi * math.sqrt(0.5 / GOLD["k_at_r_min"])
    assert period == pytest.approx(expect, rel=3e-3)
    # momentum is conserved exactly (forces antisymmetric, same kicks)
    assert v[0].sum() == pytest.approx(0.0, abs=1e-15)


def test_velocity_verlet_nve_energy_drift(orc):
    """NVE conservation of the shifted energy U - n_pairs U(r_c): the force is
    truncated, so a pair crossing r_c changes the unshifted U by U(r_c)."""
    s = W.stratified(500, 0.7, 8, T=1.0)
    uc = GOLD["U_at_2p5"]
    F, U0, _, n0 = orc.forces_cells(s.pos, s.L, 2.5)
    E0 = U0 - n0 * uc + 0.5 * (s.vel ** 2).sum()
    p, v, F, _, _ = orc.vv_run(s.pos, s.vel, s.L, 2.5, 1.0, 0.002, 100, use_cells=True, forces=F)
    _, U1, _, n1 = orc.forces_cells(p, s.L, 2.5)
    E1 = U1 - n1 * uc + 0.5 * (v ** 2).sum()
    assert abs(E1 - E0) / abs(E0) < 1e-3


def test_drift_is_round_to_nearest_even(orc):
    # a displacement of exactly k + 1/2 units rounds to the even neighbour
    L = 4.0
    dt = 1.0
    dtu = dt * TWO32 / L
    pos = np.zeros((3, 2), dtype=np.uint32)
    pos[0, 1] = 2 ** 31
    vel = np.zeros((3, 2))
    vel[0, 0] = 2.5 / dtu
    vel[1, 0] = -3.5 / dtu
    vel[2, 0] = 7.25 / dtu
    p, v, F, _, _ = orc.vv_run(pos, vel, L, 0.5, 1.0, dt, 1, use_cells=False, forces=np.zeros((3, 2)))
    assert int(p[0, 0]) == 2 and int(p[1, 0]) == TWO32 - 4 and int(p[2, 0]) == 7


# --- tuner MLP (Sec. 6: data-driven tuning) --------------------------------------

def test_mlp_gradient_matches_finite_differences(orc):
    Cn = 5
    P = orc.mlp_nparams(Cn)
    assert P == 64 * 16 + 64 + 64 * 64 + 64 + Cn * 64 + Cn
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, size=P)
    X = rng.normal(size=(7, 16))
    T = rng.normal(size=(7, Cn))
    M = (rng.random((7, Cn)) > 0.3).astype(np.float64)
    loss, g = orc.mlp_loss_grad(p, Cn, X, T, M)
    h = 1e-6
    for k in rng.choice(P, 40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (orc.mlp_loss_grad(pp, Cn, X, T, M)[0] - orc.mlp_loss_grad(pm, Cn, X, T, M)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_mlp_reduces_to_bias_when_hidden_weights_vanish(orc):
    Cn = 3
    P = orc.mlp_nparams(Cn)
    p = np.zeros(P)
    b3 = np.array([0.5, -1.0, 2.0])
    p[-Cn:] = b3
    X = np.random.default_rng(1).normal(size=(4, 16))
    np.testing.assert_array_equal(orc.mlp_forward(p, Cn, X), np.tile(b3, (4, 1)))
    T = np.zeros((4, Cn))
    M = np.ones((4, Cn))
    loss, g = orc.mlp_loss_grad(p, Cn, X, T, M)
    assert loss == pytest.approx((b3 ** 2).mean())
    np.testing.assert_allclose(g[-Cn:], 2 * b3 / Cn)        # d/db3 of the mean squared error


def test_adam_first_step_is_lr_times_sign(orc):
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    orc.adam_step(p, g, m, v, 0.01, 1, eps=0.0)
    np.testing.assert_allclose(p, [0.99, -1.99, 2.99], rtol=0, atol=1e-15)


# --- features ------------------------------------------------------------------

def test_features_of_hand_built_configuration(orc):
    L, rc, skin = 10.0, 2.5, 0.3          # nc = 4, 64 cells of edge 2.5
    pos = np.zeros((3, 8), dtype=np.uint32)
    pos[0, :] = [0, 1, 2, 3, 4, 5, 2 ** 30 + 1, 2 ** 31]   # 6 in cell 0, one in cell 1, one in cell 2
    f = orc.features(pos, L, rc, skin)
    occ = np.zeros(64)
    occ[0], occ[1], occ[2] = 6, 1, 1
    assert f[0] == pytest.approx(math.log(8 / 1000.0))
    assert f[1] == pytest.approx(math.log(8))
    assert f[2] == pytest.approx(8 / 64)
    assert f[3] == pytest.approx(occ.std())
    assert f[4] == pytest.approx(61 / 64)
    np.testing.assert_allclose(f[5:13], np.array([61, 2, 0, 1, 0, 0, 0, 0]) / 64)
    blocks = np.zeros(64)
    blocks[0], blocks[1], blocks[2] = 6, 1, 1      # top-two-bit blocks along x: 0, 1, 2
    assert f[13] == pytest.approx(blocks.std() / blocks.mean())
    assert f[14] == pytest.approx(1.0)
    assert f[15] == pytest.approx((38 / 8) * (4 / 3 * math.pi * 2.8 ** 3) / 2.5 ** 3)


# --- linked-cell half shells (readings R5 and R20) ------------------------------

def _half_shell_pairs(pos, L, r, backward):
    """Pairs found by visiting, for every particle, the forward (R5) or backward
    (R20) half shell of cells: own cell with j after (before) i in cell order,
    and the 13 cells ahead (behind) of it; written from the readings, in plain
    Python, on the oracle's cell order."""
    import oracle as orc
    n = pos.shape[1]
    nc = orc.ncells(L, r)
    perm, cs = orc.bin_cells(pos, nc)
    slot = np.empty(n, dtype=np.int64)
    slot[perm] = np.arange(n)
    R2max = orc.cut2_int(L, r)
    sgn = -1 if backward else 1
    # the 13 forward neighbour offsets (dz, dy, dx): (0,0,+1), (0,+1,*), (+1,*,*)
    fwd = [(0, 0, 1)] + [(0, 1, dx) for dx in (-1, 0, 1)] + [(1, dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    out = []
    for i in range(n):
        ci = [int((int(pos[a, i]) * nc) >> 32) for a in range(3)]
        c_lin = (ci[2] * nc + ci[1]) * nc + ci[0]
        cand = [j for j in perm[cs[c_lin]:cs[c_lin + 1]] if sgn * (slot[j] - slot[i]) > 0]
        for dz, dy, dx in fwd:
            z, y, x = (ci[2] + sgn * dz) % nc, (ci[1] + sgn * dy) % nc, (ci[0] + sgn * dx) % nc
            c2 = (z * nc + y) * nc + x
            cand += list(perm[cs[c2]:cs[c2 + 1]])
        for j in cand:
            R2 = orc.r2_int(pos[:, i], pos[:, j])
            if 0 < R2 <= R2max:
                out.append((min(i, int(j)), max(i, int(j))))
    return out


@pytest.mark.parametrize("backward", [False, True])
def test_half_shells_cover_every_pair_once(orc, backward):
    """Both half shells of the linked-cell Newton-3 orders find every pair of the
    brute force exactly once (the backward one is the forward one with the
    roles of the two cells of every pair swapped)."""
    for name, L, pos in tiny_cases():
        got = _half_shell_pairs(pos, L, 1.0, backward)
        assert len(got) == len(set(got)), name                      # no pair twice
        bf = {tuple(int(v) for v in p) for p in orc.pairs_bruteforce(pos, L, 1.0)}
        assert set(got) == bf, name


def _subcell_pairs(pos, L, r, half, backward=False):
    """Pairs found by visiting, for every particle, the 5 x 5 x 5 cells of edge
    >= r/2 around its own (the sub-cell container): all of them, or (Newton-3)
    the half after (before) the own cell in (dz, dy, dx) offset order with j
    after (before) i in the own cell; plain Python on the oracle's cell order."""
    import oracle as orc
    n = pos.shape[1]
    nc = orc.ncells(L, 0.5 * r)
    assert nc >= 5
    perm, cs = orc.bin_cells(pos, nc)
    slot = np.empty(n, dtype=np.int64)
    slot[perm] = np.arange(n)
    R2max = orc.cut2_int(L, r)
    sgn = -1 if backward else 1
    offs = [(dz, dy, dx) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)]
    if half:
        offs = [o for o in offs if (o[0], o[1], o[2]) > (0, 0, 0)]
    out = []
    for i in range(n):
        ci = [int((int(pos[a, i]) * nc) >> 32) for a in range(3)]
        c_lin = (ci[2] * nc + ci[1]) * nc + ci[0]
        own = list(perm[cs[c_lin]:cs[c_lin + 1]])
        cand = [j for j in own if sgn * (slot[j] - slot[i]) > 0] if half else [j for j in own if j != i]
        for dz, dy, dx in offs:
            if (dz, dy, dx) == (0, 0, 0):
                continue
            z, y, x = (ci[2] + sgn * dz) % nc, (ci[1] + sgn * dy) % nc, (ci[0] + sgn * dx) % nc
            c2 = (z * nc + y) * nc + x
            cand += list(perm[cs[c2]:cs[c2 + 1]])
        for j in cand:
            R2 = orc.r2_int(pos[:, i], pos[:, j])
            if 0 < R2 <= R2max:
                out.append((min(i, int(j)), max(i, int(j))))
    return out


@pytest.mark.parametrize("half,backward", [(0, False), (1, False), (1, True)])
def test_subcell_stencil_covers_every_pair(orc, half, backward):
    """The 5 x 5 x 5 stencil of cells of edge >= r_c / 2 finds every pair of the
    brute force, each once from either side (full) or exactly once (either half
    shell), on boxes of 5 to 9 cells per axis."""
    rng = np.random.default_rng(17)
    cases = [("uniform", 2.6, rng.integers(0, TWO32, size=(3, 60), dtype=np.uint64).astype(np.uint32)),
             ("uniform9", 4.6, rng.integers(0, TWO32, size=(3, 150), dtype=np.uint64).astype(np.uint32)),
             ("crowded", 3.0, rng.integers(0, 2 ** 30, size=(3, 70), dtype=np.uint64).astype(np.uint32))]
    for name, L, pos in cases:
        got = _subcell_pairs(pos, L, 1.0, half, backward)
        bf = {tuple(int(v) for v in p) for p in orc.pairs_bruteforce(pos, L, 1.0)}
        if half:
            assert len(got) == len(set(got)), name
            assert set(got) == bf, name
        else:
            assert len(got) == 2 * len(bf) and set(got) == bf, name


# --- sampled forces (the checker of the full-size GPU runs) --------------------

def _sampled_cases():
    rng = np.random.default_rng(7)
    out = []
    s = W.uniform(300, 0.8, 71)
    out.append(("uniform", s.L, s.pos))
    s = W.stratified(400, 0.5, 72)
    out.append(("stratified", s.L, s.pos))
    # pairs that interact only through a periodic face on each axis
    L = 8.0
    u = L / TWO32
    face = np.zeros((3, 6), dtype=np.uint32)
    for a in range(3):
        face[:, 2 * a] = int(round(4.0 / u))
        face[:, 2 * a + 1] = int(round(4.0 / u))
        face[a, 2 * a] = int(round(0.4 / u))
        face[a, 2 * a + 1] = TWO32 - int(round(0.9 / u))
    out.append(("faces", L, face))
    # a crowded cluster: 60 particles within 1.2 sigma of one point, in a dilute box
    s = W.stratified(200, 0.1, 73)
    crowd = (np.array([[2 ** 31], [2 ** 30], [2 ** 29]], dtype=np.int64)
             + rng.integers(-int(0.6 / (s.L / TWO32)), int(0.6 / (s.L / TWO32)), size=(3, 60)))
    pos = np.concatenate([s.pos.astype(np.int64), crowd], axis=1) % TWO32
    out.append(("crowded", s.L, pos.astype(np.uint32)))
    return out


@pytest.mark.parametrize("name,L,pos", _sampled_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_sampled_forces_equal_bruteforce_rows(orc, name, L, pos):
    """forces_sampled(idx) must be the idx columns of the brute-force forces,
    bit for bit (each row is the same ascending-j loop of Eq. 1), for any index
    subset: repeated, unordered, first and last particle included."""
    n = pos.shape[1]
    F, _, _, npairs = orc.forces_bruteforce(pos, L, 2.5)
    assert npairs > 0
    rng = np.random.default_rng(n)
    idx = np.concatenate([[0, n - 1, n - 1], rng.permutation(n)[: max(1, n // 3)], [n // 2, 0]])
    Fs = orc.forces_sampled(pos, L, 2.5, idx)
    assert Fs.shape == (3, idx.shape[0])
    assert np.array_equal(Fs, F[:, idx])
    assert np.array_equal(orc.forces_sampled(pos, L, 2.5, np.arange(n)), F)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sampled_forces_two_particle_textbook_value(orc, axis):
    """Against the printed F(r) directly (not through the brute force): both
    particles of an isolated pair at r = 2 get -/+ F(2) along the axis."""
    L = 8.0
    d = int(round(2.0 / (L / TWO32)))
    pos = two_particles(L, d, axis, base=2 ** 31)
    Fs = orc.forces_sampled(pos, L, 2.5, np.array([1, 0]))   # columns: particle 1, then particle 0
    # the radial force F(r) (positive = repulsive) acts on particle 0, the
    # lower one, along -axis
    assert Fs[axis, 1] == pytest.approx(-GOLD["F_at_2"], rel=1e-11)
    assert Fs[axis, 0] == -Fs[axis, 1]
    assert np.all(Fs[[a for a in range(3) if a != axis]] == 0.0)
    # beyond the cutoff on the sampled side too
    far = two_particles(L, int(round(2.6 / (L / TWO32))), axis)
    assert np.all(orc.forces_sampled(far, L, 2.5, np.array([0, 1])) == 0.0)
