"""Verlet cluster lists on the GPU against the oracle (Sec. 2.1.1's cluster
container; cluster sizes 4, 6 and 8 of Sec. 5.1).

The cluster order, the cluster boundaries, the cluster-pair lists and their
member masks are integer results decided by exact integer rules: the order
and boundaries are compared bit for bit, the lists as sets per cluster (the
library's search order is not defined) and each entry's mask with the
oracle's mask of the same cluster pair.  Forces of every cluster configuration are compared
with the brute force in the force-parity tests (they iterate over all
configurations); here also across rebuilds, capacity regrowth and the
full-size fluid on sampled particles."""
import numpy as np
import pytest

import oracle
from paper_2512_03565_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lj():
    from paper_2512_03565_gb300 import build as b
    b.build()
    oracle.build()
    from paper_2512_03565_gb300 import ljgb
    ljgb.load()
    return ljgb


def systems():
    rng = np.random.default_rng(41)
    out = []
    s = W.stratified(6000, 0.75, 201)
    out.append(("fluid", s.L, s.rc, s.skin, s.pos))
    s = W.slab(5000, 0.8, 0.02, 0.35, 202)
    out.append(("slab", s.L, s.rc, s.skin, s.pos))
    s = W.fcc(4000, 1.0, 203)
    out.append(("fcc", s.L, s.rc, s.skin, s.pos))
    out.append(("uniform_small", 3.3, 1.0, 0.0, rng.integers(0, 2 ** 32, size=(3, 20), dtype=np.uint64).astype(np.uint32)))
    out.append(("crowded", 4.0, 1.0, 0.2, rng.integers(0, 2 ** 30, size=(3, 300), dtype=np.uint64).astype(np.uint32)))
    z = np.repeat(rng.integers(0, 2 ** 32, size=40, dtype=np.uint64), 10)
    out.append(("dup_z", 6.0, 1.0, 0.3, np.vstack([rng.integers(0, 2 ** 32, size=(2, 400), dtype=np.uint64), z[None]]
                                                  ).astype(np.uint32)))
    return out


@pytest.mark.parametrize("M", [4, 6, 8])
@pytest.mark.parametrize("half", [0, 1])
def test_cluster_order_and_lists_bit_exact(lj, M, half):
    for name, L, rc, skin, pos in systems():
        d = lj.Domain(L, rc, skin, precision=lj.LJ_PREC_FP64)
        d.set_particles(pos)
        d.build_clusters(M, half)
        perm, _, nt = d.cells()
        cs, nt2 = d.clusters()
        lists = d.cluster_lists()
        masks = d.cluster_masks()
        vcl_pairs = d.pairs(lj.LJ_VCL)
        d.close()
        # the member pairs within r_l of the listed cluster pairs are exactly the brute-force r_l pairs
        assert np.array_equal(vcl_pairs, oracle.pairs_bruteforce(pos, L, rc + skin)), name
        perm_ref, cs_ref, lists_ref, masks_ref = oracle.vcl_lists(pos, L, rc + skin, M, half, masks=True)
        assert nt == nt2 == oracle.vcl_ntower(pos.shape[1], M), name
        assert np.array_equal(perm, perm_ref), name
        assert np.array_equal(cs, cs_ref), name
        assert len(lists) == len(lists_ref), name
        for I, (got, ref) in enumerate(zip(lists, lists_ref)):
            assert len(set(got.tolist())) == len(got), (name, I)
            assert sorted(got.tolist()) == ref.tolist(), (name, I)
            want = {int(J): int(m) for J, m in zip(ref, masks_ref[I])}
            assert {int(J): int(m) for J, m in zip(got, masks[I])} == want, (name, I)


def test_lists_follow_the_particles_across_rebuilds(lj):
    """An MD run on cluster lists rebuilds them (period and skin); after it, the
    current lists equal the oracle's for the current positions and the forces
    match the brute force."""
    s = W.stratified(5000, 0.75, 204, T=1.5)
    cfg = lj.config(lj.LJ_VCL, lj.LJ_ORD_CL_TILE, 4, lj.LJ_N3_ATOMIC)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(s.pos, s.vel)
    d.integrate(0.004, 30, cfg, rebuild_every=10)
    assert d.counters()[2] >= 3
    pos, _ = d.state()
    d.build_clusters(4, 1)
    lists = d.cluster_lists()
    _, _, ref = oracle.vcl_lists(pos, s.L, s.rc + s.skin, 4, 1)
    assert [sorted(x.tolist()) for x in lists] == [r.tolist() for r in ref]
    d.compute_forces(cfg)
    F_ref, _, _, _ = oracle.forces_bruteforce(pos, s.L, s.rc)
    rms = np.sqrt((F_ref ** 2).sum(0).mean())
    assert np.abs(d.forces() - F_ref).max() <= 1e-12 * rms
    d.close()


def test_capacity_regrowth(lj):
    """Lists sized for a dilute gas overflow when the same context gets a dense
    liquid; the build regrows the capacity and the forces stay exact."""
    dil = W.stratified(4000, 0.05, 205)
    den = W.fcc(4000, 1.1, 206)
    L = dil.L
    d = lj.Domain(L, 2.5, 0.3, precision=lj.LJ_PREC_FP64)
    d.set_particles(dil.pos)
    cfg = lj.config(lj.LJ_VCL, lj.LJ_ORD_CL_JLANE, 8, lj.LJ_N3_OFF)
    d.compute_forces(cfg)
    # the dense lattice scaled into the same box: a dense cube in one corner
    pos = (den.pos.astype(np.float64) * (den.L / L)).astype(np.uint32)
    d.set_particles(pos)
    before = d.counters()[4]
    d.compute_forces(cfg)
    assert d.counters()[4] > before
    F_ref, _, _, np_ref = oracle.forces_bruteforce(pos, L, 2.5)
    rms = np.sqrt((F_ref ** 2).sum(0).mean())
    assert np.abs(d.forces() - F_ref).max() <= 1e-12 * rms
    assert d.counters()[1] == np_ref
    d.close()


@pytest.mark.parametrize("order", ["CL_TILE", "CL_JLANE"])
def test_bench_fluid_full_size_sampled(lj, order):
    s = W.config2()
    o = lj.LJ_ORD_CL_TILE if order == "CL_TILE" else lj.LJ_ORD_CL_JLANE
    cfg = lj.config(lj.LJ_VCL, o, 8 if order == "CL_TILE" else 4, lj.LJ_N3_OFF)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP32_ACC64)
    d.set_particles(s.pos, s.vel)
    d.integrate(0.002, 12, cfg, rebuild_every=10)
    pos, _ = d.state()
    d.compute_forces(cfg)
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(s.n, 1000, replace=False))
    F_ref = oracle.forces_sampled(pos, s.L, s.rc, idx)
    rms = np.sqrt((F_ref ** 2).sum(0).mean())
    assert np.abs(d.forces()[:, idx] - F_ref).max() / rms <= 1e-5
    d.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_boxes(lj, seed):
    """Random box sizes and particle counts (1 to 9 towers per axis, a box
    of 3 to 9 cutoffs, uniform and clumped placements): cluster lists equal
    the oracle's and every cluster configuration's FP64 forces equal the
    brute force."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(30, 2500))
    L = float(rng.uniform(3.2, 9.0))
    rc, skin = 1.0, float(rng.choice([0.0, 0.2, 0.4]))
    if seed % 2:
        pos = rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    else:  # clumps: most particles in a few small regions
        centers = rng.integers(0, 2 ** 32, size=(3, 4), dtype=np.uint64)
        pick = rng.integers(0, 4, size=n)
        off = rng.integers(0, 2 ** 29, size=(3, n), dtype=np.uint64)
        pos = ((centers[:, pick] + off) % 2 ** 32).astype(np.uint32)
    F_ref, U_ref, _, np_ref = oracle.forces_bruteforce(pos, L, rc)
    scale = max(np.sqrt((F_ref ** 2).sum(0).mean()), 1e-300)
    d = lj.Domain(L, rc, skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(pos)
    for M in (4, 6, 8):
        for half in (0, 1):
            d.build_clusters(M, half)
            cs, _ = d.clusters()
            lists = d.cluster_lists()
            perm_ref, cs_ref, lists_ref = oracle.vcl_lists(pos, L, rc + skin, M, half)
            assert np.array_equal(cs, cs_ref), (seed, M, half)
            assert [sorted(x.tolist()) for x in lists] == [r.tolist() for r in lists_ref], (seed, M, half)
    for cfg in [c for c in lj.configs() if c.container == lj.LJ_VCL]:
        U, _ = d.compute_forces(cfg, energy=True)
        assert np.abs(d.forces() - F_ref).max() <= 1e-12 * scale + 1e-300, (seed, lj.config_name(cfg))
        assert abs(U - U_ref) <= 1e-12 * max(abs(U_ref), 1e-300), (seed, lj.config_name(cfg))
        assert d.counters()[1] == np_ref
    d.close()
