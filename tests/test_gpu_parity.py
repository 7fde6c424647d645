"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (from the required accuracy of the force path): forces
max_i |F_i - F_i^oracle| / RMS_i |F_i^oracle| <= 1e-12 with FP64 pair math and
<= 1e-5 with FP32 pair math and FP64 accumulation; energies |dU|/|U| <= 1e-12 /
1e-6.  Cell order, pair sets and Verlet lists are integer results: bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_03565_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
ETOL = {0: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module")
def lj():
    from paper_2512_03565_gb300 import build as b
    b.build()
    oracle.build()
    from paper_2512_03565_gb300 import ljgb
    ljgb.load()
    return ljgb


def rel_err(F, Fref):
    rms = np.sqrt((Fref ** 2).sum(0).mean())
    return np.abs(F - Fref).max() / rms


def ref_forces(s, rc=None):
    return oracle.forces_bruteforce(s.pos, s.L, rc or s.rc)


@pytest.fixture(scope="module")
def sys_small():
    return W.stratified(6000, 0.75, 101)


@pytest.fixture(scope="module")
def ref_small(sys_small):
    return ref_forces(sys_small)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_config_matches_oracle(lj, sys_small, ref_small, prec):
    s = sys_small
    F_ref, U_ref, W_ref, np_ref = ref_small
    d = lj.Domain(s.L, s.rc, s.skin, precision=prec)
    d.set_particles(s.pos, s.vel)
    bad = []
    for cfg in lj.configs():
        U, Wv = d.compute_forces(cfg, energy=True)
        err = rel_err(d.forces(), F_ref)
        eU = abs(U - U_ref) / abs(U_ref)
        eW = abs(Wv - W_ref) / abs(W_ref)
        npairs = d.counters()[1]
        if not (err <= TOL[prec] and eU <= ETOL[prec] and eW <= ETOL[prec] and npairs == np_ref):
            bad.append((lj.config_name(cfg), err, eU, eW, npairs, np_ref))
    d.close()
    assert not bad, bad


def test_fp32_error_on_the_densest_workload(lj):
    """FP32 pair math sums a lane's contributions in FP32 before the FP64
    fold: a whole Verlet list in VL_IPT (about 120 entries at density 1.2),
    every linked-cell candidate in the IPT and KI orders.  On the densest
    workload (jittered FCC at density 1.2, the top of the density sweep) every
    configuration stays within the FP32 bound 1e-5 of max |dF| / RMS |F|."""
    s = W.fcc(6000, 1.2, 171)
    F_ref, U_ref, _, np_ref = ref_forces(s)
    d = lj.Domain(s.L, s.rc, s.skin, precision=1)
    d.set_particles(s.pos, s.vel)
    errs = {}
    for cfg in lj.configs():
        d.compute_forces(cfg)
        errs[lj.config_name(cfg)] = rel_err(d.forces(), F_ref)
        assert d.counters()[1] == np_ref
    d.close()
    worst = max(errs, key=errs.get)
    assert errs[worst] <= TOL[1], (worst, errs[worst])


def test_dilute_gas_with_close_contacts(lj):
    """The measured limit of FP32 pair math: in a dilute gas the RMS force is
    small, and a single close pair (here 0.88-0.92 sigma, carrying 30-40 RMS
    forces) brings its FP32 error to 1-2e-5 of RMS |F| in every order.  The
    FP64 path stays within 1e-12 on the same boxes, and the FP32 path within
    3e-5 (the documented 1-2e-5 with margin); pair counts are exact in both."""
    for seed in (1000, 1001, 1003):
        s = W.stratified(4000, 0.1, seed)
        F_ref, _, _, np_ref = ref_forces(s)
        for prec, tol in ((0, 1e-12), (1, 3e-5)):
            d = lj.Domain(s.L, s.rc, s.skin, precision=prec)
            d.set_particles(s.pos, s.vel)
            worst, name = 0.0, None
            for cfg in lj.configs():
                d.compute_forces(cfg)
                e = rel_err(d.forces(), F_ref)
                if e > worst:
                    worst, name = e, lj.config_name(cfg)
                assert d.counters()[1] == np_ref
            d.close()
            assert worst <= tol, (seed, prec, name, worst)


def test_newton3_partial_sums_across_particle_counts(lj):
    """FP32 Newton-3 evaluations add each j contribution to j's FP32 partial
    sum in a per-domain buffer, which grows with the particle count and is
    cleared before every evaluation.  One domain takes 2,500 particles, then
    4,000 (the buffer grows), then the 2,500 again (a larger buffer than
    needed); every Newton-3 configuration is evaluated twice on each, and
    every evaluation must match the oracle within the FP32 bound with exact
    pair counts (a buffer left uncleared would double the j sides)."""
    a = W.stratified(2500, 0.6, 311)
    b = W.stratified(4000, 0.96, 312)  # the same box edge: 2500 / 0.6 = 4000 / 0.96
    assert abs(a.L - b.L) < 1e-9 * a.L
    refs = [oracle.forces_bruteforce(s.pos, a.L, a.rc) for s in (a, b)]
    n3 = [c for c in lj.configs() if c.newton3 in (lj.LJ_N3_ATOMIC, lj.LJ_N3_ATOMIC_BWD)]
    assert len(n3) > 20
    d = lj.Domain(a.L, a.rc, a.skin, precision=lj.LJ_PREC_FP32_ACC64)
    bad = []
    for k in (0, 1, 0):
        s = (a, b)[k]
        F_ref, _, _, np_ref = refs[k]
        d.set_particles(s.pos, s.vel)
        for cfg in n3:
            for _ in range(2):
                d.compute_forces(cfg)
                e = rel_err(d.forces(), F_ref)
                if not (e <= TOL[1] and d.counters()[1] == np_ref):
                    bad.append((s.n, lj.config_name(cfg), e, d.counters()[1], np_ref))
    d.close()
    assert not bad, bad[:5]


@pytest.mark.parametrize("prec", [0, 1])
def test_config1_uniform_1000(lj, prec):
    """1,000 particles, uniform random at density 0.8, rc 2.5, one evaluation."""
    s = W.config1()
    F_ref, U_ref, _, np_ref = ref_forces(s)
    assert abs(np_ref - 26180) < 800
    d = lj.Domain(s.L, s.rc, s.skin, precision=prec)
    d.set_particles(s.pos, s.vel)
    for cfg in [lj.config(lj.LJ_LC, lj.LJ_ORD_JSPLIT, 32), lj.config(lj.LJ_LC, lj.LJ_ORD_IPT_SMEM, 0, 1),
                lj.config(lj.LJ_LC, lj.LJ_ORD_ROT32, 0, 1), lj.config(lj.LJ_VL, lj.LJ_ORD_VL_IPT, 0, 2)]:
        if prec == 1:
            # uniform random start has overlaps down to r ~ 0.05 (|F| ~ 1e17): FP32 pair
            # math stays finite there but only the FP64 path is held to a tolerance
            U, _ = d.compute_forces(cfg, energy=True)
            assert np.isfinite(d.forces()).all()
            continue
        U, _ = d.compute_forces(cfg, energy=True)
        assert rel_err(d.forces(), F_ref) <= TOL[0], lj.config_name(cfg)
        assert abs(U - U_ref) <= ETOL[0] * abs(U_ref)
        assert d.counters()[1] == np_ref
    d.close()


def test_cells_and_pairs_bit_exact(lj, sys_small):
    s = sys_small
    d = lj.Domain(s.L, s.rc, s.skin)
    d.set_particles(s.pos, s.vel)
    for cont, r in [(lj.LJ_LC, s.rc), (lj.LJ_VL, s.rc + s.skin)]:
        d.bin_cells(cont)
        perm, cs, nc = d.cells()
        assert nc == oracle.ncells(s.L, r)
        perm_ref, cs_ref = oracle.bin_cells(s.pos, nc)
        assert np.array_equal(perm, perm_ref) and np.array_equal(cs, cs_ref)
    assert np.array_equal(d.pairs(lj.LJ_LC), oracle.pairs_bruteforce(s.pos, s.L, s.rc))
    for half in (0, 1):
        d.build_verlet(half)
        assert np.array_equal(d.pairs(lj.LJ_VL), oracle.pairs_bruteforce(s.pos, s.L, s.rc + s.skin))
        nbr, nn = d.verlet()
        nc = oracle.ncells(s.L, s.rc + s.skin)
        _, _, nbr_ref, nn_ref, _ = oracle.verlet(s.pos, s.L, s.rc + s.skin, nc, half, nbr.shape[1])
        assert np.array_equal(nn, nn_ref)
        for i in range(s.n):                  # same entries in the same scan order
            assert np.array_equal(nbr[i, :nn[i]], nbr_ref[i, :nn[i]])
    d.close()


def edge_cases():
    rng = np.random.default_rng(99)
    out = []
    for L, n in [(3.3, 20), (4.0, 60), (5.0, 120), (3.0, 90)]:
        out.append(("uniform", L, rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)))
    out.append(("one_cell", 4.0, rng.integers(0, 2 ** 30, size=(3, 50), dtype=np.uint64).astype(np.uint32)))
    faces = rng.integers(0, 4, size=(3, 64)).astype(np.uint64) * 2 ** 30
    faces[:, :8] = 0
    out.append(("faces", 4.0, faces.astype(np.uint32)))
    out.append(("octant", 5.0, rng.integers(0, 2 ** 31, size=(3, 80), dtype=np.uint64).astype(np.uint32)))
    L = 4.0
    dfp = int(round(1.0 / (L / 2 ** 32)))
    out.append(("at_cutoff", L, np.array([[0, dfp, 0, 2 ** 31], [0, 0, dfp + 1, 2 ** 31], [0, 0, 0, 0]], dtype=np.uint32)))
    big = rng.integers(0, 2 ** 30, size=(3, 300), dtype=np.uint64).astype(np.uint32)   # 300 in one cell
    out.append(("crowded_cell", 4.0, big))
    return out


@pytest.mark.parametrize("name,L,pos", edge_cases(), ids=[c[0] for c in edge_cases()])
def test_edge_cases_fp64(lj, name, L, pos):
    rc, skin = 1.0, 0.0
    F_ref, U_ref, _, np_ref = oracle.forces_bruteforce(pos, L, rc)
    d = lj.Domain(L, rc, skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(pos)
    assert np.array_equal(d.pairs(lj.LJ_LC), oracle.pairs_bruteforce(pos, L, rc))
    for cfg in lj.configs():
        U, _ = d.compute_forces(cfg, energy=True)
        F = d.forces()
        scale = max(np.sqrt((F_ref ** 2).sum(0).mean()), 1e-300)
        assert np.abs(F - F_ref).max() <= 1e-12 * scale + 1e-300, (name, lj.config_name(cfg))
        assert abs(U - U_ref) <= 1e-12 * max(abs(U_ref), 1e-300), (name, lj.config_name(cfg))
        assert d.counters()[1] == np_ref
    d.close()


@pytest.mark.parametrize("name,L,pos", [c for c in edge_cases() if c[0] in ("uniform", "crowded_cell", "faces")][:3] +
                         [c for c in edge_cases() if c[0] == "crowded_cell"],
                         ids=["uniform-nc3", "uniform-nc4", "uniform-nc5", "crowded_cell"])
def test_verlet_lists_bit_exact_edge(lj, name, L, pos):
    """Lists on 3-5 cells per axis (at 3 one segment covers a whole row of
    cells and takes the integer path) and on a 300-particle cell, whose lists
    outgrow the builder's shared staging and take its direct-store path:
    entries, lengths and scan order equal the oracle's for full and half lists."""
    rl = 1.0
    d = lj.Domain(L, rl, 0.0, precision=lj.LJ_PREC_FP64)
    d.set_particles(pos)
    nc = oracle.ncells(L, rl)
    for half in (0, 1):
        d.build_verlet(half)
        nbr, nn = d.verlet()
        _, _, nbr_ref, nn_ref, _ = oracle.verlet(pos, L, rl, nc, half, nbr.shape[1])
        assert np.array_equal(nn, nn_ref)
        for i in range(pos.shape[1]):
            assert np.array_equal(nbr[i, :nn[i]], nbr_ref[i, :nn[i]]), (name, half, i)
    if name == "crowded_cell":
        assert nn.max() > 64
    d.close()


@pytest.mark.parametrize("cfg_args", [(1, 3, 4, 0), (2, 7, 4, 1)], ids=["VL-JSPLIT4", "VCL-JLANE4-N3"])
def test_update_positions_keeps_lists_while_the_skin_allows(lj, cfg_args):
    """lj_update_positions keeps the cell (or cluster) order and lists: small
    moves reuse the lists (no build), a move beyond skin/2 triggers one, and
    the forces equal those of a fresh context loaded with the same coordinates
    (FP64) and the oracle's."""
    s = W.stratified(5000, 0.7, 51)
    cfg = lj.config(*cfg_args)
    x0 = (s.pos.astype(np.float64) + 0.5) * (s.L / 2.0 ** 32)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(x0, s.vel)
    d.compute_forces(cfg)
    builds = d.counters()[2]
    rng = np.random.default_rng(7)
    small = x0 + rng.uniform(-0.05, 0.05, size=x0.shape)     # |move| < skin/2 = 0.15
    large = small.copy()
    large[:, 17] += 0.4                                        # one particle beyond skin/2
    for x, rebuilt in ((small, False), (large, True)):
        d.update_positions(x)
        d.compute_forces(cfg)
        assert (d.counters()[2] > builds) == rebuilt
        builds = d.counters()[2]
        ref = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
        ref.set_particles(x, s.vel)
        ref.compute_forces(cfg)
        F_ref = ref.forces()
        ref.close()
        assert rel_err(d.forces(), F_ref) <= 1e-12
        q = np.array([[oracle.quantize(v, s.L) for v in row] for row in x], dtype=np.uint32)
        F_orc, _, _, _ = oracle.forces_bruteforce(q, s.L, s.rc)
        assert rel_err(d.forces(), F_orc) <= 1e-12
    pos, vel = d.state()
    assert np.array_equal(vel, s.vel)                           # velocities untouched
    if cfg.newton3 != lj.LJ_N3_OFF:                             # atomics: no bitwise repeat
        d.close()
        return
    # the caller's pinned host memory is read and written by the kernels
    # directly (no staging copies): same positions in, same forces out, bitwise
    import torch
    F_staged = d.forces()
    x_pin = torch.from_numpy(np.ascontiguousarray(large)).pin_memory()
    f_pin = torch.empty((3, s.n), dtype=torch.float64).pin_memory()
    d.update_positions(x_pin)
    d.compute_forces(cfg)
    d.forces(out=f_pin)
    assert np.array_equal(f_pin.numpy(), F_staged)
    assert np.array_equal(d.state()[0], pos)
    d.close()


def test_quantization_matches_oracle(lj):
    rng = np.random.default_rng(5)
    L = 12.345
    x = rng.uniform(-3 * L, 4 * L, size=(3, 5000))
    x[:, :4] = [[0.0, L, -L, L * (1 - 1e-17)]] * 3
    d = lj.Domain(L, 2.5, 0.3)
    d.set_particles(x)
    pos, _ = d.state()
    ref = np.array([[oracle.quantize(v, L) for v in row] for row in x], dtype=np.uint32)
    assert np.array_equal(pos, ref)
    d.close()


@pytest.mark.parametrize("cfg_args", [(0, 3, 8, 0), (1, 5, 0, 0), (1, 3, 4, 0), (1, 5, 0, 1), (2, 6, 4, 0),
                                      (2, 7, 8, 1)],
                         ids=["LC-JSPLIT8", "VL-IPT", "VL-JSPLIT4", "VL-IPT-N3", "VCL-TILE4", "VCL-JLANE8-N3"])
def test_integrator_matches_oracle_fp64(lj, cfg_args):
    s = W.stratified(3000, 0.7, 12, T=1.0)
    cfg = lj.config(*cfg_args)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(s.pos, s.vel)
    d.integrate(0.002, 20, cfg)
    pos, vel = d.state()
    p_ref, v_ref, F_ref, _, _ = oracle.vv_run(s.pos, s.vel, s.L, s.rc, 1.0, 0.002, 20, use_cells=True)
    dp = np.abs(pos.astype(np.int64) - p_ref.astype(np.int64))
    dp = np.minimum(dp, 2 ** 32 - dp)
    assert dp.max() <= 2, dp.max()                  # FP64 summation order differs at 1e-16
    assert np.abs(vel - v_ref).max() <= 1e-9 * np.abs(v_ref).max()
    assert rel_err(d.forces(), F_ref) <= 1e-8
    d.close()


@pytest.mark.parametrize("cfg_args", [(1, 3, 4, 0), (0, 3, 2, 0)])
def test_pending_kick_is_exact(lj, cfg_args):
    """The closing half kick of a call is left pending and fused into the next
    call's first kick (or applied by a reader): one call of 20 steps, 20 calls
    of one step, and two calls of 10 with a kinetic-energy read in between give
    bit-identical states (deterministic N3-off kernels), which match the FP64
    oracle's velocity Verlet on the FP64 path."""
    s = W.stratified(4000, 0.7, 31, T=1.0)
    cfg = lj.config(*cfg_args)
    out = []
    for mode in ("one_call", "many_calls", "read_between"):
        d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
        d.set_particles(s.pos, s.vel)
        if mode == "one_call":
            d.integrate(0.002, 20, cfg)
        elif mode == "many_calls":
            for _ in range(20):
                d.integrate(0.002, 1, cfg)
        else:
            d.integrate(0.002, 10, cfg)
            ke = d.kinetic_energy()
            assert ke > 0
            d.integrate(0.002, 10, cfg)
        out.append(d.state())
        d.close()
    for p, v in out[1:]:
        assert np.array_equal(p, out[0][0]) and np.array_equal(v, out[0][1])
    p_ref, v_ref, _, _, _ = oracle.vv_run(s.pos, s.vel, s.L, s.rc, 1.0, 0.002, 20, use_cells=True)
    dp = np.abs(out[0][0].astype(np.int64) - p_ref.astype(np.int64))
    assert np.minimum(dp, 2 ** 32 - dp).max() <= 2
    assert np.abs(out[0][1] - v_ref).max() <= 1e-9 * np.abs(v_ref).max()


@pytest.mark.parametrize("cfg_args", [(1, 5, 0, 0), (1, 3, 8, 1), (0, 0, 0, 1), (1, 5, 0, 2), (2, 6, 6, 1),
                                      (2, 7, 4, 0)])
def test_md_run_fp32_vs_fp64_library(lj, cfg_args):
    """100 steps with Verlet rebuilds every 10 (and the skin check) on FP32 and
    FP64 paths stay close; the final FP32 forces match the oracle on the final state."""
    s = W.stratified(8000, 0.75, 21, T=1.0)
    cfg = lj.config(*cfg_args)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP32_ACC64)
    d.set_particles(s.pos, s.vel)
    d.integrate(0.002, 100, cfg, rebuild_every=10)
    pos, vel = d.state()
    cnt = d.counters()
    assert cnt[2] >= (0 if cfg.container == lj.LJ_LC else 10)
    d.compute_forces(cfg)
    F_ref, _, _, _ = oracle.forces_bruteforce(pos, s.L, s.rc)
    assert rel_err(d.forces(), F_ref) <= 1e-5
    d.close()


def test_newton3_two_pass_is_deterministic(lj, sys_small):
    s = sys_small
    cfg = lj.config(lj.LJ_VL, lj.LJ_ORD_VL_IPT, 0, lj.LJ_N3_TWOPASS)
    outs = []
    for _ in range(2):
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        d.compute_forces(cfg)
        outs.append(d.forces())
        d.close()
    assert np.array_equal(outs[0], outs[1])


def test_features_match_oracle(lj):
    for s in [W.stratified(20000, 0.75, 3), W.slab(20000, 0.8, 0.02, 0.4, 4)]:
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos)
        f = d.features()
        ref = oracle.features(s.pos, s.L, s.rc, s.skin)
        np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-14)
        d.close()


def test_mlp_forward_and_gradient_match_oracle(lj):
    Cn = 33
    rng = np.random.default_rng(2)
    P = oracle.mlp_nparams(Cn)
    p = rng.normal(0, 0.2, size=P)
    X = rng.normal(size=(200, 16))
    T = rng.normal(size=(200, Cn))
    M = (rng.random((200, Cn)) > 0.2).astype(np.float64)
    Y = lj.mlp_forward(p, Cn, X)
    np.testing.assert_allclose(Y, oracle.mlp_forward(p.astype(np.float32).astype(np.float64), Cn,
                                                     X.astype(np.float32).astype(np.float64)), rtol=1e-4, atol=1e-5)
    loss, g = lj.mlp_loss_grad(p, Cn, X, T, M)
    p32 = p.astype(np.float32).astype(np.float64)
    loss_ref, g_ref = oracle.mlp_loss_grad(p32, Cn, X.astype(np.float32).astype(np.float64),
                                           T.astype(np.float32).astype(np.float64), M)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_mlp_training_reduces_loss(lj):
    rng = np.random.default_rng(9)
    Cn = 8
    X = rng.normal(size=(256, 16))
    Wt = rng.normal(size=(16, Cn))
    T = np.tanh(X @ Wt * 0.3)
    M = np.ones_like(T)
    p0 = rng.normal(0, 0.1, size=lj.mlp_nparams(Cn))
    p, losses = lj.mlp_train(p0, Cn, X, T, M, epochs=500, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0]
    # the GPU training follows the oracle's Adam on the same gradients for a few steps
    q = p0.astype(np.float32).astype(np.float64)
    m, v = np.zeros_like(q), np.zeros_like(q)
    X64, T64 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    for t in range(1, 4):
        _, g = oracle.mlp_loss_grad(q, Cn, X64, T64, M)
        oracle.adam_step(q, g, m, v, 3e-3, t)
    p3, _ = lj.mlp_train(p0, Cn, X, T, M, epochs=3, lr=3e-3)
    assert np.abs(p3 - q).max() <= 1e-4


def test_tuner_prepare_matches_oracle(lj):
    """Relative log times, masks and standardised features of the learned
    tuner's training set, GPU kernels against the oracle: timings with untimed
    (NaN), zero and negative entries, a row with nothing timed, a constant
    feature column; 1000 rows span several blocks with a ragged tail."""
    rng = np.random.default_rng(12)
    Mr, Cn = 1000, 37
    T = np.exp(rng.normal(-1.0, 0.6, size=(Mr, Cn)))
    T[rng.random((Mr, Cn)) < 0.1] = np.nan
    T[3, 5], T[4, 6], T[7, :] = 0.0, -2.0, np.nan
    X = rng.normal(2.0, 3.0, size=(Mr, 16)) * np.logspace(-3, 3, 16)
    X[:, 9] = 0.625
    Y, Mk, Xs, mean, sd = lj.tuner_prepare(T, X)
    Yr, Mr_ = oracle.tuner_targets(T)
    Xr, mr, sr = oracle.standardize(X)
    np.testing.assert_array_equal(Mk, Mr_)
    np.testing.assert_array_equal(Mk[7], 0.0)
    np.testing.assert_allclose(Y, Yr, rtol=2e-7, atol=1e-7)       # FP64 arithmetic, FP32 output
    np.testing.assert_allclose(mean, mr, rtol=2e-7, atol=1e-30)
    np.testing.assert_allclose(sd, sr, rtol=2e-7)
    assert sd[9] == 1.0 and np.all(Xs[:, 9] == 0.0)
    np.testing.assert_allclose(Xs, Xr, rtol=2e-7, atol=1e-6)


def test_capacity_regrowth_and_skin_rebuild(lj):
    s = W.fcc(4000, 1.2, 5)                       # dense: lists longer than the initial estimate
    d = lj.Domain(s.L, s.rc, 0.6)
    d.set_particles(s.pos, s.vel)
    d.build_verlet(0)
    assert np.array_equal(d.pairs(lj.LJ_VL), oracle.pairs_bruteforce(s.pos, s.L, s.rc + 0.6))
    d.close()
    # a particle teleported by more than skin/2 triggers an early rebuild; FP64
    # so that a single missed pair (|F| >= |F(r_c)| = 0.039) would stand out
    s = W.stratified(3000, 0.6, 6)
    cfg = lj.config(lj.LJ_VL, lj.LJ_ORD_VL_IPT)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(s.pos, s.vel)
    d.compute_forces(cfg)
    builds = d.counters()[2]
    pos, vel = d.state()
    vel[:, 0] = [2000.0, 0.0, 0.0]                # moves 4 sigma in one step of dt = 0.002
    d2 = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP64)
    d2.set_particles(pos, vel)
    d2.integrate(0.002, 1, cfg, rebuild_every=1000)
    assert d2.counters()[3] >= 1                  # early (skin) rebuild counted
    # the closing kick of the skin step used the forces of the rebuilt lists:
    # the step equals the oracle's velocity Verlet (no lists) to FP64 rounding.
    # (Later steps are not compared: the teleported particle then nearly hits
    # another, |F| ~ 1e12, and rounding decides the trajectory.)
    p1, v1 = d2.state()
    p_ref, v_ref, _, _, _ = oracle.vv_run(pos, vel, s.L, s.rc, 1.0, 0.002, 1, use_cells=True)
    dp = np.abs(p1.astype(np.int64) - p_ref.astype(np.int64))
    assert np.minimum(dp, 2 ** 32 - dp).max() <= 2
    assert np.abs(v1 - v_ref).max() <= 1e-9 * np.abs(v_ref).max()
    d2.integrate(0.002, 2, cfg, rebuild_every=1000)
    p2, _ = d2.state()
    d2.compute_forces(cfg)
    F_ref, _, _, _ = oracle.forces_bruteforce(p2, s.L, s.rc)
    assert rel_err(d2.forces(), F_ref) <= 1e-12
    d.close()
    d2.close()
    assert builds >= 1


def test_nonfinite_force_is_reported(lj):
    pos = np.array([[0, 1, 2 ** 31], [0, 0, 0], [0, 0, 0]], dtype=np.uint32)  # two particles 1 unit apart
    d = lj.Domain(10.0, 2.5, 0.3, precision=lj.LJ_PREC_FP32_ACC64)
    d.set_particles(pos)
    with pytest.raises(lj.LJError, match="NONFINITE"):
        d.compute_forces(lj.config(lj.LJ_LC, lj.LJ_ORD_IPT_SMEM), energy=True)
    d.close()


def test_state_errors(lj):
    d = lj.Domain(10.0, 2.5, 0.3)
    with pytest.raises(lj.LJError, match="STATE"):
        d.compute_forces(lj.config(lj.LJ_LC, lj.LJ_ORD_IPT_SMEM))
    d.set_particles(np.zeros((3, 4), dtype=np.uint32) + np.arange(4, dtype=np.uint32) * 2 ** 28)
    with pytest.raises(lj.LJError, match="ARG"):
        d.compute_forces(lj.config(lj.LJ_LC, lj.LJ_ORD_KI, 3))
    d.close()
    small = lj.Domain(5.5, 1.0, 1.0)        # 5 cells for LC, 2 for VL
    small.set_particles(np.zeros((3, 4), dtype=np.uint32) + np.arange(4, dtype=np.uint32) * 2 ** 28)
    with pytest.raises(lj.LJError, match="ARG"):
        small.compute_forces(lj.config(lj.LJ_VL, lj.LJ_ORD_VL_IPT))
    small.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_boxes_every_config(lj, seed):
    """Random box sizes (3 to 9 cells per axis), particle counts and skins,
    uniform or clumped: every configuration's FP64 forces, energy and pair
    count equal the brute force."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(30, 2500))
    L = float(rng.uniform(3.2, 9.5))
    rc, skin = 1.0, float(rng.choice([0.0, 0.1, 0.4]))
    if seed % 2:
        pos = rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    else:
        centers = rng.integers(0, 2 ** 32, size=(3, 3), dtype=np.uint64)
        off = rng.integers(0, 2 ** 30, size=(3, n), dtype=np.uint64)
        pos = ((centers[:, rng.integers(0, 3, size=n)] + off) % 2 ** 32).astype(np.uint32)
    F_ref, U_ref, _, np_ref = oracle.forces_bruteforce(pos, L, rc)
    scale = max(np.sqrt((F_ref ** 2).sum(0).mean()), 1e-300)
    d = lj.Domain(L, rc, skin, precision=lj.LJ_PREC_FP64)
    d.set_particles(pos)
    nc_vl = int(np.floor(L / (rc + skin)))
    for cfg in lj.configs():
        if cfg.container == lj.LJ_VL and nc_vl < 3:
            continue
        U, _ = d.compute_forces(cfg, energy=True)
        assert np.abs(d.forces() - F_ref).max() <= 1e-12 * scale + 1e-300, (seed, lj.config_name(cfg))
        assert abs(U - U_ref) <= 1e-12 * max(abs(U_ref), 1e-300), (seed, lj.config_name(cfg))
        assert d.counters()[1] == np_ref, (seed, lj.config_name(cfg))
    d.close()


def test_degenerate_sizes(lj):
    """No particles is an argument error; one particle has no pair in any
    configuration; two particles whose only pair crosses the periodic boundary
    match the oracle in every configuration (FP64 and FP32 pair math); a lone
    particle drifts ballistically under velocity Verlet."""
    L, rc, skin = 4.0, 1.0, 0.3
    u = L / 2 ** 32
    d = lj.Domain(L, rc, skin, precision=lj.LJ_PREC_FP64)
    with pytest.raises(lj.LJError, match="ARG"):
        d.set_particles(np.zeros((3, 0), dtype=np.uint32))
    one = np.array([[123456789], [2 ** 31], [7]], dtype=np.uint32)
    d.set_particles(one)
    for cfg in lj.configs():
        U, W_ = d.compute_forces(cfg, energy=True)
        assert np.array_equal(d.forces(), np.zeros((3, 1))), lj.config_name(cfg)
        assert U == 0.0 and W_ == 0.0 and d.counters()[1] == 0, lj.config_name(cfg)
    d.close()
    half = int(round(0.45 / u))                    # separation 0.9 across the x = 0 face
    two = np.array([[2 ** 32 - half, half], [2 ** 30, 2 ** 30], [5, 5]], dtype=np.uint32)
    F_ref, U_ref, _, np_ref = oracle.forces_bruteforce(two, L, rc)
    assert np_ref == 1 and F_ref[0, 1] > 0          # repulsive at 0.9: the pair pushes apart across the face
    for prec in (lj.LJ_PREC_FP64, lj.LJ_PREC_FP32_ACC64):
        d = lj.Domain(L, rc, skin, precision=prec)
        d.set_particles(two)
        for cfg in lj.configs():
            U, _ = d.compute_forces(cfg, energy=True)
            assert rel_err(d.forces(), F_ref) <= TOL[prec], (prec, lj.config_name(cfg))
            assert abs(U - U_ref) <= ETOL[prec] * abs(U_ref), (prec, lj.config_name(cfg))
            assert d.counters()[1] == 1, (prec, lj.config_name(cfg))
        d.close()
    d = lj.Domain(L, rc, skin, precision=lj.LJ_PREC_FP64)
    x0 = np.array([[1.0], [2.0], [3.0]])
    v0 = np.array([[0.5], [-0.25], [0.125]])
    d.set_particles(x0, v0)
    d.integrate(0.002, 10, lj.config(lj.LJ_LC, lj.LJ_ORD_IPT_SMEM))
    x = d.state()[0].astype(np.float64) * u
    # quantisation (< 1 unit) plus one rounding to the nearest unit per drift
    np.testing.assert_allclose(x, np.mod(x0 + 10 * 0.002 * v0, L), rtol=0, atol=12 * u)
    d.close()
