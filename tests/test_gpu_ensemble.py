"""Batched ensemble of independent boxes in one persistent launch (lj_ensemble_*),
checked against the FP64 oracle and against the same boxes run one at a time
through the single-box path; and its bounded-barrier failure path."""
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


def small_ensemble(nboxes=12, seed=7):
    # sizes and densities spread like the 256-box workload, scaled down; includes
    # small dense boxes with fewer than 3 cells per axis (all-pairs path)
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nboxes):
        n = int(np.exp(rng.uniform(np.log(150), np.log(4000))))
        rho = float(rng.uniform(0.1, 1.0))
        out.append(W.homogeneous(n, rho, 1000 + k, T=1.0, rc=2.5, skin=0.3))
    out.append(W.homogeneous(180, 1.0, 77, T=1.0))     # L = 5.6: two cells per axis
    return out


def rel_err(F, Fref):
    rms = np.sqrt((Fref ** 2).sum(0).mean())
    return np.abs(F - Fref).max() / rms


def test_ensemble_initial_forces_match_oracle(lj):
    boxes = small_ensemble()
    assert any(int(np.floor(s.L / 2.5)) < 3 for s in boxes)
    ens = lj.Ensemble(boxes)
    ens.run(0.002, 0)
    for s, (pos, vel, frc) in zip(boxes, ens.state()):
        assert np.array_equal(pos, s.pos)
        F_ref, _, _, _ = oracle.forces_bruteforce(s.pos, s.L, 2.5)
        assert rel_err(frc, F_ref) <= 1e-5
    ens.close()


def test_ensemble_matches_single_box_runs(lj):
    boxes = small_ensemble(seed=3)
    ens = lj.Ensemble(boxes)
    ens.run(0.002, 20, use_graph=True)
    assert ens.uses_graph(), ens.last_error()
    w = 8
    for s, (pos, vel, frc) in zip(boxes, ens.state()):
        if int(np.floor(s.L / 2.5)) >= 3:
            d = lj.Domain(s.L, 2.5, 0.3)
            d.set_particles(s.pos, s.vel)
            d.integrate(0.002, 20, lj.config(lj.LJ_LC, lj.LJ_ORD_JSPLIT, w))
            p_ref, v_ref = d.state()
            F_ref = d.forces()
            d.close()
            dp = np.abs(pos.astype(np.int64) - p_ref.astype(np.int64))
            dp = np.minimum(dp, 2 ** 32 - dp)
            assert dp.max() <= 64                  # same FP32 arithmetic; at most rounding-level drift
            assert rel_err(frc, F_ref) <= 1e-5
        F_orc, _, _, _ = oracle.forces_bruteforce(pos, s.L, 2.5)
        assert rel_err(frc, F_orc) <= 1e-5
    ens.close()


def test_ensemble_graph_replays_continue_the_run(lj):
    boxes = small_ensemble(nboxes=5, seed=11)
    a = lj.Ensemble(boxes)
    a.run(0.002, 10)
    a.run(0.002, 10)
    b = lj.Ensemble(boxes)
    b.run(0.002, 20)
    for (pa, va, fa), (pb, vb, fb) in zip(a.state(), b.state()):
        dp = np.abs(pa.astype(np.int64) - pb.astype(np.int64))
        assert np.minimum(dp, 2 ** 32 - dp).max() <= 64
    a.close()
    b.close()


def test_ensemble_autotune_picks_a_listed_shape(lj):
    ens = lj.Ensemble(small_ensemble(nboxes=6, seed=5))
    w, blk = ens.tune(0.002, 5)
    assert w in (2, 4, 8, 16) and blk in (128, 256, 512)
    ens.run(0.002, 5)
    ens.close()


def test_ensemble_barrier_timeout_is_reported(lj):
    """One block leaves before its first barrier; the others' bounded waits run
    out (about a millisecond), the launch ends and the run reports a timeout.
    The context stays usable afterwards."""
    ens = lj.Ensemble(small_ensemble(nboxes=4, seed=9))
    ens.debug(spin_limit=5000, skip_block=0)
    with pytest.raises(lj.LJError, match="TIMEOUT"):
        ens.run(0.002, 3, use_graph=False)
    ens.debug(0, -1)
    ens.run(0.002, 3)
    ens.close()


def test_ensemble_lists_initial_forces_match_oracle(lj):
    """Verlet-list mode: the lists built inside the launch (one warp per cell;
    whole-box lists for the box with fewer than 3 cells of edge r_c + skin)
    give the oracle's forces."""
    boxes = small_ensemble(seed=21)
    assert any(int(np.floor(s.L / 2.8)) < 3 for s in boxes)
    ens = lj.Ensemble(boxes)
    ens.set_lists(0.3, 10)
    ens.run(0.002, 0)
    for s, (pos, vel, frc) in zip(boxes, ens.state()):
        assert np.array_equal(pos, s.pos)
        F_ref, _, _, _ = oracle.forces_bruteforce(s.pos, s.L, 2.5)
        assert rel_err(frc, F_ref) <= 1e-5
    ens.close()


def test_ensemble_lists_match_single_box_list_runs(lj):
    """25 steps with list rebuilds at steps 10 and 20 inside the launch: each
    box follows the single-box Verlet-list path (same lists, same JSPLIT order
    and width) to rounding, and its final forces match the oracle's."""
    boxes = small_ensemble(seed=23)
    ens = lj.Ensemble(boxes)
    ens.set_lists(0.3, 10)
    ens.run(0.002, 25, use_graph=True)
    assert ens.uses_graph(), ens.last_error()
    w = 8
    for s, (pos, vel, frc) in zip(boxes, ens.state()):
        if int(np.floor(s.L / 2.8)) >= 3:
            d = lj.Domain(s.L, 2.5, 0.3)
            d.set_particles(s.pos, s.vel)
            d.integrate(0.002, 25, lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, w), rebuild_every=10)
            p_ref, v_ref = d.state()
            d.close()
            dp = np.abs(pos.astype(np.int64) - p_ref.astype(np.int64))
            assert np.minimum(dp, 2 ** 32 - dp).max() <= 64
        F_orc, _, _, _ = oracle.forces_bruteforce(pos, s.L, 2.5)
        assert rel_err(frc, F_orc) <= 1e-5
    ens.close()


def test_ensemble_lists_skin_rebuild(lj):
    """A particle moving 4 sigma per step leaves its skin in the first step:
    the launch rebuilds the lists before that step's forces, which match the
    oracle's (missing pairs of the moved particle would not)."""
    boxes = small_ensemble(nboxes=4, seed=25)
    vel = boxes[0].vel.copy()
    vel[:, 3] = [2000.0, 0.0, 0.0]
    boxes[0] = W.System(L=boxes[0].L, pos=boxes[0].pos, vel=vel, name="teleport")
    ens = lj.Ensemble(boxes)
    ens.set_lists(0.3, 1000)
    ens.run(0.002, 0)
    ens.run(0.002, 1)
    for s, (pos, _, frc) in zip(boxes, ens.state()):
        F_orc, _, _, _ = oracle.forces_bruteforce(pos, s.L, 2.5)
        assert rel_err(frc, F_orc) <= 1e-5
    ens.set_lists(0.0)                            # back to linked cells
    ens.run(0.002, 2)
    for s, (pos, _, frc) in zip(boxes, ens.state()):
        F_orc, _, _, _ = oracle.forces_bruteforce(pos, s.L, 2.5)
        assert rel_err(frc, F_orc) <= 1e-5
    ens.close()
