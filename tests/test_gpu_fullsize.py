"""Parity at the workloads' full sizes, on sampled outputs the oracle computes one
by one (each sampled particle against all others, O(N) each):

* the 1,048,576-particle fluid in the bench's launch configuration (FP32 pair
  math, Verlet lists, JSPLIT-4, Newton-3 off), at the start and after an MD run
  through lj_integrate_step with list rebuilds;
* the 2-million-particle expanding droplet (FCC sphere in a mostly empty box);
* the 256-box batch (3 M particles) in list mode after a rebuild inside the
  launch, sampled box by box.

The scale of the tolerance is the RMS force of the sample."""
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


def sampled_err(pos, L, rc, F, idx):
    F_ref = oracle.forces_sampled(pos, L, rc, idx)
    rms = np.sqrt((F_ref ** 2).sum(0).mean())
    return np.abs(F[:, idx] - F_ref).max() / rms


def test_bench_fluid_full_size(lj):
    s = W.config2()
    assert s.n == 1048576
    cfg = lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP32_ACC64)
    d.set_particles(s.pos, s.vel)
    d.compute_forces(cfg)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(s.n, 1500, replace=False))
    assert sampled_err(s.pos, s.L, s.rc, d.forces(), idx) <= 1e-5
    d.integrate(0.002, 20, cfg, rebuild_every=10)
    pos, _ = d.state()
    d.compute_forces(cfg)
    assert d.counters()[2] >= 2                      # the run rebuilt its lists
    assert sampled_err(pos, s.L, s.rc, d.forces(), idx) <= 1e-5
    d.close()


def test_droplet_full_size(lj):
    s = W.config4()
    assert s.n > 1_900_000
    cfg = lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4)
    d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP32_ACC64)
    d.set_particles(s.pos, s.vel)
    d.integrate(0.002, 10, cfg, rebuild_every=10)
    pos, _ = d.state()
    d.compute_forces(cfg)
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(s.n, 1000, replace=False))
    assert sampled_err(pos, s.L, s.rc, d.forces(), idx) <= 1e-5
    d.close()


def test_ensemble_full_size_lists(lj):
    boxes = W.config5(256)
    ens = lj.Ensemble(boxes)
    ens.set_lists(0.3, 10)
    ens.run(0.002, 12)                                # builds at steps 0 and 10
    state = ens.state()
    ens.close()
    n = np.array([s.n for s in boxes])
    rho = np.array([s.n / s.L ** 3 for s in boxes])
    pick = {int(np.argmax(n)), int(np.argmin(n)), int(np.argmax(rho)), int(np.argmin(rho)), 17, 200}
    rng = np.random.default_rng(3)
    for b in sorted(pick):
        s = boxes[b]
        pos, _, frc = state[b]
        idx = np.sort(rng.choice(s.n, min(s.n, 400), replace=False))
        assert sampled_err(pos, s.L, 2.5, frc, idx) <= 1e-5, b
