"""Run-time tuning on the GPU: full search (Sec. 2.3.2) and the learned tuner
(Sec. 6's data-driven tuning) with the committed model trained on GB300
timings of the density sweep."""
import os
import time

import numpy as np
import pytest

from paper_2512_03565_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lj():
    from paper_2512_03565_gb300 import build as b
    b.build()
    from paper_2512_03565_gb300 import ljgb
    ljgb.load()
    return ljgb


def test_full_search_returns_argmin_of_its_evidence(lj):
    s = W.stratified(60000, 0.6, 41)
    d = lj.Domain(s.L, s.rc, s.skin)
    d.set_particles(s.pos, s.vel)
    cfg, times = d.tune(0, 2)
    timed = {k: v for k, v in times.items() if not np.isnan(v)}
    assert len(timed) == 64
    assert lj.config_name(cfg) == min(timed, key=timed.get)
    d.close()


def test_learned_tuner_without_model_falls_back_to_full_search(lj):
    s = W.stratified(20000, 0.5, 42)
    d = lj.Domain(s.L, s.rc, s.skin)
    d.set_particles(s.pos, s.vel)
    cfg, times = d.tune(1, 1)
    assert lj.load().lj_config_valid(cfg)
    assert sum(not np.isnan(v) for v in times.values()) == 64
    d.close()


@pytest.mark.parametrize("system", [
    lambda: W.stratified(300000, 0.4, 999),
    lambda: W.slab(400000, 0.8, 0.02, 0.5, 998),
    lambda: W.fcc(250000, 1.0, 997),
], ids=["fluid-0.4", "slab-0.5", "fcc-1.0"])
@pytest.mark.skipif(os.environ.get("LJGB_CHECKS", "0") not in ("", "0"),
                    reason="the network ranks the production kernels; the index-check build shifts their relative cost")
def test_learned_tuner_gain_on_held_out_systems(lj, system):
    """The learned tuner as it runs (features -> network, then its three
    highest-ranked configurations timed, 3 evaluations each) is measured
    against full search on systems absent from the training data.  Its choice
    must be within 5% of the measured best (the tuner target; each
    configuration's time is the median of three full searches of 3 evaluations
    each) and no worse than the paper's default order (1/V, here
    VL:JSPLIT-32), and one call must cost a small fraction of one full search's
    tuning time.  The tuner is called five times and the median of its picks'
    times is held to the bound: on these systems the best list orders lie
    within a few percent of each other (6% on the density-0.4 fluid), about as
    far apart as two timings of one order taken seconds apart, so a single pick
    can land on either side of the line."""
    from paper_2512_03565_gb300 import tuner
    s = system()
    model = tuner.load()
    d = lj.Domain(s.L, s.rc, s.skin)
    d.set_particles(s.pos, s.vel)
    t0 = time.perf_counter()
    runs = [d.tune(0, 3)[1]]
    t_full = time.perf_counter() - t0
    runs += [d.tune(0, 3)[1] for _ in range(2)]
    times = {k: float(np.median([r[k] for r in runs])) for k in runs[0]}
    tuner.install(d, model)
    t0 = time.perf_counter()
    picks = [lj.config_name(d.tune(1, 3)[0])]
    t_learned = time.perf_counter() - t0
    picks += [lj.config_name(d.tune(1, 3)[0]) for _ in range(4)]
    d.close()
    best = min(v for v in times.values() if not np.isnan(v))
    t_l = float(np.median([times[p] for p in picks]))
    t_default = times["VL:JSPLIT-32:N3off"]
    assert t_l <= 1.05 * best, (picks, t_l, best)
    assert t_l <= t_default * 1.02
    assert t_learned < 0.1 * t_full


def test_energy_counter_and_energy_tuner(lj):
    """Sec. 2.3.3: energy per evaluation as the tuning metric.  The GPU's
    energy counter only increases; the energy tuner returns the configuration
    of least measured energy per evaluation, with finite times and energies
    for every configuration it ran."""
    e0 = lj.energy_read()
    # up to 2 s: the probe stops after 5 counter updates (about 0.5 s at the
    # GB300's 100 ms period); a counter that does not update twice in 2 s
    # cannot time a tuning batch, which is a property of the driver, not of
    # the library
    period = lj.energy_period(probe_ms=2000.0)
    e1 = lj.energy_read()
    assert e1 >= e0 > 0
    if not np.isfinite(period):
        pytest.skip("the GPU energy counter did not update twice within 2 s")
    assert 0 < period < 1000
    s = W.stratified(60000, 0.6, 43)
    d = lj.Domain(s.L, s.rc, s.skin)
    d.set_particles(s.pos, s.vel)
    cfg, ev = d.tune_energy(min_ms=5 * period)
    d.close()
    ran = {k: v for k, v in ev.items() if not np.isnan(v[1])}
    assert len(ran) == 64
    # power = energy / time per evaluation: a busy GB300 draws between its
    # idle floor and its 1.4 kW limit
    assert all(v[0] > 0 and 100.0 < v[1] / v[0] < 1500.0 for v in ran.values())
    assert lj.config_name(cfg) == min(ran, key=lambda k: ran[k][1])
