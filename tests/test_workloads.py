"""CPU checks of the synthetic input recipes: the named workloads have the
sizes, densities, shapes and velocity statistics they are documented with,
and every generator is a pure function of its seed."""
import math

import numpy as np
import pytest

from paper_2512_03565_gb300 import workloads as W

TWO32 = 2.0 ** 32


def frac(s):
    return s.pos.astype(np.float64) / TWO32


def check_velocities(s, T):
    # centre of mass at rest, temperature exactly T over 3n - 3 degrees of freedom (k_B = 1)
    v = s.vel
    assert v.shape == (3, s.n) and v.dtype == np.float64
    np.testing.assert_allclose(v.mean(axis=1), 0.0, atol=1e-12)
    T_got = s.mass * float((v * v).sum()) / (3 * s.n - 3)
    assert T_got == pytest.approx(T, rel=1e-12)


def min_image_min_distance(s):
    x = frac(s) * s.L
    best = np.inf
    for a in range(0, s.n, 512):
        d = x[:, a:a + 512, None] - x[:, None, :]
        d -= s.L * np.round(d / s.L)
        r2 = (d * d).sum(axis=0)
        idx = np.arange(a, min(a + 512, s.n))
        r2[idx - a, idx] = np.inf
        best = min(best, float(r2.min()))
    return math.sqrt(best)


def test_config1_uniform_1000():
    s = W.config1()
    assert s.n == 1000 and s.pos.dtype == np.uint32 and s.pos.shape == (3, 1000)
    assert s.L == pytest.approx(10.7722, abs=1e-4)
    assert (s.rc, s.skin, s.eps, s.sigma, s.mass) == (2.5, 0.3, 1.0, 1.0, 1.0)
    check_velocities(s, 1.0)
    # uniform: each coordinate's fractions look U[0, 1) (mean 1/2, variance 1/12)
    f = frac(s)
    np.testing.assert_allclose(f.mean(axis=1), 0.5, atol=0.04)
    np.testing.assert_allclose(f.var(axis=1), 1.0 / 12.0, atol=0.01)


def test_config2_fluid_size_and_density():
    assert W.box_edge(1048576, 0.75) == pytest.approx(111.818, abs=1e-3)
    s = W.homogeneous(8000, 0.75, 11)
    assert s.n / s.L ** 3 == pytest.approx(0.75, rel=1e-12)
    check_velocities(s, 1.0)
    # the jittered lattice keeps particles apart (no overlapping pair at start)
    assert min_image_min_distance(s) >= 0.4 * s.L / math.ceil(s.n ** (1 / 3)) - 1e-9
    # homogeneous: the 8 octants hold 1/8 of the particles each
    oct_ = (frac(s) >= 0.5).astype(int)
    counts = np.bincount(oct_[0] + 2 * oct_[1] + 4 * oct_[2], minlength=8)
    np.testing.assert_allclose(counts / s.n, 1 / 8, atol=0.01)


def test_density_sweep_recipe():
    boxes = W.config3(scale=0.02)
    assert len(boxes) == 24
    rhos = [b.n / b.L ** 3 for b in boxes[:16]]
    np.testing.assert_allclose(rhos, np.exp(np.linspace(math.log(0.05), math.log(1.2), 16)), rtol=1e-12)
    for k, b in enumerate(boxes[16:]):
        fr = 0.30 + 0.05 * k
        z = frac(b)[2]
        lo, hi = 0.5 - fr / 2, 0.5 + fr / 2
        inside = (z >= lo) & (z < hi)
        n_liq = inside.sum()
        rho_liq = n_liq / (fr * b.L ** 3)
        rho_vap = (b.n - n_liq) / ((1 - fr) * b.L ** 3)
        assert rho_liq == pytest.approx(0.8, rel=0.02)
        assert rho_vap == pytest.approx(0.02, rel=0.1)


def test_droplet_recipe():
    # the expanding droplet's radius gives 2,000,000 particles at density 0.8
    assert 4 / 3 * math.pi * 84.19 ** 3 * 0.8 == pytest.approx(2.0e6, rel=2e-3)
    s = W.droplet(12.0)
    assert s.L == pytest.approx(4 * 2 * 12.0)
    check_velocities(s, 1.2)
    x = (frac(s) - 0.5) * s.L
    r = np.sqrt((x * x).sum(axis=0))
    a = (4 / 0.8) ** (1 / 3)
    assert r.max() <= 12.0 + 0.02 * a
    assert s.n == pytest.approx(4 / 3 * math.pi * 12.0 ** 3 * 0.8, rel=0.05)
    # nearest neighbours at the FCC spacing a / sqrt(2), up to the jitter
    assert min_image_min_distance(s) >= a / math.sqrt(2) - 0.04 * a


def test_ensemble_recipe():
    boxes = W.config5()
    assert len(boxes) == 256
    ns = np.array([b.n for b in boxes])
    rhos = np.array([b.n / b.L ** 3 for b in boxes])
    assert ns.min() >= 500 and ns.max() <= 50000
    assert rhos.min() >= 0.1 - 1e-12 and rhos.max() <= 1.0 + 1e-12
    # log-uniform N: log N has mean (log 500 + log 50000) / 2, uniform rho has mean 0.55
    assert np.log(ns).mean() == pytest.approx(0.5 * (math.log(500) + math.log(50000)), abs=0.2)
    assert rhos.mean() == pytest.approx(0.55, abs=0.05)


@pytest.mark.parametrize("make", [lambda: W.uniform(500, 0.8, 3), lambda: W.stratified(500, 0.8, 3),
                                  lambda: W.fcc(500, 1.0, 3), lambda: W.slab(800, 0.8, 0.02, 0.4, 3),
                                  lambda: W.droplet(6.0, seed=3), lambda: W.exploding_cube(500, seed=3)])
def test_generators_are_pure_functions_of_the_seed(make):
    a, b = make(), make()
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.vel, b.vel)
    assert a.L == b.L


def test_fixed_point_conversion_wraps_and_floors():
    q = W._frac_to_fp(np.array([0.0, 0.5, 1.0 - 2.0 ** -40, 1.0, -0.25, 1.25]))
    np.testing.assert_array_equal(q, np.array([0, 2 ** 31, 2 ** 32 - 1, 0, 3 * 2 ** 30, 2 ** 30], dtype=np.uint32))
