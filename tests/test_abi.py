"""CPU-only checks of the C ABI library: it loads without a GPU, exports every
entry point include/ljgb.h declares, validates arguments on the host, and its
host-side tuning rule (Sec. 2.3.2 full search: reduce each configuration's
samples, take the fastest) picks the argmin of injected fake timings."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lj():
    from paper_2512_03565_gb300 import build as b
    b.build()
    from paper_2512_03565_gb300 import ljgb
    ljgb.load()
    return ljgb


def header_symbols():
    src = open(os.path.join(ROOT, "include", "ljgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lj_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lj):
    lib = C.CDLL(lj.LIB_PATH)
    names = header_symbols()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lj.exported_symbols()) == set(names)


def test_init_domain_rejects_bad_arguments_on_host(lj):
    lib = lj.load()
    h = C.c_void_p()
    box = (C.c_double * 3)(10.0, 10.0, 10.0)
    bad = [
        ((C.c_double * 3)(10.0, 11.0, 10.0), 2.5, 0.3),   # not cubic
        (box, 0.0, 0.3),                                  # cutoff <= 0
        (box, 2.5, -0.1),                                 # negative skin
        (box, 4.0, 1.1),                                  # rc + skin >= L/2
    ]
    for b, rc, skin in bad:
        assert lib.lj_init_domain(C.byref(h), b, rc, skin, 1.0, 1.0, 1, None) == lj.LJ_ERR_ARG
    assert lib.lj_init_domain(C.byref(h), box, 2.5, 0.3, 0.0, 1.0, 1, None) == lj.LJ_ERR_ARG
    assert lib.lj_init_domain(C.byref(h), box, 2.5, 0.3, 1.0, 1.0, 7, None) == lj.LJ_ERR_ARG
    assert lib.lj_init_domain(None, box, 2.5, 0.3, 1.0, 1.0, 1, None) == lj.LJ_ERR_ARG


def test_config_space(lj):
    cfgs = lj.configs()
    names = [lj.config_name(c) for c in cfgs]
    assert len(names) == len(set(names)) == 64
    assert all(lj.load().lj_config_valid(c) for c in cfgs)
    # invalid combinations are masked (cf. the paper's lc_c01, usable only without Newton3)
    for bad in [lj.config(lj.LJ_LC, lj.LJ_ORD_VL_IPT), lj.config(lj.LJ_LC, lj.LJ_ORD_KI, 3),
                lj.config(lj.LJ_LC, lj.LJ_ORD_JSPLIT, 64), lj.config(lj.LJ_LC, lj.LJ_ORD_IPT_SMEM, 0, 2),
                lj.config(lj.LJ_VL, lj.LJ_ORD_ROT32), lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4, 2),
                lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4, lj.LJ_N3_ATOMIC_BWD),
                lj.config(lj.LJ_VL, lj.LJ_ORD_VL_IPT, 0, lj.LJ_N3_ATOMIC_BWD),
                lj.config(lj.LJ_LC, lj.LJ_ORD_ROT32, 0, 4), lj.config(lj.LJ_VCL, lj.LJ_ORD_CL_TILE, 5),
                lj.config(lj.LJ_VCL, lj.LJ_ORD_JSPLIT, 4), lj.config(lj.LJ_VCL, lj.LJ_ORD_CL_JLANE, 8, 2),
                lj.config(lj.LJ_LC, lj.LJ_ORD_CL_TILE, 4), lj.config(3, 0),
                lj.config(lj.LJ_LCS, lj.LJ_ORD_JSPLIT, 32), lj.config(lj.LJ_LCS, lj.LJ_ORD_IPT_SMEM),
                lj.config(lj.LJ_LCS, lj.LJ_ORD_JSPLIT, 4, lj.LJ_N3_TWOPASS), lj.config(4, 3, 4)]:
        assert not lj.load().lj_config_valid(bad)


def test_tune_select_is_argmin_of_reduced_evidence(lj):
    rng = np.random.default_rng(3)
    for reduce in (0, 1):
        for _ in range(50):
            n_cfg, s = rng.integers(2, 40), rng.integers(1, 10)
            t = rng.uniform(0.1, 5.0, size=(n_cfg, s))
            t[rng.random((n_cfg, s)) < 0.1] = np.nan
            valid = (rng.random(n_cfg) < 0.8).astype(np.int32)
            red = np.where(np.isnan(t), np.inf if reduce else 0.0, t)
            cnt = (~np.isnan(t)).sum(1)
            v = red.min(1) if reduce else np.where(cnt > 0, red.sum(1) / np.maximum(cnt, 1), np.inf)
            v = np.where((valid == 1) & (cnt > 0), v, np.inf)
            want = int(np.argmin(v)) if np.isfinite(v).any() else -1
            assert lj.tune_select(t, valid, reduce) == want


def test_tune_select_edge_cases(lj):
    assert lj.tune_select(np.full((3, 2), np.nan)) == -1
    assert lj.tune_select(np.array([[1.0], [1.0], [0.5]]), np.array([1, 1, 0])) == 0   # ties keep the first
    assert lj.tune_select(np.array([[2.0, 0.1], [1.0, 1.0]]), reduce=1) == 0
    assert lj.tune_select(np.array([[2.0, 0.1], [1.0, 1.0]]), reduce=0) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    from paper_2512_03565_gb300 import ljgb
    mod = importlib.reload(ljgb)
    monkeypatch.setattr(mod, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mod, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mod.load()
    importlib.reload(ljgb)


def test_energy_counter_absent_is_a_status_not_a_crash():
    """Without a GPU (or NVML) the energy path returns a status code."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: covered by the GPU tests")
    from paper_2512_03565_gb300 import ljgb as lj
    with pytest.raises(lj.LJError) as e:
        lj.energy_read()
    assert e.value.status in (lj.LJ_ERR_STATE, lj.LJ_ERR_CUDA)


def test_bench_tables_cover_every_configuration(lj):
    """bench.py's per-mode figures (flops per pair) exist for every Newton-3 mode of the configuration list."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_module", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert {c.newton3 for c in lj.configs()} <= set(bench.FLOPS_PER_PAIR)
    # the roof of a launch: a Verlet-list launch (1M particles, 75.7 entries of
    # 4 B each, 25 M pairs x 23 flops) lies below the ridge, a linked-cell one
    # (positions and forces only) above it
    cfg_vl = lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4)
    cfg_lc = lj.config(lj.LJ_LC, lj.LJ_ORD_JSPLIT, 4)
    n, pairs = 1048576, 25.25e6
    vl_bytes = bench.algorithmic_bytes(cfg_vl, n, int(75.7 * n))
    assert vl_bytes == 16.0 * n + 24.0 * n + 4.0 * int(75.7 * n) + 4.0 * n
    assert bench.roofline_bound(23 * pairs, vl_bytes, 80.5, 6780.0)[0] == "hbm"
    assert bench.roofline_bound(23 * pairs, bench.algorithmic_bytes(cfg_lc, n, None), 80.5, 6780.0)[0] == "alu"
    # the committed ncu figures of the benched kernel parse, and the traffic is
    # at least the list entries and positions one launch must read
    traffic = bench.from_profiles("traffic", "VL:JSPLIT-4:N3off")
    assert traffic is not None and traffic > 303e6
    assert 0 < bench.from_profiles("l1_lsu_pct", "VL:JSPLIT-4:N3off") <= 100
    assert 0 < bench.from_profiles("issue_pct", "VL:JSPLIT-4:N3off") <= 100
    assert bench.from_profiles("traffic", "no such configuration") is None


def test_index_check_build_compiles_and_exports_the_same_symbols(lj):
    # LJGB_CHECKS=1 builds a second library whose kernels check every index
    # they follow; it must compile and keep the ABI of the default build
    import shutil
    import subprocess
    import sys
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    env = dict(os.environ, LJGB_CHECKS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "paper_2512_03565_gb300", "build.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    path = r.stdout.strip().splitlines()[-1]
    assert os.path.basename(os.path.dirname(path)) == "_build_checks" and path != lj.LIB_PATH
    lib = C.CDLL(path)
    missing = [n for n in header_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_handles_close_once_and_work_as_context_managers(lj, monkeypatch):
    # the binding's lifetime rules, without a GPU: close() destroys the handle
    # once, and leaving a with-block closes it
    calls = []

    class FakeLib:
        def lj_destroy(self, h):
            calls.append(("ctx", h.value))

        def lj_ensemble_destroy(self, h):
            calls.append(("ens", h.value))

    for cls, kind in ((lj.Domain, "ctx"), (lj.Ensemble, "ens")):
        obj = cls.__new__(cls)
        obj.lib, obj.h = FakeLib(), lj._VP(1234)
        with obj as o:
            assert o is obj
        assert calls[-1] == (kind, 1234) and not obj.h
        obj.close()
        assert len([c for c in calls if c[0] == kind]) == 1


def test_unit_rates_program_compiles(tmp_path):
    # the per-SM throughput probe behind the FP32-pair design builds for sm_103a
    import shutil
    import subprocess
    nvcc = os.environ.get("NVCC", "nvcc")
    if shutil.which(nvcc) is None:
        pytest.skip("nvcc not available")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-c",
                        os.path.join(ROOT, "paper_2512_03565_gb300", "unit_rates.cu"), "-o",
                        str(tmp_path / "unit_rates.o")], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
