"""The C-ABI library's host code built with AddressSanitizer and
UndefinedBehaviorSanitizer (host compiler only; the device code is
unchanged), driven through the CPU ABI tests: argument validation, the
configuration space, the full-search selection rule with injected timings and
the missing-energy-counter status.  Any out-of-bounds access, use after free
or undefined behaviour in that host code aborts the child process."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_abi_host_code_under_address_and_ub_sanitizers(tmp_path):
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not libasan or not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("no AddressSanitizer runtime")
    from paper_2512_03565_gb300 import build as b
    lib = b.build(out=str(tmp_path / "san"),
                  host_flags=("-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=undefined",
                              "-fno-omit-frame-pointer"))
    env = dict(os.environ, LD_PRELOAD=libasan, LJGB_LIB=lib, PYTHONPATH=ROOT,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:halt_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    env.pop("LJGB_CHECKS", None)
    # host-logic tests only: the ones that run nvcc or import the bench would
    # inherit the preloaded sanitizer runtime
    skip = "not index_check_build and not bench and not unit_rates"
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        os.path.join(ROOT, "tests", "test_abi.py"), "-k", skip],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0 and " passed" in p.stdout, (p.stdout[-3000:], p.stderr[-4000:])
    assert "ERROR: AddressSanitizer" not in p.stderr and "runtime error" not in p.stderr, p.stderr[-4000:]
