"""The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer (host
only), driven through its Python layer on small systems: cell binning, linked
cells, Verlet lists, brute force, sampled forces, velocity Verlet, features,
the MLP and the cluster lists.  Any out-of-bounds access, use after free or
undefined behaviour aborts the child process."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, oracle
from paper_2512_03565_gb300 import workloads as W
rng = np.random.default_rng(5)
for L, n in [(3.3, 20), (5.0, 120), (4.0, 300)]:
    pos = rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    oracle.forces_bruteforce(pos, L, 1.0)
    oracle.forces_sampled(pos, L, 1.0, np.arange(0, n, 3))
    nc = oracle.ncells(L, 1.0)
    oracle.bin_cells(pos, nc)
    oracle.pairs_cells(pos, L, 1.0, nc)
    oracle.pairs_bruteforce(pos, L, 1.0)
    oracle.verlet(pos, L, 1.0, nc, 0, 8)      # small capacity: the overflow path
    oracle.verlet(pos, L, 1.0, nc, 1, 256)
    oracle.forces_cells(pos, L, 1.0)
    oracle.features(pos, L, 1.0, 0.2)
    for M in (1, 4, 6, 8):
        oracle.vcl_lists(pos, L, 1.2, M, 0)
        oracle.vcl_lists(pos, L, 1.2, M, 1)
s = W.stratified(500, 0.7, 3)
oracle.vv_run(s.pos, s.vel, s.L, s.rc, 1.0, 0.002, 5, use_cells=True)
P = oracle.mlp_nparams(7)
p = rng.normal(0, 0.1, size=P)
X = rng.normal(size=(9, 16)); T = rng.normal(size=(9, 7)); Mk = np.ones((9, 7))
oracle.mlp_forward(p, 7, X)
oracle.mlp_loss_grad(p, 7, X, T, Mk)
print("sanitized oracle ok")
'''


def test_oracle_under_address_and_ub_sanitizers(tmp_path):
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not libasan or not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("no AddressSanitizer runtime")
    so = tmp_path / "liboracle_san.so"
    r = subprocess.run(["gcc", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-std=gnu11", "-o", str(so), os.path.join(ROOT, "oracle", "lj_oracle.c"), "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_PRELOAD=libasan, LJ_ORACLE_LIB=str(so), OMP_NUM_THREADS="2",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", PYTHONPATH=ROOT)
    p = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0 and "sanitized oracle ok" in p.stdout, (p.stdout[-2000:], p.stderr[-4000:])
