"""FP64 CPU oracle for the Lennard-Jones short-range force path (arXiv 2512.03565).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product
library never loads it, and it shares no code with the CUDA path: the C source
``lj_oracle.c`` is written directly from the paper's definitions (Sec. 2.1
Eq. 1, the cutoff and Newton's third law; Sec. 2.1.1 linked cells and Verlet
lists; Sec. 4.1 Algorithm 1's pair kernel, taken as textbook LJ 12-6; Sec. 6's
data-driven tuning for the MLP).

Every function here is a thin ctypes marshalling layer over ``lj_oracle.c``;
arrays are numpy, positions are uint32 fixed point (u = L / 2^32) in SoA form
``(3, n)``.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(closed forms, FCC lattice sums, invariants, brute-force equality, finite
differences).  Nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lj_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile lj_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # LJ_ORACLE_LIB: an alternative build of lj_oracle.c (the sanitizer test)
        lib = C.CDLL(os.environ.get("LJ_ORACLE_LIB") or build())
        i64, f64, u32, u64, i32 = C.c_int64, C.c_double, C.c_uint32, C.c_uint64, C.c_int
        vp = C.c_void_p
        sig = {
            "orc_num_threads": (i32, []),
            "orc_set_threads": (None, [i32]),
            "orc_cut2_int": (u64, [f64, f64]),
            "orc_r2_int": (u64, [u32, u32, u32, u32, u32, u32]),
            "orc_quantize": (u32, [f64, f64]),
            "orc_forces_bruteforce": (i64, [i64, _U32P, _U32P, _U32P, f64, f64, f64, f64,
                                            _F64P, _F64P, _F64P, vp, vp]),
            "orc_forces_sampled": (None, [i64, _U32P, _U32P, _U32P, f64, f64, f64, f64, i64,
                                          _I64P, _F64P, _F64P, _F64P]),
            "orc_pairs_bruteforce": (i64, [i64, _U32P, _U32P, _U32P, f64, f64, vp]),
            "orc_ncells": (i32, [f64, f64]),
            "orc_cell_of": (u32, [u32, u32, u32, i32]),
            "orc_bin_cells": (i32, [i64, _U32P, _U32P, _U32P, i32, _U32P, _U32P]),
            "orc_pairs_cells": (i64, [i64, _U32P, _U32P, _U32P, f64, f64, i32, vp]),
            "orc_verlet": (i32, [i64, _U32P, _U32P, _U32P, f64, f64, i32, i32, i32, _U32P, _U32P,
                                 _I32P, _I32P]),
            "orc_forces_cells": (i64, [i64, _U32P, _U32P, _U32P, f64, f64, f64, f64,
                                       _F64P, _F64P, _F64P, vp, vp]),
            "orc_vv_run": (i32, [i64, _U32P, _U32P, _U32P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                 _F64P, f64, f64, i32, f64, f64, f64, f64, i32, vp, vp]),
            "orc_features": (i32, [i64, _U32P, _U32P, _U32P, f64, f64, f64, _F64P]),
            "orc_vcl_ntower": (i32, [i64, i32]),
            "orc_vcl_order": (i64, [i64, _U32P, _U32P, _U32P, i32, _U32P, _U32P]),
            "orc_vcl_lists": (i32, [i64, _U32P, _U32P, _U32P, _U32P, _U32P, f64, f64, i32, i32, i32, _I32P, _I32P,
                                    _U64P]),
            "orc_mlp_nparams": (i64, [i32]),
            "orc_mlp_forward": (None, [_F64P, i32, i64, _F64P, _F64P]),
            "orc_mlp_loss_grad": (f64, [_F64P, i32, i64, _F64P, _F64P, _F64P, _F64P]),
            "orc_adam_step": (None, [i64, _F64P, _F64P, _F64P, _F64P, f64, f64, f64, f64, i32]),
            "orc_tuner_targets": (None, [i64, i32, _F64P, _F64P, _F64P]),
            "orc_standardize": (None, [i64, i32, _F64P, _F64P, _F64P, _F64P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _soa(pos):
    p = np.ascontiguousarray(pos, dtype=np.uint32)
    if p.ndim != 2 or p.shape[0] != 3:
        raise ValueError("positions must be uint32 of shape (3, n)")
    return np.ascontiguousarray(p[0]), np.ascontiguousarray(p[1]), np.ascontiguousarray(p[2])


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def cut2_int(L: float, r: float) -> int:
    """floor((r/u)^2), u = L/2^32, exact (reading R2)."""
    return int(_load().orc_cut2_int(float(L), float(r)))


def r2_int(pi, pj) -> int:
    return int(_load().orc_r2_int(*(int(v) for v in pi), *(int(v) for v in pj)))


def quantize(x: float, L: float) -> int:
    return int(_load().orc_quantize(float(x), float(L)))


def forces_bruteforce(pos, L, rc, eps=1.0, sigma=1.0):
    """O(N^2) minimum-image LJ (Eq. 1, cutoff, textbook 12-6).  Returns (F (3,n), U, W, npairs)."""
    x, y, z = _soa(pos)
    n = x.shape[0]
    F = np.zeros((3, n))
    fx, fy, fz = (np.zeros(n) for _ in range(3))
    U, W = C.c_double(0.0), C.c_double(0.0)
    npairs = _load().orc_forces_bruteforce(n, x, y, z, L, rc, eps, sigma, fx, fy, fz,
                                           C.addressof(U), C.addressof(W))
    F[0], F[1], F[2] = fx, fy, fz
    return F, U.value, W.value, int(npairs)


def forces_sampled(pos, L, rc, idx, eps=1.0, sigma=1.0):
    """Forces on particles idx only, each against all others.  Returns (3, len(idx))."""
    x, y, z = _soa(pos)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    fx, fy, fz = (np.zeros(idx.shape[0]) for _ in range(3))
    _load().orc_forces_sampled(x.shape[0], x, y, z, L, rc, eps, sigma, idx.shape[0], idx, fx, fy, fz)
    return np.stack([fx, fy, fz])


def pairs_bruteforce(pos, L, r):
    """All pairs i<j with 0 < R^2 <= floor((r/u)^2), lexicographic, as (m, 2) int32."""
    x, y, z = _soa(pos)
    lib = _load()
    n = x.shape[0]
    m = lib.orc_pairs_bruteforce(n, x, y, z, L, r, None)
    out = np.zeros((max(m, 1), 2), dtype=np.int32)
    lib.orc_pairs_bruteforce(n, x, y, z, L, r, out.ctypes.data)
    return out[:m]


def ncells(L, edge_min) -> int:
    return int(_load().orc_ncells(float(L), float(edge_min)))


def cell_of(p, nc) -> int:
    return int(_load().orc_cell_of(int(p[0]), int(p[1]), int(p[2]), int(nc)))


def bin_cells(pos, nc):
    """Stable counting sort by cell id (reading R3).  Returns (perm, cell_start)."""
    x, y, z = _soa(pos)
    n = x.shape[0]
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    cs = np.zeros(nc ** 3 + 1, dtype=np.uint32)
    _load().orc_bin_cells(n, x, y, z, nc, perm, cs)
    return perm[:n], cs


def pairs_cells(pos, L, r, nc):
    """Pair set of the 27-cell linked-cell scan (cells of edge >= r), as (m, 2) int32 sorted."""
    x, y, z = _soa(pos)
    lib = _load()
    n = x.shape[0]
    m = lib.orc_pairs_cells(n, x, y, z, L, r, nc, None)
    if m < 0:
        raise ValueError("need at least 3 cells per dimension")
    out = np.zeros((max(m, 1), 2), dtype=np.int32)
    lib.orc_pairs_cells(n, x, y, z, L, r, nc, out.ctypes.data)
    return out[:m]


def verlet(pos, L, rl, nc, half, cap):
    """Verlet lists in sorted-index space (reading R4).

    Returns (perm, cell_start, nbr (n, cap) int32, nnbr (n,), overflow flag)."""
    x, y, z = _soa(pos)
    n = x.shape[0]
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    cs = np.zeros(nc ** 3 + 1, dtype=np.uint32)
    nbr = np.full((max(n, 1), cap), -1, dtype=np.int32)
    nnbr = np.zeros(max(n, 1), dtype=np.int32)
    r = _load().orc_verlet(n, x, y, z, L, rl, nc, int(bool(half)), cap, perm, cs, nbr, nnbr)
    if r < 0:
        raise ValueError("need at least 3 cells per dimension")
    return perm[:n], cs, nbr[:n], nnbr[:n], bool(r)


def vcl_ntower(n, M) -> int:
    """Towers per axis of the cluster grid (reading R19): the largest k >= 1 with k^3 M <= n."""
    return int(_load().orc_vcl_ntower(int(n), int(M)))


def vcl_order(pos, M):
    """Cluster order (reading R19).  Returns (perm, cl_start): perm[k] is the
    original index of the k-th particle in cluster order, cluster c holds
    perm[cl_start[c]:cl_start[c+1]]."""
    x, y, z = _soa(pos)
    n = x.shape[0]
    perm = np.zeros(n, dtype=np.uint32)
    cls = np.zeros(n + 1, dtype=np.uint32)
    ncl = _load().orc_vcl_order(n, x, y, z, int(M), perm, cls)
    if ncl < 0:
        raise ValueError("need n >= 1 and M >= 1")
    return perm, cls[:ncl + 1].copy()


def vcl_lists(pos, L, rl, M, half, masks=False):
    """Cluster-pair lists by brute force over all cluster pairs and their
    member pairs (readings R19, R21): I lists J iff some member pair lies
    within r_l.  Returns (perm, cl_start, lists): lists[I] the ascending
    neighbour clusters of I; with masks=True also the per-entry member masks
    (bit a * M + b for the a-th member of I and the b-th of J)."""
    x, y, z = _soa(pos)
    perm, cls = vcl_order(pos, M)
    ncl = cls.shape[0] - 1
    nn = np.zeros(max(ncl, 1), dtype=np.int32)
    cap = max(ncl, 1)
    nbr = np.zeros((max(ncl, 1), cap), dtype=np.int32)
    mk = np.zeros((max(ncl, 1), cap), dtype=np.uint64)
    r = _load().orc_vcl_lists(ncl, perm, cls, x, y, z, L, rl, int(bool(half)), int(M), cap, nbr, nn, mk)
    if r != 0:
        raise ValueError("cluster lists failed")
    lists = [nbr[I, :nn[I]].copy() for I in range(ncl)]
    if masks:
        return perm, cls, lists, [mk[I, :nn[I]].copy() for I in range(ncl)]
    return perm, cls, lists


def forces_cells(pos, L, rc, eps=1.0, sigma=1.0):
    """Linked-cell FP64 forces (same definition as the brute force).  Returns (F, U, W, npairs)."""
    x, y, z = _soa(pos)
    n = x.shape[0]
    fx, fy, fz = (np.zeros(n) for _ in range(3))
    U, W = C.c_double(0.0), C.c_double(0.0)
    npairs = _load().orc_forces_cells(n, x, y, z, L, rc, eps, sigma, fx, fy, fz,
                                      C.addressof(U), C.addressof(W))
    if npairs < 0:
        raise ValueError("need at least 3 cells per dimension")
    return np.stack([fx, fy, fz]), U.value, W.value, int(npairs)


def vv_run(pos, vel, L, rc, mass, dt, nsteps, eps=1.0, sigma=1.0, use_cells=True, forces=None):
    """Velocity Verlet (Sec. 2.1).  Returns (pos, vel, F, U, W) after nsteps."""
    x, y, z = (a.copy() for a in _soa(pos))
    v = np.ascontiguousarray(vel, dtype=np.float64).copy()
    vx, vy, vz = (np.ascontiguousarray(v[a]).copy() for a in range(3))
    if forces is None:
        if use_cells:
            F, _, _, _ = forces_cells(np.stack([x, y, z]), L, rc, eps, sigma)
        else:
            F, _, _, _ = forces_bruteforce(np.stack([x, y, z]), L, rc, eps, sigma)
    else:
        F = np.asarray(forces, dtype=np.float64)
    fx, fy, fz = (np.ascontiguousarray(F[a]).copy() for a in range(3))
    U, W = C.c_double(0.0), C.c_double(0.0)
    r = _load().orc_vv_run(x.shape[0], x, y, z, vx, vy, vz, fx, fy, fz, mass, dt, nsteps, L, rc,
                           eps, sigma, int(bool(use_cells)), C.addressof(U), C.addressof(W))
    if r != 0:
        raise ValueError("vv_run failed")
    return np.stack([x, y, z]), np.stack([vx, vy, vz]), np.stack([fx, fy, fz]), U.value, W.value


def features(pos, L, rc, skin):
    """The 16 tuner features (see lj_oracle.c)."""
    x, y, z = _soa(pos)
    out = np.zeros(16)
    if _load().orc_features(x.shape[0], x, y, z, L, rc, skin, out) != 0:
        raise ValueError("bad arguments")
    return out


def mlp_nparams(C_out: int) -> int:
    return int(_load().orc_mlp_nparams(int(C_out)))


def mlp_forward(params, C_out, X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.zeros((X.shape[0], C_out))
    _load().orc_mlp_forward(np.ascontiguousarray(params, dtype=np.float64), C_out, X.shape[0], X, Y)
    return Y


def mlp_loss_grad(params, C_out, X, T, mask):
    X = np.ascontiguousarray(X, dtype=np.float64)
    g = np.zeros(mlp_nparams(C_out))
    loss = _load().orc_mlp_loss_grad(np.ascontiguousarray(params, dtype=np.float64), C_out,
                                     X.shape[0], X, np.ascontiguousarray(T, dtype=np.float64),
                                     np.ascontiguousarray(mask, dtype=np.float64), g)
    return float(loss), g


def adam_step(params, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays params, m, v."""
    _load().orc_adam_step(params.shape[0], params, np.ascontiguousarray(grad, dtype=np.float64),
                          m, v, lr, beta1, beta2, eps, int(t))


def tuner_targets(T):
    """Relative log times log(t / t_best) per row and the validity mask (NaN or
    non-positive times are not valid)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    M, Cn = T.shape
    Y, mask = np.zeros_like(T), np.zeros_like(T)
    _load().orc_tuner_targets(M, Cn, T, Y, mask)
    return Y, mask


def standardize(X):
    """Per-column mean and population standard deviation (below 1e-12: 1) and
    the standardised rows.  Returns (Xs, mean, std)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    M, F = X.shape
    Xs, mean, sd = np.zeros_like(X), np.zeros(F), np.zeros(F)
    _load().orc_standardize(M, F, X, Xs, mean, sd)
    return Xs, mean, sd
