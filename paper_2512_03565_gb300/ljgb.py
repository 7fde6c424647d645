"""Thin Python binding of the C ABI in include/ljgb.h (argument marshalling only).

Every computation runs in libljgb.so's CUDA kernels; nothing here computes
forces, cells, lists or integration steps.  The functions keep the C names
(``lj_init_domain``, ``lj_compute_forces``, ...) and ``Domain`` wraps one
context.  Arrays may be numpy arrays (host) or torch tensors (device or
host); positions and forces are SoA, shape (3, n).

If the library has not been built this module raises on load: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LJGB_CHECKS=1 selects the build with device index checks (see build.py);
# LJGB_LIB names another build of the same library (e.g. one with host-side
# sanitizers)
LIB_PATH = os.environ.get("LJGB_LIB") or os.path.join(
    _HERE, "_build_checks" if os.environ.get("LJGB_CHECKS", "0") not in ("", "0") else "_build", "libljgb.so")

# lj_status
LJ_OK, LJ_ERR_ARG, LJ_ERR_CUDA, LJ_ERR_CAPACITY, LJ_ERR_SKIN, LJ_ERR_NONFINITE, LJ_ERR_TIMEOUT, \
    LJ_ERR_STATE, LJ_ERR_OOM = range(9)
STATUS_NAMES = ["LJ_OK", "LJ_ERR_ARG", "LJ_ERR_CUDA", "LJ_ERR_CAPACITY", "LJ_ERR_SKIN",
                "LJ_ERR_NONFINITE", "LJ_ERR_TIMEOUT", "LJ_ERR_STATE", "LJ_ERR_OOM"]
LJ_PREC_FP64, LJ_PREC_FP32_ACC64 = 0, 1
LJ_LC, LJ_VL, LJ_VCL, LJ_LCS = 0, 1, 2, 3
LJ_ORD_IPT_SMEM, LJ_ORD_IPT_TMA, LJ_ORD_KI, LJ_ORD_JSPLIT, LJ_ORD_ROT32, LJ_ORD_VL_IPT, LJ_ORD_CL_TILE, \
    LJ_ORD_CL_JLANE = range(8)
LJ_N3_OFF, LJ_N3_ATOMIC, LJ_N3_TWOPASS, LJ_N3_ATOMIC_BWD = 0, 1, 2, 3
ORDER_NAMES = ["IPT_SMEM", "IPT_TMA", "KI", "JSPLIT", "ROT32", "VL_IPT", "CL_TILE", "CL_JLANE"]


class lj_config(C.Structure):
    _fields_ = [("container", C.c_int32), ("order", C.c_int32), ("param", C.c_int32), ("newton3", C.c_int32)]

    def __repr__(self):
        return config_name(self)

    def key(self):
        return (self.container, self.order, self.param, self.newton3)


def config(container, order, param=0, newton3=LJ_N3_OFF) -> lj_config:
    return lj_config(container, order, param, newton3)


def config_name(c: lj_config) -> str:
    cont = {LJ_LC: "LC", LJ_VL: "VL", LJ_VCL: "VCL", LJ_LCS: "LCS"}.get(c.container, f"c{c.container}")
    o = ORDER_NAMES[c.order] if 0 <= c.order < len(ORDER_NAMES) else f"ord{c.order}"
    p = f"-{c.param}" if c.param else ""
    n3 = ["N3off", "N3atomic", "N3twopass", "N3bwd"][c.newton3] if 0 <= c.newton3 <= 3 else f"n3={c.newton3}"
    return f"{cont}:{o}{p}:{n3}"


class LJError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


_lib = None
_lock = threading.Lock()

_VP = C.c_void_p
_SIGS = {
    "lj_init_domain": (C.c_int, [C.POINTER(_VP), C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_int, _VP]),
    "lj_set_particles": (C.c_int, [_VP, C.c_int64, _VP, _VP, C.c_double, C.c_int]),
    "lj_set_particles_fp": (C.c_int, [_VP, C.c_int64, _VP, _VP, C.c_double, C.c_int]),
    "lj_update_positions": (C.c_int, [_VP, _VP, C.c_int32]),
    "lj_bin_cells": (C.c_int, [_VP, C.c_int32]),
    "lj_build_verlet": (C.c_int, [_VP, C.c_int32]),
    "lj_build_clusters": (C.c_int, [_VP, C.c_int32, C.c_int32]),
    "lj_get_clusters": (C.c_int, [_VP, C.POINTER(C.c_int64), _VP, C.POINTER(C.c_int32)]),
    "lj_get_cluster_lists": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int32)]),
    "lj_get_cluster_masks": (C.c_int, [_VP, _VP]),
    "lj_tuner_prepare": (C.c_int, [_VP, C.c_int64, C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "lj_compute_forces": (C.c_int, [_VP, lj_config, _VP, _VP]),
    "lj_config_valid": (C.c_int32, [lj_config]),
    "lj_config_list": (C.c_int32, [_VP, C.c_int32]),
    "lj_integrate_step": (C.c_int, [_VP, C.c_double, C.c_int32, C.c_int32, lj_config]),
    "lj_tune": (C.c_int, [_VP, C.c_int32, C.c_int32, C.POINTER(lj_config), _VP]),
    "lj_energy_read": (C.c_int, [C.c_int32, C.POINTER(C.c_double)]),
    "lj_energy_period": (C.c_int, [C.c_int32, C.c_double, C.POINTER(C.c_double)]),
    "lj_tune_energy": (C.c_int, [_VP, C.c_double, C.POINTER(lj_config), _VP, _VP]),
    "lj_tune_select": (C.c_int32, [_VP, C.c_int32, C.c_int32, _VP, C.c_int32]),
    "lj_features": (C.c_int, [_VP, _VP]),
    "lj_tuner_set_model": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP, _VP]),
    "lj_mlp_forward": (C.c_int, [_VP, C.c_int32, _VP, C.c_int64, _VP, _VP]),
    "lj_mlp_loss_grad": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, C.c_int64, _VP, _VP, _VP]),
    "lj_mlp_train": (C.c_int, [_VP, _VP, _VP, C.c_int64, C.c_int32, _VP, C.c_int32, C.c_float, _VP, _VP]),
    "lj_get_forces": (C.c_int, [_VP, _VP, C.c_int32]),
    "lj_get_state": (C.c_int, [_VP, _VP, _VP, C.c_int32]),
    "lj_get_pairs": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int64), _VP]),
    "lj_get_cells": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int32)]),
    "lj_get_verlet": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int32)]),
    "lj_get_counters": (C.c_int, [_VP, _VP]),
    "lj_kinetic_energy": (C.c_int, [_VP, C.POINTER(C.c_double)]),
    "lj_timing": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP]),
    "lj_bin_cells_static": (C.c_int, [_VP, C.c_int64, C.c_int32, _VP, _VP, _VP]),
    "lj_ensemble_create": (C.c_int, [C.POINTER(_VP), C.c_int32, _VP, _VP, _VP, _VP, C.c_double, C.c_double,
                                     C.c_double, C.c_double, _VP]),
    "lj_ensemble_set_lists": (C.c_int, [_VP, C.c_double, C.c_int32, C.c_int32]),
    "lj_ensemble_run": (C.c_int, [_VP, C.c_double, C.c_int32, C.c_int32]),
    "lj_ensemble_tune": (C.c_int, [_VP, C.c_double, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lj_ensemble_get": (C.c_int, [_VP, _VP, _VP, _VP]),
    "lj_ensemble_debug": (C.c_int, [_VP, C.c_uint32, C.c_int32]),
    "lj_ensemble_size": (C.c_int64, [_VP]),
    "lj_ensemble_uses_graph": (C.c_int32, [_VP]),
    "lj_ensemble_last_error": (C.c_char_p, [_VP]),
    "lj_ensemble_pairs": (C.c_int64, [_VP]),
    "lj_ensemble_destroy": (None, [_VP]),
    "lj_last_error": (C.c_char_p, [_VP]),
    "lj_destroy": (None, [_VP]),
}


def exported_symbols():
    """Names of the entry points this binding expects the library to export."""
    return list(_SIGS)


def energy_read(device=-1):
    """The GPU's total-energy counter in millijoules (NVML), or raises LJError."""
    v = C.c_double()
    st = load().lj_energy_read(int(device), C.byref(v))
    if st != LJ_OK:
        raise LJError(st, "GPU energy counter unavailable")
    return v.value


def energy_period(device=-1, probe_ms=500.0):
    """Median update interval (ms) of the GPU's total-energy counter."""
    v = C.c_double()
    st = load().lj_energy_period(int(device), float(probe_ms), C.byref(v))
    if st != LJ_OK:
        raise LJError(st, "GPU energy counter unavailable")
    return v.value


def load():
    """Load libljgb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build() or python paper_2512_03565_gb300/build.py)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.uint32: torch.int32, np.float32: torch.float32}[dtype]
        t = x
        if dtype is np.uint32:
            if t.dtype not in (torch.int32, torch.uint32):
                raise TypeError("fixed-point positions must be a 32-bit integer tensor")
        elif t.dtype != want:
            raise TypeError(f"expected {want}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr(), int(t.is_cuda), t
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def configs():
    lib = load()
    n = lib.lj_config_list(None, 0)
    arr = (lj_config * n)()
    lib.lj_config_list(C.cast(arr, _VP), n)
    return [lj_config(a.container, a.order, a.param, a.newton3) for a in arr]


class Domain:
    """One library context: a cubic periodic box of LJ particles."""

    def __init__(self, L, rc=2.5, skin=0.3, eps=1.0, sigma=1.0, precision=LJ_PREC_FP32_ACC64, stream=None):
        self.lib = load()
        self.h = _VP()
        box = (C.c_double * 3)(L, L, L)
        st = self.lib.lj_init_domain(C.byref(self.h), box, rc, skin, eps, sigma, precision, _stream_ptr(stream))
        if st != LJ_OK:
            raise LJError(st, "lj_init_domain failed")
        self.L, self.rc, self.skin, self.eps, self.sigma, self.precision = L, rc, skin, eps, sigma, precision
        self.n = 0

    def _check(self, st):
        if st != LJ_OK:
            raise LJError(st, self.lib.lj_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.lj_destroy(self.h)
            self.h = _VP()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, pos, vel=None, mass=1.0, fixed_point=None):
        """pos: (3, n) float64 coordinates or uint32 fixed point; vel: (3, n) float64 or None."""
        if fixed_point is None:
            fixed_point = (pos.dtype == np.uint32) if not _is_torch(pos) else (str(pos.dtype) in ("torch.int32", "torch.uint32"))
        n = int(pos.shape[-1])
        pp, pdev, keep_p = _ptr(pos, np.uint32 if fixed_point else np.float64)
        vp, vdev, keep_v = _ptr(vel, np.float64)
        if vel is not None and vdev != pdev:
            raise ValueError("positions and velocities must both be on the device or both on the host")
        fn = self.lib.lj_set_particles_fp if fixed_point else self.lib.lj_set_particles
        self._check(fn(self.h, n, pp, vp, mass, pdev))
        self.n = n
        self.mass = mass

    def update_positions(self, pos):
        """New (3, n) float64 coordinates of the loaded particles (caller's
        order); cell order and Verlet lists are kept while the skin allows."""
        pp, pdev, keep = _ptr(pos, np.float64)
        self._check(self.lib.lj_update_positions(self.h, pp, pdev))

    def bin_cells(self, container):
        self._check(self.lib.lj_bin_cells(self.h, container))

    def build_verlet(self, half=False):
        self._check(self.lib.lj_build_verlet(self.h, int(bool(half))))

    def build_clusters(self, M, half=False):
        """Cluster order and cluster-pair lists for cluster size M (4, 6 or 8)."""
        self._check(self.lib.lj_build_clusters(self.h, int(M), int(bool(half))))

    def compute_forces(self, cfg, energy=False):
        """One force evaluation; with energy=True returns (U, W)."""
        if energy:
            U, W = C.c_double(), C.c_double()
            self._check(self.lib.lj_compute_forces(self.h, cfg, C.byref(U), C.byref(W)))
            return U.value, W.value
        self._check(self.lib.lj_compute_forces(self.h, cfg, None, None))
        return None

    def forces(self, out=None):
        """Forces (3, n) float64 in original order; into `out` (a device tensor, or a host tensor, written
        directly by the kernel when pinned) if given."""
        if out is not None:
            p, dev, _ = _ptr(out, np.float64)
            self._check(self.lib.lj_get_forces(self.h, p, dev))
            return out
        F = np.empty((3, self.n))
        self._check(self.lib.lj_get_forces(self.h, F.ctypes.data, 0))
        return F

    def state(self):
        pos = np.empty((3, self.n), dtype=np.uint32)
        vel = np.empty((3, self.n))
        self._check(self.lib.lj_get_state(self.h, pos.ctypes.data, vel.ctypes.data, 0))
        return pos, vel

    def integrate(self, dt, nsteps, cfg, rebuild_every=10):
        self._check(self.lib.lj_integrate_step(self.h, dt, nsteps, rebuild_every, cfg))

    def pairs(self, container):
        m = C.c_int64()
        self._check(self.lib.lj_get_pairs(self.h, container, C.byref(m), None))
        out = np.zeros((max(m.value, 1), 2), dtype=np.int32)
        self._check(self.lib.lj_get_pairs(self.h, container, C.byref(m), out.ctypes.data))
        return out[:m.value]

    def cells(self):
        nc = C.c_int32()
        self._check(self.lib.lj_get_cells(self.h, None, None, C.byref(nc)))
        perm = np.zeros(self.n, dtype=np.uint32)
        cs = np.zeros(nc.value ** 3 + 1, dtype=np.uint32)
        self._check(self.lib.lj_get_cells(self.h, perm.ctypes.data, cs.ctypes.data, C.byref(nc)))
        return perm, cs, nc.value

    def verlet(self):
        cap = C.c_int32()
        self._check(self.lib.lj_get_verlet(self.h, None, None, C.byref(cap)))
        nbr = np.zeros((self.n, cap.value), dtype=np.int32)
        nn = np.zeros(self.n, dtype=np.int32)
        self._check(self.lib.lj_get_verlet(self.h, nbr.ctypes.data, nn.ctypes.data, C.byref(cap)))
        return nbr, nn

    def clusters(self):
        """(cl_start (ncl + 1,), n_t) of the current cluster order."""
        ncl, nt = C.c_int64(), C.c_int32()
        self._check(self.lib.lj_get_clusters(self.h, C.byref(ncl), None, C.byref(nt)))
        cs = np.zeros(ncl.value + 1, dtype=np.uint32)
        self._check(self.lib.lj_get_clusters(self.h, C.byref(ncl), cs.ctypes.data, C.byref(nt)))
        return cs, nt.value

    def cluster_lists(self):
        """Neighbour cluster indices per cluster (a list of int32 arrays, library order)."""
        cs, _ = self.clusters()
        ncl = len(cs) - 1
        cap = C.c_int32()
        self._check(self.lib.lj_get_cluster_lists(self.h, None, None, C.byref(cap)))
        nbr = np.zeros((max(ncl, 1), cap.value), dtype=np.int32)
        nn = np.zeros(max(ncl, 1), dtype=np.int32)
        self._check(self.lib.lj_get_cluster_lists(self.h, nbr.ctypes.data, nn.ctypes.data, C.byref(cap)))
        return [nbr[I, :nn[I]].copy() for I in range(ncl)]


    def cluster_masks(self):
        """Member masks of the cluster-pair lists (a list of uint64 arrays, in
        the order of cluster_lists)."""
        cap = C.c_int32()
        ncl = C.c_int64()
        self._check(self.lib.lj_get_clusters(self.h, C.byref(ncl), None, None))
        nn = np.zeros(max(ncl.value, 1), dtype=np.int32)
        self._check(self.lib.lj_get_cluster_lists(self.h, None, nn.ctypes.data, C.byref(cap)))
        m = np.zeros((max(ncl.value, 1), max(cap.value, 1)), dtype=np.uint64)
        self._check(self.lib.lj_get_cluster_masks(self.h, m.ctypes.data))
        return [m[I, :nn[I]].copy() for I in range(ncl.value)]
    def counters(self):
        c = np.zeros(5, dtype=np.int64)
        self._check(self.lib.lj_get_counters(self.h, c.ctypes.data))
        return c

    def timing(self, enable=-1):
        """Returns (force-kernel ms, timed evaluations, total kernel launches); enable 1/0
        restarts/stops the force-kernel event timing, -1 leaves it as is."""
        ms, n, tot = C.c_double(), C.c_int64(), C.c_int64()
        self._check(self.lib.lj_timing(self.h, enable, C.byref(ms), C.byref(n), C.byref(tot)))
        return ms.value, n.value, tot.value

    def kinetic_energy(self):
        v = C.c_double()
        self._check(self.lib.lj_kinetic_energy(self.h, C.byref(v)))
        return v.value

    def features(self):
        f = np.zeros(16)
        self._check(self.lib.lj_features(self.h, f.ctypes.data))
        return f

    def tune(self, kind=0, samples=3):
        all_cfg = configs()
        times = np.full(len(all_cfg), np.nan)
        chosen = lj_config()
        self._check(self.lib.lj_tune(self.h, kind, samples, C.byref(chosen), times.ctypes.data))
        return chosen, dict(zip((config_name(c) for c in all_cfg), times))

    def tune_energy(self, min_ms=1000.0):
        """Full search by energy per evaluation (GPU energy counter); returns the
        chosen configuration and {name: (ms, mJ) per evaluation}."""
        all_cfg = configs()
        t = np.full(len(all_cfg), np.nan)
        e = np.full(len(all_cfg), np.nan)
        chosen = lj_config()
        self._check(self.lib.lj_tune_energy(self.h, float(min_ms), C.byref(chosen), t.ctypes.data, e.ctypes.data))
        return chosen, {config_name(c): (float(a), float(b)) for c, a, b in zip(all_cfg, t, e)}

    def set_tuner_model(self, params, C_out, mean, std, cfgs):
        p = np.ascontiguousarray(params, dtype=np.float32)
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(std, dtype=np.float32)
        arr = (lj_config * C_out)(*cfgs)
        self._check(self.lib.lj_tuner_set_model(self.h, p.ctypes.data, C_out, m.ctypes.data, s.ctypes.data,
                                                C.cast(arr, _VP)))


class Ensemble:
    """Many independent boxes advanced by one persistent launch (lj_ensemble_*)."""

    def __init__(self, systems, rc=2.5, eps=1.0, sigma=1.0, mass=1.0, stream=None):
        self.lib = load()
        self.h = _VP()
        self.systems = systems
        Ls = np.array([s.L for s in systems], dtype=np.float64)
        counts = np.array([s.n for s in systems], dtype=np.int64)
        pos = np.concatenate([np.ascontiguousarray(s.pos, dtype=np.uint32).ravel() for s in systems])
        vel = np.concatenate([np.ascontiguousarray(s.vel, dtype=np.float64).ravel() for s in systems])
        st = self.lib.lj_ensemble_create(C.byref(self.h), len(systems), Ls.ctypes.data, counts.ctypes.data,
                                         pos.ctypes.data, vel.ctypes.data, rc, eps, sigma, mass,
                                         _stream_ptr(stream))
        if st != LJ_OK:
            raise LJError(st, "lj_ensemble_create failed")
        self.counts = counts
        self.n = int(counts.sum())

    def run(self, dt, nsteps, use_graph=True):
        st = self.lib.lj_ensemble_run(self.h, dt, nsteps, int(bool(use_graph)))
        if st != LJ_OK:
            raise LJError(st, "lj_ensemble_run failed")

    def set_lists(self, skin=0.3, rebuild_every=10, cap=0):
        """Verlet-list mode (skin > 0) or linked cells (skin = 0) for the batch."""
        st = self.lib.lj_ensemble_set_lists(self.h, float(skin), int(rebuild_every), int(cap))
        if st != LJ_OK:
            raise LJError(st, self.lib.lj_ensemble_last_error(self.h).decode())

    def tune(self, dt=0.002, steps=10):
        w, b = C.c_int32(), C.c_int32()
        st = self.lib.lj_ensemble_tune(self.h, dt, steps, C.byref(w), C.byref(b))
        if st != LJ_OK:
            raise LJError(st, "lj_ensemble_tune failed")
        return w.value, b.value

    def state(self):
        pos = np.zeros(3 * self.n, dtype=np.uint32)
        vel = np.zeros(3 * self.n)
        frc = np.zeros(3 * self.n)
        st = self.lib.lj_ensemble_get(self.h, pos.ctypes.data, vel.ctypes.data, frc.ctypes.data)
        if st != LJ_OK:
            raise LJError(st, "lj_ensemble_get failed")
        out, off = [], 0
        for nb in self.counts:
            sl = slice(3 * off, 3 * (off + nb))
            out.append((pos[sl].reshape(3, nb), vel[sl].reshape(3, nb), frc[sl].reshape(3, nb)))
            off += nb
        return out

    def uses_graph(self):
        return bool(self.lib.lj_ensemble_uses_graph(self.h))

    def last_error(self):
        return self.lib.lj_ensemble_last_error(self.h).decode()

    def pairs(self):
        """Unique in-cutoff pairs over the force evaluations since the last call."""
        return int(self.lib.lj_ensemble_pairs(self.h))

    def debug(self, spin_limit=0, skip_block=-1):
        self.lib.lj_ensemble_debug(self.h, spin_limit, skip_block)

    def close(self):
        if self.h:
            self.lib.lj_ensemble_destroy(self.h)
            self.h = _VP()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_select(timings, valid=None, reduce=0) -> int:
    t = np.ascontiguousarray(timings, dtype=np.float64)
    v = None if valid is None else np.ascontiguousarray(valid, dtype=np.int32)
    return int(load().lj_tune_select(t.ctypes.data, t.shape[0], t.shape[1], None if v is None else v.ctypes.data, reduce))


def mlp_nparams(C_out: int) -> int:
    return 64 * 16 + 64 + 64 * 64 + 64 + C_out * 64 + C_out


def tuner_prepare(T, X):
    """lj_tuner_prepare: (Y, mask, Xs, mean, std), float32."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    M, Cn = T.shape
    Y, mask = np.zeros((M, Cn), dtype=np.float32), np.zeros((M, Cn), dtype=np.float32)
    Xs = np.zeros((M, X.shape[1]), dtype=np.float32)
    mean, std = np.zeros(X.shape[1], dtype=np.float32), np.zeros(X.shape[1], dtype=np.float32)
    st = load().lj_tuner_prepare(T.ctypes.data, M, Cn, X.ctypes.data, Y.ctypes.data, mask.ctypes.data,
                                 Xs.ctypes.data, mean.ctypes.data, std.ctypes.data, None)
    if st != LJ_OK:
        raise LJError(st, "lj_tuner_prepare failed")
    return Y, mask, Xs, mean, std


def mlp_forward(params, C_out, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    Y = np.zeros((X.shape[0], C_out), dtype=np.float32)
    st = load().lj_mlp_forward(p.ctypes.data, C_out, X.ctypes.data, X.shape[0], Y.ctypes.data, None)
    if st != LJ_OK:
        raise LJError(st, "lj_mlp_forward failed")
    return Y


def mlp_loss_grad(params, C_out, X, T, mask):
    X = np.ascontiguousarray(X, dtype=np.float32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    M = np.ascontiguousarray(mask, dtype=np.float32)
    g = np.zeros(p.shape[0], dtype=np.float32)
    loss = C.c_float()
    st = load().lj_mlp_loss_grad(p.ctypes.data, C_out, X.ctypes.data, T.ctypes.data, M.ctypes.data, X.shape[0],
                                 g.ctypes.data, C.byref(loss), None)
    if st != LJ_OK:
        raise LJError(st, "lj_mlp_loss_grad failed")
    return float(loss.value), g


def mlp_train(params, C_out, X, T, mask, epochs, lr):
    X = np.ascontiguousarray(X, dtype=np.float32)
    p = np.array(params, dtype=np.float32, copy=True)
    T = np.ascontiguousarray(T, dtype=np.float32)
    M = np.ascontiguousarray(mask, dtype=np.float32)
    losses = np.zeros(epochs + 1, dtype=np.float32)
    st = load().lj_mlp_train(X.ctypes.data, T.ctypes.data, M.ctypes.data, X.shape[0], C_out, p.ctypes.data,
                             epochs, lr, losses.ctypes.data, None)
    if st != LJ_OK:
        raise LJError(st, "lj_mlp_train failed")
    return p, losses
