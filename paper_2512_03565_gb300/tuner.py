"""Learned configuration tuner: data collection, training and installation.

The paper's full search (Sec. 2.3.2) times every configuration in every tuning
phase; Sec. 6 proposes knowledge-based or data-driven tuning instead.  Here the
data is the library's own full-search timings (lj_tune kind 0) on synthetic
systems shaped like the tuned workloads, the model is the 16-64-64-C network
of k_mlp.cu trained on the GPU by the library's kernels (lj_mlp_train), and
inference runs inside lj_tune kind 1.

Targets are per-row relative log times, log(t_config / t_best), so the network
ranks configurations; missing or invalid configurations are masked out of the
loss.  The network's outputs are the configurations that come within 10 % of
the best in at least one training row.  Features are standardised with the
training set's mean and standard deviation (stored with the model).  Targets,
masks and standardisation are computed by the library (lj_tuner_prepare).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import ljgb as lj

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuner_model.npz")


def config_keys(cfgs):
    return [lj.config_name(c) for c in cfgs]


def collect(systems, samples=3, snapshots=(0,), dt=0.002, cfg_run=None, log=None):
    """Full-search timings of every configuration on each system (and on later
    snapshots of a short MD run).  Returns (X (rows, 16), T (rows, C) ms with NaN
    where not timed, names of the C configurations, row labels)."""
    cfgs = lj.configs()
    names = config_keys(cfgs)
    X, T, labels = [], [], []
    run_cfg = cfg_run or lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4)
    for s in systems:
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        done = 0
        for snap in sorted(snapshots):
            if snap > done:
                d.integrate(dt, snap - done, run_cfg)
                done = snap
            f = d.features()
            _, times = d.tune(0, samples)
            X.append(f)
            T.append([times.get(nm, float("nan")) for nm in names])
            labels.append(f"{s.name} rc={s.rc} step={snap}")
            if log:
                best = min((v for v in T[-1] if not math.isnan(v)), default=float("nan"))
                log(f"{labels[-1]}: best {best:.4f} ms")
        d.close()
    return np.array(X), np.array(T, dtype=np.float64), names, labels


def valid(T):
    """Timed entries of a timing table (NaN or non-positive = not timed)."""
    return np.isfinite(T) & (T > 0)


def candidates(T, near=1.10):
    """Configurations within `near` of some row's best in the timings T: the
    only ones the network ranks (it has no evidence that the others ever win,
    and each extra output is one more chance of a wrong pick on a system
    unlike the training data)."""
    ok = valid(T)
    best = np.min(np.where(ok, T, np.inf), axis=1, keepdims=True)
    return (ok & (T <= near * best)).any(axis=0)


def prepare(X, T):
    """Training inputs on the GPU (lj_tuner_prepare): relative log times
    log(t / t_best) per row and their mask, and the standardised features with
    the columns' mean and standard deviation."""
    return lj.tuner_prepare(T, X)


def train(X, T, epochs=3000, lr=3e-3, seed=0, near=1.10):
    """Trains the network on the GPU over the candidate configurations of T
    (see `candidates`).  Returns the model dict; model["keep"] marks T's
    columns that are the network's outputs, in order."""
    keep = candidates(T, near)
    Y, M, Xs, mean, std = prepare(X, T[:, keep])
    Cn = int(keep.sum())
    rng = np.random.default_rng(seed)
    P = lj.mlp_nparams(Cn)
    p0 = np.zeros(P)
    sizes = [(64, 16), (64,), (64, 64), (64,), (Cn, 64), (Cn,)]
    off = 0
    for sh in sizes:
        k = int(np.prod(sh))
        if len(sh) == 2:
            p0[off:off + k] = rng.normal(0.0, 1.0 / math.sqrt(sh[1]), size=k)
        off += k
    params, losses = lj.mlp_train(p0, Cn, Xs, Y, M, epochs, lr)
    return {"params": params.astype(np.float32), "mean": mean, "std": std, "C": Cn, "losses": losses, "keep": keep}


def predict(model, X):
    Xs = (np.asarray(X, dtype=np.float64) - model["mean"]) / model["std"]
    return lj.mlp_forward(model["params"], int(model["C"]), Xs)


def save(model, names, path=MODEL_PATH, meta=None):
    """Saves the model with the names of its outputs (the kept columns of `names`)."""
    keep = model.get("keep")
    out_names = list(names) if keep is None else [n for n, k in zip(names, keep) if k]
    np.savez(path, params=model["params"], mean=model["mean"], std=model["std"], C=int(model["C"]),
             names=np.array(out_names), losses=model.get("losses", np.zeros(1)),
             meta=json.dumps(meta or {}))


def load(path=MODEL_PATH):
    z = np.load(path, allow_pickle=False)
    names = [str(v) for v in z["names"]]
    by_name = {lj.config_name(c): c for c in lj.configs()}
    cfgs = [by_name[n] for n in names]
    return {"params": z["params"], "mean": z["mean"], "std": z["std"], "C": int(z["C"]), "cfgs": cfgs,
            "names": names, "meta": json.loads(str(z["meta"]))}


def install(domain, model):
    """Loads the model into a context for lj_tune kind 1."""
    domain.set_tuner_model(model["params"], int(model["C"]), model["mean"], model["std"], model["cfgs"])
