"""Experiment drivers for the tuned force path (run on a GB300).

* ``density_sweep``: labelled rows for the learned tuner: the 24 density-sweep
  boxes (16 homogeneous, rho 0.05..1.2; 8 liquid/vapour slabs) at cutoffs 2.5
  and 3.0, each timed by full search (every configuration) on snapshots of a
  short MD run.
* ``leave_one_out``: trains the network without the rows of one box and ranks
  that box's configurations; reports the regret of the learned choice against
  the measured best and against a fixed default order.
* ``droplet``: the expanding droplet (FCC liquid sphere in a vacuum box)
  integrated for many steps with re-tuning every ``phase`` steps, in three arms:
  full search at every phase, the learned tuner, and the best single fixed
  configuration in hindsight (from the full-search evidence of every phase).

* ``ensemble``: the 256-box batch in one persistent launch vs the same boxes
  run one after another, on linked cells and on Verlet lists.

* ``energy``: time and energy per evaluation of every configuration on four
  systems, and whether the runtime-best and energy-best choices differ.

* ``ensemble-launch``: one direct launch of the list-mode batch (for ncu).

* ``clusters``: Verlet cluster lists (Sec. 5.1's cluster-size dimension):
  per cluster size and order, the force-kernel time on fixed lists, the
  tuning-cost time (rebuild amortised) and the candidate pairs per particle,
  beside the particle Verlet lists, on fluid, slab, dilute gas and FCC solid.

* ``traversal``: the linked-cell Newton-3 orders with the forward and the
  backward half shell (the two roles a cell can take in a cell pair, Sec.
  5.1) on homogeneous, slab and solid systems, in both pair precisions.

* ``precision``: the FP32-pair error of every configuration against the FP64
  oracle (max |dF| / RMS |F|) on the densest workloads (FCC at 1.2 and 1.0,
  the fluid at 0.75, a gas at 0.1), with the lengths over which a lane sums
  in FP32 (list entries and linked-cell candidates per particle).

* ``c2-sweep``: the 1,048,576-particle fluid MD run (100 steps, lists rebuilt
  every 10) with every valid configuration, 5 fresh runs each: the mean
  force-kernel time over steps 10-100, minimum over the runs.

* ``force-launch``: a few force evaluations of one configuration on the
  homogeneous fluid (density 0.75, r_c 2.5, skin 0.3) after a warm-up one,
  for kernel profilers (FP32 pair arithmetic unless ``--fp64``; energy and
  virial with ``--energy``); ``mlp-launch``: one forward and one gradient pass of
  the tuner network on a batch of rows; ``aux-launch``: the auxiliary kernels
  (features, pair lister, 16-bit list copy, getters, quantisation, the
  allocation-free binning, tuner training inputs, a few training epochs) once
  each on a 60,000-particle fluid.

Usage: python -m paper_2512_03565_gb300.experiments sweep|train|droplet|ensemble|ensemble-launch|energy|traversal|clusters|c2-sweep
       [options]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import ljgb as lj
from . import tuner
from . import workloads as W


def density_sweep(scale=1.0, cutoffs=(2.5, 3.0), snapshots=(0, 50, 100), samples=3, out=None, log=print,
                  vacuum=True):
    X, T, labels, box_ids = [], [], [], []
    names = None
    box = 0
    for rc in cutoffs:
        systems = W.config3(rc=rc, scale=scale) + (W.vacuum_extension(rc) if vacuum else [])
        for s in systems:
            t0 = time.time()
            x, t, nm, lb = tuner.collect([s], samples=samples, snapshots=snapshots)
            names = nm
            X.append(x)
            T.append(t)
            labels += lb
            box_ids += [box] * x.shape[0]
            box += 1
            log(f"{s.name} rc={rc}: {x.shape[0]} rows in {time.time() - t0:.1f} s")
    X, T = np.concatenate(X), np.concatenate(T)
    if out:
        np.savez(out, X=X, T=T, names=np.array(names), labels=np.array(labels), box=np.array(box_ids))
    return X, T, names, labels, np.array(box_ids)


def regret_of(pred, t_row, mask_row):
    """Time of the predicted best valid configuration over the measured best."""
    p = np.where(mask_row, pred, np.inf)
    k = int(np.argmin(p))
    best = np.nanmin(np.where(mask_row, t_row, np.nan))
    return t_row[k] / best, k


def leave_one_out(X, T, box_ids, names, epochs=2000, lr=3e-3, default="VL:JSPLIT-32:N3off", log=print):
    M = tuner.valid(T)
    res = []
    d_idx = names.index(default) if default in names else None
    for b in np.unique(box_ids):
        tr, te = box_ids != b, box_ids == b
        model = tuner.train(X[tr], T[tr], epochs=epochs, lr=lr)
        cols = np.where(model["keep"])[0]
        pred = tuner.predict(model, X[te])
        for r, row in enumerate(np.where(te)[0]):
            reg, kk = regret_of(pred[r], T[row, cols], M[row, cols])
            k = int(cols[kk])
            best = np.nanmin(np.where(M[row], T[row], np.nan))
            dflt = T[row, d_idx] / best if d_idx is not None and M[row, d_idx] else float("nan")
            res.append({"box": int(b), "row": int(row), "learned_regret": float(reg),
                        "learned_choice": names[k], "best": names[int(np.nanargmin(np.where(M[row], T[row], np.nan)))],
                        "default_regret": float(dflt)})
        log(f"box {b}: mean regret {np.mean([x['learned_regret'] for x in res if x['box'] == b]):.3f}")
    return res


def droplet(radius=84.19, steps=10000, phase=500, samples=3, arms=("exhaustive", "learned"), model_path=None,
            confirm=2, dt=0.002, log=print):
    """Expanding droplet with re-tuning every `phase` steps.  Per phase each arm
    records the tuning time and the synchronised wall time of integrating the
    phase (force kernels, list builds, binning, integration).  The hindsight
    best fixed configuration comes from the full-search evidence."""
    s = W.config4(radius)
    log(f"droplet: n={s.n} L={s.L:.1f}")
    out = {"n": s.n, "L": s.L, "steps": steps, "phase": phase, "arms": {}}
    names = [lj.config_name(c) for c in lj.configs()]
    evidence = []
    for arm in arms:
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        if arm == "learned":
            tuner.install(d, tuner.load(model_path or tuner.MODEL_PATH))
        run_ms, force_ms, tune_ms, tune_evals, choices, phase_ms = 0.0, 0.0, 0.0, 0, [], []
        for ph in range(steps // phase):
            d.counters()
            t0 = time.perf_counter()
            if arm == "exhaustive":
                cfg, times = d.tune(0, samples)
                evidence.append([times.get(nm, float("nan")) for nm in names])
                tune_evals += sum(1 for v in times.values() if not math.isnan(v)) * (samples + 1)
            else:
                cfg, times = d.tune(1, confirm)
                n_timed = sum(1 for v in times.values() if not math.isnan(v))
                tune_evals += n_timed * (3 + 1)
            tune_ms += (time.perf_counter() - t0) * 1e3
            d.timing(1)
            d.counters()
            t0 = time.perf_counter()
            d.integrate(dt, phase, cfg)
            d.counters()  # synchronises
            pm = (time.perf_counter() - t0) * 1e3
            fms, _, _ = d.timing(0)
            run_ms += pm
            force_ms += fms
            phase_ms.append(pm)
            choices.append(lj.config_name(cfg))
            log(f"{arm} phase {ph}: {lj.config_name(cfg)} run {pm:.1f} ms force {fms:.1f} ms")
        out["arms"][arm] = {"run_ms": run_ms, "force_ms": force_ms, "tune_ms": tune_ms, "tune_evals": tune_evals,
                            "tuning_step_fraction": tune_evals / steps, "choices": choices, "phase_ms": phase_ms}
        d.close()
    if evidence:
        E = np.array(evidence)
        tot = np.nansum(np.where(np.isfinite(E), E, np.inf), axis=0)
        k = int(np.argmin(tot))
        out["best_fixed_in_hindsight"] = names[k]
        out["evidence"] = {"names": names, "ms": E.tolist()}
    if "exhaustive" in out["arms"] and "learned" in out["arms"]:
        ex, le = out["arms"]["exhaustive"], out["arms"]["learned"]
        out["learned_over_exhaustive_run"] = le["run_ms"] / ex["run_ms"]
        out["learned_over_exhaustive_with_tuning"] = (le["run_ms"] + le["tune_ms"]) / (ex["run_ms"] + ex["tune_ms"])
    return out


def ensemble(nboxes=256, steps=1000, dt=0.002, seq_boxes=None, lists=False, log=print):
    """The batched ensemble: `nboxes` boxes (N log-uniform in [500, 50000], rho
    uniform in [0.1, 1.0]) for `steps` steps in one persistent launch per run,
    replayed as a CUDA graph, after the launch-shape autotuner; compared with
    the same boxes integrated one after another through the single-box path.
    lists=True runs the batch on Verlet lists (skin 0.3, rebuilt every 10
    steps inside the launch) and the single-box runs on the same list order."""
    boxes = W.config5(nboxes)
    ntot = sum(s.n for s in boxes)
    log(f"ensemble: {nboxes} boxes, {ntot} particles, {'Verlet lists' if lists else 'linked cells'}")
    ens = lj.Ensemble(boxes)
    if lists:
        ens.set_lists(0.3, 10)
    w, blk = ens.tune(dt, 10)
    ens.run(dt, 0)                   # initial forces
    ens.run(dt, 10)                  # warm-up, capture
    ens.pairs()
    t0 = time.perf_counter()
    ens.run(dt, steps, use_graph=True)
    t_ens = time.perf_counter() - t0
    pairs = ens.pairs()
    graph = ens.uses_graph()
    ens.close()
    seq = list(range(len(boxes))) if seq_boxes is None else list(seq_boxes)
    t_seq, n_seq = 0.0, 0
    cfg = lj.config(lj.LJ_VL if lists else lj.LJ_LC, lj.LJ_ORD_JSPLIT, w)
    edge = 2.8 if lists else 2.5
    for k in seq:
        s = boxes[k]
        if int(np.floor(s.L / edge)) < 3:
            continue                 # the single-box path needs >= 3 cells per axis
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        d.integrate(dt, 1, cfg)
        d.counters()
        t0 = time.perf_counter()
        d.integrate(dt, steps, cfg)
        d.counters()
        t_seq += time.perf_counter() - t0
        n_seq += s.n
        d.close()
    out = {"boxes": nboxes, "particles": ntot, "steps": steps, "lists": lists, "w": w, "block": blk, "graph": graph,
           "ensemble_s": t_ens, "pairs_per_s": pairs / t_ens, "particle_steps_per_s": ntot * steps / t_ens,
           "sequential_s": t_seq, "sequential_particles": n_seq,
           "sequential_particle_steps_per_s": n_seq * steps / t_seq if t_seq else None}
    if t_seq:
        out["speedup_vs_sequential"] = out["particle_steps_per_s"] / out["sequential_particle_steps_per_s"]
    log(json.dumps(out))
    return out


def energy(min_ms=1000.0, log=print):
    """Energy vs runtime as the tuning metric (Sec. 2.3.3, Sec. 5.2): every
    configuration's time and energy per evaluation (GPU energy counter) on a
    homogeneous fluid, a dilute gas, a dense FCC solid and a liquid/vapour
    slab; reports whether the runtime-best and energy-best choices differ."""
    period = lj.energy_period(probe_ms=1000.0)
    window = max(min_ms, 8.0 * period) if np.isfinite(period) else min_ms
    systems = [W.config2(), W.homogeneous(500_000, 0.1, W.BASE_SEED + 71), W.fcc(1_000_000, 1.0, W.BASE_SEED + 72),
               W.slab(400_000, 0.8, 0.02, 0.5, W.BASE_SEED + 73)]
    out = {"counter_period_ms": period, "window_ms": window, "systems": []}
    for s in systems:
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        cfg, ev = d.tune_energy(min_ms=window)
        d.close()
        ran = {k: v for k, v in ev.items() if not np.isnan(v[1])}
        t_best = min(ran, key=lambda k: ran[k][0])
        e_best = min(ran, key=lambda k: ran[k][1])
        r = {"system": s.name, "n": s.n, "runtime_best": t_best, "energy_best": e_best,
             "energy_of_runtime_best_over_best": ran[t_best][1] / ran[e_best][1],
             "time_of_energy_best_over_best": ran[e_best][0] / ran[t_best][0],
             "watts_runtime_best": ran[t_best][1] / ran[t_best][0], "configs": ran}
        out["systems"].append(r)
        log(f"{s.name}: runtime-best {t_best} ({ran[t_best][0]:.4f} ms, {ran[t_best][1]:.1f} mJ), "
            f"energy-best {e_best} ({ran[e_best][0]:.4f} ms, {ran[e_best][1]:.1f} mJ)")
    return out


def traversal(n=500_000, samples=5, log=print):
    """Sec. 5.1: the same pairs, with the roles of the two cells of every cell
    pair swapped.  Full-search times (rebin included, as in tuning) of every
    linked-cell order with the forward (LJ_N3_ATOMIC) and the backward
    (LJ_N3_ATOMIC_BWD) half shell; the ratio backward / forward per order and
    whether the best linked-cell configuration changes direction."""
    systems = [W.stratified(n, 0.75, W.BASE_SEED + 81), W.slab(n, 0.8, 0.02, 0.5, W.BASE_SEED + 82),
               W.slab(n, 0.8, 0.02, 0.2, W.BASE_SEED + 83), W.fcc(n, 1.0, W.BASE_SEED + 84)]
    out = []
    for s in systems:
        for prec in (lj.LJ_PREC_FP32_ACC64, lj.LJ_PREC_FP64):
            d = lj.Domain(s.L, s.rc, s.skin, precision=prec)
            d.set_particles(s.pos, s.vel)
            _, times = d.tune(0, samples)
            d.close()
            ratio = {}
            for k, v in times.items():
                if k.startswith("LC:") and k.endswith(":N3atomic"):
                    ratio[k[3:-len(":N3atomic")]] = times[k[:-len("N3atomic")] + "N3bwd"] / v
            lc = {k: v for k, v in times.items() if k.startswith("LC:") and not k.endswith("N3off")}
            best_lc = min(lc, key=lc.get)
            r = {"system": s.name, "n": s.n, "precision": prec, "bwd_over_fwd": ratio,
                 "best_lc_n3": best_lc, "best_overall": min(times, key=times.get), "times_ms": times}
            out.append(r)
            log(f"{s.name} prec={prec}: best LC Newton-3 {best_lc}; bwd/fwd " +
                " ".join(f"{k}={v:.3f}" for k, v in sorted(ratio.items())))
    return out


def c2_sweep(steps=100, skip=10, repeats=5, dt=0.002, only=None, log=print):
    """The 1,048,576-particle fluid (density 0.75, skin 0.3, lists rebuilt every
    10 steps) run with every valid configuration: `repeats` fresh MD runs of
    `steps` velocity-Verlet steps from the same start; per run the mean
    force-kernel time over steps skip..steps (CUDA events around each force
    launch), per configuration the minimum over the runs, with the whole-step
    wall time (host-synchronised) and the unique in-cutoff pairs of the last
    evaluation.  Caches are not flushed between steps.  `only`: run just the
    configurations whose name contains one of these substrings."""
    import torch
    s = W.config2()
    out = {}
    for cfg in lj.configs():
        name = lj.config_name(cfg)
        if only and not any(o in name for o in only):
            continue
        force, step, pairs = [], [], 0
        for _ in range(repeats):
            d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP32_ACC64)
            d.set_particles(s.pos, s.vel)
            d.integrate(dt, skip, cfg, rebuild_every=10)
            torch.cuda.synchronize()
            d.timing(1)
            t0 = time.perf_counter()
            d.integrate(dt, steps - skip, cfg, rebuild_every=10)
            torch.cuda.synchronize()
            step.append((time.perf_counter() - t0) / (steps - skip) * 1e3)
            ms, k, _ = d.timing(0)
            force.append(ms / max(k, 1))
            pairs = int(d.counters()[1])
            d.close()
        out[name] = {"force_ms": min(force), "force_ms_runs": force, "step_ms": min(step), "pairs": pairs}
        log(f"{name}: force {min(force):.4f} ms (min of {repeats}), step {min(step):.4f} ms, pairs {pairs}")
    return out


def clusters(samples=5, evals=20, log=print):
    """Sec. 5.1, cluster sizes: every cluster-list configuration (orders
    CL_TILE / CL_JLANE, M = 4, 6, 8, Newton-3 off / atomic) against the best
    particle Verlet-list configuration.  Per system: full-search times
    (rebuild amortised), force-kernel time on fixed lists (CUDA events over
    `evals` evaluations), and the candidate pairs per particle that the
    cluster lists hand to the kernel (sum over cluster pairs of |I| |J|,
    full lists) against the particle lists' entries."""
    systems = [W.config2(), W.slab(500_000, 0.8, 0.02, 0.5, W.BASE_SEED + 91),
               W.stratified(500_000, 0.1, W.BASE_SEED + 92), W.fcc(500_000, 1.0, W.BASE_SEED + 93)]
    out = []
    for s in systems:
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        _, times = d.tune(0, samples)
        vl = {k: v for k, v in times.items() if k.startswith("VL:")}
        best_vl = min(vl, key=vl.get)
        kernel = {}
        cfgs = [c for c in lj.configs() if c.container == lj.LJ_VCL]
        by_name = {lj.config_name(c): c for c in lj.configs()}
        for cfg in [by_name[best_vl]] + cfgs:
            d.compute_forces(cfg)
            d.timing(1)
            for _ in range(evals):
                d.compute_forces(cfg)
            ms, n, _ = d.timing(0)
            kernel[lj.config_name(cfg)] = ms / max(n, 1)
        cand, masked = {}, {}
        for M in (4, 6, 8):
            d.build_clusters(M, 0)
            cs, _ = d.clusters()
            sizes = np.diff(cs).astype(np.int64)
            lists = d.cluster_lists()
            cand[M] = float(sum(sizes[I] * sizes[l].sum() for I, l in enumerate(lists)) / s.n)
            bits = sum(int(sum(bin(int(v)).count("1") for v in m)) for m in d.cluster_masks())
            masked[M] = float(bits / s.n)
        d.build_verlet(0)
        _, nn = d.verlet()
        r = {"system": s.name, "n": s.n, "best_vl": best_vl, "times_ms": times, "kernel_ms": kernel,
             "cluster_candidates_per_particle": cand, "masked_pairs_per_particle": masked,
             "verlet_entries_per_particle": float(nn.mean())}
        out.append(r)
        vcl = {k: v for k, v in kernel.items() if k.startswith("VCL:")}
        bv = min(vcl, key=vcl.get)
        log(f"{s.name}: VL {best_vl} kernel {kernel[best_vl]:.4f} ms; best VCL {bv} {vcl[bv]:.4f} ms; "
            f"candidates/particle {cand}, masked pairs/particle {masked} vs VL entries {nn.mean():.1f}")
    return out


def precision(n=8000, log=print):
    import oracle
    oracle.build()
    systems = [W.fcc(n, 1.2, 71), W.fcc(n, 1.0, 72), W.stratified(n, 0.75, 73), W.stratified(n, 0.1, 74)]
    out = []
    for s in systems:
        F_ref, _, _, np_ref = oracle.forces_bruteforce(s.pos, s.L, s.rc)
        rms = float(np.sqrt((F_ref ** 2).sum(0).mean()))
        d = lj.Domain(s.L, s.rc, s.skin, precision=lj.LJ_PREC_FP32_ACC64)
        d.set_particles(s.pos, s.vel)
        errs = {}
        for cfg in lj.configs():
            d.compute_forces(cfg)
            errs[lj.config_name(cfg)] = float(np.abs(d.forces() - F_ref).max() / rms)
        d.build_verlet(0)
        _, nn = d.verlet()
        d.close()
        rho = s.n / s.L ** 3
        nc = int(s.L // s.rc)
        cand = 27.0 * s.n / nc ** 3
        worst = max(errs, key=errs.get)
        r = {"system": s.name, "n": s.n, "rho": rho, "pairs_in_cutoff_per_particle": 2.0 * np_ref / s.n,
             "verlet_entries_per_particle_mean": float(nn.mean()), "verlet_entries_max": int(nn.max()),
             "lc_candidates_per_particle": cand, "rms_force": rms, "worst_config": worst,
             "worst_err": errs[worst], "errors": errs}
        log(f"{s.name}: worst {worst} {errs[worst]:.3e}; list mean {nn.mean():.1f} max {nn.max()}")
        out.append(r)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["sweep", "train", "droplet", "ensemble", "ensemble-launch", "energy",
                                     "traversal", "clusters", "force-launch", "mlp-launch", "precision",
                                     "c2-sweep", "aux-launch"])
    ap.add_argument("--cfg", default="1,3,4,0", help="force-launch: container,order,param,newton3")
    ap.add_argument("--particles", type=int, default=524288)
    ap.add_argument("--evals", type=int, default=3)
    ap.add_argument("--only", default=None, help="c2-sweep: comma-separated name substrings to run")
    ap.add_argument("--fp64", action="store_true", help="force-launch: FP64 pair arithmetic")
    ap.add_argument("--energy", action="store_true", help="force-launch: also reduce energy and virial")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--data", default="tuner_data.npz")
    ap.add_argument("--model", default=tuner.MODEL_PATH)
    ap.add_argument("--out", default=None)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--phase", type=int, default=500)
    ap.add_argument("--radius", type=float, default=84.19)
    ap.add_argument("--loo", action="store_true")
    ap.add_argument("--samples", type=int, default=3, help="timed evaluations per configuration (sweep)")
    a = ap.parse_args(argv)
    from . import build as B
    B.build()
    if a.what == "sweep":
        density_sweep(scale=a.scale, samples=a.samples, out=a.data)
    elif a.what == "train":
        z = np.load(a.data)
        X, T, names, box = z["X"], z["T"], [str(v) for v in z["names"]], z["box"]
        model = tuner.train(X, T, epochs=a.epochs)
        tuner.save(model, names, a.model, meta={"rows": int(X.shape[0]), "epochs": a.epochs,
                                                "configs_timed": len(names), "outputs": int(model["C"]),
                                                "final_loss": float(model["losses"][-1])})
        print(f"trained: rows={X.shape[0]} loss {model['losses'][0]:.4f} -> {model['losses'][-1]:.4f}")
        if a.loo:
            res = leave_one_out(X, T, box, names, epochs=a.epochs)
            summ = {"mean_learned_regret": float(np.mean([r["learned_regret"] for r in res])),
                    "max_learned_regret": float(np.max([r["learned_regret"] for r in res])),
                    "mean_default_regret": float(np.nanmean([r["default_regret"] for r in res])),
                    "rows": res}
            print(json.dumps({k: v for k, v in summ.items() if k != "rows"}))
            if a.out:
                json.dump(summ, open(a.out, "w"))
    elif a.what == "ensemble":
        res = {"linked_cells": ensemble(steps=a.steps), "verlet_lists": ensemble(steps=a.steps, lists=True)}
        if a.out:
            json.dump(res, open(a.out, "w"))
    elif a.what == "ensemble-launch":
        # the 256-box batch on Verlet lists: an initial-force launch, then one
        # direct (not graph-replayed) launch of a.steps steps, for profilers
        ens = lj.Ensemble(W.config5(256))
        ens.set_lists(0.3, 10)
        ens.run(0.002, 0, use_graph=False)
        t0 = time.perf_counter()
        ens.run(0.002, a.steps, use_graph=False)
        print(json.dumps({"steps": a.steps, "ms_per_step": (time.perf_counter() - t0) / max(1, a.steps) * 1e3}))
        ens.close()
    elif a.what == "precision":
        res = precision()
        print(json.dumps([{k: v for k, v in r.items() if k != "errors"} for r in res]))
        if a.out:
            json.dump(res, open(a.out, "w"))
    elif a.what == "force-launch":
        s = W.homogeneous(a.particles, 0.75, W.BASE_SEED + 1, T=1.0, rc=2.5, skin=0.3)
        cfg = lj.config(*[int(v) for v in a.cfg.split(",")])
        prec = lj.LJ_PREC_FP64 if a.fp64 else lj.LJ_PREC_FP32_ACC64
        d = lj.Domain(s.L, s.rc, s.skin, precision=prec)
        d.set_particles(s.pos, s.vel)
        d.compute_forces(cfg, a.energy)
        d.timing(1)
        for _ in range(a.evals):
            d.compute_forces(cfg, a.energy)
        ms, k, _ = d.timing(0)
        print(json.dumps({"config": lj.config_name(cfg), "n": s.n, "evals": a.evals, "fp64": a.fp64,
                          "energy": a.energy, "force_kernel_ms": ms / max(k, 1)}))
        d.close()
    elif a.what == "aux-launch":
        # the library's auxiliary kernels, each launched at least once on a
        # 60,000-particle fluid (small enough for the 16-bit list copy)
        s = W.stratified(60000, 0.75, W.BASE_SEED + 91)
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos, s.vel)
        d.features()
        d.pairs(lj.LJ_LC)
        cfg = lj.config(lj.LJ_VL, lj.LJ_ORD_JSPLIT, 4, lj.LJ_N3_OFF)
        d.compute_forces(cfg)
        d.verlet()
        d.integrate(0.002, 2, cfg)
        d.state()
        d.kinetic_energy()
        d.forces()
        d.close()
        d = lj.Domain(s.L, s.rc, s.skin)                       # coordinates as doubles: quantised on the GPU
        d.set_particles(np.ascontiguousarray((s.pos.astype(np.float64) + 0.5) * (s.L / 2.0 ** 32)), s.vel)
        d.compute_forces(lj.config(lj.LJ_LC, lj.LJ_ORD_JSPLIT, 2, lj.LJ_N3_OFF))
        d.close()
        import torch                                           # the allocation-free binning entry point
        dev = torch.device("cuda", 0)
        nc = int(np.floor(s.L / s.rc))
        pos_d = torch.from_numpy(s.pos.view(np.int32)).to(dev).contiguous()
        perm_d = torch.zeros(s.n, dtype=torch.int32, device=dev)
        cs_d = torch.zeros(nc ** 3 + 1, dtype=torch.int32, device=dev)
        st = lj.load().lj_bin_cells_static(pos_d.data_ptr(), s.n, nc, perm_d.data_ptr(), cs_d.data_ptr(),
                                           torch.cuda.current_stream(dev).cuda_stream)
        if st != lj.LJ_OK:
            raise lj.LJError(st, "lj_bin_cells_static failed")
        torch.cuda.synchronize(dev)
        rng = np.random.default_rng(6)
        T = np.exp(rng.normal(size=(174, 64)))
        X = rng.normal(size=(174, 16))
        Y, M, Xs, _, _ = lj.tuner_prepare(T, X)
        p0 = rng.normal(0, 0.1, size=lj.mlp_nparams(64))
        lj.mlp_train(p0, 64, Xs, Y, M, 3, 3e-3)
        print(json.dumps({"n": s.n, "rows": 174}))
    elif a.what == "mlp-launch":
        model = tuner.load()
        rng = np.random.default_rng(5)
        X = rng.standard_normal((4096, 16)).astype(np.float32)
        C_out = int(model["C"])
        T = rng.standard_normal((4096, C_out)).astype(np.float32)
        M = np.ones_like(T)
        lj.mlp_forward(model["params"], C_out, X)
        lj.mlp_loss_grad(model["params"], C_out, X, T, M)
        print(json.dumps({"rows": 4096, "outputs": C_out}))
    elif a.what == "c2-sweep":
        res = c2_sweep(only=a.only.split(",") if a.only else None)
        if a.out:
            json.dump(res, open(a.out, "w"))
    elif a.what == "clusters":
        res = clusters()
        if a.out:
            json.dump(res, open(a.out, "w"))
    elif a.what == "traversal":
        res = traversal()
        if a.out:
            json.dump(res, open(a.out, "w"))
    elif a.what == "energy":
        res = energy()
        print(json.dumps({k: v for k, v in res.items() if k != "systems"}))
        if a.out:
            json.dump(res, open(a.out, "w"))
    else:
        res = droplet(a.radius, a.steps, a.phase, model_path=a.model)
        print(json.dumps({k: v for k, v in res.items() if k != "evidence"}))
        if a.out:
            json.dump(res, open(a.out, "w"))


if __name__ == "__main__":
    main()
