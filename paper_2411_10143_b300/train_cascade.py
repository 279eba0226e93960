"""Label SpMV configurations by timing them on this GPU, then train the cascade.

Offline stage of Sec. III-B: for every matrix of a training suite, time every
SpMV configuration (mean of ``reps`` back-to-back runs, as the paper averages
200 runs per configuration, Sec. III-B-2), label the fastest one per cascade
stage, and train one classifier per stage on the Table IV features with the
library's own GPU training kernels (cp_model_train).

Labelling rule: the configuration with the smallest mean time; times within 2 %
of the best count as ties, broken toward the cheaper conversion (CSR < COO <
HYB < SELL < ELL < DIA), then the smaller parameter.  By default the classifiers
train on soft targets instead, a distribution over each stage's classes with
weight exp(-(t / t_best - 1) / tau), tau = 0.02 (cp_model_train_soft): near-ties
are learned as near-ties, and a choice that costs 40 % weighs more than one that
costs 3 %.  The labels remain for the accuracy report.

Usage: python -m paper_2411_10143_b300.train_cascade [--count N] [--reps R]
writes weights/cascade.json (and weights/dataset.npz with features, times and
labels).

With --batch it trains, instead, the classifier that picks the batched solve's
threads per row (the BATCH_TPR stage), on labels from the batching autotuner:
cp_batch_tune times batches of small SPD systems (workloads.batch_suite) at
every launch shape, and those times become the soft targets.  It writes that
stage into the same weights file and weights/batch_dataset.npz.
"""
from __future__ import annotations

import argparse
import json
import time
from pathlib import Path

import numpy as np

from . import cascade as C
from . import models, workloads as W

CONV_COST_ORDER = {C.FMT_CSR: 0, C.FMT_COO: 1, C.FMT_HYB: 2, C.FMT_SELL: 3, C.FMT_ELL: 4,
                   C.FMT_DIA: 5}
TIE = 1.02


def config_space():
    """(name, Config) for every configuration the cascade can pick."""
    out = [("CSR-scalar", C.config("CSR", C.ALGO_SCALAR)),
           ("CSR-merge", C.config("CSR", C.ALGO_MERGE))]
    out += [(f"CSR-vector{t}", C.config("CSR", C.ALGO_VECTOR, tpv=t)) for t in C.TPV_CLASSES]
    out += [("COO", C.config("COO")), ("ELL", C.config("ELL"))]
    out += [(f"SELL-{s}", C.config("SELL", sigma=s)) for s in C.SIGMA_CLASSES]
    out += [("HYB", C.config("HYB")), ("DIA", C.config("DIA"))]
    return out


def time_spmv(M, cfg, reps=100, warm=5):
    """Device time (ms) of one SpMV with ``cfg``: `reps` calls captured in one
    CUDA graph on the library's stream and replayed between two events, so the
    host's launch latency (larger than a small matrix's kernel) is not timed; a
    configuration of several kernels still pays its own launches."""
    import torch
    x = torch.ones(M.ncols, dtype=torch.float64, device="cuda")
    y = torch.empty(M.nrows, dtype=torch.float64, device="cuda")
    M.convert(cfg)
    for _ in range(warm):
        M.spmv(x, y, cfg)
    torch.cuda.synchronize()
    s = M.ctx.stream
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        for _ in range(reps):
            M.spmv(x, y, cfg)
    g.replay()  # warm
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record()
        g.replay()
        e1.record()
    e1.synchronize()
    del g
    return e0.elapsed_time(e1) / reps


# one configuration per format whose conversion the cost-aware switch weighs
CONVERSIONS = [(C.FMT_COO, C.config("COO")), (C.FMT_ELL, C.config("ELL")),
               (C.FMT_SELL, C.config("SELL", sigma=32)), (C.FMT_HYB, C.config("HYB")),
               (C.FMT_DIA, C.config("DIA"))]


def conversion_times(M):
    """{format index: ms} of converting the CSR matrix to each format from
    scratch (cached formats dropped first), host clock around the call; the
    sweep adds "features": ms of the feature pass."""
    import torch
    out = {}
    for f, cfg in CONVERSIONS:
        M.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            M.convert(cfg)
        except C.CascadeError as e:
            if e.status not in (C.ERR_FOOTPRINT, C.ERR_UNSUPPORTED):
                raise
            continue
        torch.cuda.synchronize()
        out[f] = (time.perf_counter() - t0) * 1e3
    M.reset()
    return out


def sweep(ctx, A, reps=100):
    """Features, {config name: SpMV ms} (configurations over the format budget
    are absent) and {format: conversion ms} for one matrix."""
    M = ctx.load(A)
    times = {}
    for name, cfg in config_space():
        try:
            times[name] = time_spmv(M, cfg, reps)
        except C.CascadeError as e:
            if e.status != C.ERR_FOOTPRINT:
                raise
    conv = conversion_times(M)
    import torch
    M.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    feats = M.features()  # the O(nnz) Table IV pass, timed for the two-tier rule
    conv["features"] = (time.perf_counter() - t0) * 1e3
    M.free()
    return feats, times, conv


def format_best(times):
    """Fastest SpMV time of each format (CP_FMT_* index -> ms; inf if absent)."""
    inf = float("inf")
    return {
        C.FMT_CSR: min([times.get("CSR-scalar", inf), times.get("CSR-merge", inf)]
                       + [times.get(f"CSR-vector{t}", inf) for t in C.TPV_CLASSES]),
        C.FMT_COO: times.get("COO", inf),
        C.FMT_ELL: times.get("ELL", inf),
        C.FMT_SELL: min(times.get(f"SELL-{s}", inf) for s in C.SIGMA_CLASSES),
        C.FMT_HYB: times.get("HYB", inf),
        C.FMT_DIA: times.get("DIA", inf),
    }


def fit_line(x, y):
    """y = a + b x with a, b >= 0, least squares in relative error (weights
    1/y), so the small matrices' launch-bound times and the large ones'
    per-non-zero cost both fit."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if len(x) < 2:
        return (float(y.mean()) if len(y) else 0.0), 0.0
    w = 1.0 / np.maximum(y, 1e-9)
    b, a = np.polyfit(x, y, 1, w=w)
    if a < 0:
        a, b = 0.0, float(np.sum(w * w * x * y) / max(np.sum(w * w * x * x), 1e-300))
    if b < 0:
        a, b = float(np.average(y, weights=w * w)), 0.0
    return float(a), float(b)


def gate_figures(T, CV, NNZ, L):
    """The cost-aware switch's figures (cp_gate): per format the median SpMV
    speedup over CSR-scalar where the FORMAT label is that format, and linear
    fits (in millions of non-zeros) of the conversion times and of the
    CSR-scalar SpMV time."""
    mnnz = np.asarray(NNZ, np.float64) * 1e-6
    spmv_a, spmv_b = fit_line(mnnz, [t["CSR-scalar"] for t in T])
    speedup, conv_a, conv_b = [1.0] * 6, [0.0] * 6, [0.0] * 6
    for f in range(1, 6):
        ratio = [t["CSR-scalar"] / format_best(t)[f] for t, lab in zip(T, L)
                 if lab[0] == f and np.isfinite(format_best(t)[f])]
        if not ratio:  # never the label: its typical ratio where it runs
            ratio = [t["CSR-scalar"] / format_best(t)[f] for t in T
                     if np.isfinite(format_best(t)[f])]
        speedup[f] = float(np.median(ratio)) if ratio else 1.0
        xs = [x for x, c in zip(mnnz, CV) if f in c]
        ys = [c[f] for c in CV if f in c]
        conv_a[f], conv_b[f] = fit_line(xs, ys)
    feat_a, feat_b = fit_line(mnnz, [c["features"] for c in CV])
    return dict(speedup=speedup, conv_a_ms=conv_a, conv_b_ms=conv_b, spmv_a_ms=spmv_a,
                spmv_b_ms=spmv_b, feat_a_ms=feat_a, feat_b_ms=feat_b, small_rows=100_000)


GATE_K = 7  # training matrices whose speedups the gate's per-matrix estimate takes


def neighbour_figures(F, T, mu, sd, k=GATE_K):
    """The gate's per-matrix speedups (cp_gate_set_neighbours): the training
    matrices' features standardised as the cascade's inputs (log1p, then the
    FORMAT model's mu and sd) and each format's best SpMV speedup over
    CSR-scalar (0 where the format could not be built)."""
    mu = np.asarray(mu, np.float64)
    sd = np.asarray(sd, np.float64)
    z = (np.log1p(np.maximum(np.asarray(F, np.float64), 0.0)) - mu) / sd
    sp = []
    for t in T:
        fb = format_best(t)
        sp.append([t["CSR-scalar"] / fb[f] if np.isfinite(fb[f]) else 0.0 for f in range(6)])
    return dict(k=int(k), mu=mu.tolist(), sd=sd.tolist(),
                z=np.round(z.astype(np.float32), 5).tolist(),
                speedup=np.round(np.asarray(sp, np.float32), 5).tolist())


def add_neighbours(weights: Path, dataset: Path, k=GATE_K):
    """Adds the gate's neighbour figures to a trained weights file from its
    stored dataset (the training split only); needs no GPU."""
    data = json.loads(weights.read_text())
    F, _, T, _, _, _, test = load_dataset(dataset)
    fm = data["stages"]["FORMAT"]
    idx = np.flatnonzero(~np.asarray(test, bool))
    data["meta"]["gate"]["neighbours"] = neighbour_figures(
        np.asarray(F)[idx], [T[i] for i in idx], fm["mu"], fm["sd"], k)
    weights.write_text(json.dumps(data))


def _argmin_tie(cands):
    """cands: list of (time, tiebreak key, label); ties within 2 % go to the smaller key."""
    best = min(t for t, _, _ in cands)
    ok = [c for c in cands if c[0] <= best * TIE]
    return min(ok, key=lambda c: c[1])[2]


def labels_from_times(times):
    """Per-stage labels (FORMAT, CSR_ALGO, CSR_TPV, SELL_SIGMA) from one sweep."""
    inf = float("inf")
    csr_vec = {t: times.get(f"CSR-vector{t}", inf) for t in C.TPV_CLASSES}
    sell = {s: times.get(f"SELL-{s}", inf) for s in C.SIGMA_CLASSES}
    fmt_best = {
        C.FMT_CSR: min(times.get("CSR-scalar", inf), times.get("CSR-merge", inf),
                       min(csr_vec.values())),
        C.FMT_COO: times.get("COO", inf),
        C.FMT_ELL: times.get("ELL", inf),
        C.FMT_SELL: min(sell.values()),
        C.FMT_HYB: times.get("HYB", inf),
        C.FMT_DIA: times.get("DIA", inf),
    }
    fmt = _argmin_tie([(t, CONV_COST_ORDER[f], f) for f, t in fmt_best.items()])
    algo = _argmin_tie([(times.get("CSR-scalar", inf), 0, C.ALGO_SCALAR),
                        (min(csr_vec.values()), 1, C.ALGO_VECTOR),
                        (times.get("CSR-merge", inf), 2, C.ALGO_MERGE)])
    tpv = _argmin_tie([(t, i, i) for i, t in enumerate(csr_vec.values())])
    sig = _argmin_tie([(t, i, i) for i, t in enumerate(sell.values())])
    return [fmt, algo, tpv, sig]


def stage_times(times):
    """Per-stage candidate times (FORMAT, CSR_ALGO, CSR_TPV, SELL_SIGMA), in the
    class order of each stage; inf where a configuration was not timed."""
    inf = float("inf")
    csr_vec = [times.get(f"CSR-vector{t}", inf) for t in C.TPV_CLASSES]
    sell = [times.get(f"SELL-{s}", inf) for s in C.SIGMA_CLASSES]
    fb = format_best(times)
    return ([fb[f] for f in range(6)],
            [times.get("CSR-scalar", inf), min(csr_vec), times.get("CSR-merge", inf)],
            csr_vec, sell)


def soft_targets(times, tau):
    """Target distributions of the four stages from one sweep: class c gets
    weight exp(-(t_c / t_best - 1) / tau), normalised; untimed classes get 0.
    With tau = 0.02, configurations within a few percent of the fastest share
    the weight and one 10 % slower keeps under 1 % of it."""
    out = []
    for ts in stage_times(times):
        t = np.asarray(ts, np.float64)
        ok = np.isfinite(t)
        w = np.zeros(len(t))
        if ok.any():
            best = t[ok].min()
            w[ok] = np.exp(-(t[ok] / best - 1.0) / tau)
        else:
            w[:] = 1.0
        out.append(w / w.sum())
    return out


def cascade_pick_time(times, pred):
    """SpMV time of the configuration the cascade picks from per-stage classes."""
    fmt, algo, tpv, sig = pred
    if fmt == C.FMT_CSR:
        if algo == C.ALGO_VECTOR:
            return times[f"CSR-vector{C.TPV_CLASSES[tpv]}"]
        return times["CSR-merge" if algo == C.ALGO_MERGE else "CSR-scalar"]
    if fmt == C.FMT_SELL:
        return times.get(f"SELL-{C.SIGMA_CLASSES[sig]}", times["CSR-scalar"])
    return times.get(C.FORMATS[fmt], times["CSR-scalar"])


def build_dataset(ctx, suite, reps=100, log=print):
    F, L, T, CV, NNZ, names = [], [], [], [], [], []
    t0 = time.time()
    for i, (name, make) in enumerate(suite):
        A = make()
        f, times, conv = sweep(ctx, A, reps)
        F.append(f)
        L.append(labels_from_times(times))
        T.append(times)
        CV.append(conv)
        NNZ.append(A.nnz)
        names.append(name)
        if log and i % 20 == 0:
            log(f"[{i}/{len(suite)}] {name} n={A.nrows} nnz={A.nnz} "
                f"best={min(times, key=times.get)} ({time.time() - t0:.0f}s)")
    return np.array(F), np.array(L, np.int32), T, CV, NNZ, names


def train_all(ctx, F, L, h=32, epochs=3000, lr=3e-3, seed=7, targets=None):
    """One classifier per stage, on the labels L, or on soft targets (a list of
    four [N][k] arrays) when given."""
    out = {}
    for stage, name in enumerate(models.CASCADE_STAGES):
        if targets is not None:
            loss = ctx.model_train_soft(stage, F, targets[stage], h1=h, h2=h, epochs=epochs,
                                        lr=lr, seed=seed + stage)
        else:
            loss = ctx.model_train(stage, F, L[:, stage], h1=h, h2=h, epochs=epochs, lr=lr,
                                   seed=seed + stage)
        m = ctx.model_get(stage)
        out[name] = dict(dims=m["dims"], params=m["params"], mu=m["mu"], sd=m["sd"],
                         loss=loss)
    return out


def predict_classes(ctx, mdl, F):
    """Per-stage arg-max classes of the trained models, batch-evaluated on the GPU
    (cp_mlp_forward) for the training report."""
    return np.stack([stage_picks(ctx, mdl[name], F) for name in models.CASCADE_STAGES], 1)


def stage_picks(ctx, m, F):
    """Arg-max classes of one stage's model on the feature rows F (cp_mlp_forward)."""
    import torch
    d, h1, h2, k = m["dims"]
    z = (np.log1p(F) - np.asarray(m["mu"], np.float64)) / np.asarray(m["sd"], np.float64)
    X = torch.as_tensor(z.astype(np.float32), device="cuda")
    P = torch.as_tensor(np.asarray(m["params"], np.float32), device="cuda")
    logits = torch.zeros((len(F), k), device="cuda")
    scratch = torch.zeros(C.Context.mlp_scratch_floats(len(F), d, h1, h2, k), device="cuda")
    ctx.mlp_forward((d, h1, h2, k), P, X, logits, scratch)
    return logits.argmax(1).cpu().numpy()


# ------------------------------------------------------------------ batched solve
BATCH_SYSTEMS = 16  # systems in one labelling batch (one matrix, seeded right-hand sides)


def batch_labels(ctx, suite, nsys=BATCH_SYSTEMS, log=print):
    """Labels of the BATCH_TPR stage from the batching autotuner: for every
    matrix of the suite, a batch of nsys CG systems on it (b = A x*, x* seeded;
    FP32 inner solves in FP64 refinement to 1e-10, as the server batches them)
    goes through cp_batch_tune, which times every launch shape.  A class's time
    is its best over the four block sizes.  Returns the Table IV features
    [N][15], the times [N][3] (ms; threads per row 1, 4, 16) and the names."""
    import torch
    F, T, names = [], [], []
    opts = C.default_opts(tol=1e-10, inner_tol=1e-5, precision=C.PREC_FP32_IR)
    t0 = time.time()
    for i, (name, make) in enumerate(suite):
        A = make()
        M = ctx.load(A)
        f = M.features()
        bs = []
        for k in range(nsys):
            xs = torch.as_tensor(W.vector(A.nrows, 5000 + k), device="cuda")
            b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
            M.spmv(xs, b)
            bs.append(b)
        _, ms = ctx.batch_tune([M] * nsys, [0] * nsys, bs, opts)
        T.append([min(ms[(t, r)] for t in C.Context.BATCH_THREADS) for r in C.BATCH_TPR_CLASSES])
        F.append(f)
        names.append(name)
        M.free()
        if log and i % 20 == 0:
            log(f"[{i}/{len(suite)}] {name} n={A.nrows} nnz={A.nnz} ms={np.round(T[-1], 3)} "
                f"({time.time() - t0:.0f}s)")
    return np.array(F), np.array(T, np.float64), names


def batch_soft_targets(T, tau):
    """Target distributions over threads per row (1, 4, 16) from measured batch
    times: exp(-(t / t_best - 1) / tau), normalised per matrix."""
    T = np.asarray(T, np.float64)
    w = np.exp(-(T / T.min(1, keepdims=True) - 1.0) / tau)
    return w / w.sum(1, keepdims=True)


def batch_evaluate(T, picks):
    """Regret of the picks against the measured best, and their speedup over a
    thread per row everywhere (the untuned rule), geometric means."""
    T = np.asarray(T, np.float64)
    t_pick = T[np.arange(len(T)), picks]
    g = lambda v: float(np.exp(np.mean(np.log(v))))
    return dict(mean_regret=g(t_pick / T.min(1)), speedup_vs_one_thread_per_row=g(T[:, 0] / t_pick),
                picks_within_2pct=int((t_pick <= T.min(1) * TIE).sum()), n=len(T))


def train_batch_stage(ctx, F, T, test, tau=0.02, h=32, epochs=3000, seed=11):
    """The BATCH_TPR classifier on soft targets from the autotuner's times;
    returns the model and its evaluation on the held-out and training rows."""
    loss = ctx.model_train_soft(C.STAGE_BATCH_TPR, F[~test], batch_soft_targets(T[~test], tau),
                                h1=h, h2=h, epochs=epochs, lr=3e-3, seed=seed)
    m = ctx.model_get(C.STAGE_BATCH_TPR)
    mdl = dict(dims=m["dims"], params=m["params"], mu=m["mu"], sd=m["sd"], loss=loss)
    picks = stage_picks(ctx, mdl, F)
    ev = dict(test=batch_evaluate(T[test], picks[test]), train=batch_evaluate(T[~test], picks[~test]),
              test_accuracy=float((picks[test] == T[test].argmin(1)).mean()),
              label_counts=np.bincount(T.argmin(1), minlength=3).tolist(), loss=loss,
              matrices=len(F), held_out=int(test.sum()), systems_per_batch=BATCH_SYSTEMS,
              tau=tau, seed=seed)
    return mdl, ev


def evaluate(times_list, picks):
    """Geometric-mean speedups of the cascade's picks over CSR-scalar and over the
    format-only prediction, plus regret against the measured best."""
    sp_default, sp_fmt_only, regret, exact = [], [], [], 0
    for times, pred in zip(times_list, picks):
        t_pick = cascade_pick_time(times, pred)
        best = min(times.values())
        sp_default.append(times["CSR-scalar"] / t_pick)
        # format-only: the predicted format with its default algorithm / parameter
        fmt = int(pred[0])
        t_fmt = (times["CSR-scalar"] if fmt == C.FMT_CSR
                 else times.get("SELL-1" if fmt == C.FMT_SELL else C.FORMATS[fmt],
                                times["CSR-scalar"]))
        sp_fmt_only.append(t_fmt / t_pick)
        regret.append(t_pick / best)
        exact += t_pick <= best * TIE
    g = lambda v: float(np.exp(np.mean(np.log(v))))
    return dict(speedup_vs_csr_scalar=g(sp_default), speedup_vs_format_only=g(sp_fmt_only),
                mean_regret=g(regret), picks_within_2pct=exact, n=len(picks))


def load_dataset(path):
    """A dataset written by an earlier run (features, labels, timings,
    conversion times, sizes, names and its held-out split)."""
    d = np.load(path)
    T = [json.loads(t) for t in d["times"]]
    CV = [{(int(k) if k.isdigit() else k): v for k, v in json.loads(c).items()}
          for c in d["conversions"]]
    return (d["features"], d["labels"], T, CV, d["nnz"].tolist(), d["names"].tolist(),
            d["test"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=240)
    ap.add_argument("--reps", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--hidden", type=int, default=32)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--tau", type=float, default=0.02,
                    help="> 0: train on soft targets exp(-(t / t_best - 1) / tau) from the "
                         "measured times; 0: on the arg-min labels")
    ap.add_argument("--dataset", default=None,
                    help="train on a stored dataset.npz instead of timing the suite again")
    ap.add_argument("--out", default=str(models.WEIGHTS))
    ap.add_argument("--neighbours-only", action="store_true",
                    help="add the gate's neighbour figures to --out from --dataset (no GPU)")
    ap.add_argument("--batch", action="store_true",
                    help="label the batched solve's threads per row with the batching "
                         "autotuner and train the BATCH_TPR stage into --out (the cascade's "
                         "stages are kept)")
    ap.add_argument("--batch-count", type=int, default=240)
    args = ap.parse_args()
    if args.batch:
        ctx = C.Context(0)
        out = Path(args.out)
        ds = out.with_name("batch_dataset.npz")
        if args.dataset:
            d = np.load(args.dataset)
            F, T, names, test = d["features"], d["times"], d["names"].tolist(), d["test"]
        else:
            F, T, names = batch_labels(ctx, W.batch_suite(count=args.batch_count))
            test = np.random.default_rng(1).random(len(F)) < 0.2
            np.savez_compressed(ds, features=F, times=T, names=np.array(names), test=test)
        mdl, ev = train_batch_stage(ctx, F, T, test, tau=args.tau if args.tau > 0 else 0.02,
                                    h=args.hidden, epochs=args.epochs)
        models.merge(out, {"BATCH_TPR": mdl}, {"batch_tpr": ev})
        print(json.dumps(ev, indent=1))
        return
    if args.neighbours_only:
        add_neighbours(Path(args.out), Path(args.dataset or Path(args.out).with_name("dataset.npz")))
        return
    ctx = C.Context(0)
    if args.dataset:
        F, L, T, CV, NNZ, names, test = load_dataset(args.dataset)
    else:
        suite = W.training_suite(seed=77, count=args.count)
        F, L, T, CV, NNZ, names = build_dataset(ctx, suite, args.reps)
        rng = np.random.default_rng(0)
        test = rng.random(len(F)) < 0.2
    targets = None
    if args.tau > 0:
        idx = np.flatnonzero(~test)
        per = [soft_targets(T[i], args.tau) for i in idx]
        targets = [np.stack([q[st] for q in per]) for st in range(4)]
    mdl = train_all(ctx, F[~test], L[~test], h=args.hidden, epochs=args.epochs, seed=args.seed,
                    targets=targets)
    picks = predict_classes(ctx, mdl, F)
    acc = {n: float((picks[test, i] == L[test, i]).mean())
           for i, n in enumerate(models.CASCADE_STAGES)}
    ev_test = evaluate([T[i] for i in np.flatnonzero(test)], picks[test])
    ev_train = evaluate([T[i] for i in np.flatnonzero(~test)], picks[~test])
    import torch
    meta = dict(gpu=torch.cuda.get_device_name(0), matrices=len(F), test=int(test.sum()),
                reps=args.reps, epochs=args.epochs, hidden=args.hidden, seed=args.seed,
                soft_tau=args.tau,
                test_accuracy=acc, eval_test=ev_test,
                eval_train=ev_train, losses={k: v["loss"] for k, v in mdl.items()},
                gate=gate_figures([T[i] for i in np.flatnonzero(~test)],
                                  [CV[i] for i in np.flatnonzero(~test)],
                                  [NNZ[i] for i in np.flatnonzero(~test)], L[~test]))
    meta["gate"]["neighbours"] = neighbour_figures(
        F[~test], [T[i] for i in np.flatnonzero(~test)], mdl["FORMAT"]["mu"], mdl["FORMAT"]["sd"])
    # the batched solve's stage is trained separately (--batch): keep it
    prev = json.loads(Path(args.out).read_text()) if Path(args.out).exists() else {}
    if "BATCH_TPR" in prev.get("stages", {}):
        mdl["BATCH_TPR"] = prev["stages"]["BATCH_TPR"]
        meta["batch_tpr"] = prev.get("meta", {}).get("batch_tpr", {})
    models.save(mdl, Path(args.out), meta)
    np.savez_compressed(Path(args.out).with_name("dataset.npz"), features=F, labels=L,
                        names=np.array(names), test=test, nnz=np.array(NNZ),
                        times=np.array([json.dumps(t) for t in T]),
                        conversions=np.array([json.dumps({str(k): v for k, v in c.items()})
                                              for c in CV]))
    print(json.dumps(meta, indent=1))


if __name__ == "__main__":
    main()
