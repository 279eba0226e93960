"""Label SpMV configurations by timing them on this GPU, then train the cascade.

Offline stage of Sec. III-B: for every matrix of a training suite, time every
SpMV configuration (mean of ``reps`` back-to-back runs, as the paper averages
200 runs per configuration, Sec. III-B-2), label the fastest one per cascade
stage, and train one classifier per stage on the Table IV features with the
library's own GPU training kernels (cp_model_train).

Labelling rule: the configuration with the smallest mean time; times within 2 %
of the best count as ties, broken toward the cheaper conversion (CSR < COO <
HYB < SELL < ELL < DIA), then the smaller parameter.

Usage: python -m paper_2411_10143_b300.train_cascade [--count N] [--reps R]
writes weights/cascade.json (and weights/dataset.npz with features, times and
labels).
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
    """Mean time (ms) of one SpMV with ``cfg``, CUDA events on the context's stream."""
    import torch
    x = torch.ones(M.ncols, dtype=torch.float64, device="cuda")
    y = torch.empty(M.nrows, dtype=torch.float64, device="cuda")
    M.convert(cfg)
    for _ in range(warm):
        M.spmv(x, y, cfg)
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        M.spmv(x, y, cfg)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def sweep(ctx, A, reps=100):
    """{config name: ms} for one matrix (configurations over the format budget
    are absent)."""
    M = ctx.load(A)
    times = {}
    for name, cfg in config_space():
        try:
            times[name] = time_spmv(M, cfg, reps)
        except C.CascadeError as e:
            if e.status != C.ERR_FOOTPRINT:
                raise
    feats = M.features()
    M.free()
    return feats, times


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
    F, L, T, names = [], [], [], []
    t0 = time.time()
    for i, (name, make) in enumerate(suite):
        A = make()
        f, times = sweep(ctx, A, reps)
        F.append(f)
        L.append(labels_from_times(times))
        T.append(times)
        names.append(name)
        if log and i % 20 == 0:
            log(f"[{i}/{len(suite)}] {name} n={A.nrows} nnz={A.nnz} "
                f"best={min(times, key=times.get)} ({time.time() - t0:.0f}s)")
    return np.array(F), np.array(L, np.int32), T, names


def train_all(ctx, F, L, h=32, epochs=3000, lr=3e-3, seed=7):
    out = {}
    for stage, name in enumerate(models.STAGE_NAMES):
        loss = ctx.model_train(stage, F, L[:, stage], h1=h, h2=h, epochs=epochs, lr=lr,
                               seed=seed + stage)
        m = ctx.model_get(stage)
        out[name] = dict(dims=m["dims"], params=m["params"], mu=m["mu"], sd=m["sd"],
                         loss=loss)
    return out


def predict_classes(ctx, mdl, F):
    """Per-stage arg-max classes of the trained models, batch-evaluated on the GPU
    (cp_mlp_forward) for the training report."""
    import torch
    preds = []
    for name in models.STAGE_NAMES:
        m = mdl[name]
        d, h1, h2, k = m["dims"]
        z = (np.log1p(F) - np.asarray(m["mu"], np.float64)) / np.asarray(m["sd"], np.float64)
        X = torch.as_tensor(z.astype(np.float32), device="cuda")
        P = torch.as_tensor(np.asarray(m["params"], np.float32), device="cuda")
        logits = torch.zeros((len(F), k), device="cuda")
        scratch = torch.zeros(C.Context.mlp_scratch_floats(len(F), d, h1, h2, k), device="cuda")
        ctx.mlp_forward((d, h1, h2, k), P, X, logits, scratch)
        preds.append(logits.argmax(1).cpu().numpy())
    return np.stack(preds, 1)


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=240)
    ap.add_argument("--reps", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--out", default=str(models.WEIGHTS))
    args = ap.parse_args()
    ctx = C.Context(0)
    suite = W.training_suite(seed=77, count=args.count)
    F, L, T, names = build_dataset(ctx, suite, args.reps)
    rng = np.random.default_rng(0)
    test = rng.random(len(F)) < 0.2
    mdl = train_all(ctx, F[~test], L[~test], epochs=args.epochs)
    picks = predict_classes(ctx, mdl, F)
    acc = {n: float((picks[test, i] == L[test, i]).mean()) for i, n in enumerate(models.STAGE_NAMES)}
    ev_test = evaluate([T[i] for i in np.flatnonzero(test)], picks[test])
    ev_train = evaluate([T[i] for i in np.flatnonzero(~test)], picks[~test])
    import torch
    meta = dict(gpu=torch.cuda.get_device_name(0), matrices=len(F), test=int(test.sum()),
                reps=args.reps, epochs=args.epochs, test_accuracy=acc, eval_test=ev_test,
                eval_train=ev_train, losses={k: v["loss"] for k, v in mdl.items()})
    models.save(mdl, Path(args.out), meta)
    np.savez_compressed(Path(args.out).with_name("dataset.npz"), features=F, labels=L,
                        names=np.array(names), test=test,
                        times=np.array([json.dumps(t) for t in T]))
    print(json.dumps(meta, indent=1))


if __name__ == "__main__":
    main()
