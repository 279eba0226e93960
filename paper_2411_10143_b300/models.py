"""Cascade-stage weights: storage format and installation into a context.

Weights trained on this GPU by ``train_cascade.py`` are kept in
``weights/cascade.json``: for every stage its layer sizes, the flat FP32
parameter vector (layout of include/cascade.h) and the feature
standardisation (mu, sd of log(1 + f)).  Without that file every stage is
absent and the cascade keeps the default CSR kernel.
"""
from __future__ import annotations

import json
from pathlib import Path

import numpy as np

WEIGHTS = Path(__file__).resolve().parent / "weights" / "cascade.json"
STAGE_NAMES = ("FORMAT", "CSR_ALGO", "CSR_TPV", "SELL_SIGMA", "BATCH_TPR")
CASCADE_STAGES = STAGE_NAMES[:4]  # the cascade proper; BATCH_TPR serves the batched solve


def save(models: dict, path: Path = WEIGHTS, meta: dict | None = None) -> None:
    path.parent.mkdir(parents=True, exist_ok=True)
    out = {"meta": meta or {}, "stages": {}}
    for name, m in models.items():
        out["stages"][name] = {
            "dims": [int(v) for v in m["dims"]],
            "params": [float(v) for v in np.asarray(m["params"], np.float32)],
            "mu": [float(v) for v in np.asarray(m["mu"], np.float32)],
            "sd": [float(v) for v in np.asarray(m["sd"], np.float32)],
        }
    path.write_text(json.dumps(out))


def merge(path: Path, stages: dict, meta: dict) -> None:
    """Write the given stages and meta entries into the weights file at path,
    keeping every other stage and meta entry it holds."""
    data = json.loads(path.read_text()) if path.exists() else {"meta": {}, "stages": {}}
    for name, m in stages.items():
        data["stages"][name] = {
            "dims": [int(v) for v in m["dims"]],
            "params": [float(v) for v in np.asarray(m["params"], np.float32)],
            "mu": [float(v) for v in np.asarray(m["mu"], np.float32)],
            "sd": [float(v) for v in np.asarray(m["sd"], np.float32)],
        }
    data["meta"].update(meta)
    path.parent.mkdir(parents=True, exist_ok=True)
    path.write_text(json.dumps(data))


def load(path: Path = WEIGHTS) -> dict:
    if not path.exists():
        return {}
    data = json.loads(path.read_text())
    out = dict(data.get("stages", {}))
    gate = data.get("meta", {}).get("gate")
    if gate:
        out["_gate"] = gate
    return out


def install(ctx, models: dict) -> list:
    """Load every stage present in ``models`` into the context; returns their names."""
    import warnings

    from . import cascade as C
    done = []
    for i, name in enumerate(STAGE_NAMES):
        m = models.get(name)
        if not m:
            continue
        d, h1, h2, k = m["dims"]
        if k != C.STAGE_CLASSES[i]:
            warnings.warn(f"stage {name}: stored model has {k} classes, the library expects "
                          f"{C.STAGE_CLASSES[i]}; stage left without a model (retrain)")
            continue
        ctx.model_load(i, h1, h2, k, np.asarray(m["params"], np.float32),
                       np.asarray(m["mu"], np.float32), np.asarray(m["sd"], np.float32))
        done.append(name)
    if models.get("_gate"):  # the cost-aware switch's figures, measured with the labels
        ctx.gate_set(C.Gate.from_dict(models["_gate"]))
        done.append("GATE")
        nb = models["_gate"].get("neighbours")
        if nb:  # per-matrix speedups from the nearest training matrices
            ctx.gate_set_neighbours(nb["z"], nb["speedup"], nb["mu"], nb["sd"], nb["k"])
            done.append("GATE_NEIGHBOURS")
    return done


def load_default(ctx) -> list:
    return install(ctx, load())
