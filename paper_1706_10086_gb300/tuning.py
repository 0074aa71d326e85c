"""Autotuning workflow around the C-ABI: timing database, cost-model training
on the GPU, prediction and regret.

* :func:`collect` runs ``alp_tune(EXHAUSTIVE)`` for every (shape, path) not
  yet in the JSONL database (the library appends one record per sweep, so an
  interrupted collection resumes where it stopped).
* :func:`dataset` turns records into targets ``ln(t_config / t_best)`` with a
  mask for configs that could not run.
* :func:`train` fits the MLP with the library's feature, forward, backward and
  Adam kernels (full batch, float32).
* :func:`predict` / :func:`evaluate` choose a config per held-out shape and
  report its regret ``t(chosen) / t(best) - 1`` against the exhaustive sweep,
  next to two choices without the network: one fixed config tuned once (the
  paper's method, Sect. 3: one tile size per architecture, tuned at one matrix
  size) and the winner of the nearest training shape.

Everything numeric runs in the library's kernels; this module moves arrays.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import alp, inputs

PATHS = {"native": alp.ALP_PATH_NATIVE, "emul": alp.ALP_PATH_EMUL}


def config_lists():
    nat = [alp.alp_config_at(alp.ALP_PATH_NATIVE, i).astuple()
           for i in range(alp.alp_config_count(alp.ALP_PATH_NATIVE))]
    emu = [alp.alp_config_at(alp.ALP_PATH_EMUL, i).astuple()
           for i in range(alp.alp_config_count(alp.ALP_PATH_EMUL))]
    return nat, emu


def load_db(path):
    recs = []
    if not os.path.exists(path):
        return recs
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line:
                recs.append(json.loads(line))
    return recs


def collect(shapes, paths, db_path, runs=2, log_every=0):
    """Exhaustive sweeps of every (M, N, K) in ``shapes`` for each path name in
    ``paths``, skipping those already in the database."""
    os.environ["ALP_TUNE_DB"] = db_path
    os.environ["ALP_TUNE_RUNS"] = str(runs)
    have = {(r["M"], r["N"], r["K"], r["path"]) for r in load_db(db_path)}
    done = 0
    for (M, N, K) in shapes:
        for pname in paths:
            if (int(M), int(N), int(K), pname) in have:
                continue
            if pname == "emul" and K > 32768:
                continue
            alp.alp_tune(int(M), int(N), int(K), PATHS[pname], alp.ALP_TUNE_EXHAUSTIVE)
            done += 1
            if log_every and done % log_every == 0:
                print(f"collect: {done} sweeps", flush=True)
    return done


def _record_times(rec, nat, emu):
    """Per-output times (ms) of one record, NaN where not measured."""
    C = len(nat) + len(emu)
    t = np.full(C, np.nan)
    index = {c: i for i, c in enumerate(nat)} if rec["path"] == "native" else \
        {c: len(nat) + i for i, c in enumerate(emu)}
    for row in rec["configs"]:
        key = tuple(int(v) for v in row[:6])
        est = row[6]
        if key in index and est is not None and math.isfinite(est):
            t[index[key]] = est
    return t


def dataset(records):
    nat, emu = config_lists()
    C = len(nat) + len(emu)
    M = np.array([r["M"] for r in records], dtype=np.int64)
    N = np.array([r["N"] for r in records], dtype=np.int64)
    K = np.array([r["K"] for r in records], dtype=np.int64)
    P = np.array([1 if r["path"] == "emul" else 0 for r in records], dtype=np.int32)
    times = np.stack([_record_times(r, nat, emu) for r in records]) if records else \
        np.zeros((0, C))
    best = np.nanmin(times, axis=1)
    T = np.log(times / best[:, None])
    Mask = np.isfinite(T).astype(np.float32)
    T = np.where(Mask > 0, T, 0.0).astype(np.float32)
    return {"M": M, "N": N, "K": K, "path": P, "times": times, "T": T, "Mask": Mask, "C": C}


def init_params(C, seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from the
    seeded generator (passed to the kernels as inputs)."""
    shapes = [(64, 7), (64,), (64, 64), (64,), (C, 64), (C,)]
    out, off = [], 0
    for shp in shapes:
        n = int(np.prod(shp))
        if len(shp) == 2:
            a = inputs.uniform(seed, off, shp) / math.sqrt(shp[1])
        else:
            a = np.zeros(shp)
        out.append(a)
        off += n
    return np.concatenate([a.ravel() for a in out]).astype(np.float32)


class Trainer:
    """Device state of one training run."""

    def __init__(self, ds, seed=1706 + 4):
        import torch
        self.torch = torch
        dev = torch.device("cuda")
        self.C = ds["C"]
        self.B = len(ds["M"])
        t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        self.dM, self.dN, self.dK = (t(ds[k], torch.int64) for k in ("M", "N", "K"))
        self.dpath = t(ds["path"], torch.int32)
        self.Xraw = torch.empty(self.B, 7, dtype=torch.float32, device=dev)
        self.X = torch.empty(self.B, 7, dtype=torch.float32, device=dev)
        self.mean = torch.empty(7, dtype=torch.float32, device=dev)
        self.std = torch.empty(7, dtype=torch.float32, device=dev)
        alp.alp_mlp_features(self.B, self.dM, self.dN, self.dK, self.dpath, None, None, self.Xraw)
        alp.alp_mlp_feature_stats(self.B, self.Xraw, self.mean, self.std)
        alp.alp_mlp_features(self.B, self.dM, self.dN, self.dK, self.dpath, self.mean, self.std,
                             self.X)
        self.T = t(ds["T"], torch.float32)
        self.Mask = t(ds["Mask"], torch.float32)
        self.nparam = alp.alp_mlp_param_count(self.C)
        self.params = t(init_params(self.C, seed), torch.float32)
        self.grads = torch.zeros(self.nparam, dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.grads)
        self.v = torch.zeros_like(self.grads)
        self.Y = torch.empty(self.B, self.C, dtype=torch.float32, device=dev)
        self.cache = torch.empty(self.B, 128, dtype=torch.float32, device=dev)
        self.work = torch.empty(self.B * (self.C + 128), dtype=torch.float32, device=dev)
        self.loss = torch.zeros(2, dtype=torch.float32, device=dev)
        self.step = 0

    def epoch(self, lr):
        alp.alp_mlp_forward(self.params, self.C, self.X, self.B, self.Y, self.cache)
        alp.alp_mlp_backward(self.params, self.C, self.X, self.B, self.cache, self.Y, self.T,
                             self.Mask, self.grads, self.work, self.loss)
        self.step += 1
        alp.alp_mlp_adam(self.params, self.grads, self.m, self.v, self.nparam, self.step, lr)

    def current_loss(self):
        alp.alp_mlp_forward(self.params, self.C, self.X, self.B, self.Y, self.cache)
        alp.alp_mlp_backward(self.params, self.C, self.X, self.B, self.cache, self.Y, self.T,
                             self.Mask, self.grads, self.work, self.loss)
        return float(self.loss[0].item())

    def model(self):
        return (self.params.cpu().numpy().copy(), self.mean.cpu().numpy().copy(),
                self.std.cpu().numpy().copy())


def train(ds, epochs=3000, lr=3e-3, seed=1706 + 4, log_every=0):
    tr = Trainer(ds, seed)
    hist = [tr.current_loss()]
    for e in range(epochs):
        tr.epoch(lr if e < epochs * 0.7 else lr * 0.1)
        if log_every and (e + 1) % log_every == 0:
            hist.append(tr.current_loss())
    hist.append(tr.current_loss())
    return tr.model(), hist


def predict(model, M, N, K, path):
    """Predicted outputs (n x C) for shapes with the library's forward kernel."""
    import torch
    params, mean, std = model
    dev = torch.device("cuda")
    n = len(M)
    C = (len(params) - 4672) // 65
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    X = torch.empty(n, 7, dtype=torch.float32, device=dev)
    alp.alp_mlp_features(n, t(M, torch.int64), t(N, torch.int64), t(K, torch.int64),
                         t(path, torch.int32), t(mean, torch.float32), t(std, torch.float32), X)
    Y = torch.empty(n, C, dtype=torch.float32, device=dev)
    cache = torch.empty(n, 128, dtype=torch.float32, device=dev)
    alp.alp_mlp_forward(t(params, torch.float32), C, X, n, Y, cache)
    return Y.cpu().numpy()


def _valid_range(path, n_nat, C):
    return (0, n_nat) if path == 0 else (n_nat, C)


def choose_by_model(model, ds):
    nat, _ = config_lists()
    Y = predict(model, ds["M"], ds["N"], ds["K"], ds["path"])
    out = np.empty(len(Y), dtype=np.int64)
    for i, y in enumerate(Y):
        lo, hi = _valid_range(ds["path"][i], len(nat), ds["C"])
        out[i] = lo + int(np.argmin(y[lo:hi]))
    return out


def regret(ds, choice):
    t = ds["times"][np.arange(len(choice)), choice]
    best = np.nanmin(ds["times"], axis=1)
    r = t / best - 1.0
    return np.where(np.isfinite(r), r, np.nan)


def fixed_config_choice(train_ds, test_ds, tuning_shape=None, tuning_ds=None):
    """One config per path for every shape.  With tuning_ds (the sweep of the
    tuning shape, e.g. N = 10240 as in the paper's Sect. 3) it is that sweep's
    winner; with only tuning_shape, the winner of the nearest training shape;
    otherwise the config with the lowest mean ln(t / t_best) over training."""
    nat, _ = config_lists()
    out = np.empty(len(test_ds["M"]), dtype=np.int64)
    for p in (0, 1):
        lo, hi = _valid_range(p, len(nat), train_ds["C"])
        sel = train_ds["path"] == p
        if not sel.any():
            continue
        if tuning_ds is not None and (tuning_ds["path"] == p).any():
            row = tuning_ds["times"][np.where(tuning_ds["path"] == p)[0][0]]
            c = lo + int(np.nanargmin(row[lo:hi]))
        elif tuning_shape is not None:
            d = (np.log2(train_ds["M"][sel]) - math.log2(tuning_shape[0])) ** 2 + \
                (np.log2(train_ds["N"][sel]) - math.log2(tuning_shape[1])) ** 2 + \
                (np.log2(train_ds["K"][sel]) - math.log2(tuning_shape[2])) ** 2
            row = train_ds["times"][sel][int(np.argmin(d))]
            c = lo + int(np.nanargmin(row[lo:hi]))
        else:
            T = np.where(train_ds["Mask"][sel] > 0, train_ds["T"][sel], np.inf)[:, lo:hi]
            c = lo + int(np.argmin(np.mean(np.where(np.isfinite(T), T, 10.0), axis=0)))
        out[test_ds["path"] == p] = c
    return out


def nearest_shape_choice(train_ds, test_ds):
    f = lambda d: np.stack([np.log2(d["M"]), np.log2(d["N"]), np.log2(d["K"])], axis=1)
    a, b = f(train_ds), f(test_ds)
    out = np.empty(len(b), dtype=np.int64)
    nat, _ = config_lists()
    for i in range(len(b)):
        same = train_ds["path"] == test_ds["path"][i]
        idx = np.where(same)[0]
        j = idx[int(np.argmin(((a[idx] - b[i]) ** 2).sum(axis=1)))]
        lo, hi = _valid_range(test_ds["path"][i], len(nat), train_ds["C"])
        out[i] = lo + int(np.nanargmin(train_ds["times"][j][lo:hi]))
    return out


def summarize(r):
    r = r[np.isfinite(r)]
    return {"mean": float(np.mean(r)), "median": float(np.median(r)),
            "p90": float(np.percentile(r, 90)), "max": float(np.max(r)), "n": int(len(r))}


def evaluate(model, train_ds, test_ds, tuning_shape=(10240, 10240, 10240), tuning_ds=None):
    res = {"mlp": summarize(regret(test_ds, choose_by_model(model, test_ds))),
           "fixed_tuned_once": summarize(regret(test_ds, fixed_config_choice(
               train_ds, test_ds, tuning_shape, tuning_ds))),
           "fixed_best_mean": summarize(regret(test_ds, fixed_config_choice(train_ds, test_ds))),
           "nearest_shape": summarize(regret(test_ds, nearest_shape_choice(train_ds, test_ds)))}
    return res


def validate_full_runs(model, train_ds, test_ds, tuning_ds=None, count=50, max_flops=4e11,
                       seed=1706 + 7, runs=2):
    """Checks the proxy-based regret on whole problems: for up to `count`
    held-out (shape, path) cases with 2MNK <= max_flops (chosen with a seeded
    generator), times on the full problem the configs chosen by the MLP, by
    the config tuned once, by the nearest training shape and the proxy
    sweep's winner, and returns per choice the mean and p90 of the proxy
    regret and of the full-run regret against the fastest of those four, plus
    how often the proxy winner is the fastest on the full run."""
    nat, emu = config_lists()
    allc = nat + emu
    flops = 2.0 * test_ds["M"] * test_ds["N"] * test_ds["K"]
    idx = np.where(flops <= max_flops)[0]
    pick = idx[np.argsort(inputs.uniform(seed, 0, (len(idx),)))[:count]]
    sub = {k: (v[pick] if isinstance(v, np.ndarray) and len(v) == len(test_ds["M"]) else v)
           for k, v in test_ds.items()}
    choices = {"mlp": choose_by_model(model, sub),
               "fixed_tuned_once": fixed_config_choice(train_ds, sub, tuning_ds=tuning_ds,
                                                       tuning_shape=(10240, 10240, 10240)),
               "nearest_shape": nearest_shape_choice(train_ds, sub),
               "proxy_best": np.array([int(np.nanargmin(r)) for r in sub["times"]])}
    full = {name: np.empty(len(pick)) for name in choices}
    for i in range(len(pick)):
        M, N, K, p = (int(sub["M"][i]), int(sub["N"][i]), int(sub["K"][i]), int(sub["path"][i]))
        cache = {}
        for name, ch in choices.items():
            c = int(ch[i])
            if c not in cache:
                cache[c] = alp.alp_tune_time_config(M, N, K, alp.ALP_PATH_EMUL if p else
                                                    alp.ALP_PATH_NATIVE, allc[c], False, runs)
            full[name][i] = cache[c]
    best_full = np.min(np.stack(list(full.values())), axis=0)
    res = {"cases": int(len(pick)), "max_flops": max_flops,
           "proxy_winner_fastest_on_full_run": float(np.mean(full["proxy_best"] <= best_full))}
    for name, ch in choices.items():
        res[name] = {"proxy": summarize(regret(sub, ch)),
                     "full_run_vs_best_of_four": summarize(full[name] / best_full - 1.0)}
    return res


def tune_batched_classes(M, N, K, pA, pB, pC, alpha=1.5, beta=0.5, runs=3,
                         tiles=(32, 64, 128), bks=(16, 32), log=None):
    """Autotunes the batched GEMM's tile per size class: for every class
    present in the batch, times the class's own problems (alp_gemm_batched_varsize
    on that sub-batch, CUDA events, best of ``runs`` after a warm-up) with each
    candidate (bm, bn, bk) and installs the fastest with
    alp_batched_set_class_config.  M, N, K, pA, pB, pC are host arrays (sizes and
    device addresses of row-major operands with tight leading dimensions).
    Returns {class: ((bm, bn, bk), ms, {candidate: ms})}."""
    import torch
    dev = torch.device("cuda")
    M, N, K = (np.ascontiguousarray(a, dtype=np.int64) for a in (M, N, K))
    cls = np.array([alp.alp_batched_class_of(int(m), int(n)) for m, n in zip(M, N)])
    stream = torch.cuda.current_stream(dev)
    out = {}
    for c in sorted(set(cls.tolist())):
        idx = np.where(cls == c)[0]
        hM, hN, hK = M[idx].copy(), N[idx].copy(), K[idx].copy()
        t = lambda a, dt=torch.int64: torch.tensor(np.asarray(a), dtype=dt, device=dev)
        n = len(idx)
        args = (n, t(hM), t(hN), t(hK), t(np.full(n, alpha), torch.float64),
                t(np.asarray(pA)[idx]), t(hK), t(np.asarray(pB)[idx]), t(hN),
                t(np.full(n, beta), torch.float64), t(np.asarray(pC)[idx]), t(hN), hM, hN, hK)
        ws = alp.alp_gemm_batched_workspace(n, hM, hN, hK)
        work = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)
        old = alp.alp_batched_get_class_config(c)
        times = {}
        for bm in tiles:
            for bn in tiles:
                for bk in bks:
                    alp.alp_batched_set_class_config(c, bm, bn, bk)
                    alp.alp_gemm_batched_varsize(*args, work, ws, stream=stream)
                    best = float("inf")
                    for _ in range(runs):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        alp.alp_gemm_batched_varsize(*args, work, ws, stream=stream)
                        e1.record(stream)
                        e1.synchronize()
                        best = min(best, e0.elapsed_time(e1))
                    times[(bm, bn, bk)] = best
        win = min(times, key=lambda k: (times[k], k))
        alp.alp_batched_set_class_config(c, *win)
        out[c] = (win, times[win], times)
        if log:
            log(f"class {c}: {n} problems, default {old} {times.get(tuple(old), float('nan')):.3f} ms"
                f" -> {win} {times[win]:.3f} ms")
    # Each class was timed alone; in one batch the largest tile of any class
    # decides the persistent kernel's variant (128: one block per SM, 64: two,
    # 32: three).  Time the whole batch with the per-class winners and with the
    # best tiles of at most 64 and of at most 32, and keep the fastest table.
    def capped(cap):
        return {c: min((k for k in v[2] if max(k[0], k[1]) <= cap), key=lambda k: (v[2][k], k))
                for c, v in out.items()}
    tables = [{c: v[0] for c, v in out.items()}]
    for cap in (64, 32):
        if min(tiles) <= cap and capped(cap) not in tables:
            tables.append(capped(cap))
    if len(tables) > 1:
        n = len(M)
        t = lambda a, dt=torch.int64: torch.tensor(np.asarray(a), dtype=dt, device=dev)
        args = (n, t(M), t(N), t(K), t(np.full(n, alpha), torch.float64), t(np.asarray(pA)),
                t(K), t(np.asarray(pB)), t(N), t(np.full(n, beta), torch.float64),
                t(np.asarray(pC)), t(N), M, N, K)
        ws = alp.alp_gemm_batched_workspace(n, M, N, K)
        work = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)

        def whole(table):
            for c, cfg in table.items():
                alp.alp_batched_set_class_config(c, *cfg)
            alp.alp_gemm_batched_varsize(*args, work, ws, stream=stream)
            best = float("inf")
            for _ in range(runs):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                alp.alp_gemm_batched_varsize(*args, work, ws, stream=stream)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            return best
        ts = [whole(tb) for tb in tables]
        if log:
            log("whole batch: " + ", ".join(f"{max(max(k[0], k[1]) for k in tb.values())}-wide "
                                            f"{t:.3f} ms" for tb, t in zip(tables, ts)))
        chosen = tables[int(np.argmin(ts))]
        for c, cfg in chosen.items():
            alp.alp_batched_set_class_config(c, *cfg)
            out[c] = (cfg, out[c][2][cfg], out[c][2])
    return out


def run(db, n_train=2000, n_test=500, lo=64, hi=16384, paths=("native", "emul"), runs=2,
        epochs=3000, lr=3e-3, out=None, log_every=100, validate=0):
    """The whole predictor workload: sweep, train on the GPU, evaluate."""
    import time
    seed = inputs.workload_seed("mlp_predictor")
    train_sh = inputs.shapes(seed, n_train, lo, hi)
    test_sh = inputs.shapes(seed + 1, n_test, lo, hi)
    t0 = time.time()
    collect(train_sh, paths, db, runs=runs, log_every=log_every)
    collect(test_sh, paths, db, runs=runs, log_every=log_every)
    # the paper's tuning sizes (Sect. 3): N = 10240, control N = 7168
    tuning_shapes = [(10240, 10240, 10240), (7168, 7168, 7168)]
    collect(tuning_shapes, paths, db, runs=runs)
    t_collect = time.time() - t0
    recs = load_db(db)
    tuning_ds = dataset([r for r in recs if (r["M"], r["N"], r["K"]) == tuning_shapes[0]])
    key = lambda r: (r["M"], r["N"], r["K"])
    train_keys = {tuple(int(v) for v in s) for s in train_sh}
    test_keys = {tuple(int(v) for v in s) for s in test_sh}
    train_ds = dataset([r for r in recs if key(r) in train_keys])
    test_ds = dataset([r for r in recs if key(r) in test_keys and key(r) not in train_keys])
    t0 = time.time()
    model, hist = train(train_ds, epochs=epochs, lr=lr, log_every=max(1, epochs // 10))
    t_train = time.time() - t0
    res = {"n_train": int(len(train_ds["M"])), "n_test": int(len(test_ds["M"])),
           "collect_s": round(t_collect, 1), "train_s": round(t_train, 2),
           "loss_history": [round(h, 5) for h in hist]}
    for pname, pid in (("all", None), ("native", 0), ("emul", 1)):
        sel = np.ones(len(test_ds["M"]), bool) if pid is None else test_ds["path"] == pid
        if not sel.any():
            continue
        sub = {k: (v[sel] if isinstance(v, np.ndarray) and len(v) == len(sel) else v)
               for k, v in test_ds.items()}
        res[pname] = evaluate(model, train_ds, sub, tuning_ds=tuning_ds)
    if validate:
        t0 = time.time()
        res["full_run_validation"] = validate_full_runs(model, train_ds, test_ds, tuning_ds,
                                                        count=validate)
        res["full_run_validation"]["seconds"] = round(time.time() - t0, 1)
    control = dataset([r for r in recs if (r["M"], r["N"], r["K"]) == tuning_shapes[1]])
    nat, _ = config_lists()
    res["tuning_shape_winners"] = {
        f"{tuning_shapes[i][0]}^3 {'native' if p == 0 else 'emul'}":
            list((nat + config_lists()[1])[int(np.nanargmin(d["times"][j]))])
        for i, d in enumerate((tuning_ds, control)) for j, p in enumerate(d["path"])}
    if out:
        with open(out, "w") as f:
            json.dump(res, f, indent=1)
        np.savez(out + ".model.npz", params=model[0], mean=model[1], std=model[2])
    return res, model


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="tile-config predictor workload")
    ap.add_argument("--db", required=True)
    ap.add_argument("--out", default=None)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=500)
    ap.add_argument("--runs", type=int, default=2)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--paths", default="native,emul")
    ap.add_argument("--validate", type=int, default=0,
                    help="held-out cases also timed on whole problems")
    a = ap.parse_args()
    res, _ = run(a.db, a.train, a.test, paths=tuple(a.paths.split(",")), runs=a.runs,
                 epochs=a.epochs, out=a.out, validate=a.validate)
    print(json.dumps({k: v for k, v in res.items() if k != "loss_history"}))
