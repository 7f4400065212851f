"""Learned dispatch for perm_auto: timings measured by this library, a cost model
trained on the GPU by the library's own MLP kernels, and its evaluation.

The paper tunes two linear hyperplanes in (m/n, n) at build time (Algorithm
"Optimized Algorithm Selection", p1..p8).  Here a small perceptron predicts
log2(seconds) of every candidate from features of the matrix (order, shape,
density, dtype, log work counts; ``capi.perm_auto_features``) and perm_auto runs
the argmin.  This module:

* times candidates on a seeded grid of (m, n, density, dtype) cells
  (``measure_grid``), extrapolating sweeps too long to run from a timed term range;
* trains the model with ``capi.perm_mlp_train`` and installs it with
  ``capi.perm_set_cost_model``;
* refits the paper's rule (``PaperRule``) on the same timings as a baseline;
* scores policies on a held-out batch against exhaustive timing (``evaluate``).

Usage (on a GPU):  python -m paper_2510_03421_gb300.costmodel --cells 600 --eval 10000
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import capi, inputs

CANDS = ("combinatoric", "ryser", "glynn", "glynn_fixed")
DTYPES = {"f64": capi.PERM_F64, "c128": capi.PERM_C128, "u8": capi.PERM_U8}
DIMS = (capi.PERM_NFEATURES, 64, capi.PERM_NCAND)
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "costmodel_gb300.npz")

# candidates that exist per dtype
AVAILABLE = {
    capi.PERM_F64: (True, True, True, True),
    capi.PERM_C128: (True, False, True, False),
    capi.PERM_U8: (True, False, True, False),
}

BUDGET_S = 0.02        # longest run timed in full; longer ones are extrapolated
TERM_SAMPLE = 1 << 22  # terms timed for an extrapolated sweep


def make_matrix(m, n, density, dtype, seed):
    if dtype == "f64":
        return inputs.sparse_real(m, n, density, seed)
    if dtype == "c128":
        return inputs.sparse_complex(m, n, density, seed)
    return inputs.sparse01(m, n, density, seed)


def _log2_nodes(m, n, d):
    total, term = 0.0, 1.0
    for k in range(1, m + 1):
        term *= (n - k + 1) * d
        total += term
    return math.log2(total) if total > 1 else 0.0


def work_log2(m, n, density, cand):
    """log2 of the work count of a candidate (terms x width)."""
    if cand == 0:
        return _log2_nodes(m, n, max(density, 1e-3))
    if cand == 1:
        return n + math.log2(max(m, 1))
    if cand == 3 and m < n:
        return (m - 1) + math.log2(n - m + 1) + math.log2(n)
    return (n - 1) + math.log2(max(n, 1))


class Timer:
    def __init__(self, dev):
        import torch
        self.torch = torch
        self.dev = dev
        self.stream = torch.cuda.Stream(dev)
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def run(self, fn, reps=2):
        best = float("inf")
        with self.torch.cuda.stream(self.stream):
            fn()  # warm-up (and first-use setup)
            for _ in range(reps):
                self.e0.record(self.stream)
                fn()
                self.e1.record(self.stream)
                self.e1.synchronize()
                best = min(best, self.e0.elapsed_time(self.e1) * 1e-3)
        return best


def time_candidate(timer, dA, m, n, density, code, cand):
    """Seconds for candidate `cand` on the device matrix dA (m <= n), or None if the
    candidate does not exist for the dtype.  Long sweeps are timed on a term range
    and scaled; long combinatoric searches are scaled from the node count."""
    if not AVAILABLE[code][cand]:
        return None
    s = timer.stream
    big = dict(max_terms=1 << 62)
    if cand == 0:
        lw = work_log2(m, n, density, 0)
        if lw > 30:  # about a second or more: scale from a smaller search of the same density
            return None
        return timer.run(lambda: capi.perm_combinatoric(dA, stream=s, opts=big))
    if cand == 1:
        total = 1 << n
        if total <= TERM_SAMPLE * 4:
            return timer.run(lambda: capi.perm_ryser(dA, stream=s, opts=big))
        if m > n:
            return None
        part = timer.run(lambda: capi.perm_ryser_partial(dA, 0, TERM_SAMPLE, stream=s, opts=big))
        return part * total / TERM_SAMPLE
    if cand == 3 and m < n:
        # the integer-pipe candidate walks a rectangle grouped: 2^(m-1) (n-m+1) terms of
        # n columns; a long walk is timed on its first mm rows and scaled by the terms
        opts = dict(big, arith=capi.PERM_ARITH_MIXED)
        steps = (1 << (m - 1)) * (n - m + 1)
        if steps <= TERM_SAMPLE * 4:
            return timer.run(lambda: capi.perm_glynn(dA, stream=s, opts=opts))
        mm = m
        while mm > 1 and (1 << (mm - 1)) * (n - mm + 1) > TERM_SAMPLE:
            mm -= 1
        sub = dA[:mm]
        part = timer.run(lambda: capi.perm_glynn(sub, stream=s, opts=opts))
        return part * steps / ((1 << (mm - 1)) * (n - mm + 1))
    opts = dict(big, arith=capi.PERM_ARITH_MIXED if cand == 3 else capi.PERM_ARITH_FP64)
    total = 1 << (n - 1)
    if total <= TERM_SAMPLE * 4:
        return timer.run(lambda: capi.perm_glynn(dA, stream=s, opts=opts))
    part = timer.run(lambda: capi.perm_glynn_partial(dA, 0, TERM_SAMPLE, stream=s, opts=opts))
    return part * total / TERM_SAMPLE


def grid_cells(count, seed):
    """A seeded sample of the (m, n, density, dtype) grid: m in 2..40, n in m..60."""
    g = inputs.rng(seed)
    cells = []
    pairs = [(m, n) for m in range(2, 41) for n in range(m, 61)]
    for _ in range(count):
        m, n = pairs[int(g.integers(len(pairs)))]
        d = float(g.choice([0.1, 0.5, 1.0]))
        dt = str(g.choice(list(DTYPES)))
        cells.append((m, n, d, dt))
    return cells


def measure_grid(dev, cells, seed0=0, log=None):
    """Features, log2-seconds targets and masks for the cells."""
    import torch
    timer = Timer(dev)
    X, T, Mk, rows = [], [], [], []
    for k, (m, n, d, dt) in enumerate(cells):
        A = make_matrix(m, n, d, dt, seed0 + k)
        dA = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
        code = DTYPES[dt]
        nnz = float(np.count_nonzero(A)) / A.size
        t = np.zeros(capi.PERM_NCAND, dtype=np.float32)
        mk = np.zeros(capi.PERM_NCAND, dtype=np.float32)
        for c in range(capi.PERM_NCAND):
            try:
                sec = time_candidate(timer, dA, m, n, nnz, code, c)
            except capi.PermError:
                sec = None
            if sec is not None and sec > 0:
                t[c] = math.log2(sec)
                mk[c] = 1.0
        X.append(capi.perm_auto_features(m, n, nnz, code))
        T.append(t)
        Mk.append(mk)
        rows.append((m, n, nnz, dt))
        if log and k % 100 == 0:
            log("measured %d/%d cells" % (k, len(cells)))
    return np.array(X, np.float32), np.array(T, np.float32), np.array(Mk, np.float32), rows


def fill_combinatoric(X, T, Mk, rows):
    """Label the combinatoric searches too long to time: log2 seconds = log2 nodes +
    the per-dtype offset fitted on the timed searches of at least 2^16 nodes."""
    offs = {}
    for (m, n, d, dt), t, mk in zip(rows, T, Mk):
        lw = work_log2(m, n, d, 0)
        if mk[0] and lw >= 16:
            offs.setdefault(dt, []).append(t[0] - lw)
    for i, ((m, n, d, dt), mk) in enumerate(zip(rows, Mk)):
        if not mk[0] and dt in offs:
            T[i, 0] = work_log2(m, n, d, 0) + float(np.median(offs[dt]))
            Mk[i, 0] = 1.0
    return T, Mk


def train(dev, X, T, Mk, epochs=600, batch=128, lr=3e-3, seed=7):
    import torch
    tX = torch.from_numpy(X).to(dev)
    tT = torch.from_numpy(T).to(dev)
    tM = torch.from_numpy(Mk).to(dev)
    w, hist = capi.perm_mlp_train(tX, tT, tM, DIMS, epochs, batch, lr, seed)
    torch.cuda.synchronize(dev)
    return w.cpu().numpy(), hist.cpu().numpy()


def predict(weights, X):
    """Host evaluation of the perceptron (the same arithmetic perm_auto runs)."""
    in_dim, hid, out = DIMS
    w = np.asarray(weights, np.float64)
    k = 0
    W1 = w[k:k + in_dim * hid].reshape(in_dim, hid); k += in_dim * hid
    b1 = w[k:k + hid]; k += hid
    W2 = w[k:k + hid * hid].reshape(hid, hid); k += hid * hid
    b2 = w[k:k + hid]; k += hid
    W3 = w[k:k + hid * out].reshape(hid, out); k += hid * out
    b3 = w[k:k + out]
    h = np.maximum(np.asarray(X, np.float64) @ W1 + b1, 0)
    h = np.maximum(h @ W2 + b2, 0)
    return h @ W3 + b3


class PaperRule:
    """The paper's selection rule (Algorithm "Optimized Algorithm Selection") refit on
    our timings: for n <= p8 = 13, combinatoric if square and n <= p4 or if
    p1 r + p2 n + p3 > 0, else Glynn; for n > p8, Glynn if p5 r + p6 n + p7 > 0, else
    Ryser.  The hyperplanes are fitted by logistic regression on (r, n)."""

    P8 = 13

    def __init__(self):
        self.p = np.zeros(8)

    @staticmethod
    def _fit(F, y, iters=3000, lr=0.5):
        w = np.zeros(F.shape[1] + 1)
        Fb = np.hstack([F, np.ones((F.shape[0], 1))])
        for _ in range(iters):
            z = np.clip(Fb @ w, -30, 30)
            pr = 1 / (1 + np.exp(-z))
            w -= lr * Fb.T @ (pr - y) / max(len(y), 1)
        return w

    def fit(self, rows, T, Mk):
        small, small_y, large, large_y = [], [], [], []
        p4 = 0
        for (m, n, d, dt), t, mk in zip(rows, T, Mk):
            r = m / n
            if n <= self.P8 and mk[0] and mk[2]:
                small.append((r, n / 64))
                small_y.append(1.0 if t[0] < t[2] else 0.0)
                if m == n and t[0] < t[2]:
                    p4 = max(p4, n)
            if n > self.P8 and mk[1] and mk[2]:
                large.append((r, n / 64))
                large_y.append(1.0 if t[2] < t[1] else 0.0)
        w1 = self._fit(np.array(small), np.array(small_y)) if small else np.array([0, 0, -1.0])
        w2 = self._fit(np.array(large), np.array(large_y)) if large else np.array([0, 0, 1.0])
        self.p = np.array([w1[0], w1[1], w1[2], p4, w2[0], w2[1], w2[2], self.P8])
        return self

    def choose(self, m, n, code):
        r = m / n
        p = self.p
        if n <= self.P8:
            if (m == n and n <= p[3]) or (p[0] * r + p[1] * n / 64 + p[2] > 0):
                return 0
            return 2
        if code != capi.PERM_F64:
            return 2
        return 2 if p[4] * r + p[5] * n / 64 + p[6] > 0 else 1


def evaluate(dev, weights, rule, count, seed, log=None, max_best_s=0.01):
    """Held-out matrices from cells whose best time is at most max_best_s: time every
    candidate (exhaustive), and score each policy by sum time(choice) / sum time(best)."""
    import torch
    capi.perm_set_cost_model(None, None)  # perm_auto_choice then reports the built-in rule
    timer = Timer(dev)
    g = inputs.rng(seed)
    pairs = [(m, n) for m in range(2, 41) for n in range(m, 61)]
    totals = {"best": 0.0, "model": 0.0, "paper_rule": 0.0, "always_glynn": 0.0, "builtin": 0.0}
    agree, k, tries = 0, 0, 0
    while k < count and tries < 20 * count:
        tries += 1
        m, n = pairs[int(g.integers(len(pairs)))]
        if (1 << (n - 1)) > (1 << 24):  # keep exhaustive timing of every candidate cheap
            continue
        d = float(g.choice([0.1, 0.5, 1.0]))
        dt = str(g.choice(list(DTYPES)))
        A = make_matrix(m, n, d, dt, seed * 7919 + tries)
        dA = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
        code = DTYPES[dt]
        nnz = float(np.count_nonzero(A)) / A.size
        times = []
        for c in range(capi.PERM_NCAND):
            try:
                s = time_candidate(timer, dA, m, n, nnz, code, c)
            except capi.PermError:
                s = None
            times.append(math.inf if s is None else s)
        best = min(times)
        if not math.isfinite(best) or best > max_best_s:
            continue
        x = capi.perm_auto_features(m, n, nnz, code)
        y = predict(weights, x[None, :])[0]
        y = [y[c] if math.isfinite(times[c]) else math.inf for c in range(capi.PERM_NCAND)]
        choice = int(np.argmin(y))
        builtin, _ = capi.perm_auto_choice(dA)
        totals["best"] += best
        totals["builtin"] += times[builtin] if math.isfinite(times[builtin]) else times[2]
        totals["model"] += times[choice]
        totals["paper_rule"] += times[rule.choose(m, n, code)] if math.isfinite(times[rule.choose(m, n, code)]) \
            else times[2]
        totals["always_glynn"] += times[3] if code == capi.PERM_F64 else times[2]
        agree += int(times[choice] == best)
        k += 1
        if log and k % 500 == 0:
            log("evaluated %d/%d" % (k, count))
    ratio = {p: totals[p] / totals["best"] for p in totals if p != "best"}
    return {"matrices": k, "ratio_to_exhaustive": ratio, "model_picks_best": agree / max(k, 1),
            "total_best_s": totals["best"]}


def save(path, weights, meta):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, weights=np.asarray(weights, np.float32), dims=np.array(DIMS), meta=json.dumps(meta))


def load(path=MODEL_PATH):
    """(weights, dims, meta) of a saved model; ValueError if the file is damaged."""
    try:
        z = np.load(path, allow_pickle=False)
        w = np.asarray(z["weights"], np.float32)
        dims = tuple(int(v) for v in z["dims"])
        meta = json.loads(str(z["meta"]))
    except Exception as e:  # unreadable archive, missing array, bad metadata
        raise ValueError("cost model file %s is damaged: %s" % (path, e)) from None
    in_dim, hid, out = dims if len(dims) == 3 else (0, 0, 0)
    if (in_dim, out) != (capi.PERM_NFEATURES, capi.PERM_NCAND) or \
            w.size != in_dim * hid + hid + hid * hid + hid + hid * out + out or not np.all(np.isfinite(w)):
        raise ValueError("cost model file %s does not hold a %d -> %d perceptron" % (path, capi.PERM_NFEATURES,
                                                                                 capi.PERM_NCAND))
    return w, dims, meta


def install(path=MODEL_PATH, device=0):
    """Install a saved model as perm_auto's cost model on `device`."""
    w, dims, _ = load(path)
    capi.perm_set_cost_model(w, dims, device)
    return w


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=600)
    ap.add_argument("--eval", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--report", default=None)
    a = ap.parse_args()
    import torch
    dev = torch.device("cuda:0")
    log = lambda s: print(s, flush=True)  # noqa: E731
    t0 = time.time()
    cells = grid_cells(a.cells, inputs.SEED_BASE + 5)
    X, T, Mk, rows = measure_grid(dev, cells, seed0=inputs.SEED_BASE * 10, log=log)
    T, Mk = fill_combinatoric(X, T, Mk, rows)
    t1 = time.time()
    w, hist = train(dev, X, T, Mk, epochs=a.epochs)
    t2 = time.time()
    rule = PaperRule().fit(rows, T, Mk)
    res = evaluate(dev, w, rule, a.eval, inputs.SEED_BASE + 6, log=log)
    meta = {"cells": a.cells, "epochs": a.epochs, "final_loss": float(hist[-1]), "measure_s": t1 - t0,
            "train_s": t2 - t1, "paper_rule": [float(v) for v in rule.p], "evaluation": res,
            "device": torch.cuda.get_device_name(dev)}
    save(a.out, w, meta)
    print(json.dumps(meta), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump({"meta": meta, "loss_history": [float(v) for v in hist]}, f)


if __name__ == "__main__":
    main()
