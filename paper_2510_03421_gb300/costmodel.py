"""Learned dispatch for perm_auto: timings measured by this library, a cost model
trained on the GPU by the library's own MLP kernels, and its evaluation.

The paper tunes two linear hyperplanes in (m/n, n) at build time (Algorithm
"Optimized Algorithm Selection", p1..p8).  Here a small perceptron predicts
log2(seconds) of every candidate -- an algorithm together with a kernel configuration
(arithmetic: FP64, integer pipes, mixed; chunk starts per thread or from the FP64
tensor-core contraction; chunk length) -- from features of the matrix (order, shape,
density, dtype, log work counts; ``capi.perm_auto_features``) and perm_auto runs the
argmin.  This module:

* times candidates on a seeded grid of (m, n, density, dtype) cells
  (``measure_grid``), extrapolating sweeps too long to run from a timed term range;
* trains the model with ``capi.perm_mlp_train`` on each cell's regret (log2 time over
  the cell's fastest candidate) and installs it with ``capi.perm_set_cost_model``;
* refits the paper's rule (``PaperRule``) on the same timings as a baseline;
* scores policies on a held-out batch against exhaustive timing (``evaluate``).

Usage (on a GPU):  python -m paper_2510_03421_gb300.costmodel --cells 3000 --eval 10000
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import capi, inputs

CANDS = ("combinatoric", "ryser", "glynn", "glynn_mixed", "ryser_fp64", "glynn_fp64_tensor_core_start",
         "glynn_integer_only", "glynn_short_chunks_or_complex_fp64")
DTYPES = {"f64": capi.PERM_F64, "c128": capi.PERM_C128, "u8": capi.PERM_U8}
DIMS = (capi.PERM_NFEATURES, 64, capi.PERM_NCAND)
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "costmodel_gb300.npz")

# candidates that exist per dtype (shape limits are applied in time_candidate, as in
# the library's own feasibility test)
AVAILABLE = {
    capi.PERM_F64: (True,) * 8,
    capi.PERM_C128: (True, False, True, False, False, False, False, True),
    capi.PERM_U8: (True, False, True, False, False, False, False, False),
}


def cand_opts(cand, code):
    """(entry point, opts) perm_auto runs for candidate `cand` on dtype `code`."""
    real = code == capi.PERM_F64
    if cand == 1:
        return "ryser", {}
    if cand == 2:
        return "glynn", dict(arith=capi.PERM_ARITH_FP64) if real else {}
    if cand == 3:
        return "glynn", dict(arith=capi.PERM_ARITH_MIXED)
    if cand == 4:
        return "ryser", dict(arith=capi.PERM_ARITH_FP64)
    if cand == 5:
        return "glynn", dict(arith=capi.PERM_ARITH_FP64, start=capi.PERM_START_DMMA)
    if cand == 6:
        return "glynn", dict(arith=capi.PERM_ARITH_FIXED)
    if cand == 7:
        return "glynn", dict(arith=capi.PERM_ARITH_MIXED, chunk_log2=6) if real else dict(arith=capi.PERM_ARITH_FP64)
    raise ValueError(cand)


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


def _esym(m, n):
    """The integer pipes take a real rectangle with the padding in closed form (m n
    multiply-adds per sign vector) when m <= 32 and n - m >= 3 or m <= 8."""
    return m < n and m <= 32 and (n - m >= 3 or m <= 8)


def _ryser_by_size(m, n):
    if m >= n:
        return None
    by_size = sum(math.comb(n, s) for s in range(1, m + 1))
    return by_size if 3 * by_size < (1 << n) else None


def work_log2(m, n, density, cand):
    """log2 of the work count of a candidate (terms x width)."""
    if cand == 0:
        return _log2_nodes(m, n, max(density, 1e-3))
    if cand in (1, 4):
        bs = _ryser_by_size(m, n)
        return math.log2(bs) + math.log2(max(m, 1)) if bs else n + math.log2(max(m, 1))
    if cand in (3, 6, 7) and m < n:
        if _esym(m, n):
            return (m - 1) + math.log2(m * n)
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

    def run(self, fn, reps=3):
        """Median of `reps` timed runs after a warm-up (robust to a stray slow run)."""
        times = []
        with self.torch.cuda.stream(self.stream):
            fn()  # warm-up (and first-use setup)
            for _ in range(reps):
                self.e0.record(self.stream)
                fn()
                self.e1.record(self.stream)
                self.e1.synchronize()
                times.append(self.e0.elapsed_time(self.e1) * 1e-3)
        return float(np.median(times))


def time_candidate(timer, dA, m, n, density, code, cand, reps=3):
    """Seconds for candidate `cand` on the device matrix dA (m <= n), or None if the
    candidate does not exist for the dtype and shape.  Long sweeps are timed on a term
    range (squares) or a leading block of rows (rectangles) and scaled by the work
    count; long combinatoric searches are labelled later from the node count."""
    if not AVAILABLE[code][cand]:
        return None
    if cand == 5 and (m != n or n > 48):
        return None
    if cand == 7 and code == capi.PERM_C128 and m != n:
        return None
    s = timer.stream
    big = dict(max_terms=1 << 62)
    if cand == 0:
        if work_log2(m, n, density, 0) > 30:  # about a second or more
            return None
        return timer.run(lambda: capi.perm_combinatoric(dA, stream=s, opts=big), reps)
    fn, opts = cand_opts(cand, code)
    opts = dict(big, **opts)
    full = getattr(capi, "perm_" + fn)
    lw = work_log2(m, n, density, cand)
    if lw <= math.log2(TERM_SAMPLE) + 2 + math.log2(max(n, 1)):
        return timer.run(lambda: full(dA, stream=s, opts=opts), reps)
    if fn == "glynn" and m == n:
        part = timer.run(lambda: capi.perm_glynn_partial(dA, 0, TERM_SAMPLE, stream=s, opts=opts), reps)
        return part * (1 << (n - 1)) / TERM_SAMPLE
    if fn == "ryser" and cand == 4 and _ryser_by_size(m, n) is None:
        part = timer.run(lambda: capi.perm_ryser_partial(dA, 0, TERM_SAMPLE, stream=s, opts=opts), reps)
        return part * (1 << n) / TERM_SAMPLE
    # a smaller problem of the same kind: fewer rows (rectangular Glynn), or fewer
    # columns (Ryser), scaled by the ratio of the work counts
    mm, nn = m, n
    while work_log2(mm, nn, density, cand) > math.log2(TERM_SAMPLE) + math.log2(max(nn, 1)):
        if fn == "glynn" and mm > 1:
            mm -= 1
        elif nn > mm + 1:
            nn -= 1
        elif mm > 1:
            mm -= 1
            nn -= 1
        else:
            break
    sub = dA[:mm, :nn]
    part = timer.run(lambda: full(sub, stream=s, opts=opts), reps)
    return part * 2.0 ** (lw - work_log2(mm, nn, density, cand))


def grid_cells(count, seed, small_frac=0.5, small_n=26):
    """A seeded sample of the (m, n, density, dtype) grid: m in 2..40, n in m..60; a
    fraction `small_frac` drawn from n <= small_n, where the candidates' times are
    close, every candidate is timed in full and most matrices of a mixed batch are."""
    g = inputs.rng(seed)
    cells = []
    pairs = [(m, n) for m in range(2, 41) for n in range(m, 61)]
    small = [(m, n) for (m, n) in pairs if n <= small_n]
    for k in range(count):
        pool = small if k < small_frac * count else pairs
        m, n = pool[int(g.integers(len(pool)))]
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


def regret(T, Mk):
    """Targets relative to each cell's fastest candidate (log2 time - log2 best): the
    choice depends only on these differences, and the absolute scale (2^-15 .. 2^10 s
    across the grid) would otherwise take the model's capacity."""
    T = T.copy()
    for i in range(len(T)):
        live = Mk[i] > 0
        if live.any():
            T[i, live] -= T[i, live].min()
    return T


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


def evaluate(dev, weights, rule, count, seed, log=None, max_best_s=0.01, reps=3, max_n=24):
    """Held-out matrices from cells whose best time is at most max_best_s (and n <=
    max_n, so that timing every candidate stays cheap): time every candidate
    (exhaustive, median of `reps`), and score each policy by sum time(choice) / sum
    time(best), overall and per dtype."""
    import torch
    capi.perm_set_cost_model(None, None)  # perm_auto_choice then reports the built-in rule
    timer = Timer(dev)
    g = inputs.rng(seed)
    pairs = [(m, n) for m in range(2, 41) for n in range(m, 61)]
    policies = ("best", "model", "paper_rule", "always_glynn", "builtin")
    totals = {p: 0.0 for p in policies}
    per_dtype = {dt: {p: 0.0 for p in policies} for dt in DTYPES}
    counts = {dt: 0 for dt in DTYPES}
    agree, k, tries = 0, 0, 0
    while k < count and tries < 20 * count:
        tries += 1
        m, n = pairs[int(g.integers(len(pairs)))]
        if n > max_n:
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
                s = time_candidate(timer, dA, m, n, nnz, code, c, reps=reps)
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
        pr = rule.choose(m, n, code)
        row = {"best": best, "model": times[choice],
               "builtin": times[builtin] if math.isfinite(times[builtin]) else times[2],
               "paper_rule": times[pr] if math.isfinite(times[pr]) else times[2],
               "always_glynn": times[3] if code == capi.PERM_F64 else times[2]}
        for p in policies:
            totals[p] += row[p]
            per_dtype[dt][p] += row[p]
        counts[dt] += 1
        agree += int(times[choice] == best)
        k += 1
        if log and k % 500 == 0:
            log("evaluated %d/%d" % (k, count))
    ratio = {p: totals[p] / totals["best"] for p in totals if p != "best"}
    by_dtype = {dt: {p: per_dtype[dt][p] / per_dtype[dt]["best"] for p in policies if p != "best"}
                for dt in DTYPES if counts[dt]}
    return {"matrices": k, "per_dtype_matrices": counts, "ratio_to_exhaustive": ratio,
            "ratio_to_exhaustive_by_dtype": by_dtype, "model_picks_best": agree / max(k, 1),
            "total_best_s": totals["best"], "timing": "median of %d after a warm-up" % reps}


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
    ap.add_argument("--cells", type=int, default=3000)
    ap.add_argument("--eval", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=1500)
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
    w, hist = train(dev, X, regret(T, Mk), Mk, epochs=a.epochs)
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
