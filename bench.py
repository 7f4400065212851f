#!/usr/bin/env python
"""Benchmark: Glynn Gray-code terms/s for the permanent of a 36 x 36 float64
matrix (entries i.i.d. uniform[-1, 1], fixed seed), through the C ABI.

One step = one full perm_glynn call on the matrix (all 2^35 Gray-code terms:
chunk-start rebuilds, the sweep, the reductions and the normalisation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 36] [--arith auto|fp64|fixed]

Prints one JSON line (rank 0).  Under torchrun each rank computes its own copy of
the workload on its own GPU (weak scaling, no data-path collective); ``value`` is
the terms of all ranks divided by the slowest rank's time.  ``--impl reference``
times the CPU oracle on the host cores on a bounded sample of the same terms.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Glynn Gray-code terms/s (n=36 FP64) & batched perms/s vs plain FP64 at stated err"
UNIT = "terms/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=36, help="matrix order (36 is the benchmark workload)")
    ap.add_argument("--dtype", default="f64", choices=["f64", "c128"],
                    help="c128: the 32x32 complex workload (profiling runs)")
    ap.add_argument("--arith", default="auto", choices=["auto", "fp64", "fixed", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 100,000-matrix leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 sweep comparison")
    ap.add_argument("--batch-count", type=int, default=100000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--precision-only", action="store_true",
                    help="run only the precision study (digits lost) and print it as one JSON line")
    ap.add_argument("--cauchy-only", action="store_true",
                    help="run only the Cauchy (Borchardt) leg and print its figures as one JSON line")
    return ap.parse_args()


def workload(n: int, dtype: str = "f64"):
    from paper_2510_03421_gb300 import inputs
    if dtype == "c128":
        A = inputs.complex_gaussian(n, n, inputs.SEED_BASE + 2)
        return A, "glynn %dx%d complex128 Gaussian/sqrt(n) seed %d (2^%d Gray-code terms per step)" % (
            n, n, inputs.SEED_BASE + 2, n - 1)
    if n == 36:
        A = inputs.square36_f64()
    else:
        A = inputs.uniform_real(n, n, inputs.SEED_BASE + 2)
    desc = "glynn %dx%d float64 uniform[-1,1] seed %d (2^%d Gray-code terms per step)" % (
        n, n, inputs.SEED_BASE + 2, n - 1)
    return A, desc


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- CPU oracle timing
def cpu_oracle_rate(A, seconds: float, cores: int):
    """Oracle Glynn partial sums (double, as it stands) on disjoint term ranges, one
    per host thread; returns (terms/s, terms timed, wall seconds)."""
    import oracle
    oracle.build()
    n = A.shape[0]
    T = 1 << (n - 1)
    probe = 1 << 10
    t0 = time.perf_counter()
    oracle.glynn_partial(A, 0, probe, prec="f64")
    per_term = (time.perf_counter() - t0) / probe
    per_thread = max(probe, int(seconds / per_term))
    per_thread = min(per_thread, T // cores)
    starts = [(T // cores) * k for k in range(cores)]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda s: oracle.glynn_partial(A, s, s + per_thread, prec="f64"), starts))
    wall = time.perf_counter() - t0
    terms = per_thread * cores
    return terms / wall, terms, wall


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r[1:5]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    A, desc = workload(args.n)
    cores = os.cpu_count() or 1
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_rate(A, per_step / 4, cores)
    rates, terms_total, wall_total = [], 0, 0.0
    for _ in range(args.steps):
        r, t, w = cpu_oracle_rate(A, per_step, cores)
        rates.append(r)
        terms_total += t
        wall_total += w
    value = terms_total / wall_total
    sample = "%d oracle Glynn terms per step (double, O(n^2) per term as the paper's base algorithm), %d threads" % (
        terms_total // max(1, args.steps), cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": args.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batched leg
# Per padded order N of the mixed integer-pipe sweep glynn_fx_kernel<N, K, false>: thread
# instructions per term (ncu smsp__inst_executed.sum x 32 / terms), DRAM bytes per launch
# and pipe utilisations, from one ncu capture of this kernel (label says which); the
# bench times the kernel itself and scales by its own terms/s.
ISSUE_PROFILE = {
    36: {"instructions_per_term": 887.7, "dram_bytes_per_launch": 90112,
         "pipes": {"alu": 0.634, "fp64": 0.618, "fma": 0.272, "issue": 0.571},
         "label": "ncu --set full capture of glynn_fx_kernel<36, 8, false> at n = 34 (2^33 terms: 2.383e11 warp "
                  "instructions, 32.0 threads per instruction; instructions scale per term, DRAM traffic does "
                  "not grow with the term count)"},
}


BATCH_CHECK = {}  # results of the batched leg kept for the oracle check of the CPU leg


def run_batched(args, dev, stream):
    """100,000 complex128 n x n blocks of Haar unitaries (n uniform in 4..20): one
    perm_batched graph launch per step, against one perm_glynn call per matrix."""
    import numpy as np
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    count = args.batch_count
    sizes, packed, offsets = inputs.batched_haar(count, 4, 20, inputs.SEED_BASE + 4)
    M = sizes.astype(np.int32)
    tp = torch.from_numpy(packed).to(dev)
    to = torch.from_numpy(offsets).to(dev)
    tM = torch.from_numpy(M).to(dev)
    out = torch.empty((count, 2), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        # the first call tunes the launch settings on a sample of the batch
        capi.perm_batched(tp, to, tM, tM, out=out, stream=stream, opts=dict(exhaustive=1))
        for _ in range(max(1, args.warmup)):
            capi.perm_batched(tp, to, tM, tM, out=out, stream=stream)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            ev[k][0].record(stream)
            capi.perm_batched(tp, to, tM, tM, out=out, stream=stream)
            ev[k][1].record(stream)
        stream.synchronize()
    batched_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # plain: one perm_glynn call per matrix (its own kernel launches, default arithmetic),
    # on a sample of the batch, captured once into a CUDA graph and replayed, so that the
    # time is the kernels' and not the host's; the same again with opts.arith = FP64
    sample = min(count, 10000)
    views = [tp[int(offsets[b]): int(offsets[b]) + int(sizes[b]) ** 2].view(int(sizes[b]), int(sizes[b]))
             for b in range(sample)]
    plain = {}
    for key, opts in (("default", None), ("fp64", dict(arith=capi.PERM_ARITH_FP64))):
        res = torch.empty((sample, 2), dtype=torch.float64, device=dev)
        outs = [res[b] for b in range(sample)]
        for b in range(sample):  # eager pass: per-call set-up, and the workspace sized
            capi.perm_glynn(views[b], out=outs[b], stream=stream, opts=opts)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
            for b in range(sample):
                capi.perm_glynn(views[b], out=outs[b], stream=stream, opts=opts)
        graph.replay()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(max(1, args.steps // 4)):
                graph.replay()
            e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / max(1, args.steps // 4)
        plain[key] = {"perms_per_s": sample / (ms * 1e-3), "ms_per_sample": ms, "values": res.cpu().numpy()}
        del graph
    a = out.cpu().numpy()
    p = plain["default"]["values"]
    za, zp = a[:sample, 0] + 1j * a[:sample, 1], p[:, 0] + 1j * p[:, 1]
    rel = float(np.max(np.abs(za - zp) / np.maximum(np.abs(zp), 1e-300)))
    BATCH_CHECK["batched"] = a
    BATCH_CHECK["plain"] = p
    BATCH_CHECK["sizes"], BATCH_CHECK["packed"], BATCH_CHECK["offsets"] = sizes, packed, offsets
    batched_rate = count / (batched_ms * 1e-3)
    terms = float(np.sum(2.0 ** (sizes.astype(np.float64) - 1)))
    # algorithmic work of the complex Glynn sweep: 8n - 4 FP64-equivalent operations per term
    flops = float(np.sum(2.0 ** (sizes.astype(np.float64) - 1) * (8.0 * sizes - 4.0)))
    return {"workload": "%d complex128 n x n leading blocks of Haar unitaries (order 64), n uniform in 4..20" % count,
            "perms_per_s": count / (batched_ms * 1e-3), "ms_per_batch": batched_ms,
            "terms_per_s": terms / (batched_ms * 1e-3),
            "fp64_equiv_tflops": flops / (batched_ms * 1e-3) / 1e12,
            "plain_kernel": {"perms_per_s": plain["default"]["perms_per_s"],
                             "fp64_perms_per_s": plain["fp64"]["perms_per_s"], "sample": sample,
                             "how": "one perm_glynn per matrix (default arithmetic; and opts.arith = FP64) for the "
                                    "first %d matrices, captured in one CUDA graph, replayed, CUDA events" % sample},
            "speedup_vs_plain_kernel": batched_rate / plain["default"]["perms_per_s"],
            "speedup_vs_plain_fp64_kernel": batched_rate / plain["fp64"]["perms_per_s"],
            "max_rel_diff_vs_plain": rel,
            "arith": "n >= 13: integer pipes (fixed-point column sums, complex software-float products, 192-bit "
                     "accumulation; the tuner may put part of each product on the FP64 unit); below: FP64, "
                     "Kahan-compensated",
            "launch": "one CUDA graph (size-class kernels on parallel branches)"}


def run_batched_real(args, dev, stream):
    """The same batch shape with real entries (uniform[-1,1]): 100,000 matrices, n uniform in
    4..20, one tuned perm_batched graph launch per step."""
    import numpy as np
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    count = args.batch_count
    g = inputs.rng(inputs.SEED_BASE + 6)
    sizes = g.integers(4, 21, count).astype(np.int32)
    offsets = np.zeros(count, np.int64)
    offsets[1:] = np.cumsum(sizes.astype(np.int64) ** 2)[:-1]
    packed = g.uniform(-1.0, 1.0, int(offsets[-1] + int(sizes[-1]) ** 2))
    tp, to, tM = [torch.from_numpy(x).to(dev) for x in (packed, offsets, sizes)]
    out = torch.empty(count, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        capi.perm_batched(tp, to, tM, tM, out=out, stream=stream, opts=dict(exhaustive=1))
        for _ in range(max(1, args.warmup)):
            capi.perm_batched(tp, to, tM, tM, out=out, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            ev[k][0].record(stream)
            capi.perm_batched(tp, to, tM, tM, out=out, stream=stream)
            ev[k][1].record(stream)
        stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    return {"workload": "%d float64 n x n matrices, uniform[-1,1], n uniform in 4..20, seed %d" % (
                count, inputs.SEED_BASE + 6),
            "perms_per_s": count / (ms * 1e-3), "ms_per_batch": ms}


def run_sbp(args, dev, stream, count=1000000, n=12, N=24):
    """SBP coefficients c_m = per(C P) (Eq. SBGpermanent): one real n x N coefficient
    matrix, `count` random occupation bitstrings with n of N states occupied, one
    perm_sbp call per step (columns gathered inside the kernel)."""
    import numpy as np
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    g = inputs.rng(inputs.SEED_BASE + 7)
    C = g.uniform(-1.0, 1.0, (n, N))
    cols = np.argsort(g.random((count, N)), axis=1)[:, :n]
    occ = np.bitwise_or.reduce(np.left_shift(np.uint64(1), cols.astype(np.uint64)), axis=1)
    dC = torch.from_numpy(C).to(dev)
    docc = torch.from_numpy(occ.view(np.int64)).to(dev)
    out = torch.empty(count, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            capi.perm_sbp(dC, docc, out=out, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            ev[k][0].record(stream)
            capi.perm_sbp(dC, docc, out=out, stream=stream)
            ev[k][1].record(stream)
        stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    return {"workload": "%d occupation bitstrings, %d of %d states occupied, real coefficients uniform[-1,1], "
                        "seed %d" % (count, n, N, inputs.SEED_BASE + 7),
            "coefficients_per_s": count / (ms * 1e-3), "terms_per_s": count * 2.0 ** (n - 1) / (ms * 1e-3),
            "ms_per_call": ms}


def run_batched_int(args, dev, stream):
    """Exact batches: 100,000 0/1 matrices (Bernoulli(0.5)) and 100,000 Gaussian-integer
    matrices (parts uniform in -2..2), n uniform in 4..20, one perm_batched call each
    (one warp per matrix, int128)."""
    import numpy as np
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    count = args.batch_count
    g = inputs.rng(inputs.SEED_BASE + 8)
    sizes = g.integers(4, 21, count).astype(np.int32)
    offsets = np.zeros(count, np.int64)
    offsets[1:] = np.cumsum(sizes.astype(np.int64) ** 2)[:-1]
    total = int(offsets[-1] + int(sizes[-1]) ** 2)
    res = {}
    for kind, packed, fn in (("0/1", (g.random(total) < 0.5).astype(np.uint8), capi.perm_batched),
                             ("gaussian", g.integers(-2, 3, 2 * total).astype(np.int64), capi.perm_batched_gaussian)):
        tp, to, tM = (torch.from_numpy(a).to(dev) for a in (packed, offsets, sizes))
        with torch.cuda.stream(stream):
            out = fn(tp, to, tM, tM, stream=stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for k in range(args.steps):
                ev[k][0].record(stream)
                fn(tp, to, tM, tM, out=out, stream=stream)
                ev[k][1].record(stream)
            stream.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        res[kind] = {"perms_per_s": count / (ms * 1e-3), "ms_per_batch": ms}
    res["workload"] = "%d matrices per kind, n uniform in 4..20, seed %d; exact int128" % (count, inputs.SEED_BASE + 8)
    return res


def run_cauchy(args, dev, stream, count=1216, n=36):
    """Cauchy permanents by Borchardt's theorem (perm_cauchy): `count` matrices
    c_ij = 1 / (x_i - y_j) of order n with the points of the paper's accuracy tests
    (x ~ U[0.25, 0.75], y ~ U[-0.75, -0.25]), one call per step; plus one matrix of
    order 36 and one of order 64 alone (latency)."""
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    seed = inputs.SEED_BASE + 15
    x, y = inputs.cauchy_points(n, seed, count=count)

    def timed(xh, yh, steps):
        dx, dy = torch.from_numpy(xh).to(dev), torch.from_numpy(yh).to(dev)
        out = torch.empty(xh.shape[0], dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                capi.perm_cauchy(dx, dy, out=out, stream=stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                ev[k][0].record(stream)
                capi.perm_cauchy(dx, dy, out=out, stream=stream)
                ev[k][1].record(stream)
            stream.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps, out
    ms, out = timed(x, y, args.steps)
    ms36, _ = timed(x[:1], y[:1], args.steps)
    x64, y64 = inputs.cauchy_points(64, seed + 1)
    ms64, _ = timed(x64, y64, args.steps)
    return {"workload": "%d Cauchy matrices of order %d, x ~ U[0.25,0.75], y ~ U[-0.75,-0.25], seed %d" % (
                count, n, seed),
            "matrices_per_s": count / (ms * 1e-3), "ms_per_call": ms, "first": float(out[0].item()),
            "ms_one_matrix_n36": ms36, "ms_one_matrix_n64": ms64}


def run_precision(dev, stream, cases=((8, 8), (16, 16), (24, 24), (32, 32), (8, 16), (16, 32))):
    """The paper's precision study (Eq. digits_lost, d = log10(|eval - true| / |true|) -
    log10(eps)) on its three matrix families: all ones (per = n!/(n-m)!), the identity
    padded with zero columns (per = 1) and Cauchy matrices c_ij = 1/(x_i - y_j) (square;
    truth: perm_cauchy, Borchardt's theorem rounded to double).  Each algorithm reports
    d and whether its stated error bound covers the error."""
    import math

    import numpy as np
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    eps = float(np.finfo(np.float64).eps)
    algos = {"glynn": ("perm_glynn", capi.PERM_ARITH_AUTO), "glynn_fp64": ("perm_glynn", capi.PERM_ARITH_FP64),
             "ryser": ("perm_ryser", capi.PERM_ARITH_AUTO)}

    def digits(v, t):
        e = abs(v - t)
        return None if e == 0 else round(math.log10(e / abs(t)) - math.log10(eps), 2)

    rows = []
    for m, n in cases:
        fams = [("ones", np.ones((m, n)), math.factorial(n) / math.factorial(n - m)),
                ("identity", np.eye(m, n), 1.0)]
        if m == n:
            x, y = inputs.cauchy_points(n, inputs.SEED_BASE + 20 + n, draws=100)
            dx, dy = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
            tout = capi.perm_cauchy(dx, dy, stream=stream)
            stream.synchronize()  # the result is written on `stream`; read it after that
            t = float(tout[0].item())
            fams.append(("cauchy", 1.0 / (x[0][:, None] - y[0][None, :]), t))
        for name, A, truth in fams:
            row = {"matrix": "%s %dx%d" % (name, m, n), "true": truth}
            dA = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
            for key, (fn, arith) in algos.items():
                out = torch.empty(1, dtype=torch.float64, device=dev)
                err = torch.empty(1, dtype=torch.float64, device=dev)
                getattr(capi, fn)(dA, out=out, stream=stream, opts={"arith": arith, "err": err})
                stream.synchronize()
                v, e = float(out.item()), float(err.item())
                row[key] = {"d": digits(v, truth), "bound_holds": (e < 0) or abs(v - truth) <= e}
            rows.append(row)
    return {"metric": "digits lost, Eq. digits_lost (None = exact)", "cases": rows}


def _oracle_glynn(A):
    import oracle
    return complex(oracle.glynn(A))


def batched_oracle_check():
    """CPU leg: both arms of the batched comparison against the long-double oracle, two
    matrices of every order 4..20 from the plain arm's sample (spawned processes)."""
    import multiprocessing

    import numpy as np
    sizes, packed, offsets = BATCH_CHECK["sizes"], BATCH_CHECK["packed"], BATCH_CHECK["offsets"]
    sample = len(BATCH_CHECK["plain"])
    picks = []
    for n in range(4, 21):
        idx = np.nonzero(sizes[:sample] == n)[0]
        if len(idx):
            picks += sorted({int(idx[0]), int(idx[-1])})
    mats = [np.ascontiguousarray(packed[offsets[b]: offsets[b] + int(sizes[b]) ** 2].reshape(int(sizes[b]),
                                                                                         int(sizes[b])))
            for b in picks]
    t0 = time.time()
    with multiprocessing.get_context("spawn").Pool(min(len(mats), os.cpu_count() or 1)) as pool:
        truth = pool.map(_oracle_glynn, mats)
    res = {}
    for arm in ("batched", "plain"):
        v = BATCH_CHECK[arm]
        errs = [abs(complex(v[b, 0], v[b, 1]) - t) / abs(t) for b, t in zip(picks, truth)]
        res["max_rel_err_vs_oracle_" + arm] = float(max(errs))
    res["checked"] = "%d matrices, two of every order 4..20, oracle in long double (%.0f s)" % (len(picks),
                                                                                          time.time() - t0)
    return res


CHUNK_STUDY = {}  # GPU partial sums kept for the oracle comparison of the CPU leg


def run_chunk_start_study(dev, stream, span=4096, chunk_log2=6):
    """GPU part of the chunk-start precision study on the 36x36 float64 and 32x32
    complex128 workloads: term ranges at the start, middle and end of the Gray walk,
    summed by each variant (FP64 with per-thread chunk starts, FP64 with the starts
    from the tensor-core contraction, integer pipes, mixed); chunks of 2^6 terms, so
    each range holds 64 chunk starts.  Also the whole 32x32 all-ones matrix (per =
    32!, Eq. digits_lost) by each variant."""
    import math

    import torch

    from paper_2510_03421_gb300 import capi, inputs
    variants = {"fp64_thread_start": dict(arith=capi.PERM_ARITH_FP64, start=capi.PERM_START_SCALAR),
                "fp64_tensor_core_start": dict(arith=capi.PERM_ARITH_FP64, start=capi.PERM_START_DMMA),
                "integer_pipes": dict(arith=capi.PERM_ARITH_FIXED), "mixed": dict(arith=capi.PERM_ARITH_MIXED)}
    cvariants = {"fp64": dict(arith=capi.PERM_ARITH_FP64), "integer_pipes": dict(arith=capi.PERM_ARITH_FIXED),
                 "mixed": dict(arith=capi.PERM_ARITH_MIXED)}
    out = {}
    for wname, A, vs in (("36x36 float64", inputs.square36_f64(), variants),
                         ("32x32 complex128", inputs.square32_c128(), cvariants)):
        n = A.shape[0]
        T = 1 << (n - 1)
        ranges = [(0, span), (T // 3 + 77, T // 3 + 77 + span), (T - span, T)]
        dA = torch.from_numpy(A).to(dev)
        rows = {}
        for vname, opts in vs.items():
            vals = []
            for a, b in ranges:
                o = capi.perm_glynn_partial(dA, a, b, stream=stream, opts=dict(opts, chunk_log2=chunk_log2))
                stream.synchronize()
                v = o.cpu().numpy()
                vals.append(float(v[0] + v[1]) if A.dtype.kind == "f" else complex(v[0] + v[1], v[2] + v[3]))
            rows[vname] = vals
        out[wname] = {"ranges": ranges, "values": rows}
        CHUNK_STUDY[wname] = (A, ranges, rows)
    ones = torch.ones((32, 32), dtype=torch.float64, device=dev)
    exact = float(math.factorial(32))
    eps = 2.0 ** -52
    digits = {}
    for vname, opts in variants.items():
        r = capi.perm_glynn(ones, stream=stream, opts=opts)
        stream.synchronize()
        e = abs(float(r.item()) - exact)
        digits[vname] = None if e == 0 else round(math.log10(e / exact) - math.log10(eps), 2)
    return {"metric": "chunk-start variants: partial sums on sampled term ranges (errors against the "
                      "long-double oracle in the CPU leg) and digits lost on the 32x32 all-ones matrix",
            "chunk_log2": chunk_log2, "span": span, "ones_32x32_digits_lost": digits}


def chunk_start_oracle_check():
    """CPU leg: each variant's sampled-range partial sums against the oracle's, in units
    of the range's sum of |term| (the scale of any evaluation's rounding)."""
    import oracle
    res = {}
    for wname, (A, ranges, rows) in CHUNK_STUDY.items():
        truth = [oracle.glynn_partial(A, a, b) for a, b in ranges]
        scale = [oracle.glynn_partial_abs(A, a, b) for a, b in ranges]
        res[wname] = {v: max(abs(x - t) / s for x, t, s in zip(vals, truth, scale)) for v, vals in rows.items()}
    return {"max_error_over_sum_abs": res}


# ----------------------------------------------------------------------------- other configs
def run_configs(dev, stream, reps=3):
    """Time each of the other workloads (CUDA events, best of `reps` after a warm-up):
    16x16 float64 by Glynn, Ryser and the combinatoric algorithm (16! injective maps);
    32x32 complex128 by Glynn; 20x40 float64 by Glynn (padding summed in closed form)
    and by rectangular Ryser (2^40 Gray-ordered subsets on the integer pipes); 26x26 0/1
    (exact int128) by Glynn."""
    import torch

    from paper_2510_03421_gb300 import capi, inputs
    A16, R = inputs.square16_f64(), inputs.rect20x40_f64()
    cases = [("16x16 float64 uniform[-1,1], Glynn", "perm_glynn", A16, None, 1 << 15, reps),
             ("16x16 float64 uniform[-1,1], Ryser", "perm_ryser", A16, None, 1 << 16, reps),
             ("16x16 float64 uniform[-1,1], combinatoric (16! leaves)", "perm_combinatoric", A16,
              dict(max_terms=1 << 46), 20922789888000, 1),
             ("32x32 complex128 Gaussian / sqrt(2n), Glynn", "perm_glynn", inputs.square32_c128(), None, 1 << 31,
              reps),
             ("20x40 float64 uniform[0,1], Glynn (padding in closed form: 2^19 sign vectors)", "perm_glynn", R, None,
              1 << 19, reps),
             ("20x40 float64 uniform[0,1], Ryser (2^40 subsets, 6.19e11 of size <= 20)", "perm_ryser", R, None,
              1 << 40, 1),
             ("26x26 0/1 Bernoulli(0.5), exact, Glynn", "perm_glynn", inputs.square26_01(), None, 1 << 25, reps)]
    res = {}
    for name, fn, A, opts, terms, nrep in cases:
        dA = torch.from_numpy(A).to(dev)
        out = torch.empty(2 if A.dtype.kind in "ciu" else 1, dtype=torch.float64 if A.dtype.kind != "u" else
                          torch.int64, device=dev)
        err = torch.empty(1, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            best = float("inf")
            if nrep > 1:
                getattr(capi, fn)(dA, out=out, stream=stream, opts=opts)
            for _ in range(nrep):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                getattr(capi, fn)(dA, out=out, stream=stream, opts=opts)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        row = {"ms": best, "terms_per_s": terms / (best * 1e-3)}
        if A.dtype.kind == "f" and nrep > 1:  # the result with its stated bound (short legs)
            o = dict(opts or {}, err=err)
            getattr(capi, fn)(dA, out=out, stream=stream, opts=o)
            stream.synchronize()
            row["result"], row["err_bound"] = float(out[0].item()), float(err.item())
        elif A.dtype.kind == "f":
            row["result"] = float(out[0].item())
        res[name] = row
    return res


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)  # before the process group, so each rank's NCCL uses its own GPU
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2510_03421_gb300 import capi

    if args.cauchy_only:
        print(json.dumps(run_cauchy(args, dev, torch.cuda.Stream(dev))), flush=True)
        return
    if args.precision_only:
        print(json.dumps(run_precision(dev, torch.cuda.Stream(dev))), flush=True)
        return
    A, desc = workload(args.n, args.dtype)
    n = args.n
    terms = 1 << (n - 1)
    arith = {"auto": capi.PERM_ARITH_AUTO, "fp64": capi.PERM_ARITH_FP64, "fixed": capi.PERM_ARITH_FIXED,
             "mixed": capi.PERM_ARITH_MIXED}[args.arith]
    dA = torch.from_numpy(A).to(dev)
    out = torch.empty(2 if args.dtype == "c128" else 1, dtype=torch.float64, device=dev)
    err = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = capi.perm_opts(arith=arith)
    opts_err = capi.perm_opts(arith=arith, err=err.data_ptr())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2

    # roofline denominator: FP64 FMA issue rate measured now, on this GPU
    dfma = capi.perm_probe_rate(capi.PROBE_DFMA, local, stream)
    peak_flops = 2.0 * dfma

    for _ in range(args.warmup):
        capi.perm_glynn(dA, out=out, stream=stream, opts=opts)
    if args.dtype == "c128":  # the complex integer-pipe sweep states no bound
        capi.perm_glynn(dA, out=out, stream=stream, opts=opts)
        torch.cuda.synchronize(dev)
        result, err_bound = [float(v) for v in out.cpu()], None
    else:
        capi.perm_glynn(dA, out=out, stream=stream, opts=opts_err)  # result and its stated error bound
        torch.cuda.synchronize(dev)
        result, err_bound = float(out.item()), float(err.item())

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            capi.perm_glynn(dA, out=out, stream=stream, opts=opts)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    clock_summary = clocks.summary()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * terms * args.steps / (total_ms * 1e-3)

    # end to end through the C ABI with host (pinned) buffers, copies inside the timed region
    hA = torch.from_numpy(A).pin_memory()
    hout = torch.empty(out.numel(), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        capi.perm_glynn(hA, out=hout, stream=stream, opts=opts)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * terms * args.steps / e2e_s

    flops_per_term = 2 * n  # n additions, n-1 multiplications, one accumulation
    achieved = flops_per_term * terms / (ms_per_step * 1e-3)
    fixed = args.arith in ("auto", "fixed", "mixed")  # auto takes the integer-pipe sweep for n >= 10
    if fixed and n < 10:
        fixed = args.arith in ("fixed", "mixed")
    mixed = fixed and args.arith in ("auto", "mixed")
    launches_per_step = 3 if fixed else 2  # [fixed-point table,] sweep, final reduction
    props = torch.cuda.get_device_properties(dev)
    if fixed:
        # The integer-pipe sweep is bound by instruction issue (ncu: issue ahead of every
        # pipe).  Peak: one warp instruction per scheduler per clock, 4 schedulers per SM,
        # at the maximum SM clock; achieved: thread instructions per term (ncu, below)
        # times terms/s.
        sm_max = (clock_summary or {}).get("sm_max_mhz") or 2070.0
        issue_peak = props.multi_processor_count * 4 * 32 * sm_max * 1e6
        prof = ISSUE_PROFILE.get((n + 3) & ~3) if (mixed and args.dtype == "f64") else None
        roof = {"bound": "alu", "pipe": "instruction issue (integer ALU + IMAD, a share of each product on the "
                                        "FP64 unit)" if mixed else "instruction issue (integer ALU + IMAD)",
                "achieved": None, "peak": issue_peak / 1e12, "unit": "T thread-instructions/s", "frac": None,
                "traffic": None,
                "peak_source": "%d SMs x 4 schedulers x 32 lanes x %.0f MHz (maximum SM clock)" % (
                    props.multi_processor_count, sm_max)}
        if prof:
            ipt = prof["instructions_per_term"]
            roof["achieved"] = ipt * terms / (ms_per_step * 1e-3) / 1e12
            roof["frac"] = roof["achieved"] * 1e12 / issue_peak
            roof["instructions_per_term"] = ipt
            roof["traffic"] = prof["dram_bytes_per_launch"]
            roof["pipes_ncu"] = prof["pipes"]
            roof["evidence"] = prof["label"]
        roof["fp64_equivalent"] = {"achieved_tflops": achieved / 1e12, "fp64_peak_tflops": peak_flops / 1e12,
                                   "ratio": achieved / peak_flops, "flops_per_term": flops_per_term,
                                   "peak_source": "measured now: 2 x DFMA issue rate (perm_probe_rate)"}
    else:
        roof = {"bound": "alu", "pipe": "fp64", "achieved": achieved / 1e12, "peak": peak_flops / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak_flops, "traffic": None,
                "peak_source": "measured now: 2 x DFMA issue rate (perm_probe_rate)",
                "flops_per_term": flops_per_term}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "n": n, "m": n,
                   "arith": (("mixed: exact int64 fixed-point column sums; products in a 64-bit-mantissa "
                              "software float on the integer pipes, a few columns per term on the FP64 unit "
                              "beside them; 192-bit accumulation") if mixed else
                             ("fixed: exact int64 fixed-point column sums, 64-bit-mantissa products, 192-bit "
                              "accumulation") if fixed else
                             "fp64: FP64 column sums re-anchored every 2^14 terms, Kahan accumulation"),
                   "l2": "flushed between steps (256 MiB write, outside the timed events)",
                   "parallelism": "replica per GPU" if world > 1 else "1 GPU"},
        "result": result, "err_bound": err_bound,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(A.nbytes),
                "d2h_bytes_per_step": 8 * out.numel()},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clock_summary,
    }
    if args.dtype == "c128":
        line["dtype"] = "c128"
        line["roofline"] = None  # complex runs are profiling runs; the headline is the real workload
    if fixed and not args.no_fp64 and args.dtype == "f64":
        # the plain FP64 sweep on the same matrix, for comparison at stated error
        o64 = capi.perm_opts(arith=capi.PERM_ARITH_FP64)
        o64e = capi.perm_opts(arith=capi.PERM_ARITH_FP64, err=err.data_ptr())
        capi.perm_glynn(dA, out=out, stream=stream, opts=o64e)
        torch.cuda.synchronize(dev)
        r64, e64 = float(out.item()), float(err.item())
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev64[k][0].record(stream)
            capi.perm_glynn(dA, out=out, stream=stream, opts=o64)
            ev64[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ms64 = sum(a.elapsed_time(b) for a, b in ev64) / args.steps
        a64 = flops_per_term * terms / (ms64 * 1e-3)
        line["fp64_sweep"] = {"value": terms / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "result": r64,
                              "err_bound": e64, "achieved_tflops": a64 / 1e12, "frac_of_fp64_peak": a64 / peak_flops,
                              "speedup_of_default": ms64 / ms_per_step,
                              "abs_diff_to_default": abs(r64 - result)}
    if not args.no_batched:
        side = torch.cuda.Stream(dev)
        line["batched"] = run_batched(args, dev, side)
        line["batched"]["frac_of_fp64_peak"] = line["batched"]["fp64_equiv_tflops"] * 1e12 / peak_flops
        line["batched_real"] = run_batched_real(args, dev, side)
        line["sbp"] = run_sbp(args, dev, side)
        line["batched_int"] = run_batched_int(args, dev, side)
        line["cauchy"] = run_cauchy(args, dev, side)
        line["precision"] = run_precision(dev, side)
        line["precision"]["chunk_start"] = run_chunk_start_study(dev, side)
        line["other_configs"] = run_configs(dev, side)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if "batched" in line and BATCH_CHECK:
            line["batched"]["accuracy"] = batched_oracle_check()
        if CHUNK_STUDY:
            line["precision"]["chunk_start"].update(chunk_start_oracle_check())
        cores = os.cpu_count() or 1
        rate, tt, wall = cpu_oracle_rate(A, args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d Glynn terms of the same matrix (oracle in double, O(n^2) per term), "
                                          "%.1f s wall on %d threads" % (tt, wall, cores)}
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
