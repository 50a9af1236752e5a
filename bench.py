#!/usr/bin/env python3
"""Benchmark of the masked S-format product C = P_S(A A) (Eq. (product), Sec. 4.1).

Workload (default ``matern12_3d_1m``): N = 2^20 points uniform in [0,1]^3, Matern-1/2
kernel with lengthscale 0.1 scaled by 1/N, samplets with vanishing moments up to degree 3
(20 moments), leaf size 32, eta = 1.0, a-posteriori threshold 1e-8; C on A's own pattern.
Inputs are prepared before timing (cluster tree and pattern on the host, values on the
device) and stay resident in HBM.

One step = one masked product in the mixed arithmetic (float inputs, float products,
compensated float accumulation).  ``value`` is useful GFLOP/s (exact flop count of the
symbolic phase, no padding).  The same product in FP64 is run once for the comparison
and the relative Frobenius error of the mixed result against it is reported.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the plain-C FP64 oracle on the host cores on a bounded sample
of output blocks of the same workload.  Under torchrun every rank runs its own replica
(the product does not shard across GPUs here) and rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# the input builder's OpenMP threads sleep when idle instead of spinning (spinning host threads
# slowed the pinned host-to-device copies of the end-to-end measurement)
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "masked S-product GFLOP/s & HBM GB/s, N=2^20 d=3; mixed vs FP64 at 1e-6 rel err"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="matern12_3d_1m")
    ap.add_argument("--n", type=int, default=0, help="override N (smaller runs for checks)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", type=int, default=256, help="matrices of the batched workload")
    ap.add_argument("--batch-log2", default="10,16", help="batched workload: N log-uniform in [2^a, 2^b]")
    ap.add_argument("--precisions", default="fp64,fp64_df,mixed", help="drivers mode: arithmetic forms to run")
    ap.add_argument("--tau", type=float, default=None, help="override the workload's threshold")
    ap.add_argument("--variant", type=int, default=-1,
                    help="float kernel variant to time (default: the autotuner's choice)")
    ap.add_argument("--sizes", default=None,
                    help="paper_mult_2d/3d (default 5000,...,1000000) and selinv_2d (default its N): the N of the "
                         "sweep")
    ap.add_argument("--mus", default="1e-2,1e-4,1e-6", help="selinv workload: ridge parameters")
    ap.add_argument("--nodes", type=int, default=7, help="contour workload: quadrature nodes of Eq. (ContInt)")
    ap.add_argument("--product", choices=["fp32", "tf32x3", "bf16x3"], default="fp32",
                    help="arithmetic of the timed product: compensated float (default) or a split "
                         "tensor-core form")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
def workload_config(w, n, pat, triples, flops):
    nnz = pat.nnz
    return {
        "workload": w.name, "n": n, "d": w.d, "domain": w.domain, "kernel": "matern-%g" % w.nu, "ell": w.ell,
        "kernel_scale": "1/N", "nugget": w.nugget, "q": w.q, "leaf": w.leaf, "eta": w.eta, "tau": w.tau,
        "blocks": pat.nblocks, "nnz": nnz, "triples": triples, "flops_per_product": flops,
        "l2": "inputs larger than L2 (A is %.2f GB in float), no flush" % (nnz * 4 / 1e9),
        "product": "C = P_S(A A) on A's pattern",
    }


def build_input(w, n):
    import workloads as W
    from paper_2211_11681_gb300.builder import Builder
    x = W.points(w, n)
    t0 = time.time()
    b = Builder(x, w.leaf, w.q, w.eta)
    t1 = time.time()
    pat, vals = b.values(w.nu, w.ell, 1.0 / n, w.nugget, w.tau)
    t2 = time.time()
    return b, pat, vals, {"host_s": round(t1 - t0, 2), "values_s": round(t2 - t1, 2)}


def compression_error(b, pat, vals, w, n, seed=23):
    """||T K T^T y - K^eta y|| / ||T K T^T y|| for y = T x, x a seeded Gaussian vector: the
    uncompressed kernel matrix applied on the device (every entry evaluated), the samplet
    transform on the host, the compressed matrix by s_spmm."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import sformat as sf
    x = W.random_vector(n, seed)
    t0 = time.time()
    tkx = b.transform(b.kernel_matvec(w.nu, w.ell, 1.0 / n, w.nugget, x))
    tx = torch.from_numpy(b.transform(x)).cuda().reshape(1, n)
    ky = torch.empty_like(tx)
    sf.spmm(pat, vals, tx, ky)
    ref = torch.from_numpy(tkx).cuda()
    e = float((ref - ky[0]).norm() / ref.norm())
    return {"value": e, "seconds": round(time.time() - t0, 2),
            "how": "||T K x - K^eta T x|| / ||T K x||, x ~ N(0, I) (seed %d), K x with every entry evaluated" % seed}


def algorithmic_bytes(pat, width):
    # each operand read once, C written once, plus the pattern's index arrays
    bo, rp, ci = pat.arrays()
    idx = 8 * (len(bo) + len(rp)) + 4 * len(ci)
    return width * 3 * pat.nnz + 3 * idx


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [s.strip() for s in ln.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and f[0] != self.uuid and any(r[0] == self.uuid for r in rows):
                continue
            rows.append(f)
        mine = [r for r in rows if r[0] == self.uuid] or rows
        if not mine:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in mine if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in mine if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in mine for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(mine)}


def kernel_traffic(record="mul_f32_nt_traffic.json", source="mul_nt.cu"):
    """Per-launch DRAM bytes of the product kernel from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", record)
    src = os.path.join(ROOT, "paper_2211_11681_gb300", "csrc", source)
    try:
        with open(path) as f:
            rec = json.load(f)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("source_sha256") != sha:
            return None
        return rec.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def aggregate_ranks(ms, units, dist=None, device="cpu"):
    """Whole-job throughput of replicas: every rank did `units` of work in its own `ms`; the
    job time is the slowest rank's (max over ranks), the value is all ranks' units over it
    (GFLOP/s when units are flops).  Returns (max ms, value)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units * world / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------------------
def oracle_sample(pat, vals_host, cpu_seconds, seed=0):
    """Time the plain-C FP64 oracle on a bounded random sample of output blocks, using all
    host cores.  Returns (GFLOP/s, cores, description, seconds)."""
    from oracle import product as oprod
    from oracle.sformat import BlockCSR
    bo, rp, ci = pat.arrays()
    A = BlockCSR(np.diff(bo), rp, ci.astype(np.int64), vals_host)
    cores = len(os.sched_getaffinity(0))
    rng = np.random.Generator(np.random.PCG64(seed))
    order = rng.permutation(A.nblocks)
    # calibrate on a small sample, then size the sample for about cpu_seconds
    k = max(64, A.nblocks // 2000)
    sub = np.sort(order[:k])
    t0 = time.time()
    oprod.mul_masked(A, A, A, subset=sub, nthreads=cores)
    dt = max(time.time() - t0, 1e-3)
    k2 = int(min(A.nblocks, max(k, k * cpu_seconds / dt)))
    sub = np.sort(order[:k2])
    _, fl = oprod.mul_count(A, A, A, subset=sub)
    t0 = time.time()
    oprod.mul_masked(A, A, A, subset=sub, nthreads=cores)
    dt = time.time() - t0
    desc = "%d of %d output blocks (%.2f%%), uniform random (seed %d), %.3g useful flops" % (
        k2, A.nblocks, 100.0 * k2 / A.nblocks, seed, fl)
    return fl / dt / 1e9, cores, desc, dt


def run_reference(args, w, n, rank, world):
    import torch
    if rank != 0:
        return
    b, pat, vals, prep = build_input(w, n)
    vals_host = vals.cpu().numpy()
    del vals, b
    torch.cuda.empty_cache()
    times, cores, desc = [], 0, ""
    for i in range(args.warmup + args.steps):
        v, cores, desc, dt = oracle_sample(pat, vals_host, args.cpu_seconds / 2, seed=i)
        if i >= args.warmup:
            times.append(v)
    value = statistics.median(times)
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "d": w.d, "nnz": pat.nnz, "blocks": pat.nblocks},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def run_batch(args, rank, world):
    """256 independent matrices, N log-uniform in [2^10, 2^16], concatenated into one pattern:
    one graph-replayed persistent launch per batched step, against a loop of one launch per
    matrix (same kernel variant).  Metric: masked products per second.  The values of each
    matrix are built on the device and kept in float only, in slices of one buffer."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    lo, hi = (int(v) for v in args.batch_log2.split(","))
    ws = W.batch_workloads(count=args.batch, nmin_log2=lo, nmax_log2=hi)
    t0 = time.time()
    pats, parts = [], []
    t_host = t_dev = 0.0
    for w in ws:
        ta = time.time()
        b = Builder(W.points(w), w.leaf, w.q, w.eta)
        tb = time.time()
        p, v = b.values(w.nu, w.ell, 1.0 / w.n, w.nugget, 0.0)
        pats.append(p)
        parts.append(v.float())
        del b, v
        t_host += tb - ta
        t_dev += time.time() - tb
    P = sf.concat(pats)
    A = torch.empty(max(P.nnz, 1), dtype=torch.float32, device="cuda")
    offs = [0]
    for v in parts:
        A[offs[-1]:offs[-1] + v.numel()].copy_(v)
        offs.append(offs[-1] + v.numel())
    del parts
    torch.cuda.empty_cache()
    prep = time.time() - t0
    C = torch.empty_like(A)
    plan = sf.Plan(P, P, P, "fp32")
    plan.set_symmetric_a(True)                 # every part is a symmetric kernel matrix
    triples, flops = plan.stats()
    t1 = time.time()
    shape = plan.autotune(A, A, C)
    tune_s = time.time() - t1
    g = plan.graph(A, A, C)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        g.launch()
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            g.launch()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    variant = plan.variant_index
    del g, plan
    torch.cuda.empty_cache()
    # one launch per matrix, same variant, on slices of the same buffers
    plans = []
    for p in pats:
        q = sf.Plan(p, p, p, "fp32")
        q.set_symmetric_a(True)
        q.set_variant(variant)
        plans.append(q)
    views = [(A[offs[i]:offs[i + 1]], C[offs[i]:offs[i + 1]]) for i in range(len(pats))]
    for _ in range(args.warmup):
        for q, (a, c) in zip(plans, views):
            q.mul(a, a, c)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for q, (a, c) in zip(plans, views):
            q.mul(a, a, c)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1) / args.steps
    n = len(ws)
    line = {"metric": "batched masked S-products/s (%d matrices, N log-uniform 2^%d..2^%d)" % (n, lo, hi),
            "value": n / (ms * 1e-3), "unit": "products/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "matern32_2d_batch", "matrices": n, "n_total": int(sum(w.n for w in ws)),
                       "n_min": int(min(w.n for w in ws)), "n_max": int(max(w.n for w in ws)),
                       "nnz": P.nnz, "blocks": P.nblocks, "triples": triples, "flops_per_step": flops,
                       "prep_seconds": round(prep, 1), "host_builder_s": round(t_host, 1),
                       "device_values_s": round(t_dev, 1), "autotune_s": round(tune_s, 1),
                       "l2": "inputs larger than L2, no flush"},
            "gflops": flops / (ms * 1e-3) / 1e9, "autotuned_variant": shape, "variant_index": variant,
            "loop": {"ms_per_step": round(ms_loop, 3), "products_per_s": n / (ms_loop * 1e-3),
                     "launches_per_step": n},
            "batched_speedup_vs_loop": ms_loop / ms, "clocks": clk.summary(), "gpu_launches": args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_paper_mult(args, rank, world):
    """The multiplication benchmark of Sec. 5.1: K (.) K~ with K the compressed exponential
    kernel exp(-r)/N (q+1 = 4 vanishing moments, eta = 1.25, tau = 1e-5/N) on uniform points
    in [0,1]^d and K~ = K (1 + 0.1 u); the formatted product on K's a-posteriori pattern in
    FP64 and in compensated float, timed, and its error e_F(K K~ - K (.) K~) = ||(..) X||_F /
    ||X||_F with X in R^{N x 10} uniform.  One JSON line per N, then a summary line."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    w = W.WORKLOADS[args.workload]
    sizes = args.sizes or ",".join(str(v) for v in W.PAPER_MULT_NS)
    ns = [args.n] if args.n else [int(v) for v in sizes.split(",")]
    stream = torch.cuda.current_stream()
    rows = []

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for n in ns:
        t0 = time.time()
        x = W.points(w, n)
        b = Builder(x, w.leaf, w.q, w.eta)
        pat, K = b.values(w.nu, w.ell, 1.0 / n, w.nugget, W.tau_of(w, n))
        apriori = b.nnz_apriori
        del b
        prep = time.time() - t0
        g = torch.Generator(device="cuda")
        g.manual_seed(w.seed + 100)
        Kt = K * (1.0 + 0.1 * torch.rand(K.numel(), dtype=torch.float64, device="cuda", generator=g))
        g.manual_seed(99)
        X = torch.rand((10, n), dtype=torch.float64, device="cuda", generator=g)
        p64 = sf.Plan(pat, pat, pat, "fp64")
        triples, flops = p64.stats()
        C64 = torch.empty_like(K)
        ms64 = timed(lambda: p64.mul(K, Kt, C64), 1 if flops > 2e12 else 3)
        T1, T2, T3 = (torch.empty_like(X) for _ in range(3))
        sf.spmm(pat, Kt, X, T1)
        sf.spmm(pat, K, T1, T2)                      # K (K~ X): the exact product applied to X
        sf.spmm(pat, C64, X, T3)
        xn = float(X.norm())
        ef64 = float((T2 - T3).norm()) / xn
        del p64
        K32, Kt32 = K.float(), Kt.float()
        C32 = torch.empty_like(K32)
        p32 = sf.Plan(pat, pat, pat, "fp32")
        shape = p32.autotune(K32, Kt32, C32)
        ms32 = timed(lambda: p32.mul(K32, Kt32, C32), 3)
        C32d = C32.double()
        sf.spmm(pat, C32d, X, T3)
        ef32 = float((T2 - T3).norm()) / xn
        rel32 = float((C32d - C64).norm() / C64.norm())
        row = {"n": n, "d": w.d, "apriori_nnz": apriori, "nnz": pat.nnz, "blocks": pat.nblocks, "triples": triples,
               "flops": flops, "prep_s": round(prep, 2),
               "fp64": {"ms": round(ms64, 3), "tflops": flops / ms64 / 1e9, "e_F": ef64},
               "f32": {"ms": round(ms32, 3), "tflops": flops / ms32 / 1e9, "e_F": ef32, "rel_frob_vs_fp64": rel32,
                       "shape": shape},
               "norm_KKtX": float(T2.norm()) / xn}
        rows.append(row)
        if rank == 0:
            print(json.dumps({"paper_mult_point": row}), flush=True)
        del K, Kt, K32, Kt32, C32, C32d, C64, X, T1, T2, T3, p32, pat
        torch.cuda.empty_cache()
    line = {"metric": "formatted product K (.) K~ on the a-posteriori pattern (Sec. 5.1): ms, TFLOP/s, e_F",
            "value": rows[-1]["f32"]["ms"], "unit": "ms per product (float, largest N)", "higher_is_better": False,
            "n_gpus": world, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "kernel": "exp(-r)/N (Matern-1/2, ell=1)", "q": w.q,
                       "eta": w.eta, "tau": "1e-5/N", "leaf": w.leaf, "perturbation": "K~ = K (1 + 0.1 u), u ~ U[0,1]",
                       "estimator": "e_F(M) = ||M X||_F/||X||_F, X in R^{N x 10} uniform [0,1]"},
            "points": rows,
            "paper_context": "Sec. 5.1 plots e_F between 1e-8 and 2e-6 for N = 5e3..1e6 (point values not in the source)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_selinv(args, rank, world):
    """Selected inversion on the compression pattern (Sec. 4.2, Eq. (blockInv); the inversion
    experiment of Sec. 5.2): (K + mu I)^{-1} on the a-posteriori pattern of K, the compressed
    exponential kernel exp(-r)/N (q+1 = 4 vanishing moments, eta = 1.25, tau = 1e-5/N) on
    uniform points in [0,1]^2, for ridge parameters mu = 1e-2, 1e-4, 1e-6.  Timed: one block
    LDL^T factorization and one selected inversion (FP64, CUDA events), and the paper's error
    e_F(Z (K + mu I) - I) with X in R^{N x 10} uniform.  One JSON line per N, then a summary."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import selinv as si
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    w = W.WORKLOADS[args.workload]
    ns = [args.n] if args.n else ([int(v) for v in args.sizes.split(",")] if args.sizes else [w.n])
    mus = [float(v) for v in args.mus.split(",")]
    stream = torch.cuda.current_stream()
    peak64 = sf.peak_fma("fp64")
    rows = []
    for n in ns:
        x = W.points(w, n)
        b = Builder(x, w.leaf, w.q, w.eta)
        pat, K = b.values(w.nu, w.ell, 1.0 / n, 0.0, W.tau_of(w, n))
        del b
        t0 = time.time()
        inv = si.SelInv(pat)
        sym_s = time.time() - t0
        st = inv.stats()
        flops = st["flops_factor"] + st["flops_invert"]
        g = torch.Generator(device="cuda")
        g.manual_seed(99)
        X = torch.rand((10, n), dtype=torch.float64, device="cuda", generator=g)
        T1, T2 = torch.empty_like(X), torch.empty_like(X)
        Z = torch.empty_like(K)
        pts = []
        for mu in mus:
            inv.factor(K, mu)
            inv.invert(Z)
            inv.status()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            reps = max(1, args.steps)
            fac = ivt = 0.0
            for _ in range(reps):
                e[0].record(stream)
                inv.factor(K, mu)
                e[1].record(stream)
                inv.invert(Z)
                e[2].record(stream)
                torch.cuda.synchronize()
                fac += e[0].elapsed_time(e[1])
                ivt += e[1].elapsed_time(e[2])
            inv.status()
            fac, ivt = fac / reps, ivt / reps
            sf.spmm(pat, K, X, T1)
            T1 += mu * X                                  # (K + mu I) X
            sf.spmm(pat, Z, T1, T2)                       # Z (K + mu I) X
            ef = float((T2 - X).norm() / X.norm())
            pts.append({"mu": mu, "factor_ms": round(fac, 3), "invert_ms": round(ivt, 3),
                        "gflops": flops / ((fac + ivt) * 1e6), "frac_fp64_peak": flops / ((fac + ivt) * 1e-3) / peak64,
                        "e_F": ef})
        row = {"n": n, "nnz": pat.nnz, "blocks": pat.nblocks, "l_blocks": st["l_blocks"],
               "l_entries": st["l_entries"], "levels": st["levels"], "flops_factor": st["flops_factor"],
               "flops_invert": st["flops_invert"], "symbolic_s": round(sym_s, 3), "points": pts}
        rows.append(row)
        if rank == 0:
            print(json.dumps({"selinv_point": row}), flush=True)
        del inv, K, Z, X, T1, T2, pat
        torch.cuda.empty_cache()
    last = rows[-1]
    best = min(last["points"], key=lambda p: p["factor_ms"] + p["invert_ms"])
    line = {"metric": "selected inversion (K + mu I)^{-1} on the a-posteriori pattern (Sec. 4.2, 5.2): ms per "
                      "factorization + inversion",
            "value": round(best["factor_ms"] + best["invert_ms"], 3), "unit": "ms (FP64, largest N)",
            "higher_is_better": False, "n_gpus": world, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "kernel": "exp(-r)/N (Matern-1/2, ell=1)", "q": w.q,
                       "eta": w.eta, "tau": "1e-5/N", "leaf": w.leaf, "mu": mus,
                       "estimator": "e_F(Z (K + mu I) - I), X in R^{N x 10} uniform [0,1]"},
            "roofline": {"bound": "fp64", "achieved": best["gflops"] / 1e3, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                         "frac": best["frac_fp64_peak"],
                         "peak_source": "s_peak_fma FP64 (FMA chains on every lane), measured in this run"},
            "points": rows,
            "paper_context": "Sec. 5.2 (Pardiso, 16 Xeon cores): e_F falls with growing mu; times plotted, "
                             "point values not in the source"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_contour(args, rank, world):
    """Eq. (ContInt), the matrix-function experiment of Sec. 5.3: A = K + mu I with K the
    compressed exp(-2r)/N kernel matrix (q+1 = 4, eta = 1.25, tau = 1e-5/N) on points of a
    closed surface (the unit sphere standing in for the 3D scan), mu = 1e-4, c_lo = mu,
    c_hi = 1, n = 7 nodes: A^{-1/2} on S by seven shifted selected inversions, A^{1/2} =
    P_S(A A^{-1/2}) by the masked product, and e_F(A^{1/2} A^{1/2} - A); the Newton-Schulz
    square root on the same S beside it."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import selinv as si
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    w = W.WORKLOADS[args.workload]
    n = args.n or w.n
    mu, nodes = w.nugget, args.nodes
    stream = torch.cuda.current_stream()
    x = W.points(w, n)
    b = Builder(x, w.leaf, w.q, w.eta)
    pat, A = b.values(w.nu, w.ell, 1.0 / n, mu, W.tau_of(w, n))
    del b
    t0 = time.time()
    inv = si.SelInv(pat)
    sym_s = time.time() - t0
    st = inv.stats()
    Zi = torch.empty_like(A)
    inv.invsqrt(A, mu, 1.0, nodes, Zi)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    p64 = sf.Plan(pat, pat, pat, "fp64")
    R = torch.empty_like(A)
    e0.record(stream)
    inv.invsqrt(A, mu, 1.0, nodes, Zi)
    e1.record(stream)
    p64.mul(A, Zi, R)
    e2.record(stream)
    torch.cuda.synchronize()
    ms_inv, ms_mul = e0.elapsed_time(e1), e1.elapsed_time(e2)
    g = torch.Generator(device="cuda")
    g.manual_seed(99)
    X = torch.rand((10, n), dtype=torch.float64, device="cuda", generator=g)
    T1, T2, T3 = (torch.empty_like(X) for _ in range(3))
    sf.spmm(pat, R, X, T1)
    sf.spmm(pat, R, T1, T2)
    sf.spmm(pat, A, X, T3)
    ef = float((T2 - T3).norm() / X.norm())
    F = torch.empty_like(A)
    t1 = time.time()
    sf.funm(pat, "sqrt", A, F, steps=25)
    torch.cuda.synchronize()
    ns_s = time.time() - t1
    sf.spmm(pat, F, X, T1)
    sf.spmm(pat, F, T1, T2)
    ef_ns = float((T2 - T3).norm() / X.norm())
    flops = nodes * (st["flops_factor"] + st["flops_invert"])
    peak64 = sf.peak_fma("fp64")
    line = {"metric": "A^{1/2} by the contour integral Eq. (ContInt) with selected inversion: ms",
            "value": round(ms_inv + ms_mul, 3), "unit": "ms (FP64)", "higher_is_better": False, "n_gpus": world,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "kernel": "exp(-2r)/N (Matern-1/2, ell=0.5)", "q": w.q,
                       "eta": w.eta, "tau": "1e-5/N", "mu": mu, "c_lo": mu, "c_hi": 1.0, "nodes": nodes,
                       "points": "unit sphere (stand-in for the 3D scan)"},
            "invsqrt_ms": round(ms_inv, 3), "sqrt_product_ms": round(ms_mul, 3),
            "selinv": {"nnz": pat.nnz, "l_blocks": st["l_blocks"], "l_entries": st["l_entries"],
                       "levels": st["levels"], "symbolic_s": round(sym_s, 3)},
            "roofline": {"bound": "fp64", "achieved": flops / (ms_inv * 1e-3) / 1e12, "peak": peak64 / 1e12,
                         "unit": "TFLOP/s", "frac": flops / (ms_inv * 1e-3) / peak64,
                         "peak_source": "s_peak_fma FP64, measured in this run"},
            "e_F_sqrt_sqrt_minus_A": ef, "newton_schulz": {"steps": 25, "wall_s": round(ns_s, 3), "e_F": ef_ns},
            "rel_frob_contour_vs_ns": float((R - F).norm() / F.norm()),
            "paper_context": "Table (Sec. 5.3), 3D scan, K = 7: e_F 1.43e-3 (N = 5000) .. 2.82e-4 (N = 100000)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_grad(args, rank, world):
    """Differentiation through k Newton-Schulz steps (uniform [0,1]^3, Matern-3/2, ell = 0.15,
    q = 2, eta = 1.25): L(ell) = z^T P_S(A(ell)^{1/2}) z with z = T g, g ~ N(0, I), the
    mixed-precision iteration (float, float checkpoints) differentiated in float
    (s_funm_sqrt_backward_prec) under torch.autograd, then dL/dell = <dL/dA, dA/dell> with
    dA/dell = P_S(T dK/dell T^T) from the builder.  Reports the time and device memory of the
    forward and reverse passes, and the same in double when --precisions holds fp64."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.autograd import QuadForm, SqrtmNS
    from paper_2211_11681_gb300.builder import Builder
    w = W.WORKLOADS["matern32_3d_grad"]
    n = args.n or w.n
    steps = 10
    tau = args.tau if args.tau is not None else w.tau
    t0 = time.time()
    x = W.points(w, n)
    b = Builder(x, w.leaf, w.q, w.eta)
    pat, A = b.values(w.nu, w.ell, 1.0 / n, w.nugget, tau)
    dAdl = b.values_dell(pat, w.nu, w.ell, 1.0 / n)
    z = torch.from_numpy(b.transform(W.random_vector(n, 17))).cuda()
    apriori = b.nnz_apriori
    del b
    prep = time.time() - t0
    lam = sf.norm_est(pat, A, 50)
    c = 1.01 * lam
    free0, total = torch.cuda.mem_get_info()
    out = {}
    for prec in [p_ for p_ in args.precisions.split(",") if p_ in ("fp32", "fp64")]:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        ck_bytes = 2 * steps * pat.nnz * (4 if prec == "fp32" else 8)
        free, _ = torch.cuda.mem_get_info()
        if ck_bytes + 8 * pat.nnz * 8 > free:     # checkpoints + about eight work matrices
            out[prec] = {"skipped": "the %.0f GB of checkpoints and work buffers exceed the %.0f GB of free device "
                                    "memory" % ((ck_bytes + 64 * pat.nnz) / 1e9, free / 1e9),
                         "checkpoint_gb": round(ck_bytes / 1e9, 2)}
            continue
        Ar = A.clone().requires_grad_(True)
        t1 = time.time()
        X = SqrtmNS.apply(Ar, pat, steps, c, prec)
        L = QuadForm.apply(X, pat, z)
        torch.cuda.synchronize()
        t2 = time.time()
        free1, _ = torch.cuda.mem_get_info()
        L.backward()
        torch.cuda.synchronize()
        t3 = time.time()
        dl = float(torch.dot(Ar.grad, dAdl))
        out[prec] = {"loss": float(L.detach()), "dloss_dell": dl, "forward_s": round(t2 - t1, 3),
                     "backward_s": round(t3 - t2, 3),
                     "device_gb_in_use_after_forward": round((total - free1) / 1e9, 2),
                     "checkpoint_gb": round(2 * steps * pat.nnz * (4 if prec == "fp32" else 8) / 1e9, 2)}
        del Ar, X, L
        torch.cuda.empty_cache()
    if "dloss_dell" in out.get("fp32", {}) and "dloss_dell" in out.get("fp64", {}):
        out["fp32"]["dloss_dell_rel_vs_fp64"] = abs(out["fp32"]["dloss_dell"] / out["fp64"]["dloss_dell"] - 1)
    line = {"metric": "d/dell of z^T P_S(A(ell)^{1/2}) z through %d Newton-Schulz steps" % steps,
            "value": out.get("fp32", {}).get("backward_s"), "unit": "s per reverse pass (mixed)",
            "higher_is_better": False, "n_gpus": world, "dtype": "f32 (+f64 comparison)", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "d": w.d, "kernel": "matern-1.5", "ell": w.ell, "q": w.q,
                       "eta": w.eta, "tau": tau, "apriori_nnz": apriori, "nnz": pat.nnz, "blocks": pat.nblocks,
                       "lambda_max": lam, "c": c, "prep_seconds": round(prep, 1),
                       "device_gb_in_use_before": round((total - free0) / 1e9, 2)},
            "grad": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_drivers(args, rank, world):
    """Matrix functions at full size (N = 2^18 points on the sphere, Matern-5/2, ell = 0.3,
    nugget 1e-2, q = 2, eta = 1.25): A^{1/2} by 25 Newton-Schulz steps and exp(-A) by
    Taylor-8 with scaling and squaring, in double, double-float and mixed precision (float
    iterations with double residual correction / double squarings)."""
    import torch
    import workloads as W
    from paper_2211_11681_gb300 import sformat as sf
    w = W.WORKLOADS["matern52_sphere"]
    n = args.n or w.n
    b, pat, vals, prep = build_input(w, n)
    plan = sf.Plan(pat, pat, pat, "fp64")
    triples, flops = plan.stats()
    lam = sf.norm_est(pat, vals, 50)
    c = 1.01 * lam
    out = {}
    F = {}
    want = set(args.precisions.split(","))
    forms = [f for f in (("fp64", "fp64", 0), ("fp64_df", "fp64_df", 0), ("mixed", "fp32", 2)) if f[0] in want]
    for name, prec, refine in forms:
        Fx = torch.empty_like(vals)
        torch.cuda.synchronize()
        t0 = time.time()
        res = sf.funm(pat, "sqrt", vals, Fx, steps=25, prec=prec, scale=c, refine=refine, residual=True)
        torch.cuda.synchronize()
        out["sqrt_" + name] = {"s": round(time.time() - t0, 3), "residual": res,
                               "products": 75 + 2 * refine}
        F[name] = Fx
    for name in ("fp64_df", "mixed"):
        if name in F and "fp64" in F:
            out["sqrt_" + name]["rel_frob_vs_fp64"] = float((F[name] - F["fp64"]).norm() / F["fp64"].norm())
            out["sqrt_" + name]["speedup_vs_fp64"] = out["sqrt_fp64"]["s"] / out["sqrt_" + name]["s"]
    del F
    E = {}
    for name, prec in [(f[0], f[1]) for f in forms]:
        Ex = torch.empty_like(vals)
        torch.cuda.synchronize()
        t0 = time.time()
        sf.funm(pat, "exp_neg", vals, Ex, prec=prec, scale=lam)
        torch.cuda.synchronize()
        out["expneg_" + name] = {"s": round(time.time() - t0, 3)}
        E[name] = Ex
    for name in ("fp64_df", "mixed"):
        if name in E and "fp64" in E:
            out["expneg_" + name]["rel_frob_vs_fp64"] = float((E[name] - E["fp64"]).norm() / E["fp64"].norm())
            out["expneg_" + name]["speedup_vs_fp64"] = out["expneg_fp64"]["s"] / out["expneg_" + name]["s"]
    line = {"metric": "A^{1/2} (25 Newton-Schulz steps) and exp(-A) on S, N=%d sphere" % n,
            "value": out.get("sqrt_mixed", {}).get("s"), "unit": "s per A^{1/2} (mixed)", "higher_is_better": False,
            "n_gpus": world, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config(w, n, pat, triples, flops), lambda_max=lam, prep_seconds=prep),
            "drivers": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    import torch
    import workloads as W
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "matern52_sphere":
        run_drivers(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload == "matern32_3d_grad":
        run_grad(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload.startswith("paper_mult"):
        run_paper_mult(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload.startswith("selinv") or args.workload.startswith("contour"):
        (run_selinv if args.workload.startswith("selinv") else run_contour)(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload == "matern32_2d_batch":
        run_batch(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    w = W.WORKLOADS[args.workload]
    n = args.n or w.n
    if args.impl == "reference":
        run_reference(args, w, n, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    from paper_2211_11681_gb300 import sformat as sf
    bld, pat, vals, prep = build_input(w, n)
    t0 = time.time()
    plan32 = sf.Plan(pat, pat, pat, args.product)
    plan32.set_symmetric_a(True)      # A = T K T^T (+ mu I) is symmetric
    triples, flops = plan32.stats()
    prep["plan_s"] = round(time.time() - t0, 2)
    A32 = vals.float()
    C32 = torch.empty_like(A32)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    if args.variant >= 0 and args.product == "fp32":
        plan32.set_variant(args.variant)         # fixed shape (profiling runs)
        shape = plan32.variant()
    else:
        shape = plan32.autotune(A32, A32, C32)  # kernel shape for this pattern
    prep["autotune_s"] = round(time.time() - t0, 2)
    for _ in range(args.warmup):
        plan32.mul(A32, A32, C32)
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for e0, e1 in evs:
            e0.record(stream)
            plan32.mul(A32, A32, C32)          # one launch of the product kernel
            e1.record(stream)
        stop.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = start.elapsed_time(stop)
    launch_ms = [a.elapsed_time(c) for a, c in evs]
    ms = total_ms / args.steps
    ms, value = aggregate_ranks(ms, flops, dist, "cuda")
    clocks = clk.summary()

    # FP64 product once, and the error of the mixed result against it
    fp64 = None
    if not args.no_fp64:
        plan64 = sf.Plan(pat, pat, pat, "fp64")
        C64 = torch.empty_like(vals)
        plan64.mul(vals, vals, C64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            plan64.mul(vals, vals, C64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / 3
        err = float((C32.double() - C64).norm() / C64.norm())
        fp64 = {"ms": round(ms64, 3), "gflops": flops / (ms64 * 1e-3) / 1e9,
                "mixed_rel_frob_err_vs_fp64": err, "mixed_speedup_vs_fp64": ms64 / ms}
        # double-float (float-pair) product: double-accurate, on the float pipes
        plandf = sf.Plan(pat, pat, pat, "fp64_df")
        Cdf = torch.empty_like(vals)
        plandf.mul(vals, vals, Cdf)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            plandf.mul(vals, vals, Cdf)
        e1.record(stream)
        torch.cuda.synchronize()
        msdf = e0.elapsed_time(e1) / 3
        fp64["fp64_df"] = {"ms": round(msdf, 3), "gflops": flops / (msdf * 1e-3) / 1e9,
                           "rel_frob_err_vs_fp64": float((Cdf - C64).norm() / C64.norm()),
                           "speedup_vs_fp64": ms64 / msdf}
        del Cdf, plandf
        # split-bfloat16 (mma.sync) and split-TF32 (tcgen05) tensor-core products, float in and out
        Cbf = torch.empty_like(A32)
        for name in ("bf16x3", "tf32x3"):
            planbf = sf.Plan(pat, pat, pat, name)
            planbf.set_symmetric_a(True)
            planbf.mul(A32, A32, Cbf)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                planbf.mul(A32, A32, Cbf)
            e1.record(stream)
            torch.cuda.synchronize()
            msbf = e0.elapsed_time(e1) / 3
            fp64[name] = {"ms": round(msbf, 3), "gflops": flops / (msbf * 1e-3) / 1e9,
                          "rel_frob_err_vs_fp64": float((Cbf.double() - C64).norm() / C64.norm()),
                          "speedup_vs_fp64": ms64 / msbf}
            del planbf
            torch.cuda.empty_cache()
        del C64, plan64, Cbf
        torch.cuda.empty_cache()

    # compression error of the input (needs the builder), then release the builder: while its
    # host state was alive the pinned host-to-device copies ran at a fraction of their rate
    comp_err = compression_error(bld, pat, vals, w, n) if not args.no_fp64 else None
    del bld
    import gc
    gc.collect()

    # end to end through the C ABI with host buffers (pinned): every step copies its input A
    # host -> device and its result C device -> host inside the timed region; two device
    # buffers and separate copy / compute streams let step i+1's upload and step i-1's
    # download overlap step i's product
    Ah = torch.empty(A32.numel(), dtype=torch.float32, pin_memory=True)
    Ah.copy_(A32)
    Ch = [torch.empty(A32.numel(), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    Ad = [torch.empty_like(A32) for _ in range(2)]
    Cd = [C32, torch.empty_like(A32)]
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    e2e_steps = max(2, args.steps)

    def pipeline(steps):
        """`steps` end-to-end steps; returns the milliseconds from the first upload to the last
        download."""
        ev = lambda: torch.cuda.Event(enable_timing=True)
        up = [ev() for _ in range(steps)]
        done = [ev() for _ in range(steps)]
        down = [ev() for _ in range(steps)]
        h2d0 = [ev() for _ in range(steps)]
        d2h0 = [ev() for _ in range(steps)]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_h2d.wait_event(e0)
        for i in range(steps):
            b = i % 2
            with torch.cuda.stream(s_h2d):
                if i >= 2:
                    s_h2d.wait_event(done[i - 2])        # buffer b no longer read by step i-2
                h2d0[i].record(s_h2d)
                Ad[b].copy_(Ah, non_blocking=True)
                up[i].record(s_h2d)
            stream.wait_event(up[i])
            if i >= 2:
                stream.wait_event(down[i - 2])           # C buffer b downloaded
            plan32.mul(Ad[b], Ad[b], Cd[b], stream=stream)
            done[i].record(stream)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(done[i])
                d2h0[i].record(s_d2h)
                Ch[b].copy_(Cd[b], non_blocking=True)
                down[i].record(s_d2h)
        stream.wait_event(down[steps - 1])
        e1.record(stream)
        torch.cuda.synchronize()
        copy_ms[0] = statistics.median(h2d0[i].elapsed_time(up[i]) for i in range(steps))
        copy_ms[1] = statistics.median(d2h0[i].elapsed_time(down[i]) for i in range(steps))
        return e0.elapsed_time(e1)

    copy_ms = [0.0, 0.0]

    # warm-up steps: the first DMA through freshly pinned host pages runs at a small fraction of
    # the warm rate (measured 10 GB/s cold against 211 GB/s warm), a one-time cost of the buffers
    pipeline(max(2, args.warmup))
    e2e_ms = pipeline(e2e_steps) / e2e_steps
    e2e = {"value": flops * world / (e2e_ms * 1e-3) / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": int(Ah.numel() * 4), "d2h_bytes_per_step": int(Ch[0].numel() * 4),
           "ms_per_step": round(e2e_ms, 3), "steps": e2e_steps,
           "pipelined": "two buffers; uploads and downloads on their own streams overlap neighbouring products",
           "warmup_steps": max(2, args.warmup),
           "copy_ms_median": {"h2d": round(copy_ms[0], 2), "d2h": round(copy_ms[1], 2)}}
    del Ah, Ch, Ad, Cd

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    achieved = flops / (statistics.mean(launch_ms) * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probe = {"fp32_tflops": sf.peak_fma("fp32") / 1e12, "fp64_tflops": sf.peak_fma("fp64") / 1e12,
             "how": "s_peak_fma: independent FMA chains on every lane, CUDA events"}
    if args.product == "fp32":
        fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12      # TFLOP/s from unit counts and clock
        nt = tuple(shape["micro"]) == (0, 0)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": kernel_traffic() if nt else kernel_traffic("mul_f32_traffic.json", "mul.cu"),
                "kernel": "sf::mul_f32_nt_kernel (K-major operands, one bulk copy per lambda block, "
                          "split-K half-warps)" if nt else
                          "sf::mul_f32_kernel<tile %d, micro %dx%d, transposed A>" % (shape["tile"], *shape["micro"]),
                "peak_source": "%d SMs (device attribute) x 128 FP32 lanes x 2 flop x %g MHz sm_max (derived)"
                               % (sms, sm_max),
                "frac_of_probe": achieved / probe["fp32_tflops"], "probe": probe}
        launches = 1
    else:
        # tensor-core forms: useful flops against the dense peak of the operand type (bf16
        # measured; TF32 as the measured bf16 burst times the nominal TF32 / bf16 ratio 1.1 / 2.25)
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        tpeak = bf16 * (1.1 / 2.25) if args.product == "tf32x3" else bf16
        roof = {"bound": "tensor", "achieved": achieved, "peak": tpeak, "unit": "TFLOP/s",
                "frac": achieved / tpeak, "traffic": None,
                "kernel": "mul_tf32x3_kernel (tcgen05.mma kind::tf32, three products per term)"
                if args.product == "tf32x3" else "mul_bf16x3_kernel (mma.sync bf16, six products per term)",
                "peak_source": ("measured bf16 burst x 1.1/2.25 (nominal TF32/bf16), of measured"
                                if args.product == "tf32x3" else "measured bf16 burst, of measured")}
        launches = 2                                          # operand split + product
    dtype = {"fp32": "f32", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[args.product]
    qbytes = algorithmic_bytes(pat, 4)
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": dict(workload_config(w, n, pat, triples, flops), parallelism="replicas" if world > 1 else "1 GPU",
                       arithmetic=args.product, prep_seconds=prep, compression_error_estimate=comp_err),
        "hbm_gbs_algorithmic": qbytes / (ms * 1e-3) / 1e9,
        "fp64": fp64,
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": args.steps * launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, desc, dt = oracle_sample(pat, vals.cpu().numpy(), args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": desc,
                                "seconds": round(dt, 2)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
