"""Benchmark: refinement sweeps per second on the dense n = 16384, k = 128
workload (A = Q diag(lambda) Q^T, Q a product of 64 seeded Householder
reflectors, the 128 largest-|lambda| eigenvalues separated by 1e-3 ||A||),
through the eigref C ABI.

One step = one full sweep of Algorithm 4 (product, Gram products, k x k stage,
update, normalisation, stopping test).  Timed on the device with CUDA events
around exactly --steps sweeps after --warmup untimed sweeps.  A (2.1 GB) is
larger than L2, so no flush is needed between sweeps.

  python bench.py [--steps K] [--warmup W] [--precision bf16|fp64]
  python bench.py --impl reference      # the CPU oracle, same workload
  torchrun --nproc-per-node N bench.py --gpus N   # N independent replicas

Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "refine-steps/s & % roofline at 1e-13 angle: split-precision TC vs plain FP64"
UNIT = "refine-steps/s"
WORKLOAD = ("dense symmetric n=16384, k=128: A = Q diag(lambda) Q^T, Q = 64 seeded Householder "
            "reflectors, 128 largest |lambda| = 1 - 1e-3 i (random signs), graded tail 0.8*10^(-6u); "
            "X0 = orth(fp32(q) + N(0,1e-7))")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 pipe: 2 DFMA a clock and SM, the nominal 1.25 TFLOP/s over 152 SMs at
# the 2070 MHz maximum clock (1.25e12 / (152 x 2.07e9 x 2) = 1.99)
SMS, DFMA_PER_CLK, SM_MAX_MHZ = 152, 2, 2070.0


def fp64_peak(clocks):
    """FP64 arithmetic peak (TFLOP/s) from the unit count and the SM clock
    sampled during the timed region (the maximum clock when unsampled)."""
    mhz = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
    return SMS * DFMA_PER_CLK * 2 * mhz * 1e6 / 1e12


FP64_NOTE = "FP64 pipe: 152 SMs x 2 DFMA/clk x sampled SM clock (nominal 1.25 TFLOP/s at 2070 MHz)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def source_hash(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(kernel_file, precision):
    """DRAM bytes per launch of the product kernel from the committed ncu
    summary, or None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except OSError:
        return None
    ent = tab.get(precision)
    if not ent:
        return None
    if ent.get("source_sha256_16") != source_hash(os.path.join(ROOT, "paper_2602_23778_gb300", "csrc", kernel_file)):
        return None
    return ent.get("dram_bytes_per_launch")


def summarize_launches(path):
    """Per-kernel launches, total time and share from an ncu launch list
    (``--metrics gpu__time_duration.sum --csv``)."""
    import collections
    import csv
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3,
             "s": 1e6, "second": 1e6}
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, mi, vi, ui = (h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"),
                      h.index("Metric Unit"))
    agg = collections.OrderedDict()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki].split("(")[0].split("<")[0].replace("void ", "").replace("eigref::", "")
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += float(r[vi].replace(",", "")) * scale[r[ui]]
    tot = sum(v[1] for v in agg.values())
    lines = ["%-34s %8s %12s %8s" % ("kernel", "launches", "total_us", "share")]
    for name, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        lines.append("%-34s %8d %12.1f %7.2f%%" % (name[:34], c, t, 100 * t / tot))
    lines.append("%-34s %8d %12.1f" % ("TOTAL", sum(v[0] for v in agg.values()), tot))
    return "\n".join(lines)


def library_peaks():
    """Library (cuBLAS through torch) rates on this GPU for the dtypes the
    roofline needs: FP64 and INT8 are not in the measured-peaks file."""
    import torch

    def best(fn, iters):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(iters):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return min(ts)
    n = 8192
    out = {}
    a = torch.randn(n, n, device="cuda", dtype=torch.float64)
    b = torch.randn(n, n, device="cuda", dtype=torch.float64)
    out["fp64_gemm_tflops"] = 2 * n ** 3 / best(lambda: a @ b, 5) / 1e9
    del a, b
    a = torch.randint(-127, 127, (n, n), device="cuda", dtype=torch.int8)
    b = torch.randint(-127, 127, (n, n), device="cuda", dtype=torch.int8)
    out["int8_gemm_tops"] = 2 * n ** 3 / best(lambda: torch._int_mm(a, b.t()), 10) / 1e9
    del a, b
    a = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    b = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    out["bf16_gemm_tflops"] = 2 * n ** 3 / best(lambda: a @ b, 10) / 1e9
    out["gpu"] = torch.cuda.get_device_name(0)
    out["torch"] = torch.__version__
    return out


def workload(seed=3000, n=16384, k=128):
    from workloads import configs as C
    return C.config3(seed=seed, n=n, k=k)


def max_angle(X, Q):
    """max_j sin angle(x_j, q_j) in FP64 (absolute error ~1e-16)."""
    Xn = X / np.linalg.norm(X, axis=0)
    Qn = Q / np.linalg.norm(Q, axis=0)
    c = np.sum(Xn * Qn, axis=0)
    return float(np.max(np.linalg.norm(Xn - Qn * c[None, :], axis=0)))


def shard_indices(count, rank, world):
    """Problems of a batch that rank `rank` of `world` refines: r, r + N, ...
    (independent problems, no exchange between ranks)."""
    return list(range(rank, count, world))


def max_over_ranks(value, device):
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def orth_max(X, rows=32):
    """max |X^T X - I| with the row sum split into blocks of `rows` and the
    block Gram matrices added by Neumaier's compensated summation: the
    rounding of the measure is at most about rows * u (a plain FP64 X^T X over
    n = 16384 rows carries up to n * u, far above the 1e-14 being checked)."""
    n, k = X.shape
    S = np.zeros((k, k))
    C = np.zeros((k, k))
    for r0 in range(0, n, rows):
        B = X[r0:r0 + rows]
        G = B.T @ B
        t = S + G
        C += np.where(np.abs(S) >= np.abs(G), (S - t) + G, (G - t) + S)
        S = t
    return float(np.abs((S + C) - np.eye(k)).max())


def cpu_oracle_rate(p, sweeps):
    """The CPU oracle (as it stands) on this host: sweeps/s over a bounded sample."""
    from oracle import refine as R
    op = R.dense_operator(p.A)
    X = np.asfortranarray(p.X0)
    t0, c0 = time.perf_counter(), time.process_time()
    R.refine(op, X, p.normA, 0.0, max_iters=sweeps)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return sweeps / wall, max(1, round(cpu / wall)), wall


def dense_config(n, k, world):
    """The dense workload as both arms name it (the workload only; how it is
    computed goes under "method")."""
    return {"workload": WORKLOAD, "n": n, "k": k, "seed": 3000,
            "l2": "inputs larger than L2 (A is 2.1 GB); no flush",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, rank):
    if rank != 0:
        return
    p = workload(n=args.n, k=args.k)
    rate_w, _, _ = cpu_oracle_rate(p, args.warmup) if args.warmup > 0 else (0, 0, 0)
    rate, cores, wall = cpu_oracle_rate(p, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dense_config(p.n, p.k, args.gpus),
            "method": {"form": "CPU oracle, paper-literal Algorithm 4 (FP64)"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d oracle sweeps of the full n=16384, k=128 workload (%.1f s)" % (args.steps, wall)},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


LAPLACE = ("sparse CSR 5-point Dirichlet Laplacian on a 1024 x 1000 grid (n=1,024,000, nnz=5,115,952), "
           "a_x=1, a_y=sqrt(2); the 16 smallest eigenpairs via B = A - sigma I, sigma = (||A||_inf + lambda_17)/2; "
           "X0 = orth(fp32(sin x sin) + N(0, (1e-5/sqrt(n))^2))")


def run_laplacian(args, world, rank, local):
    out = measure_laplacian(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_laplacian(args, world, rank, local, steps=None):
    """Sweeps/s on the sparse workload: FP64 SpMM, the Gram products on the
    tensor cores (split form, default) or in FP64, FP64 k x k stage and update."""
    import torch
    import paper_2602_23778_gb300 as eigref
    from workloads import configs as C
    steps = steps or args.steps or 100
    precision = args.precision or "bf16"
    torch.cuda.set_device(local)
    p = C.config4(per_column=True)
    rp, ci, val = (torch.from_numpy(a).cuda() for a in (p.row_ptr, p.col_idx, p.val))
    X0 = torch.from_numpy(np.ascontiguousarray(p.X0.T)).cuda().t()
    stream = torch.cuda.Stream()
    h = eigref.Handle(local, stream)
    kw = dict(norm_a=p.normA, target="smallest", shift=p.lam_kp1, precision=precision)

    def timed(form_kw, steps):
        h.refine_csr(rp, ci, val, X0.clone(), max_iters=args.warmup, check_every=max(2, args.warmup), **form_kw)
        torch.cuda.synchronize()
        X = X0.clone()
        r = h.refine_csr(rp, ci, val, X, max_iters=steps, check_every=steps, profile=True, **form_kw)
        torch.cuda.synchronize()
        return r

    with ClockSampler(local) as clk:
        rep = timed(kw, steps)
    ms_step = rep["sweeps_ms"] / rep["iterations"]
    if world > 1:
        ms_step = max_over_ranks(ms_step, "cuda")
    nnz, n, k = len(p.val), p.n, p.k
    bytes_launch = 12.0 * nnz + 4.0 * (n + 1) + 2 * 8.0 * n * k
    flops_launch = 2.0 * nnz * k
    launch_ms = rep["product_ms"] / max(1, rep["product_launches"])
    pk, pk_kind = peaks()
    gbs = bytes_launch / (launch_ms * 1e-3) / 1e9
    tfs = flops_launch / (launch_ms * 1e-3) / 1e12
    clocks = clk.summary()
    peak64 = fp64_peak(clocks)
    out = {"metric": METRIC, "value": world * 1000.0 / ms_step, "unit": UNIT, "n_gpus": world,
           "steps": rep["iterations"], "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f64+bf16-slices",
           "data": "synthetic",
           "config": {"workload": LAPLACE, "n": n, "k": k, "nnz": nnz,
                      "form": "FP64 SpMM, " + ("FP64 Gram products" if precision == "fp64" else
                                               "Gram products and row update as digit planes on the tensor cores"),
                      "split_k_gram": rep["ksplit"] or None,
                      "l2": "inputs larger than L2 (CSR 65 MB + X 131 MB + P 131 MB per SpMM); no flush"},
           "roofline": {"bound": "alu", "kernel": "spmm_csr_vec2_kernel", "achieved": tfs, "peak": peak64,
                        "unit": "TFLOP/s", "frac": tfs / peak64, "traffic": traffic_for("spmm.cu", "csr"),
                        "launch_ms": launch_ms, "algorithmic_flops_per_launch": flops_launch,
                        "peak_note": FP64_NOTE,
                        "hbm": {"achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                                "algorithmic_bytes_per_launch": bytes_launch}},
           "gpu_launches": int(rep["kernel_launches"]), "clocks": clocks,
           "status": rep["status_string"]}
    if rank == 0 and precision != "fp64" and not args.no_fp64_compare:
        r64 = timed(dict(kw, precision="fp64"), steps)
        v64 = 1000.0 * r64["iterations"] / r64["sweeps_ms"]
        out["fp64_form"] = {"value": v64, "unit": UNIT, "ms_per_step": r64["sweeps_ms"] / r64["iterations"],
                            "split_over_fp64": out["value"] / world / v64}
    h.close()
    return out


BATCH = ("256 dense problems, n log-uniform on [256, 4096], k uniform on {4..64} (seed 5000); "
         "A = Q diag(lambda) Q^T with 16 seeded Householder reflectors, lambda evenly spaced on [-1, 1]; "
         "the k algebraically largest via B = A - alpha I, alpha = (lambda_{k+1} - 1)/2; X0 = orth(fp32(Q_k))")


def run_batched(args, world, rank, local):
    out = measure_batched(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_batched(args, world, rank, local, steps=None):
    """Batch sweeps/s: one sweep of every problem per step, all problems in one
    graph replay (split form), beside per-problem calls of the plain FP64 form."""
    import torch
    import paper_2602_23778_gb300 as eigref
    from paper_2602_23778_gb300 import sliced_info
    from workloads import configs as C
    steps = steps or args.steps or 40
    torch.cuda.set_device(local)
    shapes = C.config5_shapes(count=args.count)
    # weak scaling over ranks: rank r takes problems r, r + world, ...
    mine = shard_indices(len(shapes), rank, world)
    ps = [C.config5_problem(i, *shapes[i]) for i in mine]
    stream = torch.cuda.Stream()
    h = eigref.Handle(local, stream)
    A = [torch.from_numpy(p.A).cuda() for p in ps]
    X0 = [torch.from_numpy(np.ascontiguousarray(p.X0.T)).cuda().t() for p in ps]

    def items():
        return [{"A": a, "X": x.clone(), "target": "shift", "shift": p.shift, "norm_a": p.normA}
                for a, x, p in zip(A, X0, ps)]

    prec = args.precision or "bf16"
    h.refine_batched(items(), max_iters=args.warmup, precision=prec)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        st, reps = h.refine_batched(items(), max_iters=steps, precision=prec)
        torch.cuda.synchronize()
    ms_step = reps[0]["sweeps_ms"] / steps
    if world > 1:
        ms_step = max_over_ranks(ms_step, "cuda")
    pk, pk_kind = peaks()
    if prec == "fp64":
        flops = sum(2.0 * p.n * p.n * p.k for p in ps)
        peak = fp64_peak(clk.summary())
        roof = {"bound": "alu", "peak_note": FP64_NOTE}
    else:
        flops = sum(sliced_info(prec, p.n, p.k)["executed_flops"] for p in ps)
        peak = pk["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "peak_note": "sustained BF16, of %s" % pk_kind}
    ach = flops / (ms_step * 1e-3) / 1e12
    roof.update({"kernel": "whole batch sweep (products of every problem)", "achieved": ach, "peak": peak,
                 "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                 "algorithmic_flops_per_step": flops})
    out = {"metric": METRIC, "value": world * 1000.0 / ms_step, "unit": "batch sweeps/s (every problem once)",
           "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == "fp64" else prec + "-slices+f64", "data": "synthetic",
           "config": {"workload": BATCH, "problems": len(ps) * world, "form": prec,
                      "l2": "A of all problems 6.5 GB, larger than L2; no flush"},
           "roofline": roof, "gpu_launches": int(reps[0]["kernel_launches"]), "clocks": clk.summary(),
           "status": eigref.status_string(st), "problem_sweeps_per_s": len(ps) * 1000.0 / ms_step}
    if rank == 0 and not args.no_fp64_compare:
        # per-problem calls of the plain FP64 form: the launch pattern a caller
        # without the batched entry point has
        steps64 = 4
        its = items()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for it in its:
            h.refine_dense(it["A"], it["X"], max_iters=steps64, norm_a=it["norm_a"], target="shift",
                           shift=it["shift"])
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps64
        out["fp64_per_problem_calls"] = {"value": 1000.0 / ms, "unit": out["unit"], "ms_per_step": ms,
                                         "steps": steps64, "batched_over_this": (1000.0 / ms_step) / (1000.0 / ms),
                                         "note": "includes each call's set-up (sign fix, graph capture)"}
    h.close()
    return out


DENSE2 = ("dense symmetric n=8192, k=64: A = Q diag(lambda) Q^T, Q = 64 seeded Householder reflectors, "
          "lambda = sign * 10^(-6u) (graded, random signs), the 64 largest |lambda|; X0 = orth(fp32(q) + N(0,1e-7)); "
          "run until ||R||_F <= 1e-14 ||A||")


def measure_dense_n8192(args, local):
    """The n = 8192, k = 64 graded workload: sweeps/s of both forms over a
    bounded sample, and the split form run to ||R||_F <= 1e-14 ||A|| with the
    sweep count set beside the linear rate gamma = |lambda_65| / |lambda_64|
    (end of Section 3.2).  The FP64 form at this gamma would need about the
    same number of sweeps, minutes of GPU time, so only its rate is timed."""
    import torch
    import paper_2602_23778_gb300 as eigref
    from workloads import configs as C
    torch.cuda.set_device(local)
    p = C.config2()
    gamma = p.gamma   # max |lambda| off the targets / min |lambda| on them
    A = torch.from_numpy(p.A).cuda()
    X0 = torch.from_numpy(np.ascontiguousarray(p.X0.T)).cuda().t()
    h = eigref.Handle(local, torch.cuda.Stream())
    out = {"workload": DENSE2, "n": p.n, "k": p.k, "gamma": gamma}
    for form, steps in (("bf16", 200), ("fp64", 30)):
        kw = dict(norm_a=p.normA, target="largest_mag", precision=form)
        h.refine_dense(A, X0.clone(), max_iters=args.warmup, check_every=args.warmup, **kw)
        r = h.refine_dense(A, X0.clone(), max_iters=steps, check_every=steps, **kw)
        torch.cuda.synchronize()
        out[form] = {"value": 1000.0 * r["iterations"] / r["sweeps_ms"], "unit": UNIT,
                     "ms_per_step": r["sweeps_ms"] / r["iterations"], "steps": r["iterations"]}
    out["split_over_fp64"] = out["bf16"]["value"] / out["fp64"]["value"]
    kw = dict(norm_a=p.normA, target="largest_mag", precision="bf16")
    r = h.refine_dense(A, X0.clone(), max_iters=60000, tol=1e-14, stop="residual", check_every=1024,
                       history=True, **kw)
    torch.cuda.synchronize()
    hr = np.asarray(r["hist_residual"])
    T = len(hr)
    # the asymptotic linear rate: the residual's decay per sweep over the last
    # fifth of the run (where the slowest non-target component dominates),
    # beside gamma = max |lambda| off the targets / min |lambda| on them
    t0, t1 = int(0.8 * T), T - 1
    rate = float(np.exp((np.log(hr[t1]) - np.log(hr[t0])) / (t1 - t0))) if T > 10 else float("nan")
    out["to_tolerance"] = {
        "form": "bf16", "status": r["status_string"], "sweeps": r["iterations"],
        "final_rel_residual": r["final_rel_residual"], "first_rel_residual": float(hr[0]) if T else None,
        "measured_rate": rate, "gamma": gamma, "rate_over_gamma": rate / gamma,
        "rate_note": "residual decay per sweep over the last fifth of the run; the end of Section 3.2 predicts gamma",
        "seconds": r["sweeps_ms"] * 1e-3}
    h.close()
    return out


def measure_dense_n512(args, local):
    """The n = 512, k = 8 workload (10 sweeps): launch- and latency-bound; us a sweep of both forms."""
    import torch
    import paper_2602_23778_gb300 as eigref
    from workloads import configs as C
    torch.cuda.set_device(local)
    p = C.config1()
    A = torch.from_numpy(p.A).cuda()
    X0 = torch.from_numpy(np.ascontiguousarray(p.X0.T)).cuda().t()
    h = eigref.Handle(local, torch.cuda.Stream())
    out = {"workload": "dense n=512, k=8, 16 Householder reflectors, lambda evenly spaced on [-1, 1], the 8 "
                       "algebraically largest via B = A - alpha I; 10 sweeps a call", "n": p.n, "k": p.k}
    for form in ("bf16", "fp64"):
        kw = dict(norm_a=p.normA, target="shift", shift=p.shift, precision=form)
        h.refine_dense(A, X0.clone(), max_iters=10, check_every=10, **kw)
        calls = []
        for _ in range(5):
            X = X0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.refine_dense(A, X, max_iters=10, check_every=10, **kw)
            torch.cuda.synchronize()
            calls.append(time.perf_counter() - t0)
        # steady state: one long call, chunks of 100 graph-replayed sweeps
        r = h.refine_dense(A, X0.clone(), max_iters=1000, check_every=100, **kw)
        us = 1000.0 * r["sweeps_ms"] / r["iterations"]
        out[form] = {"call_ms": 1000.0 * float(np.median(calls)), "us_per_sweep": us, "value": 1e6 / us,
                     "unit": UNIT, "note": "call_ms: one call of the 10-sweep workload, wall clock with set-up and "
                                           "graph capture (median of 5); us_per_sweep: device time a sweep over a "
                                           "1000-sweep call"}
    h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="eigref", choices=["eigref", "reference"])
    ap.add_argument("--precision", default=None, choices=["bf16", "fp64", "int8"])
    ap.add_argument("--slices", type=int, default=0, help="digit planes of the split form (0: library default)")
    ap.add_argument("--product-tile", type=int, default=0, choices=[0, 32, 64],
                    help="columns of the split product's output tile (0: the library default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in K decomposition (the product's equal-work plan) instead of timing candidates")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sweeps", type=int, default=60, help="oracle sweeps timed for cpu_baseline (about 10 s)")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the plain FP64 form beside the split form")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--n", type=int, default=16384, help="smaller n / k only for profiling captures")
    ap.add_argument("--k", type=int, default=128)
    ap.add_argument("--count", type=int, default=256, help="batched workload: number of problems")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="dense run: skip the Laplacian, batched, n=8192 and n=512 measurements")
    ap.add_argument("--workload", default="dense", choices=["dense", "laplacian", "batched"],
                    help="dense: the n=16384, k=128 matrix (default); laplacian: the 1024 x 1000 CSR Laplacian, k=16; "
                         "batched: 256 dense problems of uneven n and k")
    ap.add_argument("--summarize-launches", metavar="CSV", help="summarise an ncu launch list and exit")
    ap.add_argument("--peaks", action="store_true", help="measure library FP64/INT8/BF16 GEMM rates and exit")
    args = ap.parse_args()
    if args.summarize_launches:
        print(summarize_launches(args.summarize_launches))
        return
    if args.peaks:
        print(json.dumps(library_peaks()))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.steps is None:
            args.steps = 10
        run_reference(args, rank)
        return

    import torch
    import paper_2602_23778_gb300 as eigref

    if args.workload == "laplacian":
        run_laplacian(args, world, rank, local)
        return
    if args.workload == "batched":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        run_batched(args, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return
    precision = args.precision or "bf16"
    if args.steps is None:
        args.steps = 40 if precision == "fp64" else 400
    assert args.warmup >= 3, "at least 3 warm-up sweeps"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    p = workload(n=args.n, k=args.k)
    A = torch.from_numpy(p.A).cuda()
    X0 = torch.from_numpy(np.ascontiguousarray(p.X0.T)).cuda().t()  # column-major n x k
    stream = torch.cuda.Stream()
    h = eigref.Handle(local, stream)
    kw = dict(norm_a=p.normA, target="largest_mag", precision=precision)
    if precision != "fp64":
        kw["slices"] = args.slices
        if args.no_autotune:
            kw["autotune"] = False
        if args.product_tile:
            kw["product_tile"] = args.product_tile

    def refine(X, iters, **extra):
        return h.refine_dense(A, X, max_iters=iters, check_every=max(2, iters), **kw, **extra)

    # warm-up (untimed): builds graphs, touches A, runs the same kernels
    refine(X0.clone(), args.warmup)
    torch.cuda.synchronize()

    X = X0.clone()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        rep = refine(X, args.steps, profile=True)
        torch.cuda.synchronize()
        call_s = time.perf_counter() - t0
    if dist:
        dist.barrier()
    assert rep["iterations"] == args.steps, rep
    ms_step = rep["sweeps_ms"] / args.steps
    if dist:
        ms_step = max_over_ranks(ms_step, "cuda")
    value = world * 1000.0 / ms_step

    pk, pk_kind = peaks()
    n, k = p.n, p.k
    prod_ms = rep["product_ms"] / max(1, rep["product_launches"])
    if precision == "fp64":
        flops = 2.0 * n * n * k
        peak = fp64_peak(clk.summary())
        roof = {"bound": "alu", "kernel": "gemm_fp64_kernel", "peak_note": FP64_NOTE}
        kfile = "fp64.cu"
    else:
        from paper_2602_23778_gb300 import sliced_info
        info = sliced_info(precision, n, k, slices=args.slices or 8, product_tile=args.product_tile)
        flops = info["executed_flops"]
        # the kernel runs unthrottled at the maximum SM clock inside a sub-second
        # timed region (see "clocks"): the burst BF16 rate is its peak
        peak = pk["bf16_tflops"]
        roof = {"bound": "tensor", "kernel": info["kernel"],
                "peak_note": "burst BF16 (cuBLAS 8192^3), of %s; executed digit-pair flops" % pk_kind}
        kfile = "sliced.cu"
    achieved = flops / (prod_ms * 1e-3) / 1e12
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": traffic_for(kfile, precision), "launch_ms": prod_ms,
                 "algorithmic_flops_per_launch": flops})

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if precision == "fp64" else precision + "-slices+f64",
           "data": "synthetic",
           "config": dense_config(n, k, world),
           "method": {"form": precision,
                      "slices": (args.slices or 8) if precision != "fp64" else None,
                      # columns of the split product's output tile (128 x 64 wherever k allows it)
                      "product_tile": (args.product_tile or (64 if (k + 31) // 32 % 2 == 0 else 32))
                      if precision != "fp64" else None,
                      # product: 1..4 equal K splits a tile, 8 the equal-work plan (whole CTA rounds)
                      "split_k": {"product": rep["psplit"], "gram": rep["ksplit"]} if precision != "fp64" else None},
           "setup_ms": rep["setup_ms"], "call_s": call_s, "roofline": roof,
           "gpu_launches": int(rep["kernel_launches"]), "clocks": clk.summary()}

    def accuracy(form_kw):
        def measures(Xt):
            Xh = Xt.cpu().numpy()
            return {"max_sin_angle": max_angle(Xh, p.Xtrue), "orth_max": orth_max(Xh)}
        Xa = X0.clone()
        # run to the residual level of the n = 8192 workload's rule, 1e-14 ||A||
        ra = h.refine_dense(A, Xa, max_iters=600, tol=1e-14, stop="residual", check_every=50, **form_kw)
        acc = {"sweeps": ra["iterations"], "status": ra["status_string"],
               "final_rel_residual": ra["final_rel_residual"], "target_angle": 1e-13, "target_orth": 1e-14}
        # the result with the optional reorthogonalisation of Section 3.1.3 (reorth=1)
        Xr = Xa.clone()
        h.refine_dense(A, Xr, max_iters=0, reorth=True, **form_kw)
        acc.update(measures(Xr))
        acc["without_reorth"] = measures(Xa)
        # as many sweeps again, no reorthogonalisation: the level the iteration settles at
        rf = h.refine_dense(A, Xa, max_iters=ra["iterations"], check_every=50, **form_kw)
        acc["settled"] = {"sweeps": ra["iterations"] + rf["iterations"],
                          "final_rel_residual": rf["final_rel_residual"], **measures(Xa)}
        return acc

    if rank == 0 and not args.no_accuracy:
        out["accuracy"] = accuracy(kw)

    if rank == 0 and precision != "fp64" and not args.no_fp64_compare:
        # the plain FP64 form on the same input, same timing rules, fewer sweeps
        kw64 = dict(norm_a=p.normA, target="largest_mag", precision="fp64")
        h.refine_dense(A, X0.clone(), max_iters=args.warmup, check_every=args.warmup, **kw64)
        torch.cuda.synchronize()
        r64 = h.refine_dense(A, X0.clone(), max_iters=args.fp64_steps, check_every=args.fp64_steps,
                             profile=True, **kw64)
        torch.cuda.synchronize()
        v64 = 1000.0 * r64["iterations"] / r64["sweeps_ms"]
        out["fp64_form"] = {"value": v64, "unit": UNIT, "steps": r64["iterations"],
                            "ms_per_step": r64["sweeps_ms"] / r64["iterations"],
                            "split_over_fp64": value / world / v64}
        if not args.no_accuracy:
            out["fp64_form"]["accuracy"] = accuracy(kw64)

    if rank == 0 and not args.no_e2e:
        # pinned host buffers (page-locked, as a serving host keeps its inputs)
        Ah = torch.from_numpy(np.ascontiguousarray(p.A)).pin_memory()
        Xh = torch.from_numpy(np.ascontiguousarray(p.X0.T)).pin_memory().t()   # column-major n x k
        # untimed warm-up call with host buffers (the handle keeps its device
        # staging buffer for A, as a serving process would)
        Xw = torch.from_numpy(np.ascontiguousarray(p.X0.T)).pin_memory().t()
        h.refine_dense(Ah, Xw, max_iters=args.warmup, **kw)
        t0 = time.perf_counter()
        # the library's default chunking (a CUDA graph of 32 sweeps, replayed,
        # the stop flag read between replays), as a caller would use it
        re = h.refine_dense(Ah, Xh, max_iters=args.steps, **kw)
        e2e_s = time.perf_counter() - t0
        nb_a, nb_x = Ah.numel() * 8, Xh.numel() * 8
        out["e2e"] = {"value": re["iterations"] / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": (nb_a + nb_x) / args.steps,
                      "d2h_bytes_per_step": (nb_x + 8 * k) / args.steps,
                      "note": "pinned host A and X through eigref_refine_dense after one untimed warm-up call; "
                              "the H2D copies of A and X, slicing of A, all set-up and the D2H copy of X inside "
                              "the timed call"}

    if rank == 0 and world == 1 and not args.no_other_workloads and args.n == 16384 and args.k == 128:
        # the other workloads of the benchmark set, measured in the same run
        saved = args.steps
        args.steps = None
        out["workloads"] = {"laplacian": measure_laplacian(args, 1, 0, local, steps=100),
                            "batched": measure_batched(args, 1, 0, local, steps=40),
                            "dense_n8192_k64": measure_dense_n8192(args, local),
                            "dense_n512_k8": measure_dense_n512(args, local)}
        args.steps = saved

    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, wall = cpu_oracle_rate(p, args.cpu_sweeps)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "%d oracle sweeps of the same workload (%.1f s)" % (args.cpu_sweeps, wall)}
    h.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
