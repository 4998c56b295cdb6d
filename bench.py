#!/usr/bin/env python
"""Benchmark: batched exp(A) by parallel shifted solves (Blanes, arXiv:2210.03714).

Workload (one step): 4096 real dense matrices, d drawn uniformly from
{16, 32, ..., 256}, entries N(0,1)/sqrt(d), each scaled to ||A||_1 ~ U[0.5, 8];
the R8 set (8 nonzero nodes, Sec. 4.2) with scaling and squaring.  A step is
one fm_expm_batched call over the whole batch (norm, s, scaling, B^2, the four
+-c node pairs as one system I - c^2 B^2 each, the combination, s squarings).

Printed: one JSON line (rank 0).  value = matrices per second of the mixed
precision form (batched grid path: each system solved by residual correction,
every product a double-accurate BF16 digit product on the tensor cores); the
double form (one-CTA path, FP64 LU) is timed in the same run (fp64_value) and
the largest relative difference between the two over the batch is reported.
Inputs (784 MB) are larger than L2 (129 MB), so no flush is needed between steps.

--impl reference times the CPU oracle (oracle/, plain C, FP64) on a bounded
sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched f(A)/f(A)V evals/sec at ≤1e-12 rel err, mixed vs FP64 GPU; % roofline"
WORKLOAD = ("batched expm: 4096 real dense matrices, d uniform in {16,32,...,256}, "
            "entries N(0,1)/sqrt(d), ||A||_1 ~ U[0.5,8], R8 coefficient set (8 nodes: 4 +-c pairs)")
BATCH = 4096
SEED = 1000
DIMS = tuple(range(16, 257, 16))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# DRAM bytes (read + write) of the dominant kernel on the full workload, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum); None until
# captured for the current kernel.  "grid": the 21 tile launches of one step,
# captured on the 1024-matrix batch (17.43 GB) and scaled by the entries of
# the 4096-matrix batch (sum of d^2, x3.92), profiles/oz_tiles_dram_batch1024.md.
TRAFFIC = {"mixed": None, "fp64": None, "grid": 45.2e9}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def make_batch():
    import numpy as np
    from paper_2210_03714_gb300 import workloads as wl
    dims = wl.batch_dims(BATCH, SEED, DIMS)
    norms = np.random.default_rng(SEED + 7919).uniform(0.5, 8.0, size=BATCH)
    flat = wl.batch_flat(dims, norms, SEED)
    return dims, norms, flat


def method_flops(dims, s):
    """Algorithmic flops of one evaluation (per matrix): B^2 once (2 d^3), then
    the R8 nodes +-c as 4 pairs, each one system I - c^2 B^2 factored and solved
    with d right-hand sides (Sec. 1: 8/3 d^3 per inverse, one inverse per pair),
    and s squarings at 2 d^3."""
    import numpy as np
    d3 = np.asarray(dims, dtype=np.float64) ** 3
    return float(np.sum((2.0 + 4 * (8.0 / 3.0)) * d3 + 2.0 * np.asarray(s, dtype=np.float64) * d3))


def pipe_work(dims, s, precision, systems=4, max_ir=2, digits=7):
    """Algorithmic work of the persistent kernel per pipe, per launch (flops).

    R8 in the roundoff form: its 8 nonzero nodes are 4 pairs +-c, each solved as
    one system I - c^2 B^2 (one factorization, d right-hand sides), after one
    product B^2.
    double path: every product, factorization, solve and squaring on the FP64
      pipe (2 d^3 + systems (2/3 + 2) d^3 + 2 s d^3).
    mixed path: FP32 pipe: the factorizations (2/3 d^3) and 1 + max_ir solves
      with d right-hand sides (2 d^3 each); tensor pipe (BF16 digit products):
      B^2, systems * max_ir residual products and s squarings, each
      digits (digits+1)/2 = 28 digit-pair products of 2 d^3.
    Elementwise work is O(d^2) and left out."""
    import numpy as np
    d3 = np.asarray(dims, dtype=np.float64) ** 3
    sv = np.asarray(s, dtype=np.float64)
    if precision == "fp64":
        return {"fp64": float(np.sum((2.0 + systems * (8.0 / 3.0)) * d3 + 2.0 * sv * d3))}
    pairs = digits * (digits + 1) // 2
    return {"fp32": float(np.sum(systems * (2.0 / 3.0 + 2.0 * (1 + max_ir)) * d3)),
            "tensor_bf16": float(np.sum((1 + systems * max_ir + sv) * pairs * 2.0 * d3))}


MEASURED = {}  # peaks measured in this run (measure_peaks)


def measure_peaks(dev):
    """FP64 and FP32 dense peaks of this GPU, measured at the start of the run:
    the best of several torch.matmul calls (cuBLAS DGEMM 4096^3, SGEMM 8192^3
    with TF32 off), each timed with CUDA events on the current stream."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n, reps in (("fp64", torch.float64, 4096, 3), ("fp32", torch.float32, 8192, 5)):
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            c = a @ b
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                torch.matmul(a, b, out=c)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name] = (2.0 * n ** 3 / (best / 1000.0) / 1e12,
                         "measured: torch.matmul %s %d^3 (cuBLAS), best of %d, CUDA events"
                         % (str(dt).replace("torch.", ""), n, reps))
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    MEASURED.update(out)
    return out


def pipe_peaks(peaks):
    """TFLOP/s per pipe.  BF16 tensor: the driver's measured burst figure; FP64
    and FP32: measured in this run by measure_peaks (cuBLAS through torch), else
    derived from unit counts and the maximum SM clock (152 SMs; 128 FP32 lanes
    and, on GB300, about 2 FP64 FMA per SM per clock)."""
    mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32 = MEASURED.get("fp32", (152 * 128 * 2 * mhz * 1e6 / 1e12,
                                 "derived: 152 SMs x 128 lanes x 2 x max clock"))
    fp64 = MEASURED.get("fp64", (152 * 2 * 2 * mhz * 1e6 / 1e12,
                                 "derived: 152 SMs x 2 DFMA x 2 x max clock"))
    return {"fp32": fp32, "fp64": fp64,
            "tensor_bf16": ((peaks["bf16_tflops"], "measured burst") if "bf16_tflops" in peaks
                            else (1900.0, "fallback"))}


def counted_flops(dims, s, k=8):
    """The method's algorithmic count per matrix: k shifted systems (the R8 nodes), each an inverse of 8/3 d^3 flops (Sec. 1:
    LU and d triangular solves), and s squarings of 2 d^3: (8/3 k + 2 s) d^3,
    summed over the batch.  (The fused +-c pairs do less work than this count.)"""
    import numpy as np
    d3 = np.asarray(dims, dtype=np.float64) ** 3
    return float(np.sum((8.0 / 3.0 * k + 2.0 * np.asarray(s, dtype=np.float64)) * d3))


def roofline_of(work, ms, peaks):
    """The pipe with the largest lower-bound time sets the roofline; every pipe's
    achieved rate and fraction is listed beside it."""
    pk = pipe_peaks(peaks)
    t = ms / 1000.0
    pipes = {}
    for name, flops in work.items():
        peak, src = pk[name]
        ach = flops / t / 1e12
        pipes[name] = {"achieved": ach, "peak": peak, "peak_source": src, "frac": ach / peak,
                       "flops_per_launch": flops}
    bound = max(pipes, key=lambda n: pipes[n]["flops_per_launch"] / pipes[n]["peak"])
    b = pipes[bound]
    return {"bound": "tensor" if bound == "tensor_bf16" else "alu", "pipe": bound,
            "achieved": b["achieved"], "peak": b["peak"], "unit": "TFLOP/s",
            "frac": b["frac"], "traffic": None, "pipes": pipes}


def oracle_leg(fn, unit, sample):
    """The CPU baseline leg of a configuration line: the oracle as it stands,
    timed on a bounded sample (fn runs it and returns its result).  Returns
    (result, cpu_baseline object); the result also serves the line's error
    against the oracle."""
    import oracle
    oracle.lib()
    t0 = time.perf_counter()
    res = fn(oracle)
    dt = time.perf_counter() - t0
    return res, {"value": 1.0 / dt, "unit": unit, "cores": oracle.num_threads(),
                 "kind": "oracle", "sample": sample}


def cpu_baseline(dims, norms, sample, gpu_F=None, P=None):
    """The oracle (plain C, FP64, OpenMP over matrices) on a bounded sample."""
    import numpy as np
    import oracle
    from paper_2210_03714_gb300 import workloads as wl
    rng = np.random.default_rng(99)
    idx = np.sort(rng.choice(BATCH, sample, replace=False))
    mats = [wl.dense_scaled(int(dims[b]), float(norms[b]), SEED + 1 + int(b), scale_sqrt=True)
            for b in idx]
    oracle.lib()
    t0 = time.perf_counter()
    outs, s, info = oracle.expm_batched(mats, np.ones(len(mats)), "R8")
    dt = time.perf_counter() - t0
    errs = None
    if gpu_F is not None:
        errs = []
        for j, b in enumerate(idx[:64]):
            got = P.get(gpu_F, int(b)).cpu().numpy()
            errs.append(float(np.linalg.norm(got - outs[j]) / np.linalg.norm(outs[j])))
    return dict(value=len(mats) / dt, unit="evals/s", cores=oracle.num_threads(), kind="oracle",
                sample="%d matrices drawn uniformly from the 4096-matrix batch (same d and norm "
                       "distribution), R8, one pass" % len(mats),
                seconds=dt), errs


def run_single(args, emit=True):
    """One large matrix on the grid path: the Hermitian action (A = -iH, d = 4096,
    V complex 4096 x 256, spectral radius 20, R8, N = 206) or exp of one real
    dense matrix of order --dim (entries N(0,1)/sqrt(d), ||A||_1 = 4, R8); or
    the diffusion batch: phi_1(t_b A_b) and exp(t_b A_b) of 512 matrices of
    order 512 on the batched grid path (A_b = -L + 0.1 N_b, t_b log-uniform in
    [1e-4, 1e-2], R8 with the R8 phi_1 weights, s = 11..17 doublings)."""
    import numpy as np
    import torch
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import workloads as wl
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    fm.lib()
    cs = fm.Coeffs("R8")
    units = 1
    if args.workload == "diffusion":
        mats, ts, _, _ = wl.diffusion_batch(batch=512)
        units = len(mats)
        Pd = fm.Packed([torch.from_numpy(m) for m in mats], device=dev)
        td = torch.tensor(ts, dtype=torch.float64, device=dev)
        cp = fm.Coeffs("R8_phi1")
        call = lambda prec: fm.phi1_batched(Pd, td, cs, cp, precision=prec)[0]
        workload = ("phi_1(t A) and exp(t A) of 512 matrices of order 512: A = -L + 0.1 N, "
                    "L = trid{-1,2,-1}/h^2, N N(0,1)/sqrt(d), t log-uniform in [1e-4, 1e-2], "
                    "R8 and its phi_1 weights")
        metric = ("batched phi_1 evals/sec within the doubling bound 2^(s+3) u of s = 11..17 "
                  "doublings (batched grid path)")
        ref = lambda: fm.phi1_batched(Pd, td, cs, cp, precision="fp64")[0]
    elif args.workload == "hermitian":
        # the scale to spectral radius 20 stored with the oracle's result, so the
        # comparison below sees the same A bit for bit
        gpath = os.path.join(ROOT, "tests", "golden", "hermitian_d4096.npz")
        scale = float(np.load(gpath)["scale"]) if os.path.exists(gpath) else None
        A, V, rho = wl.hermitian_action(d=4096, m=256, rho=20.0, seed=2000, scale=scale)
        Ad = torch.tensor(A, dtype=torch.complex128, device=dev)
        Vd = torch.tensor(V, dtype=torch.complex128, device=dev)
        call = lambda prec: fm.expmv(Ad, Vd, 1.0, cs, precision=prec, anorm=rho)[0]
        workload = ("exp(-iH) V: H dense Hermitian d=4096 (G complex N(0,1)/sqrt(d), "
                    "spectral radius 20), V complex 4096x256, R8, anorm=20 (N=206 steps)")
        metric = "complex action evals/sec at <=1e-12 rel err (grid path)"
        ref = lambda: fm.expmv(Ad, Vd, 1.0, cs, precision="fp64", anorm=rho)[0]
    else:
        d = args.dim
        A = wl.dense_scaled(d, 4.0, 9, scale_sqrt=True)
        Ad = torch.tensor(A, dtype=torch.float64, device=dev)
        call = lambda prec: fm.expm(Ad, 1.0, cs, precision=prec)[0]
        workload = "exp(A): one real dense matrix d=%d, N(0,1)/sqrt(d) scaled to ||A||_1=4, R8" % d
        metric = "dense exp evals/sec at <=1e-12 rel err (grid path)"
        ref = lambda: fm.expm(Ad, 1.0, cs, precision="fp64")[0]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        call(args.precision)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    per = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = call(args.precision)
        e1.record(stream)
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    st = fm.last_stats()
    ms = sum(per) / len(per)
    peaks = load_peaks()
    pk = pipe_peaks(peaks)
    # the method's algorithmic flops per call (8/3 d^3 per inverse, 2 d^3 per product; complex
    # arithmetic as 4 real flops per multiply-add)
    if args.workload == "diffusion":
        _, _, _, s_d = fm.phi1_batched(Pd, td, cs, cp, precision=args.precision)
        sv = s_d.cpu().numpy().astype(float)
        alg = float(np.sum((8.0 / 3.0 * 8 + 4.0 * sv) * 512.0 ** 3))
    elif args.workload == "hermitian":
        dd, mm, NN = 4096.0, 256.0, 206.0
        alg = 8 * (8.0 / 3.0) * 4 * dd ** 3 + NN * (1 + 8) * 8 * dd * dd * mm
    else:
        _, _, s_d = fm.expm(Ad, 1.0, cs, precision=args.precision)
        alg = (8.0 / 3.0 * 8 + 2.0 * s_d) * float(args.dim) ** 3
    if args.precision == "mixed":
        pipe, work = "tensor_bf16", st["digit_flops"]
    else:
        pipe, work = "fp64", st["product_flops"]
    step_ach = alg / (ms / 1000.0) / 1e12
    kern_s = st["tile_ms"] / 1000.0
    ach = alg / kern_s / 1e12 if (pipe == "tensor_bf16" and kern_s > 0) else step_ach
    roofline = {"bound": "tensor" if pipe == "tensor_bf16" else "alu",
                "kernel": "oz_tiles" if pipe == "tensor_bf16" else "all",
                "pipe": pipe, "achieved": ach, "peak": pk[pipe][0], "peak_source": pk[pipe][1],
                "unit": "TFLOP/s", "frac": ach / pk[pipe][0], "traffic": None,
                "flops_per_call": alg, "kernel_ms": st["tile_ms"], "step_achieved": step_ach,
                "step_frac": step_ach / pk[pipe][0],
                "vs_fp64_peak": ach / pk["fp64"][0],
                "note": "the method's algorithmic flops per call over the tile launches' "
                        "CUDA-event time (tensor) or the whole call (fp64); step_* over the "
                        "whole call"}
    if pipe == "tensor_bf16" and kern_s > 0:
        roofline["tensor_busy"] = {"achieved": work / kern_s / 1e12,
                                   "frac": work / kern_s / 1e12 / pk[pipe][0],
                                   "note": "digit-pair products issued over the tile time"}
    # against the oracle: the stored full-size result (three columns) for the
    # Hermitian action, one matrix for the diffusion batch, one for dense exp
    err_oracle = None
    cpu = None
    if args.workload == "hermitian":
        # the oracle's stored result (tests/golden, written by the oracle alone)
        gpath = os.path.join(ROOT, "tests", "golden", "hermitian_d4096.npz")
        if os.path.exists(gpath):
            g = np.load(gpath)
            Wc = out.cpu().numpy()[:, g["cols"]]
            err_oracle = float(np.linalg.norm(Wc - g["W_full"]) / np.linalg.norm(g["W_full"]))
    elif args.workload == "diffusion" and not args.no_cpu_baseline:
        res, cpu = oracle_leg(lambda o: o.phi1(mats[0], ts[0], "R8", "R8_phi1"), "evals/s",
                              "1 matrix of the batch (phi_1 and exp)")
        got = Pd.get(out, 0).cpu().numpy()
        err_oracle = float(np.linalg.norm(got - res[0]) / np.linalg.norm(res[0]))
    diff = None
    fp64_ms = None
    if not args.no_fp64 and args.precision == "mixed":
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R = ref()
        torch.cuda.synchronize()
        fp64_ms = (time.perf_counter() - t0) * 1e3
        if units > 1:  # the largest relative difference over the batch
            diff = max(float(((Pd.get(out, b) - Pd.get(R, b)).norm() / Pd.get(R, b).norm()).item())
                       for b in range(units))
        else:
            diff = float(((out - R).norm() / R.norm()).item())
    line = {"metric": metric, "value": units * 1000.0 / ms, "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "replicas", "vs_baseline": None,
            "dtype": "bf16 digits, f64 accumulate" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": {"workload": workload, "precision": args.precision,
                                             "path": "grid" if args.precision == "mixed"
                                             else ("one-CTA" if units > 1 else "grid"),
                                             "l2": "working set > L2"},
            "roofline": roofline, "products": st["products"],
            "corrections": st["corrections"], "fp64_ms": fp64_ms,
            "rel_err_vs_oracle": err_oracle, "cpu_baseline": cpu,
            "rel_diff_vs_fp64": diff, "clocks": clk}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def run_trid(args, emit=True):
    """The tridiagonal action: 32768 systems of order 1000 (the paper's d for
    trid{-1,2,-1}, Sec. 5 Fig. 4), R10 in the roundoff form (the paper's R'_10,
    13d flops per shifted solve and step) or the plain form (R_10, 8d), with
    ||t A||_1 = 8 (N = 36 steps).  One step is one fm_trid_expmv_batched call."""
    import numpy as np
    import torch
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import workloads as wl
    rank = int(os.environ.get("RANK", "0"))
    dev = torch.device("cuda", torch.cuda.current_device())
    fm.lib()
    batch, d, eta = args.trid_batch, 1000, 8.0
    form = "plain" if args.form == "plain" else "roundoff"
    penta = args.workload == "penta"
    if penta:  # half bandwidth 2: fm_band_expmv_batched
        diags, v, t = wl.penta_batch(batch, d, eta=eta, seed=6000)
        Dg, Vd, Td = (torch.tensor(x, dtype=torch.float64, device=dev) for x in (diags, v, t))
        dense_of = lambda b: wl.band_dense(diags, b)
        host_in = (diags, v, t)
        dev_in = (Dg, Vd, Td)
    else:
        dl, dd, du, v, t = wl.trid_batch(batch, d, eta=eta, seed=5000)
        Dl, Dd, Du, Vd, Td = (torch.tensor(x, dtype=torch.float64, device=dev)
                              for x in (dl, dd, du, v, t))
        dense_of = lambda b: wl.trid_dense(dl, dd, du, b)
        host_in = (dl, dd, du, v, t)
        dev_in = (Dl, Dd, Du, Vd, Td)
    cs = fm.Coeffs("R10")
    if penta:
        call = lambda: fm.band_expmv_batched(Dg, Vd, Td, cs, form=form)
    else:
        call = lambda: fm.trid_expmv_batched(Dl, Dd, Du, Vd, Td, cs, form=form)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        W, info, N = call()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    bad = int((info != 0).sum().item())
    Ns = N.cpu().numpy().astype(np.float64)
    k = sum(1 for c in cs.as_dict()["c_re"] if c != 0)
    # algorithmic work (the paper's count): per step and system k shifted
    # solves of 13d flops (roundoff: B v and the Thomas solve) or 8d (plain);
    # the kernel's traffic per step: per node and element three factors read
    # and z written and read back, plus v, the diagonals and the output
    # pentadiagonal (Sec. 1): 15d per solve and 9d per product; per step and
    # node the kernel reads five factors and writes and reads z
    if penta:
        per_solve = 24.0 if form == "roundoff" else 15.0
        nbytes = float(Ns.sum()) * d * 8.0 * (7 * k + 8) + batch * d * 8.0 * (5 * k + 6)
    else:
        per_solve = 13.0 if form == "roundoff" else 8.0
        nbytes = float(Ns.sum()) * d * 8.0 * (5 * k + 6) + batch * d * 8.0 * (3 * k + 4)
    flops = float(Ns.sum()) * k * per_solve * d
    peaks = load_peaks()
    pk = pipe_peaks(peaks)
    sec = ms / 1000.0
    fp64 = {"achieved": flops / sec / 1e12, "peak": pk["fp64"][0], "peak_source": pk["fp64"][1],
            "unit": "TFLOP/s"}
    fp64["frac"] = fp64["achieved"] / fp64["peak"]
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm = {"achieved": nbytes / sec / 1e9, "peak": hbm_peak,
           "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "unit": "GB/s"}
    hbm["frac"] = hbm["achieved"] / hbm["peak"]
    bound = "hbm" if hbm["frac"] > fp64["frac"] else "alu"
    b = hbm if bound == "hbm" else fp64
    roofline = {"bound": bound, "kernel": "band_steps" if penta else "trid_steps",
                "achieved": b["achieved"],
                "peak": b["peak"], "unit": b["unit"], "frac": b["frac"], "traffic": None,
                "pipes": {"fp64": fp64, "hbm": hbm},
                "note": "whole call (the factorization launch included); fp64: the paper's "
                        "flop count, peak derived from unit counts; hbm: the kernel's design "
                        "traffic over the measured copy bandwidth"}
    # the CPU baseline leg: one sampled system by the oracle (dense LU of the
    # same matrix), timed, and the GPU's result for it against the oracle's
    err, cpu = None, None
    if not args.no_cpu_baseline:
        Wh = W[:, 7].cpu().numpy()
        res, cpu = oracle_leg(lambda o: o.expmv(dense_of(7), v[:, 7], t[7], "R10",
                                                o.PLAIN if form == "plain" else o.ROUNDOFF),
                              "systems/s", "1 system of the batch (dense LU of the same matrix)")
        err = float(np.linalg.norm(Wh - res[0]) / np.linalg.norm(res[0]))
    # end to end with host buffers: inputs in, result and status out, per step
    pins = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in host_in]
    W_host = torch.empty((d, batch), dtype=torch.float64).pin_memory()
    info_host = torch.empty(batch, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    for q in range(e2e_steps + 1):
        if q == 1:
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
        for dst, src in zip(dev_in, pins):
            dst.copy_(src, non_blocking=True)
        W, info, N = call()
        W_host.copy_(W, non_blocking=True)
        info_host.copy_(info, non_blocking=True)
    a1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a0.elapsed_time(a1) / e2e_steps
    e2e = {"value": batch / (e2e_ms / 1000.0), "unit": "systems/s",
           "h2d_bytes_per_step": int(sum(x.numel() * 8 for x in pins)),
           "d2h_bytes_per_step": int(W_host.numel() * 8 + info_host.numel() * 4)}
    kind_name = "pentadiagonal" if penta else "tridiagonal"
    line = {"metric": "%s action evals/sec (systems/s) at <=1e-12 rel err" % kind_name,
            "value": batch / sec, "unit": "systems/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "replicas", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (("exp(t A) v: %d pentadiagonal A of order 1000, the "
                                    "fourth-order stencil (-1, 16, -30, 16, -1)/12 with each "
                                    "entry times 1 + 0.05 N(0,1), v unit random, ||t A||_1 = 8, "
                                    "R10 %s form" % (batch, form)) if penta else
                                   ("exp(t A) v: %d tridiagonal A of order 1000, "
                                    "A = -trid{1+e, 2(1+e), 1+e} (e ~ 0.05 N(0,1)), v unit "
                                    "random, ||t A||_1 = 8, R10 %s form (N = 36)" % (batch, form))),
                       "l2": "working set (GBs) larger than L2"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": 2 * args.steps,
            "status_nonzero": bad, "rel_err_vs_oracle_sample": err, "cpu_baseline": cpu,
            "clocks": clk}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def run_small(args, emit=True):
    """The two latency-bound configurations: exp of one real d = 64 matrix in
    double (N(0,1) scaled to ||A||_1 = 2, R4, s = 10) on the team path (one
    cooperative launch over many SMs; the one-CTA kernel's time is reported
    beside it), and the gradient batch on the one-CTA kernels (256 matrices of
    order 128, N(0,1)/sqrt(d), R8 action with N from each matrix's norm,
    forward and adjoint in one call)."""
    import numpy as np
    import torch
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import workloads as wl
    rank = int(os.environ.get("RANK", "0"))
    dev = torch.device("cuda", torch.cuda.current_device())
    fm.lib()
    peaks = load_peaks()
    fp64_peak = pipe_peaks(peaks)["fp64"][0]
    if args.workload == "single":
        A, _ = wl.single_d64()
        Ad = torch.tensor(A, dtype=torch.float64, device=dev)
        cs = fm.Coeffs("R4")
        call = lambda prec: fm.expm(Ad, 1.0, cs, precision=prec, status=False)
        units, d = 1, 64
        metric = "exp of one d=64 matrix, evals/sec at <=1e-12 rel err (plain FP64)"
        workload = "exp(A): one real d=64 matrix, N(0,1) scaled to ||A||_1 = 2, R4 (s = 10)"
    else:
        A, v, y = wl.grad_batch(batch=256)
        d = A.shape[1]
        P = fm.Packed([torch.from_numpy(a) for a in A], device=dev)
        vd = torch.tensor(v.ravel(), dtype=torch.float64, device=dev)
        cs = fm.Coeffs("R8")
        W0, info0, N0 = fm.expmv_batched(P, vd, 1, 1.0, cs, precision="fp64")
        Ns = [int(x) for x in N0.cpu().numpy()]
        wbar = 2 * (W0 - torch.tensor(y.ravel(), dtype=torch.float64, device=dev))
        call = lambda prec: fm.expmv_adjoint_batched(P, vd, wbar, Ns, 1.0, cs)
        units = len(A)
        metric = "gradient of an R8 action, items/sec (forward + adjoint, one CTA per item)"
        workload = ("d/dA, d/dv of <wbar, r(B)^N v>: 256 matrices of order 128, N(0,1)/sqrt(d), "
                    "R8, N = ceil(||A||_1/theta) per matrix (mean %.0f)" % np.mean(Ns))
    stream = torch.cuda.current_stream()
    prec = "fp64"  # the plain method in double (config 0) and the FP64 adjoint
    for _ in range(args.warmup):
        out = call(prec)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = call(prec)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    extra = {}
    if args.workload == "single":
        F, _, s = fm.expm(Ad, 1.0, cs, precision=prec)
        # B^2, the two +-c pairs of R4 (one LU and a d-column solve each), s squarings
        flops = (2.0 + 2 * 8.0 / 3.0) * d ** 3 + 2.0 * s * d ** 3
        ach = flops / (ms / 1000.0) / 1e12
        roofline = {"bound": "latency", "pipe": "fp64", "achieved": ach, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": None,
                    "note": "the paper's flop count over the GPU's measured FP64 peak; the "
                            "path is a chain of about 14 grid-wide barriers (B^2, two "
                            "factorizations on two blocks, the solves, 10 squarings) on a "
                            "d = 64 problem: latency-bound"}
        # the same call on one thread block (the one-CTA kernel), for context
        for _ in range(2):
            fm.expm(Ad, 1.0, cs, precision=prec, path="cta", status=False)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            fm.expm(Ad, 1.0, cs, precision=prec, path="cta", status=False)
        c1.record(stream)
        torch.cuda.synchronize()
        extra["one_cta_ms"] = c0.elapsed_time(c1) / args.steps
        if not args.no_cpu_baseline:
            res, extra["cpu_baseline"] = oracle_leg(lambda o: o.expm(A, 1.0, "R4"), "evals/s",
                                                    "the matrix itself")
            extra["rel_err_vs_oracle"] = float(np.linalg.norm(F.cpu().numpy() - res[0]) /
                                               np.linalg.norm(res[0]))
        extra["s"] = s
    else:
        Nv = np.array(Ns, dtype=np.float64)
        k = 8
        # forward: k LUs and N steps of k solves and one product; reverse: N
        # steps of k transposed solves, k rank-one updates and two products
        flops = float(np.sum(k * (2.0 / 3.0) * d ** 3 + Nv * (k * 2 * d * d + 2 * d * d)
                             + Nv * (k * 2 * d * d + k * 2 * d * d + 4 * d * d)))
        ach = flops / (ms / 1000.0) / 1e12
        roofline = {"bound": "alu", "pipe": "fp64", "achieved": ach, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": None,
                    "note": "model flop count of the forward map and its adjoint over the "
                            "derived FP64 peak; the factors are reused N times from the "
                            "CTA's scratch, so the path is latency-bound"}
        extra["status_nonzero"] = int((out[3] != 0).sum().item())
    line = {"metric": metric, "value": units * 1000.0 / ms, "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "replicas", "vs_baseline": None,
            "dtype": ("f32+f64" if prec == "mixed" else "f64"), "data": "synthetic",
            "config": {"workload": workload, "precision": prec,
                       "path": "team" if args.workload == "single" else "one-CTA",
                       "l2": "working set within L2 (latency-bound)"},
            "roofline": roofline, "clocks": clk}
    line.update(extra)
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    dims, norms, _ = make_batch()
    vals = []
    cb = None
    for it in range(args.warmup + args.steps):
        cb, _ = cpu_baseline(dims, norms, args.ref_sample)
        if it >= args.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * args.ref_sample / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": BATCH, "sample": args.ref_sample},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(args, fm, torch, flat, dims, cs, stream, barrier, max_over_ranks, world, dev):
    """The metric through the public API with host buffers: every step copies
    its input in from pinned host memory, evaluates the batch and copies the
    result and status back, all inside the timed region.  The steps run as a
    stream of batches would: the input of step k + 1 is copied in on one copy
    stream and the result of step k goes out on another while the next step
    computes (two device buffers per direction); the region ends when the
    last result is on the host."""
    nbuf = 2
    A_host = torch.from_numpy(flat).pin_memory()
    t_host = torch.ones(BATCH, dtype=torch.float64).pin_memory()
    F_host = [torch.empty_like(A_host).pin_memory() for _ in range(nbuf)]
    info_host = [torch.empty(BATCH, dtype=torch.int32).pin_memory() for _ in range(nbuf)]
    A_dev = [torch.empty(flat.size, dtype=torch.float64, device=dev) for _ in range(nbuf)]
    F_dev = [torch.empty(flat.size, dtype=torch.float64, device=dev) for _ in range(nbuf)]
    t_dev = [torch.empty(BATCH, dtype=torch.float64, device=dev) for _ in range(nbuf)]
    Pe = [fm.Packed(dims=[int(d) for d in dims], flat=A_dev[i]) for i in range(nbuf)]
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def h2d(i):
        with torch.cuda.stream(up):
            A_dev[i].copy_(A_host, non_blocking=True)
            t_dev[i].copy_(t_host, non_blocking=True)
        return up.record_event()

    def d2h(i, Fo, inf):
        down.wait_event(stream.record_event())
        with torch.cuda.stream(down):
            F_host[i].copy_(Fo, non_blocking=True)
            info_host[i].copy_(inf, non_blocking=True)
        inf.record_stream(down)

    # one step untimed, then the pipelined steps
    stream.wait_event(h2d(0))
    Fo, inf, _ = fm.expm_batched(Pe[0], t_dev[0], cs, precision=args.precision, out=F_dev[0])
    d2h(0, Fo, inf)
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(1, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    up.wait_event(e0)
    loaded = [h2d(0), None]
    done = [None, None]  # the compute of the last step that used each input buffer
    sent = [None, None]  # the copy-out of the last result in each output buffer
    for k in range(e2e_steps):
        i = k % nbuf
        if k + 1 < e2e_steps:  # the next input, once its buffer's last user is done
            if done[1 - i] is not None:
                up.wait_event(done[1 - i])
            loaded[1 - i] = h2d(1 - i)
        stream.wait_event(loaded[i])
        if sent[i] is not None:  # the output buffer is free once its last copy-out is done
            stream.wait_event(sent[i])
        Fo, inf, _ = fm.expm_batched(Pe[i], t_dev[i], cs, precision=args.precision,
                                     out=F_dev[i])
        done[i] = stream.record_event()
        d2h(i, Fo, inf)
        sent[i] = down.record_event()
    stream.wait_stream(down)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps)
    if int((info_host[(e2e_steps - 1) % nbuf] != 0).sum()) != 0:
        raise RuntimeError("end-to-end run: nonzero status")
    h2d_bytes = A_host.numel() * 8 + t_host.numel() * 8
    d2h_bytes = F_host[0].numel() * 8 + info_host[0].numel() * 4
    return {"value": world * BATCH / (e2e_ms / 1000.0), "unit": "evals/s",
            "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
            "steps": e2e_steps,
            "note": "per step: pinned host input -> device, the batched call, result and "
                    "status -> pinned host; step k + 1's input copy and step k's result copy "
                    "run on two copy streams beside the compute stream (double-buffered)"}


# ---- multi-rank host logic: one process per GPU, each running the whole batch
# (weak scaling, no collective on the data path); the timing is the maximum
# over ranks and the value counts every rank's matrices.
def ranks_setup(backend):
    """(world, rank, local rank) from the torchrun environment; joins the
    process group when world > 1 (and selects the local GPU for nccl)."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def rank_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_max(x, world, device):
    """Largest x over the ranks (the whole job's step time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, batch, ms):
    """Matrices per second of the whole job: every rank's batch over the
    slowest rank's step time."""
    return world * batch / (ms / 1000.0)


def other_configs(args):
    """Short runs of the other configurations in the default run (a few steps
    each, mixed form; the value, the roofline fraction and the error against
    the oracle).  Each entry is the line the --workload run prints, reduced."""
    import copy
    import torch
    out = {}
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config",
            "roofline", "rel_err_vs_oracle", "rel_diff_vs_fp64", "rel_err_vs_oracle_sample",
            "e2e", "cpu_baseline", "clocks", "s", "status_nonzero", "one_cta_ms")
    plan = (("single_d64_R4", "single", run_small, dict(steps=10, warmup=3)),
            ("gradient_256x128", "adjoint", run_small, dict(steps=3, warmup=1)),
            ("hermitian_action_d4096", "hermitian", run_single, dict(steps=2, warmup=1)),
            ("diffusion_phi1_512x512", "diffusion", run_single, dict(steps=2, warmup=1)),
            ("trid_action_32768x1000", "trid", run_trid, dict(steps=3, warmup=1)),
            ("penta_action_32768x1000", "penta", run_trid, dict(steps=3, warmup=1)))
    for name, wl_name, fn, kw in plan:
        a = copy.copy(args)
        a.workload = wl_name
        a.no_fp64 = True
        for k, v in kw.items():
            setattr(a, k, v)
        try:
            r = fn(a, emit=False)
            out[name] = {k: r[k] for k in keep if k in r}
        except Exception as e:  # report, do not lose the main line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def main():
    global BATCH, DIMS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=512)
    ap.add_argument("--ref-sample", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="matrices per step (default 4096; smaller values are for profiling)")
    ap.add_argument("--dims", default=None,
                    help="comma-separated orders d is drawn from (default 16,32,...,256)")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "hermitian", "dense", "diffusion", "trid", "penta",
                             "single", "adjoint"],
                    help="batch: the 4096-matrix exp batch (default); hermitian: exp(-iH)V, "
                         "d = 4096, V 4096 x 256, N = 206 steps; dense: exp(A), one real "
                         "matrix of order --dim (both on the grid path); diffusion: phi_1 "
                         "of 512 matrices of order 512 (batched grid path); trid: exp(tA)v "
                         "for 32768 tridiagonal A of order 1000 (Thomas solves); penta: the "
                         "same with pentadiagonal A (banded LU); single: exp "
                         "of one d = 64 matrix; adjoint: the gradient batch (256 x 128^2)")
    ap.add_argument("--trid-batch", type=int, default=32768,
                    help="systems of order 1000 for --workload trid")
    ap.add_argument("--form", default="roundoff", choices=["roundoff", "plain"],
                    help="form of the rational approximant for --workload trid")
    ap.add_argument("--dim", type=int, default=2048)
    ap.add_argument("--path", default="auto", choices=["auto", "cta", "grid"],
                    help="execution path of the mixed form for the batch (the double form "
                         "always runs one CTA per matrix)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip fm_autotune (FM_PATH_AUTO then takes its fixed rule)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the short runs of the other configurations in the default run")
    args = ap.parse_args()
    if args.workload != "batch" and args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the "
                          "oracle on the default batch workload only"}), flush=True)
        return 0
    if args.workload in ("trid", "penta"):
        run_trid(args)
        return 0
    if args.workload in ("single", "adjoint"):
        run_small(args)
        return 0
    if args.workload != "batch":
        run_single(args)
        return 0
    if args.batch != BATCH or args.dims:
        BATCH = args.batch
        if args.dims:
            DIMS = tuple(int(x) for x in args.dims.split(","))
        WORKLOAD = ("batched expm (reduced case): %d real dense matrices, d uniform in {%s}, "
                    "entries N(0,1)/sqrt(d), ||A||_1 ~ U[0.5,8], R8" %
                    (BATCH, ",".join(map(str, DIMS))))
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2210_03714_gb300 as fm

    world, rank, local = ranks_setup("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        rank_barrier(world)

    def max_over_ranks(x):
        return rank_max(x, world, dev)

    fm.lib()
    measure_peaks(dev)
    # the autotuner: which orders of the batch take the one-CTA kernels (below
    # d*) and which the batched grid path; FM_PATH_AUTO below uses it
    tune = None
    if args.path == "auto" and not args.no_autotune:
        fm.lib().fm_autotune_reset()
        dstar, table = fm.autotune("expm", "R8", dmax=max(DIMS))
        tune = {"dstar": dstar, "table_us_per_matrix": [
            {"d": d, "one_cta": round(a, 3), "grid": round(b, 3)} for d, a, b in table]}
    dims, norms, flat = make_batch()
    P = fm.Packed(dims=[int(d) for d in dims], flat=torch.from_numpy(flat).to(dev))
    F = torch.empty_like(P.flat)
    t_dev = torch.ones(BATCH, dtype=torch.float64, device=dev)
    cs = fm.Coeffs("R8")
    stream = torch.cuda.current_stream()

    def step(prec, out):
        path = args.path if prec == "mixed" else "cta"
        return fm.expm_batched(P, t_dev, cs, precision=prec, out=out, path=path)

    def timed(prec, out, steps, warmup):
        for _ in range(warmup):
            step(prec, out)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for k in range(steps):
            _, info, s = step(prec, out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        barrier()
        return per, info, s

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    per, info, s = timed(args.precision, F, args.steps, args.warmup)
    clk = clocks.stop()
    st = fm.last_stats()  # the last timed call
    ms = max_over_ranks(sum(per) / len(per))
    bad = int((info != 0).sum().item())
    s_host = s.cpu().numpy()
    value = whole_job_value(world, BATCH, ms)

    # the same batch with the fixed rule (no tuned split), for context
    untuned_value = None
    if tune is not None and not args.no_fp64:
        fm.lib().fm_autotune_reset()
        per_u, _, _ = timed(args.precision, F, max(1, min(args.steps, 5)), 1)
        untuned_value = whole_job_value(world, BATCH, max_over_ranks(sum(per_u) / len(per_u)))
        # restore the tuned d* for the rest of the run
        fm.lib().fm_autotune_reset()
        fm.autotune("expm", "R8", dmax=max(DIMS))

    # the plain double form on the same GPU, same batch
    F64 = torch.empty_like(P.flat)
    fp64_ms = None
    maxdiff = None
    if not args.no_fp64:
        per64, info64, _ = timed("fp64", F64, max(1, min(args.steps, 2)), 1)
        fp64_ms = max_over_ranks(sum(per64) / len(per64))
        # largest relative Frobenius difference, mixed vs double, over the batch
        diffs = []
        for b in range(BATCH):
            x, y = P.get(F, b), P.get(F64, b)
            diffs.append((x - y).norm() / y.norm())
        maxdiff = float(torch.stack(diffs).max().item())

    # end to end through the public API: pinned host input, H2D, call, D2H
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, fm, torch, flat, dims, cs, stream, barrier, max_over_ranks, world,
                      dev)

    # roofline.  Grid path (the automatic choice for this batch): every product
    # of the step is tensor-core digit work, counted by the library
    # (fm_last_stats); the rate is taken over the whole step, so it bounds the
    # tile kernel's own rate from below.  One-CTA path: the per-pipe model of
    # the persistent kernel.
    peaks = load_peaks()
    achieved = method_flops(dims, s_host) / (ms / 1000.0) / 1e12
    grid_path = st["products"] > 0
    if grid_path:
        # the dominant kernel: the tensor-core tile launches, timed by the
        # library with CUDA events on their stream (fm_last_stats.tile_ms, the
        # last timed call)
        pk = pipe_peaks(peaks)["tensor_bf16"]
        tile_s = st["tile_ms"] / 1000.0
        # with a tuned split the tile kernel sees only the orders from d*
        gmask = np.asarray(dims) >= (tune["dstar"] if tune else 1)
        alg = counted_flops(np.asarray(dims)[gmask], np.asarray(s_host)[gmask])
        ach = alg / tile_s / 1e12 if tile_s > 0 else 0.0
        busy = st["digit_flops"] / tile_s / 1e12 if tile_s > 0 else 0.0
        step_ach = alg / (ms / 1000.0) / 1e12
        fp64_pk = pipe_peaks(peaks)["fp64"]
        roofline = {"bound": "tensor", "kernel": "oz_tiles", "pipe": "tensor_bf16",
                    "achieved": ach, "peak": pk[0], "peak_source": pk[1], "unit": "TFLOP/s",
                    "frac": ach / pk[0], "traffic": TRAFFIC.get("grid") if BATCH == 4096 and not args.dims else None,
                    "traffic_unit": "bytes per step (the tile launches of one call)",
                    "flops_per_step": alg, "flops_count": "(8/3 k + 2 s) d^3 per matrix, k = 8, "
                                                          "over the matrices on the grid path",
                    "kernel_ms_per_step": st["tile_ms"], "step_achieved": step_ach,
                    "step_frac": step_ach / pk[0],
                    "vs_fp64_peak": ach / fp64_pk[0], "fp64_peak": fp64_pk[0],
                    "fp64_peak_source": fp64_pk[1],
                    "tensor_busy": {"achieved": busy, "frac": busy / pk[0],
                                    "digit_flops_per_step": st["digit_flops"],
                                    "products_per_step": st["products"],
                                    "note": "digit-pair products the tile kernel issues (28 "
                                            "pairs per product flop at full accuracy, fewer on "
                                            "level-capped corrections) over its event time"},
                    "note": "achieved = the method's algorithmic flops per step over the tile "
                            "launches' CUDA-event time (each product is emulated by BF16 digit "
                            "products, so the tensor pipe does ~28x this work: tensor_busy); "
                            "step_* over the whole step"}
    else:
        roofline = roofline_of(pipe_work(dims, s_host, args.precision), ms, peaks)
        roofline["traffic"] = TRAFFIC.get(args.precision) if BATCH == 4096 and not args.dims else None
    fp64_roofline = (roofline_of(pipe_work(dims, s_host, "fp64"), fp64_ms, peaks)
                     if fp64_ms else None)
    # the mixed form on the one-CTA path, for context
    cta_value = None
    if grid_path and not args.no_fp64:
        Fc = torch.empty_like(P.flat)
        old = args.path
        args.path = "cta"
        perc, _, _ = timed("mixed", Fc, max(1, min(args.steps, 2)), 1)
        args.path = old
        cta_value = world * BATCH / (max_over_ranks(sum(perc) / len(perc)) / 1000.0)

    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("bf16 digits+f64" if grid_path else "f32+f64") if args.precision == "mixed"
                     else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": BATCH, "precision": args.precision,
                       "coeffs": "R8", "l2": "inputs (784 MB) larger than L2, no flush",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": (st["launches"] if grid_path else 2) * args.steps,
            "gpu_launches_note": ("over the timed steps: the grid path's launches per step "
                                  "(splits, tile products, epilogues, elementwise), as counted "
                                  "by the library, times the steps"
                                  if grid_path else
                                  "over the timed steps: per step the batch-ordering kernel and "
                                  "the persistent kernel"),
            "status_nonzero": bad,
            "fp64_value": (world * BATCH / (fp64_ms / 1000.0)) if fp64_ms else None,
            "fp64_ms_per_step": fp64_ms,
            "speedup_vs_fp64": (fp64_ms / ms) if fp64_ms else None,
            "max_rel_diff_vs_fp64": maxdiff,
            "method_tflops": achieved,
            "fp64_roofline": fp64_roofline,
            "path": "grid" if grid_path else "cta",
            "mixed_cta_path_value": cta_value,
            "autotune": tune, "value_fixed_rule": untuned_value,
            "clocks": clk}
    line["peaks_measured"] = {k: {"tflops": v[0], "source": v[1]} for k, v in MEASURED.items()}
    if rank == 0 and not args.no_cpu_baseline:
        cb, errs = cpu_baseline(dims, norms, args.cpu_sample, F, P)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        if errs:
            line["max_rel_err_vs_oracle_sample"] = max(errs)
    if world == 1 and not args.no_configs:
        del F64, P, F
        torch.cuda.empty_cache()
        line["configs"] = other_configs(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
