#!/usr/bin/env python3
"""Benchmark of the batched 2x2 SVD library on one node.

A step is one pass of the whole hot path -- scaling (Eq. 2), URV (Eq. 4 -
Eq. 11), SVD of R (Eq. 13 - Eq. 17), assembly of U and V (Eq. 29) and the
stores -- over one batch of synthetic input.  The default workload is the
FP32-vs-FP64 batch of n = 2^26 real matrices (90% i.i.d. N(0,1) entries, 10%
R(t1) diag(1, 10^-u) R(t2)^T with u uniform in [2, 12], generated in FP64 and
rounded to FP32) in the FP32 form that takes the tangent step of Eq. 6 - Eq. 7
in FP64 where the matrix is ill-conditioned, generated by the seeded generator
in ``paper_2005_07403_gb300.inputs`` and resident in HBM before the timed
region.  Its 1 GiB of input (4 GiB moved per step) is far larger than the
129 MB L2, so no flush is needed between steps.  The line also carries the
comparison with the FP64 form on the same inputs (matrices/s and the FP32
forms' singular-value errors against it); the supplementary measurements
(threshold sweeps, complex128, batching, differentiation, layouts,
Kogbetliantz step) go to stderr as one JSON object, or to ``--report FILE``.

Multi-GPU (torchrun): every rank processes its own batch of the same size
(independent problems, weak scaling); there is no data-path collective, only a
barrier and a max-reduction of the timing.

``--impl reference`` times the CPU oracle (the step-by-step scalar method in
plain C, OpenMP over the host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2x2 SVDs/sec and achieved HBM GB/s vs peak, FP64 vs FP32 at stated error"
FALLBACK_HBM_GBS = 6800.0

# Workloads.  Algorithmic bytes per matrix: one read of A, one write of U, V,
# Sigma' and s (int32).  The default is the complex128 batch; the others are
# the FP32-vs-FP64 batch of n = 2^26 (90% N(0,1), 10% ill-conditioned, rounded
# to FP32; the FP64 form runs on its exact widening) in each form.
WORKLOADS = {
    "complex128": dict(rows=8, n=2**24, bytes_per=64 + 128 + 16 + 4, kind="z", form="plain",
                       dtype="f64",
                       desc="complex128 n=2^24, parts U[-1,1]*2^e, e in [-500,500] per matrix, "
                            "1% rank-deficient"),
    "real-fp64": dict(rows=4, n=2**26, bytes_per=32 + 64 + 16 + 4, kind="d", form="plain",
                      dtype="f64",
                      desc="real FP64 n=2^26 (FP32-vs-FP64 batch widened exactly)"),
    "real-fp32": dict(rows=4, n=2**26, bytes_per=16 + 32 + 8 + 4, kind="s", form="plain",
                      dtype="f32", desc="real FP32 n=2^26 (FP32-vs-FP64 batch), no re-run"),
    "real-fp32-tan64": dict(rows=4, n=2**26, bytes_per=16 + 32 + 8 + 4, kind="s", form="tan64",
                            dtype="f32",
                            desc="real FP32 n=2^26 (90% N(0,1), 10% R(t1) diag(1, 10^-u) R(t2)^T, "
                                 "u in [2,12]), FP64 tangent step (Eq. 6 - Eq. 7) where "
                                 "|r''22| < 2^-3 r11"),
    "real-fp32-rerun": dict(rows=4, n=2**26, bytes_per=16 + 32 + 8 + 4, kind="s", form="rerun",
                            dtype="f32",
                            desc="real FP32 n=2^26 with FP64 re-run below tau = 2^-8"),
    # forward (with back-scaling) plus the adjoint: fwd 116 / 60 B, adjoint 192 / 96 B
    "grad-fp64": dict(rows=4, n=2**22, bytes_per=116 + 192, kind="d", form="grad", dtype="f64",
                      desc="real FP64 n=2^22 forward + adjoint: A = R(t1) diag(s1, s2) R(t2)^T, "
                           "s1 ~ U[0.5, 2], relative gap log-uniform in [1e-3, 1] (90%) and "
                           "[1e-12, 1e-6] (10%), upstream gradients N(0,1)"),
    "grad-fp32": dict(rows=4, n=2**22, bytes_per=60 + 96, kind="s", form="grad", dtype="f32",
                      desc="real FP32 n=2^22 forward + adjoint (the FP64 workload rounded "
                           "to FP32)"),
    "complex64": dict(rows=8, n=2**25, bytes_per=32 + 64 + 8 + 4, kind="c", form="plain",
                      dtype="f32",
                      desc="complex FP32 n=2^25 (90% N(0,1), 10% ill-conditioned), no re-run"),
    "complex64-rerun": dict(rows=8, n=2**25, bytes_per=32 + 64 + 8 + 4, kind="c", form="rerun",
                            dtype="f32",
                            desc="complex FP32 n=2^25 (90% N(0,1), 10% ill-conditioned) with "
                                 "FP64 re-run below tau = 2^-8"),
}


def make_input(name, n, rank):
    """The workload's A; for the differentiation workloads a dict with A and the
    upstream gradients gU, gV, gS."""
    from paper_2005_07403_gb300 import inputs
    if name.startswith("grad-"):
        g = inputs.grad_batch(n, seed=inputs.SEED_CFG5 + rank)
        dt = np.float64 if name == "grad-fp64" else np.float32
        return {k: np.ascontiguousarray(g[k].astype(dt)) for k in ("A", "gU", "gV", "gS")}
    if name == "complex128":
        return inputs.complex_scaled(n, seed=inputs.SEED_CFG2 + rank)
    if name in ("complex64", "complex64-rerun"):
        return inputs.complex_fp32_illcond(n, seed=inputs.SEED_CFG3 + 100 + rank)[0]
    A32, _ = inputs.real_fp32_illcond(n, seed=inputs.SEED_CFG3 + rank)
    return A32.astype(np.float64) if name == "real-fp64" else A32


# threshold of the FP32 forms (log2): the tangent step's default and the re-run's
TAN64_TAU_LOG2 = -3
RERUN_TAU_LOG2 = -8
DEFAULT_WORKLOAD = "real-fp32-tan64"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--n", type=int, default=0,
                   help="override the batch size (small cases for profiling only)")
    p.add_argument("--no-tune", action="store_true",
                   help="keep the library's default launch shape")
    p.add_argument("--launch", default="",
                   help="block,mpt,unroll,waves: this launch shape for the workload's kernel "
                        "(no tuning; for profiling a given shape)")
    p.add_argument("--no-compare", action="store_true",
                   help="skip the FP32-vs-FP64 comparison and the supplementary report")
    p.add_argument("--report", default="",
                   help="write the supplementary report (JSON) to this file instead of stderr")
    p.add_argument("--multi-batches", type=int, default=0,
                   help="profiling mode: time only the multi-batch launch on the first K "
                        "batches of the 2048-batch sequence and print one JSON line")
    p.add_argument("--multi-grid", type=int, default=0,
                   help="with --multi-batches: 0 = one block per tile, G > 0 = a grid of G "
                        "blocks walking the tiles (persistent when G is at most the resident count)")
    p.add_argument("--multi-shape", default="256,1,1",
                   help="with --multi-batches: block,mpt,unroll of the launch")
    p.add_argument("--grad", choices=["fp64", "fp32", "complex128", "complex64"], default="",
                   help="profiling mode: time only the forward and the adjoint of this type "
                        "(n = --n if given, else 2^22) and print one JSON line")
    p.add_argument("--kog", choices=[c[0] for c in KOG_CASES], default="",
                   help="profiling mode: time only the Kogbetliantz step of this type "
                        "(m x m, m = --n if given) and print one JSON line")
    return p.parse_args()


def dist_env():
    from paper_2005_07403_gb300 import distributed as D
    return D.env()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return GB300_SM_MAX_MHZ


# The FP64 forms are bound by the FP64 pipe, not by HBM: GB300 executes 2 FP64
# add/mul/fma per SM per clock (1.25 TFLOP/s nominal = 152 SMs x 2 fma x 2 flops
# x 2.07 GHz).  Their roofline counts the method's FP64 add, mul and fma per
# matrix (divisions and square roots run on the integer and FP32 pipes and are
# not counted); sign, exponent, min/max and pivot steps are bit operations.
# Counted from the formulas: complex 3 add + 36 fma + 50 mul (8 hypot, Eq. 4,
# Eq. 6 - Eq. 9, Fig. 10, the expansion of Eq. 29); real 3 add + 14 fma + 17
# mul.  The ncu opcode counts of the kernels agree exactly.
GB300_SMS = 152
GB300_FP64_PER_SM_CLK = 2
GB300_SM_MAX_MHZ = 2070.0
FP64_OPS_PER_MATRIX = {"z": 89, "d": 34}
# the values-only complex method skips Eq. 29 (U: 12 fma + 21 mul; V: 5 mul)
FP64_OPS_VALUES_Z = 89 - 38


# The translation units each workload's kernels are built from (the
# differentiation step: the forward kernel's and the adjoint's); every digest
# also covers the shared headers, the C header and the build script.
KERNEL_SOURCES = {"complex128": "svd2_fwd_z.cu", "real-fp64": "svd2_fwd_d.cu",
                  "real-fp32": "svd2_fwd_s.cu", "real-fp32-rerun": "svd2_rerun.cu",
                  "real-fp32-tan64": "svd2_tan64.cu",
                  "grad-fp64": ("svd2_fwd_d.cu", "svd2_bwd.cu"),
                  "grad-fp32": ("svd2_fwd_s.cu", "svd2_bwd.cu"),
                  "complex64": "svd2_fwd_c.cu", "complex64-rerun": "svd2_rerun.cu"}


def sources_digest(workload):
    """SHA-256 over the code (comments and blank space removed) of the
    workload's kernel sources: the DRAM traffic recorded under profiles/ holds
    only for this exact digest."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join("paper_2005_07403_gb300", "csrc")
    tus = KERNEL_SOURCES[workload]
    tus = (tus,) if isinstance(tus, str) else tus
    files = [os.path.join("include", "svd2.h"), os.path.join("paper_2005_07403_gb300", "build.py")]
    files += [os.path.join(csrc, tu) for tu in tus]
    files += sorted(os.path.join(csrc, f) for f in os.listdir(os.path.join(ROOT, csrc))
                    if f.endswith(".cuh"))
    import re
    for rel in files:
        h.update(rel.encode())
        with open(os.path.join(ROOT, rel)) as f:
            text = f.read()
        # the code only: comments and blank space do not change a kernel
        if rel.endswith(".py"):
            text = re.sub(r'(?s)""".*?"""', "", text)
            text = re.sub(r"#[^\n]*", "", text)
        else:
            text = re.sub(r"(?s)/\*.*?\*/", "", text)
            text = re.sub(r"//[^\n]*", "", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload, n):
    """DRAM bytes (read + write) per launch of the workload's kernel, scaled from
    the ncu capture in profiles/dram_traffic.txt to n matrices; None when no
    capture exists for the current sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    digest = sources_digest(workload)
    for ln in lines:
        f = ln.split()
        if len(f) >= 6 and not ln.startswith("#") and f[0] == workload and f[1] == digest:
            n_cap, rd, wr = int(f[3]), float(f[4]), float(f[5])
            return (rd + wr) * n / n_cap
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smmax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smmax) if smmax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    """Host cores available to this process (an inherited OMP_NUM_THREADS, which
    torchrun sets to 1, does not limit the oracle's timing)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_form(W, cores):
    """The oracle's counterpart of the workload's form, as a function of one
    (rows, n) host batch (a dict of A and the gradients for "grad")."""
    import oracle
    if W["form"] == "grad":
        def fwd_bwd(g):
            r = oracle.svd2(g["A"], backscale=True, nthreads=cores)
            dl = 64 * float(np.finfo(g["A"].dtype).eps)
            return oracle.bwd(r["U"], r["V"], r["smax"], r["smin"], g["gU"], g["gV"],
                              g["gS"][0], g["gS"][1], dl)
        return fwd_bwd
    if W["form"] == "rerun":
        return lambda a: oracle.svd2_rerun(a, RERUN_TAU_LOG2, nthreads=cores)
    if W["form"] == "tan64":
        return lambda a: oracle.svd2_tan64(a, TAN64_TAU_LOG2, nthreads=cores)
    return lambda a: oracle.svd2(a, nthreads=cores)


def _head(A, m):
    """The first m matrices of a workload's input (an array, or the dict of the
    differentiation workloads)."""
    if isinstance(A, dict):
        return {k: np.ascontiguousarray(v[..., :m]) for k, v in A.items()}
    return np.ascontiguousarray(A[:, :m])


def cpu_baseline(A, W, min_seconds=10.0, sample=2**21):
    """The oracle as it stands, in the workload's form, on all host cores, over a
    bounded sample of the workload (the first `sample` matrices), repeated for
    at least min_seconds."""
    cores = host_cores()
    run = oracle_form(W, cores)
    S = _head(A, sample)
    run(_head(S, 1024))                              # build/load outside the timing
    reps, t0 = 0, time.perf_counter()
    while True:
        run(S)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return {"value": reps * S.shape[1] / el, "unit": "matrices/s", "cores": cores,
            "kind": "oracle",
            "sample": f"first {sample} matrices of the workload, {reps} passes, {el:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    W = WORKLOADS[args.workload]
    sample = 2**21
    A = make_input(args.workload, sample, 0)
    run = oracle_form(W, cores)
    run(_head(A, 1024))
    for _ in range(args.warmup):
        run(A)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(A)
    el = time.perf_counter() - t0
    value = args.steps * sample / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": W["dtype"], "data": "synthetic",
            "config": {"workload": W["desc"], "sample_per_step": sample},
            "cpu_baseline": {"value": value, "unit": "matrices/s", "kind": "oracle",
                             "cores": cores,
                             "sample": f"{sample} matrices of the workload per step"},
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _caller(S, W, Ad, out, workspace, G=None):
    if W["form"] == "grad":
        import torch
        gA = torch.empty_like(Ad)
        dl = S.default_rel_delta(Ad.dtype)

        def step():
            S.svd2(Ad, backscale=True, out=out)
            S.svd2_bwd(out.U, out.V, out.smax, out.smin, G["gU"], G["gV"], G["gS"][0],
                       G["gS"][1], dl, out=gA)
        return step
    if W["form"] == "rerun":
        return lambda: S.svd2_rerun(Ad, tau_log2=RERUN_TAU_LOG2, out=out, workspace=workspace)
    if W["form"] == "tan64":
        return lambda: S.svd2_tan64(Ad, tau_log2=TAN64_TAU_LOG2, out=out)
    return lambda: S.svd2(Ad, out=out)


def time_steps(torch, call, steps, warmup, stream):
    for _ in range(max(warmup, 3)):
        call()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _quantile(torch, x, q):
    """The q-quantile of a tensor (the k-th smallest, k = ceil(q * numel)), by a
    device sort (torch.kthvalue takes ~0.7 s on 2^26 elements)."""
    k = max(1, int(np.ceil(q * x.numel())))
    return float(torch.sort(x.flatten()).values[k - 1])


def error_metrics(torch, A, r):
    """Per-matrix error metrics of Sec. 8 on a real batch: rho (Eq. 33, normwise
    relative backward error of U Sigma V^T), delta and eta (Eq. 34, Eq. 35,
    departure from orthogonality of U and V), evaluated in FP64 on the exact
    widening of the outputs (Sigma = 2^-s Sigma').  A is (4, n) in the split
    layout: element (i, j) is row i + 2 j.  Returns max and 99th percentile."""
    d = lambda t: t.double()
    a = [d(A[e]) for e in range(4)]
    u = [d(r.U[e]) for e in range(4)]
    v = [d(r.V[e]) for e in range(4)]
    sc = -r.s.clamp(max=4096).double()
    sg = (torch.ldexp(d(r.smax), sc), torch.ldexp(d(r.smin), sc))
    num = torch.zeros_like(a[0])
    for i in range(2):
        for j in range(2):
            m = u[i] * sg[0] * v[j] + u[i + 2] * sg[1] * v[j + 2]
            num += (m - a[i + 2 * j]) ** 2
    den = sum(x * x for x in a)
    rho = torch.nan_to_num(torch.sqrt(num) / torch.sqrt(den), nan=0.0)

    def orth(w):
        c11 = w[0] * w[0] + w[1] * w[1]
        c22 = w[2] * w[2] + w[3] * w[3]
        c12 = w[0] * w[2] + w[1] * w[3]
        return torch.sqrt((c11 - 1) ** 2 + 2 * c12 ** 2 + (c22 - 1) ** 2)

    out = {}
    for name, x in (("rho", rho), ("delta", orth(u)), ("eta", orth(v))):
        out[name + "_max"] = float(x.max())
        out[name + "_p99"] = _quantile(torch, x, 0.99)
    return out


def compare_precisions(torch, S, steps, warmup, stream, n=2**26):
    """The FP32 forms against the FP64 form on the same inputs (the FP32-vs-FP64
    batch of n = 2^26: 90% N(0,1), 10% ill-conditioned with sigma ratio 10^-u,
    u in [2, 12], rounded to FP32; the FP64 form runs on the exact widening).
    Each form's matrices/s, and its singular values' error against the FP64
    form (which reproduces the double method bit for bit) in units of
    u = 2^-24: max and 99th percentile, sigma'_min separately for the
    well- and the ill-conditioned class.  Returns (summary, report): a flat
    dict of scalars for the bench line and the detailed report with the
    threshold sweeps of the two forms that use double precision."""
    from paper_2005_07403_gb300 import inputs, tune
    A32, ill = inputs.real_fp32_illcond(n)
    A32d = torch.from_numpy(A32).cuda()
    A64d = A32d.double()
    illd = torch.from_numpy(ill).cuda()
    del A32
    o64 = S.empty_result(4, n, torch.float64, A64d.device)
    o32 = S.empty_result(4, n, torch.float32, A32d.device)
    ws = S.rerun_workspace(n)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    shapes = {"fp64": tune.tune(A64d, o64, reps=3), "fp32": tune.tune(A32d, o32, reps=3)}
    u = 2.0**-24
    ms = {"fp64": time_steps(torch, lambda: S.svd2(A64d, out=o64), steps, warmup, stream)}
    torch.cuda.synchronize()
    sx64 = torch.ldexp(o64.smax, -o64.s.double())
    sn64 = torch.ldexp(o64.smin, -o64.s.double())
    nz = (o64.smax > 0) & (sn64 > 0)
    q99 = lambda x: _quantile(torch, x, 0.99) if x.numel() else 0.0

    def errors(o):
        sx = torch.ldexp(o.smax.double(), -o.s.double())
        sn = torch.ldexp(o.smin.double(), -o.s.double())
        ex = ((sx - sx64).abs() / sx64)[o64.smax > 0] / u
        en = ((sn - sn64).abs() / torch.where(nz, sn64, torch.ones_like(sn64))) / u
        ew, ei = en[nz & ~illd], en[nz & illd]
        return {"smax_max": float(ex.max()), "smax_p99": q99(ex),
                "smin_max_normal": float(ew.max()), "smin_p99_normal": q99(ew),
                "smin_max_illcond": float(ei.max()), "smin_p99_illcond": q99(ei)}

    forms = {
        "fp32_plain": lambda: S.svd2(A32d, out=o32),
        "fp32_tan64": lambda: S.svd2_tan64(A32d, tau_log2=TAN64_TAU_LOG2, out=o32),
        "fp32_rerun": lambda: S.svd2_rerun(A32d, tau_log2=RERUN_TAU_LOG2, out=o32, workspace=ws),
    }
    err, metrics = {}, {"fp64": error_metrics(torch, A64d, o64)}
    frac = {}
    for name, f in forms.items():
        ms[name] = time_steps(torch, f, steps, warmup, stream)
        cnt.zero_()
        if name == "fp32_tan64":
            S.svd2_tan64(A32d, tau_log2=TAN64_TAU_LOG2, out=o32, count=cnt)
        else:
            f()
        torch.cuda.synchronize()
        if name == "fp32_tan64":
            frac[name] = int(cnt.item()) / n
        elif name == "fp32_rerun":
            frac[name] = S.rerun_count(ws) / n
        err[name] = errors(o32)
        metrics[name] = error_metrics(torch, A32d, o32)
    # the threshold sweeps: throughput, share of matrices in double, sigma errors
    sweep = {"fp32_tan64": [], "fp32_rerun": []}
    for t in (-1, -2, -3, -4, -6, -8, -10, -12):
        f = lambda: S.svd2_tan64(A32d, tau_log2=t, out=o32)
        m = time_steps(torch, f, 5, 3, stream)
        cnt.zero_()
        S.svd2_tan64(A32d, tau_log2=t, out=o32, count=cnt)
        torch.cuda.synchronize()
        sweep["fp32_tan64"].append(dict(tau_log2=t, matrices_per_s=n / (m / 1e3),
                                        double_fraction=int(cnt.item()) / n, **errors(o32)))
    for t in (-4, -8, -12):
        f = lambda: S.svd2_rerun(A32d, tau_log2=t, out=o32, workspace=ws)
        m = time_steps(torch, f, 5, 3, stream)
        f()
        torch.cuda.synchronize()
        sweep["fp32_rerun"].append(dict(tau_log2=t, matrices_per_s=n / (m / 1e3),
                                        double_fraction=S.rerun_count(ws) / n, **errors(o32)))
    peak, _ = measured_peaks()
    fp64_peak = GB300_SMS * GB300_FP64_PER_SM_CLK * sm_max_mhz() / 1e3
    rate = {k: n / (v / 1e3) for k, v in ms.items()}
    summary = {
        "n": n, "u": "2^-24",
        "fp64_matrices_per_s": rate["fp64"],
        "fp64_fp64_pipe_frac": FP64_OPS_PER_MATRIX["d"] * rate["fp64"] / 1e9 / fp64_peak,
        "fp32_plain_matrices_per_s": rate["fp32_plain"],
        "fp32_plain_hbm_frac": 60 * rate["fp32_plain"] / 1e9 / peak,
        "fp32_tan64_matrices_per_s": rate["fp32_tan64"],
        "fp32_tan64_hbm_frac": 60 * rate["fp32_tan64"] / 1e9 / peak,
        "fp32_tan64_tau_log2": TAN64_TAU_LOG2,
        "fp32_tan64_double_fraction": frac["fp32_tan64"],
        "fp32_rerun_matrices_per_s": rate["fp32_rerun"],
        "fp32_rerun_tau_log2": RERUN_TAU_LOG2,
        "fp32_rerun_double_fraction": frac["fp32_rerun"],
    }
    for name in forms:
        e = err[name]
        summary[name + "_smax_err_max_u"] = e["smax_max"]
        summary[name + "_smin_err_max_u"] = max(e["smin_max_normal"], e["smin_max_illcond"])
        summary[name + "_smin_err_p99_illcond_u"] = e["smin_p99_illcond"]
        summary[name + "_rho_max"] = metrics[name]["rho_max"]
    summary["fp64_rho_max"] = metrics["fp64"]["rho_max"]
    metrics["evaluated_in"] = ("FP64 on the exact widening of each form's outputs (Eq. 32 - "
                               "Eq. 35); the FP64 form's values are at the level of that "
                               "evaluation's own rounding")
    report = {"n": n, "tuned_shapes": shapes, "ms": ms, "errors_vs_fp64_u": err,
              "error_metrics": metrics, "tau_sweep": sweep}
    del A32d, A64d, o64, o32, ws, illd
    torch.cuda.empty_cache()
    return summary, report


def bench_multi(torch, S, stream, replays=20):
    """The Kogbetliantz batching workload: 2048 batches with lengths log-uniform
    in [16, 2^20], real FP64 / complex128 at random, N(0,1) entries (drawn on
    the device); the autotuner picks the launch shape, the persistent launch is
    captured in a CUDA graph and each replay is timed; the median is reported."""
    from paper_2005_07403_gb300 import inputs
    lens, cplx = inputs.kog_batches()
    dev = [inputs.normal_batch_device(int(n), 8 if c else 4, 5000 + i)
           for i, (n, c) in enumerate(zip(lens, cplx))]
    total = int(lens.sum())
    mb = S.MultiBatch(dev)
    best = mb.autotune(reps=3)
    g = mb.graph()
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    times = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(replays):
        e0.record(stream)
        g.launch(stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    g.close()
    med = float(np.median(times))
    nbytes = int(sum(n * (212 if c else 116) for n, c in zip(lens, cplx)))
    out = {"batches": int(len(lens)), "matrices": total, "complex_fraction": float(cplx.mean()),
           "tuned_shape": best, "graph_replays": replays, "median_ms": med,
           "matrices_per_s": total / (med / 1e3), "algorithmic_GBps": nbytes / (med / 1e3) / 1e9}
    del dev, mb
    torch.cuda.empty_cache()
    return out


# The adjoint kernels' algorithmic traffic per matrix: U, V, s1, s2, gU, gV,
# g1, g2 read and gA written once (real: 20 + 4 values, complex: 36 + 8), and
# the real FP64 adjoint's FP64 add/mul/fma per matrix counted from its
# formulas (J and K 8, a and b 2, s1 + s2 1, the gap 4, p and q 6, M 2, U M 8,
# (U M) V^T 8; its three divisions run on the integer pipe, and so do 10 of
# its 18 products: those of p, q, the gap and (U M) V^T).
BWD_BYTES = {"fp64": 24 * 8, "fp32": 24 * 4, "complex128": 44 * 8, "complex64": 44 * 4}
BWD_FP64_OPS_REAL = 39
BWD_INT_PIPE_PRODUCTS_REAL = 10


def bench_grad(torch, S, stream, steps=10, warmup=3, n=2**22, only=""):
    """The differentiation workload: A = R(t1) diag(s1, s2) R(t2)^T, 10% with
    relative gaps in [1e-12, 1e-6], N(0,1) upstream gradients (complex: N(0,1)
    parts drawn on the device).  Per dtype: the forward kernel (with
    back-scaling) and the adjoint kernel timed each on its own with CUDA
    events, their sum as the step, and the adjoint's roofline: HBM bytes for
    every form, FP64-pipe operations for real FP64."""
    from paper_2005_07403_gb300 import inputs
    peak, _ = measured_peaks()
    fp64_peak = GB300_SMS * GB300_FP64_PER_SM_CLK * sm_max_mhz() / 1e3
    g = inputs.grad_batch(n) if only in ("", "fp64", "fp32") else None
    out = {"n": n}
    cases = []
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        cases.append((name, 4, lambda dt=dt: (torch.from_numpy(g["A"]).to("cuda", dt),
                                               torch.from_numpy(g["gU"]).to("cuda", dt),
                                               torch.from_numpy(g["gV"]).to("cuda", dt),
                                               torch.from_numpy(g["gS"]).to("cuda", dt))))
    for name, dt in (("complex128", torch.float64), ("complex64", torch.float32)):
        cases.append((name, 8, lambda dt=dt: (inputs.normal_batch_device(n, 8, 151, "cuda", dt),
                                               inputs.normal_batch_device(n, 8, 152, "cuda", dt),
                                               inputs.normal_batch_device(n, 8, 153, "cuda", dt),
                                               inputs.normal_batch_device(n, 2, 154, "cuda", dt))))
    for name, rows, make in cases:
        if only and name != only:
            continue
        A, gU, gV, gS = make()
        r = S.empty_result(rows, n, A.dtype, A.device)
        gA = torch.empty_like(A)
        fwd = lambda: S.svd2(A, backscale=True, out=r)
        bwd = lambda: S.svd2_bwd(r.U, r.V, r.smax, r.smin, gU, gV, gS[0], gS[1], out=gA)
        msf = time_steps(torch, fwd, steps, warmup, stream)
        fwd()
        msb = time_steps(torch, bwd, steps, warmup, stream)
        res = {"fwd_ms": msf, "bwd_ms": msb, "fwd_bwd_matrices_per_s": n / ((msf + msb) / 1e3),
               "bwd_matrices_per_s": n / (msb / 1e3), "bwd_bytes_per_matrix": BWD_BYTES[name],
               "bwd_hbm_frac": BWD_BYTES[name] * n / (msb / 1e3) / 1e9 / peak}
        if name == "fp64":
            res["bwd_fp64_ops_per_matrix"] = BWD_FP64_OPS_REAL
            res["bwd_int_pipe_products_per_matrix"] = BWD_INT_PIPE_PRODUCTS_REAL
            res["bwd_fp64_pipe_frac"] = BWD_FP64_OPS_REAL * n / (msb / 1e3) / 1e9 / fp64_peak
        out[name] = res
        del A, gU, gV, gS, r, gA
    torch.cuda.empty_cache()
    return out


def bench_host_link(torch, stream, nbytes=1 << 30, reps=5):
    """The host link as the e2e measurement sees it: copy-engine rates of one
    GiB between pinned host memory and the device in each direction and in
    both at once (two streams), timed with CUDA events, and the NUMA nodes
    (with their CPUs) this process can run on."""
    import glob
    nodes = {}
    for d in sorted(glob.glob("/sys/devices/system/node/node[0-9]*")):
        try:
            nodes[os.path.basename(d)] = open(os.path.join(d, "cpulist")).read().strip()
        except OSError:
            pass
    h = torch.empty(nbytes // 4, dtype=torch.float32).pin_memory()
    h2 = torch.empty(nbytes // 4, dtype=torch.float32).pin_memory()
    d = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    d2 = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    h.fill_(1.0)
    other = torch.cuda.Stream()

    def rate(f):
        f()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            f()
        e1.record(stream)
        torch.cuda.synchronize()
        return nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9

    def both():
        ev = torch.cuda.Event()
        ev.record(stream)
        other.wait_event(ev)
        with torch.cuda.stream(other):
            h2.copy_(d2, non_blocking=True)
        d.copy_(h, non_blocking=True)
        done = torch.cuda.Event()
        done.record(other)
        stream.wait_event(done)

    out = {"numa_nodes": nodes, "process_cpus": len(os.sched_getaffinity(0)),
           "h2d_GBps": rate(lambda: d.copy_(h, non_blocking=True)),
           "d2h_GBps": rate(lambda: h.copy_(d, non_blocking=True)),
           "both_directions_GBps": 2 * rate(both)}
    del h, h2, d, d2
    torch.cuda.empty_cache()
    return out


def bench_complex128(torch, S, stream, steps=10, warmup=3):
    """The complex128 workload (n = 2^24, parts U[-1,1] 2^e, e in [-500, 500]
    per matrix, 1% rank-deficient) on the plain FP64 form: matrices/s, the
    fraction of the FP64 pipe (89 add/mul/fma per matrix) and of HBM (212 B)."""
    from paper_2005_07403_gb300 import tune
    W = WORKLOADS["complex128"]
    n = W["n"]
    Ad = torch.from_numpy(make_input("complex128", n, 0)).cuda()
    out = S.empty_result(8, n, Ad.dtype, Ad.device)
    shape = tune.tune(Ad, out, reps=3)
    ms = time_steps(torch, lambda: S.svd2(Ad, out=out), steps, warmup, stream)
    peak, _ = measured_peaks()
    fp64_peak = GB300_SMS * GB300_FP64_PER_SM_CLK * sm_max_mhz() / 1e3
    rate = n / (ms / 1e3)
    res = {"n": n, "ms": ms, "matrices_per_s": rate, "tuned_shape": shape,
           "fp64_pipe_frac": FP64_OPS_PER_MATRIX["z"] * rate / 1e9 / fp64_peak,
           "hbm_frac": W["bytes_per"] * rate / 1e9 / peak}
    del Ad, out
    torch.cuda.empty_cache()
    return res


def bench_variants(torch, S, stream, steps=10, warmup=3):
    """The singular-values-only forms and the interleaved (n, 2, 2) layout on
    the bench's two main shapes: complex128 n = 2^24 and real FP32 n = 2^26,
    N(0,1) entries drawn on the device.  Per form: matrices/s, algorithmic
    bytes per matrix and the fraction of the measured HBM copy bandwidth
    (complex128: also of the FP64 pipe, with the method's FP64 add/mul/fma)."""
    from paper_2005_07403_gb300 import inputs
    peak, _ = measured_peaks()
    fp64_peak = GB300_SMS * GB300_FP64_PER_SM_CLK * sm_max_mhz() / 1e3
    out = {}
    for name, rows, n, dt, cdt in (("complex128", 8, 2**24, torch.float64, torch.complex128),
                                   ("real_fp32", 4, 2**26, torch.float32, torch.float32)):
        A = inputs.normal_batch_device(n, rows, 131, "cuda", dt)
        if rows == 8:   # (n, 2, 2) complex from the split rows (Re, Im of a11, a21, a12, a22)
            el = [torch.complex(A[2 * e], A[2 * e + 1]) for e in range(4)]
        else:
            el = [A[e] for e in range(4)]
        M = torch.stack([el[0], el[2], el[1], el[3]], dim=1).reshape(n, 2, 2).to(cdt).contiguous()
        res = {}
        vals = S.svd2_values(A)
        es = torch.finfo(dt).bits // 8
        b_vals = rows * es + 2 * es + 4
        b_full = 3 * rows * es + 2 * es + 4
        for form, fn, bpm in (
                ("values_only", lambda: S.svd2_values(A, out=vals), b_vals),
                ("interleaved", lambda: S.svd2_interleaved(M), b_full),
                ("interleaved_values_only", lambda: S.svd2_interleaved(M, values_only=True), b_vals)):
            ms = time_steps(torch, fn, steps, warmup, stream)
            r = {"matrices_per_s": n / (ms / 1e3), "ms": ms, "bytes_per_matrix": bpm,
                 "hbm_frac": bpm * n / (ms / 1e3) / 1e9 / peak}
            res[form] = r
        if rows == 8:
            zv, zf = FP64_OPS_VALUES_Z, FP64_OPS_PER_MATRIX["z"]
            res["values_only"]["fp64_pipe_frac"] = zv * n / (res["values_only"]["ms"] / 1e3) / 1e9 / fp64_peak
            res["interleaved"]["fp64_pipe_frac"] = zf * n / (res["interleaved"]["ms"] / 1e3) / 1e9 / fp64_peak
        out[name] = dict(n=n, **res)
        del A, M, vals
        torch.cuda.empty_cache()
    return out


KOG_CASES = (("complex128", 8192, "complex128", 48, 16),
             ("real_fp64", 8192, "float64", 12, 4),
             ("real_fp32", 16384, "float32", 16, 0))


def bench_kog(torch, S, stream, steps=10, warmup=3, only="", m_override=0):
    """One parallel Kogbetliantz step (Sec. 1) on m x m matrices of N(0,1)
    entries drawn on the device: complex128 and real FP64 with m = 8192
    (column-major), real FP32 with m = 16384; with the pivot pairs (2i, 2i+1)
    (contiguous 2x2 blocks) and with one round-robin step (gathered rows and
    columns).  G is updated in place every step (the transformation is
    unitary, so the values stay bounded).  Per case: steps/s, the update's
    algorithmic bytes (G read and written once) against the HBM copy peak and,
    in FP64, the operations it issues on the FP64 pipe against that pipe's
    peak: 12 of the 16 per real 2x2 block and 48 of the 64 per complex one,
    the rest leading products of the fma chains run on the integer pipe
    (their count is reported beside)."""
    from paper_2005_07403_gb300 import inputs
    peak, _ = measured_peaks()
    fp64_peak = GB300_SMS * GB300_FP64_PER_SM_CLK * sm_max_mhz() / 1e3
    out = {}
    for name, m, dt, ops, int_ops in KOG_CASES:
        if only and name != only:
            continue
        m = m_override or m
        dt = getattr(torch, dt)
        g = torch.Generator(device="cuda")
        g.manual_seed(141)
        G = torch.randn((m, m), generator=g, device="cuda", dtype=dt).T   # column-major
        ws = S.kog_workspace(G)
        res = {"m": m}
        for order, pairs in (("adjacent", torch.arange(m, dtype=torch.int32, device="cuda")),
                             ("round_robin", torch.from_numpy(inputs.round_robin_pairs(m, 1)).cuda())):
            ms = time_steps(torch, lambda: S.kog_step(G, pairs, workspace=ws), steps, warmup, stream)
            nbytes = 2 * m * m * G.element_size()
            r = {"steps_per_s": 1e3 / ms, "ms": ms, "bytes_per_step": nbytes,
                 "hbm_frac": nbytes / (ms / 1e3) / 1e9 / peak}
            if dt != torch.float32:
                r["fp64_pipe_ops_per_block"] = ops
                r["int_pipe_products_per_block"] = int_ops
                r["fp64_pipe_frac"] = ops * (m // 2) ** 2 / (ms / 1e3) / 1e9 / fp64_peak
            res[order] = r
        out[name] = res
        del G, ws
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    from paper_2005_07403_gb300 import svd2 as S

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    n = args.n or W["n"]
    A = make_input(args.workload, n, rank)
    G = None
    if W["form"] == "grad":
        G = {k: torch.from_numpy(v).cuda() for k, v in A.items()}
        Ad = G["A"]
    else:
        Ad = torch.from_numpy(A).cuda()
    out = S.empty_result(W["rows"], n, Ad.dtype, Ad.device)
    workspace = S.rerun_workspace(n) if W["form"] == "rerun" else None
    call = _caller(S, W, Ad, out, workspace, G)
    S.lib()
    tuned = None
    kind_launch = {"tan64": "s_tan64"}.get(W["form"], W["kind"])
    if args.launch:
        S.set_launch(kind_launch, *(int(x) for x in args.launch.split(",")))
    elif not args.no_tune:
        from paper_2005_07403_gb300 import tune
        # launch shape from the autotuner (cached)
        tuned = tune.tune(Ad, out, reps=3, form="tan64" if W["form"] == "tan64" else "plain")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        call()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    ms_per_step = ms_max / args.steps
    value = world * n * args.steps / (ms_max / 1e3)
    # our kernels per call: the batch kernel and its fix-up pass (plus a memset
    # of the flag word); the re-run form also the list compaction and the
    # re-run pass
    launches_per_step = {"rerun": 4, "grad": 3}.get(W["form"], 2)

    # end to end through the C ABI with host buffers (svd2_batch_host): every
    # step reads A from and writes every output to pinned host memory
    e2e = None
    if not args.no_e2e and W["form"] in ("plain", "tan64"):
        t64 = W["form"] == "tan64"
        Ah = torch.from_numpy(A).pin_memory()
        outs_h = S.empty_host_result(W["rows"], n, Ah.dtype)
        h2d = Ah.numel() * Ah.element_size()
        d2h = sum(t.numel() * t.element_size()
                  for t in (outs_h.U, outs_h.V, outs_h.smax, outs_h.smin, outs_h.s))
        ke = max(2, min(args.steps, 5))
        S.svd2_host(Ah, out=outs_h, tan64=t64)        # warm-up: creates the staging buffers
        barrier()
        e0.record(stream)
        for _ in range(ke):
            S.svd2_host(Ah, out=outs_h, tan64=t64)
        e1.record(stream)
        barrier()
        ems = e0.elapsed_time(e1)
        et = torch.tensor([ems], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(et, op=dist.ReduceOp.MAX)
        secs = float(et.item()) / 1e3
        e2e = {"value": world * n * ke / secs, "unit": "matrices/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "svd2_batch_host on pinned host arrays (the kernel reads and writes them "
                      "directly across the host link)",
               "host_link_GBps": (h2d + d2h) * ke / secs / 1e9}
        del Ah, outs_h

    peak, peak_src = measured_peaks()
    bytes_launch = W["bytes_per"] * n
    achieved = bytes_launch / (ms_per_step / 1e3) / 1e9
    traffic = recorded_traffic(args.workload, n)
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": traffic,
           "note": f"peak {peak_src}; algorithmic {W['bytes_per']} B/matrix x {n} per launch"
                   + ("; traffic from profiles/dram_traffic.txt scaled to n" if traffic else "")}
    if W["kind"] in FP64_OPS_PER_MATRIX:
        ops = FP64_OPS_PER_MATRIX[W["kind"]] + (BWD_FP64_OPS_REAL if W["form"] == "grad" else 0)
        fp64_peak = GB300_SMS * GB300_FP64_PER_SM_CLK * sm_max_mhz() / 1e3   # G op/s
        fp64_achieved = ops * n / (ms_per_step / 1e3) / 1e9
        # products of the method that the kernels run on the integer pipe
        # (counted in ops, the method's algorithmic count, not on the FP64 pipe)
        on_int = (8 if W["kind"] == "z" and W["form"] == "plain" else 0) + \
            (BWD_INT_PIPE_PRODUCTS_REAL if W["form"] == "grad" else 0)
        roofline = {"bound": "alu", "achieved": fp64_achieved, "peak": fp64_peak,
                    "unit": "G FP64 op/s", "frac": fp64_achieved / fp64_peak,
                    "traffic": traffic,
                    "note": f"FP64 pipe: {ops} FP64 add/mul/fma per matrix (the method's count; "
                            f"{on_int} of them products run on the integer pipe) x {n} per "
                            f"launch; peak derived: {GB300_SMS} SMs x {GB300_FP64_PER_SM_CLK} "
                            f"per clock x {sm_max_mhz():.0f} MHz",
                    "hbm": hbm}
    else:
        roofline = hbm
    line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": W["dtype"], "data": "synthetic",
            "config": {"workload": W["desc"], "n_per_gpu": n,
                       "l2": "inputs larger than L2 (>= 1 GiB per step)",
                       "launch": "block %d, mpt %d, unroll %d, waves %d" % S.get_launch(kind_launch),
                       "launch_from": ("given" if args.launch else
                                       "autotuner" if tuned else "default")},
            "roofline": roofline, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clk}
    if W["form"] == "tan64":
        line["config"]["tau_log2"] = TAN64_TAU_LOG2
    report = None
    if rank == 0 and world == 1 and not args.no_compare and args.workload == DEFAULT_WORKLOAD \
            and not args.n:
        del Ad, out
        torch.cuda.empty_cache()
        summary, prec = compare_precisions(torch, S, max(3, min(args.steps, 10)), args.warmup,
                                           stream)
        line["fp32_vs_fp64"] = summary
        # the comparison also as scalars in config, which records of the line
        # keep where they reduce nested keys to their names
        for k in ("fp64_matrices_per_s", "fp64_fp64_pipe_frac", "fp32_plain_matrices_per_s",
                  "fp32_plain_smin_err_max_u", "fp32_tan64_smax_err_max_u",
                  "fp32_tan64_smin_err_max_u", "fp32_tan64_double_fraction",
                  "fp32_rerun_matrices_per_s", "fp32_rerun_smin_err_max_u"):
            line["config"]["vs_" + k] = summary[k]
        line["config"]["compare"] = (
            "same n=2^26 inputs: FP64 %.1f G/s (%.2f of FP64 pipe); FP32 %.1f G/s (%.2f of HBM), "
            "sigma'_min err vs FP64 up to %.3g u; FP32 + FP64 tangent step %.1f G/s (%.2f of HBM), "
            "sigma'_max err <= %.1f u, sigma'_min <= %.1f u; FP32 + full FP64 re-run %.1f G/s, "
            "sigma'_min <= %.1f u (u = 2^-24)" % (
                summary["fp64_matrices_per_s"] / 1e9, summary["fp64_fp64_pipe_frac"],
                summary["fp32_plain_matrices_per_s"] / 1e9, summary["fp32_plain_hbm_frac"],
                summary["fp32_plain_smin_err_max_u"],
                summary["fp32_tan64_matrices_per_s"] / 1e9, summary["fp32_tan64_hbm_frac"],
                summary["fp32_tan64_smax_err_max_u"], summary["fp32_tan64_smin_err_max_u"],
                summary["fp32_rerun_matrices_per_s"] / 1e9, summary["fp32_rerun_smin_err_max_u"]))
        report = {"precision": prec,
                  "host_link": bench_host_link(torch, stream),
                  "complex128": bench_complex128(torch, S, stream),
                  "multi_batch": bench_multi(torch, S, stream),
                  "differentiation": bench_grad(torch, S, stream),
                  "variants": bench_variants(torch, S, stream),
                  "kogbetliantz_step": bench_kog(torch, S, stream)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, W)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        if report is not None:
            # the supplementary measurements: a file, or one JSON line on stderr
            if args.report:
                with open(args.report, "w") as f:
                    json.dump(report, f, indent=1)
            else:
                print(json.dumps({"report": report}), file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)


def run_multi_profile(args):
    """The multi-batch launch alone on the first K batches of the 2048-batch
    sequence (the Kogbetliantz batching workload), in one launch shape and
    grid, timed with CUDA events over --steps launches after --warmup; for
    comparing one block per tile with a persistent grid under a profiler."""
    import torch
    from paper_2005_07403_gb300 import inputs
    from paper_2005_07403_gb300 import svd2 as S
    lens, cplx = inputs.kog_batches()
    k = min(args.multi_batches, len(lens))
    lens, cplx = lens[:k], cplx[:k]
    dev = [inputs.normal_batch_device(int(n), 8 if c else 4, 5000 + i)
           for i, (n, c) in enumerate(zip(lens, cplx))]
    block, mpt, unroll = (int(x) for x in args.multi_shape.split(","))
    mb = S.MultiBatch(dev, block=block, mpt=mpt, unroll=unroll)
    stream = torch.cuda.current_stream()
    ms = time_steps(torch, lambda: mb.run(grid=args.multi_grid), args.steps, args.warmup, stream)
    total = int(lens.sum())
    nbytes = int(sum(n * (212 if c else 116) for n, c in zip(lens, cplx)))
    print(json.dumps({"multi_batches": k, "matrices": total, "complex_fraction": float(cplx.mean()),
                      "shape": [block, mpt, unroll], "grid": args.multi_grid, "tiles": mb.tiles,
                      "ms": ms, "matrices_per_s": total / (ms / 1e3),
                      "algorithmic_GBps": nbytes / (ms / 1e3) / 1e9}), flush=True)


def main():
    if "--sources-digest" in sys.argv:
        for w in KERNEL_SOURCES:
            print(w, sources_digest(w))
        return
    args = parse()
    if args.multi_batches > 0:
        run_multi_profile(args)
        return
    if args.grad:
        import torch
        from paper_2005_07403_gb300 import svd2 as S
        out = bench_grad(torch, S, torch.cuda.current_stream(), args.steps, args.warmup,
                         n=args.n or 2**22, only=args.grad)
        print(json.dumps({"differentiation": out}), flush=True)
        return
    if args.kog:
        import torch
        from paper_2005_07403_gb300 import svd2 as S
        out = bench_kog(torch, S, torch.cuda.current_stream(), args.steps, args.warmup,
                        only=args.kog, m_override=args.n)
        print(json.dumps({"kogbetliantz_step": out}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
