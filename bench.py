#!/usr/bin/env python3
"""Throughput of the transposition-free tensor contraction on GB300.

Default workload: the FP64 coupled-cluster-style contraction
    C[a,b,i,j] = 0.5 * sum_{c,d} A[c,a,d,b] * B[i,c,j,d] + 1.0 * C[a,b,i,j]
with a, b, c, d = 96 and i, j = 24 in general column-major layout (a 9216 x 576
x 9216 matrix product in disguise, 9.78e10 flops per step).  One step = one
tc_contract call (scatter-vector build + FP64 mainloop with fused epilogue).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun (N > 1) every rank runs an
independent replica of the workload (the contraction needs no exchange between
GPUs); `value` sums the work of all ranks over the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import paper_1607_00291_gb300 as tc  # noqa: E402
from paper_1607_00291_gb300 import _lib as L  # noqa: E402
from paper_1607_00291_gb300 import workloads as W  # noqa: E402

METRIC = "contraction TFLOP/s and % of tensor-pipe peak per precision, at stated error"
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cc4x4_f64",
                    choices=sorted(W.SPECS) + ["batch512", "tccg"] + sorted(W.PAPER_SHAPES))
    ap.add_argument("--mode", choices=["f64", "bf16x3", "bf16x6"], default=None,
                    help="override the workload's arithmetic")
    ap.add_argument("--access", choices=["auto", "box", "block", "scatter", "packed"],
                    default="auto",
                    help="tensor-core operand access: the library's choice (auto), TMA boxes "
                         "where tiles are boxes and "
                         "block-scatter gathers elsewhere (box), block-scatter gathers only "
                         "(block), element gathers only (scatter), or both operands packed "
                         "once before the mainloop (packed)")
    ap.add_argument("--profile", action="store_true",
                    help="after the timed region, run one more step between cudaProfilerStart "
                         "and cudaProfilerStop (for ncu --profile-from-start off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune-cache", default=None,
                    help="batch512: the autotuner's cache file (default: a file in the system's "
                         "temporary directory; the plans are tuned when it holds no record)")
    ap.add_argument("--no-ttgt", action="store_true", help="skip the TTGT comparison leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the secondary configurations (precision "
                         "form, forward + backward, batch) added to the line under 'configs'")
    return ap.parse_args()


# ---- process group ----------------------------------------------------------------

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks ------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- peaks ---------------------------------------------------------------------------

def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def fp64_peak_tflops() -> float:
    """FP64 denominator: cuBLAS DGEMM 4096^3 (best of 3) on this GPU, measured
    here outside the timed region (the pool's peak file carries no FP64 figure)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def mixed_roofline(per_problem, kernel_ms, pipe_peak, pipe_src, prods, kernel, traffic):
    """Roofline of a launch that runs several independent contractions.
    per_problem: (algorithmic bytes, flops) of each -- A and B read once, C
    written once; flops counted once (x `prods` products on the pipe).  Each
    problem's floor is the larger of its bytes at the measured copy bandwidth
    and its products at the pipe's peak; the line is bound by whichever of the
    two sums is larger, and `floors` gives the sum of the per-problem floors
    against the kernel time."""
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    t_hbm = [b / (hbm_peak * 1e9) * 1e3 for b, _ in per_problem]
    t_pipe = [prods * f / (pipe_peak * 1e12) * 1e3 for _, f in per_problem]
    nbytes = float(sum(b for b, _ in per_problem))
    flops = float(sum(f for _, f in per_problem))
    floor = sum(max(a, b) for a, b in zip(t_hbm, t_pipe))
    if sum(t_hbm) >= sum(t_pipe):
        ach, peak, unit, bound = nbytes / (kernel_ms * 1e-3) / 1e9, hbm_peak, "GB/s", "hbm"
        src, alg = "MEASURED_PEAKS.json hbm_gbs", f"{nbytes / 1e6:.1f} MB per launch (A, B read, C written once)"
    else:
        ach, peak, unit, bound = prods * flops / (kernel_ms * 1e-3) / 1e12, pipe_peak, "TFLOP/s", "tensor"
        src, alg = pipe_src, f"{flops:.4g} flops per launch (x{prods} products)"
    return {"bound": bound, "kernel": kernel, "achieved": round(ach, 5), "peak": round(peak, 5),
            "unit": unit, "frac": round(ach / peak, 4), "peak_source": src,
            "kernel_ms": round(kernel_ms, 4), "traffic": traffic, "algorithmic": alg,
            "floors": {"sum_floor_ms": round(floor, 4), "frac": round(floor / kernel_ms, 4),
                       "hbm_floor_ms": round(sum(t_hbm), 4), "pipe_floor_ms": round(sum(t_pipe), 4),
                       "note": "per problem the larger of its HBM floor and its pipe floor"}}


def profiled_step(args, fn):
    """--profile: one untimed step inside a profiler range, after the timed region."""
    if not args.profile:
        return
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    fn()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


KERNELS = {"packed": "k_pack+k_tcp", "gather": "k_tc", "box": "k_tc", "pair": "k_tc"}


def tc_forms(calls, mode):
    """The tensor-core mainloop form of each call (A, labA, B, labB, C, labC,
    ...) under the current settings, or None in the FP64 mode."""
    if mode == "f64":
        return None
    return [tc.operand_form(c[0], c[1], c[2], c[3], c[4], c[5], mode) for c in calls]


def kernel_name(mode, forms):
    if mode == "f64":
        return "k_f64"
    return "+".join(sorted({KERNELS[f] for f in forms}))


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source
    is unchanged since the counters were taken; else None."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except OSError:
        return None
    e = t.get(f"{kernel}:{workload}")
    if not e:
        return None
    src = os.path.join(ROOT, "paper_1607_00291_gb300", "csrc", e["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return e["dram_bytes_per_launch"] if h == e["source_sha256_16"] else None


# ---- workload -------------------------------------------------------------------------

def bundle_lengths(spec):
    """m, n, k of a workload: the products of the extents of the labels that A
    and C, B and C, A and B share (Section 4); computed from the labels alone,
    so that the reference arm never loads the product library."""
    prod = lambda labs: int(np.prod([spec.ext[x] for x in labs], dtype=np.int64))  # noqa: E731
    a, b, c = set(spec.labA), set(spec.labB), set(spec.labC)
    return prod(a & c), prod(b & c), prod(a & b)


def workload_config(spec, extra=None):
    m, n, k = bundle_lengths(spec)
    desc = (f"{spec.name}: {spec.labC} <- {spec.labA}.{spec.labB}, extents "
            + ",".join(f"{k}={v}" for k, v in sorted(spec.ext.items()))
            + f", column-major, alpha={spec.alpha}, beta={spec.beta}, mode={spec.mode}")
    cfg = {"workload": desc, "m": m, "n": n, "k": k, "mode": spec.mode}
    if extra:
        cfg.update(extra)
    return cfg


def _cm(spec, lab):
    acc, st = 1, []
    for x in lab:
        st.append(acc)
        acc *= spec.ext[x]
    return tuple(spec.ext[x] for x in lab), tuple(st)


def to_device(t, dtype):
    return torch.empty_strided(t.shape, t.stride(), dtype=dtype, device="cuda").copy_(t.to(dtype))


def host_bytes(spec):
    es = torch.tensor([], dtype=spec.dtype).element_size()
    n = lambda lab: int(np.prod(spec.shape(lab)))
    return es * n(spec.labA), es * n(spec.labB), es * n(spec.labC)


# ---- TTGT comparison (transpose-transpose-GEMM-transpose, Section 3) ----------------------

class CublasBf16x9:
    """cuBLAS's FP32 GEMM emulated on the bf16 tensor cores (each FP32 input
    split into three bf16 values, nine products: CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
    emulation forced), called through its C API on torch's stream; `unavailable`
    holds the reason when the library or the compute type is missing."""
    COMPUTE_32F_EMULATED_16BFX9, EMULATION_EAGER, R_32F, OP_N, GEMM_DEFAULT = 78, 2, 0, 0, -1

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.unavailable = None
        self.handle = ctypes.c_void_p()
        try:
            torch.matmul(torch.ones(8, 8, device="cuda"), torch.ones(8, 8, device="cuda"))
            self.lib = ctypes.CDLL("libcublas.so.13")
            if self.lib.cublasCreate_v2(ctypes.byref(self.handle)) != 0:
                raise RuntimeError("cublasCreate failed")
            if self.lib.cublasSetEmulationStrategy(self.handle, self.EMULATION_EAGER) != 0:
                raise RuntimeError("cublasSetEmulationStrategy failed")
        except (OSError, AttributeError, RuntimeError) as e:
            self.unavailable = str(e).splitlines()[0][:120]

    def close(self):
        torch.cuda.synchronize()
        if self.handle.value:
            self.lib.cublasDestroy_v2(self.handle)
            self.handle = self.ct.c_void_p()

    def matmul(self, A, B):
        """A (m x k) @ B (k x n), both row-major FP32 on the device, into a new tensor."""
        ct = self.ct
        m, k = A.shape
        n = B.shape[1]
        C = torch.empty(m, n, dtype=torch.float32, device=A.device)
        self.lib.cublasSetStream_v2(self.handle, ct.c_void_p(torch.cuda.current_stream().cuda_stream))
        one, zero = ct.c_float(1.0), ct.c_float(0.0)
        # row-major C = A B is column-major C^T = B^T A^T
        st = self.lib.cublasGemmEx(self.handle, self.OP_N, self.OP_N, n, m, k, ct.byref(one),
                                   ct.c_void_p(B.data_ptr()), self.R_32F, n,
                                   ct.c_void_p(A.data_ptr()), self.R_32F, k, ct.byref(zero),
                                   ct.c_void_p(C.data_ptr()), self.R_32F, n,
                                   self.COMPUTE_32F_EMULATED_16BFX9, self.GEMM_DEFAULT)
        if st != 0:
            raise RuntimeError(f"cublasGemmEx (BF16x9 emulation) returned status {st}")
        return C


def ttgt_contract(A, labA, B, labB, C, labC, alpha, beta, gemm=torch.matmul):
    """The contraction the way the paper's TTGT baseline computes it: copy A
    and B into matrix order (I, P) and (P, J), one library GEMM (cuBLAS via
    torch.matmul, or `gemm`), then a strided copy of the product back into
    C's layout.  Returns the bytes of the temporary matrices."""
    I = [x for x in labC if x in labA]
    J = [x for x in labC if x in labB]
    P = [x for x in labA if x in labB]
    ext = {x: n for lab, T in ((labA, A), (labB, B), (labC, C)) for x, n in zip(lab, T.shape)}
    size = lambda xs: int(np.prod([ext[x] for x in xs])) if xs else 1  # noqa: E731
    At = A.permute(*[labA.index(x) for x in I + P]).contiguous().reshape(size(I), size(P))
    Bt = B.permute(*[labB.index(x) for x in P + J]).contiguous().reshape(size(P), size(J))
    Ct = gemm(At, Bt)
    back = Ct.reshape([ext[x] for x in I + J]).permute(*[(I + J).index(x) for x in labC])
    if beta == 0.0:
        C.copy_(back).mul_(alpha)
    else:
        C.mul_(beta).add_(back, alpha=alpha)
    return (At.numel() + Bt.numel() + Ct.numel()) * At.element_size()


def time_ttgt(problems, warm: int, K: int, flops: float, ws: int, gemm=torch.matmul):
    """Device time of the TTGT form of one step (all `problems`), with the
    temporaries' bytes and the time of each problem; FP32 GEMMs in full FP32
    (no TF32) unless `gemm` says otherwise."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        extra = 0
        for _ in range(warm):
            extra = sum(ttgt_contract(*p, gemm=gemm) for p in problems)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(problems) + 1)] for _ in range(K)]
        for i in range(K):
            for j, p in enumerate(problems):
                ev[i][j].record()
                ttgt_contract(*p, gemm=gemm)
            ev[i][-1].record()
        torch.cuda.synchronize()
        ms = max_over_ranks(float(np.mean([row[0].elapsed_time(row[-1]) for row in ev])), ws)
        per = [round(float(np.mean([row[j].elapsed_time(row[j + 1]) for row in ev])), 4)
               for j in range(len(problems))]
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return {"value": round(ws * flops / (ms * 1e-3) / 1e12, 5), "unit": "TFLOP/s",
            "ms_per_step": round(ms, 4), "ms_per_problem": per, "temporary_bytes": int(extra),
            "what": "torch permute().contiguous() + torch.matmul (cuBLAS, FP64 or full FP32) + "
                    "strided copy back, same inputs, device time"}


def ttgt_legs(problems, warm, K, flops, ws, ms_ours, fp32):
    """The TTGT comparison line: full-precision GEMM, and for FP32 data also
    cuBLAS's BF16x9-emulated FP32 GEMM (the vendor's split-bf16 tensor-core
    path) between the same transposition copies."""
    tt = time_ttgt(problems, warm, K, flops, ws)
    tt["ours_over_ttgt_speed"] = round(tt["ms_per_step"] / ms_ours, 3)
    if fp32:
        em = CublasBf16x9()
        if em.unavailable:
            tt["bf16x9"] = {"unavailable": em.unavailable}
        else:
            try:
                t9 = time_ttgt(problems, warm, K, flops, ws, gemm=em.matmul)
                tt["bf16x9"] = {"ms_per_step": t9["ms_per_step"], "value": t9["value"],
                                "ours_over_ttgt_speed": round(t9["ms_per_step"] / ms_ours, 3),
                                "what": "the same TTGT step with cublasGemmEx in "
                                        "CUBLAS_COMPUTE_32F_EMULATED_16BFX9 (emulation forced)"}
            except RuntimeError as e:
                tt["bf16x9"] = {"unavailable": str(e)[:120]}
            finally:
                em.close()
    return tt


# ---- CPU oracle baseline -----------------------------------------------------------------

def oracle_sample(spec, host, seconds: float, out_count=None):
    """Time the CPU oracle on the first S output elements of the workload, S
    chosen to take about `seconds`.  Returns (flops, seconds, S, cores, C, mag)."""
    import oracle
    a, b = host["A"].numpy(), host["B"].numpy()
    k = 1
    for x in set(spec.labA) & set(spec.labB):
        k *= spec.ext[x]
    cores = oracle.num_threads()
    c = np.array(host["C"].numpy(), copy=True)
    probe = min(max(cores * 8, 64), c.size)
    t0 = time.perf_counter()
    oracle.contract_(spec.alpha, a, spec.labA, b, spec.labB, spec.beta, c, spec.labC, mag=False,
                     begin=0, end=probe)
    dt = time.perf_counter() - t0
    S = out_count or int(min(c.size, max(probe, probe * seconds / max(dt, 1e-6))))
    c = np.array(host["C"].numpy(), copy=True)
    t0 = time.perf_counter()
    mag = oracle.contract_(spec.alpha, a, spec.labA, b, spec.labB, spec.beta, c, spec.labC,
                           begin=0, end=S)
    dt = time.perf_counter() - t0
    return 2.0 * k * S, dt, S, cores, c, mag


def err_windows(numel: int, k: int, seconds: float, seed: int, extra=()):
    """Windows [b, e) of output elements (colexicographic over C's dims) for an
    oracle check of about `seconds` on the host cores: the first and the last
    elements, four seeded windows in between, and any `extra` windows."""
    budget = int(max(64, min(numel, 3.0e9 * seconds / (2.0 * max(k, 1)))))
    w = max(1, budget // 6)
    rng = np.random.default_rng(seed)
    wins = [(0, min(w, numel)), (max(0, numel - w), numel)]
    for _ in range(4):
        b = int(rng.integers(0, max(1, numel - w)))
        wins.append((b, min(numel, b + w)))
    wins.extend(extra)
    return wins


def oracle_err(alpha, hA, labA, hB, labB, beta, hC0, labC, got, windows):
    """Max normalised error |got - oracle| / mag of `got` (the device result,
    FP64 numpy array of C's shape) over the output windows.  Returns (err,
    elements checked)."""
    import oracle
    a, b = np.asarray(hA, dtype=np.float64), np.asarray(hB, dtype=np.float64)
    gflat = np.asarray(got, dtype=np.float64).ravel(order="F")
    err, count = 0.0, 0
    for (lo, hi) in windows:
        if hi <= lo:
            continue
        c = np.array(np.asarray(hC0, dtype=np.float64), copy=True)
        mag = oracle.contract_(alpha, a, labA, b, labB, beta, c, labC, begin=lo, end=hi)
        r = c.ravel(order="F")[lo:hi]
        m = mag.ravel(order="F")[lo:hi] if mag.ndim else mag.reshape(1)
        g = gflat[lo:hi]
        err = max(err, float(np.max(np.abs(g - r) / np.maximum(m, 1e-300))))
        count += hi - lo
    return err, count


# ---- our arm ---------------------------------------------------------------------------------

def batch_roofline(probs, dt, mode, kms, kernel, traffic):
    """The batch's roofline: most of its 512 problems have a short side, so
    their bytes, not their products, bound them (mixed_roofline)."""
    if mode == "f64":
        peak, src, prods = fp64_peak_tflops(), "cuBLAS DGEMM 4096^3 measured in this run", 1
    else:
        peak = measured_peaks().get("bf16_tflops", 1900.0)
        src, prods = "MEASURED_PEAKS.json bf16_tflops (burst)", (3 if mode == "bf16x3" else 6)
    es = torch.tensor([], dtype=dt).element_size()
    per = [(es * sum(int(np.prod([p.ext[x] for x in lab])) for lab in (p.labA, p.labB, p.labC)), p.flops())
           for p in probs]
    return mixed_roofline(per, kms, peak, src, prods, kernel, traffic)


def run_batch(args, ws, rank, local):
    """512 independent contractions (ranks 2-6, extents 8..64, random layouts)
    as one planned batch, replayed from a CUDA graph: scatter builder +
    persistent mainloop (+ split reduction) per step."""
    mode = args.mode or "f64"
    lean = getattr(args, "lean", False)
    dt = torch.float64 if mode == "f64" else torch.float32
    warm, K = max(3, args.warmup), max(1, args.steps)
    probs = W.batch_problems(seed=1004)
    host = [W.make_random_inputs(p, seed=5000 + i, dtype=dt) for i, p in enumerate(probs)]
    dev = [(to_device(h["A"], dt), p.labA, to_device(h["B"], dt), p.labB, to_device(h["C"], dt),
            p.labC, 1.0, 0.0) for p, h in zip(probs, host)]
    flops = sum(p.flops() for p in probs)
    lib = L.lib()
    # tuned plans: tile per shape class and the k-split balance of the batch
    import tempfile
    cache = args.autotune_cache or os.environ.get("TC_AUTOTUNE_CACHE") or \
        os.path.join(tempfile.gettempdir(), "tc_autotune_cache.txt")
    os.environ["TC_AUTOTUNE_CACHE"] = cache
    t_plan = time.perf_counter()
    plan = tc.Plan(dev, mode=mode)
    bkernel = {"f64": "k_f64_batched", "packed": "k_pack+k_tcp", "gather": "k_tc"}[plan.form]
    t_plan = time.perf_counter() - t_plan
    cfgs = [plan.config(i) for i in range(len(dev))]
    tuned = {"cache": cache, "plan_create_s": round(t_plan, 2), "balance_divisor": cfgs[0]["balance"],
             "split_problems": sum(c["splits"] > 1 for c in cfgs),
             "tiles": {f"{a}x{b}": n for (a, b), n in
                       __import__("collections").Counter((c["bm"], c["bn"]) for c in cfgs).items()}}
    plan.execute()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.execute()
    for _ in range(warm):
        graph.replay()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier(ws)
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.tc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    e0.record(cur)
    for _ in range(K):
        graph.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if not lean:
        profiled_step(args, graph.replay)
    # graph replays launch libtc's kernels without passing through the library;
    # count them from one direct execution
    l0 = lib.tc_launch_count()
    plan.execute()
    torch.cuda.synchronize()
    per_step = lib.tc_launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1) / K, ws)
    # the mainloop alone, timed with events around it
    ka, kb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ka.record(); kb.record(); torch.cuda.synchronize()
    kms = []
    for _ in range(3):
        lib.tc_set_mainloop_events(L.c_vp(ka.cuda_event), L.c_vp(kb.cuda_event))
        plan.execute()
        torch.cuda.synchronize()
        kms.append(ka.elapsed_time(kb))
    kms = max_over_ranks(min(kms), ws)
    err_code = tc.device_error()
    # oracle check of sampled outputs: sixteen problems spread over the batch,
    # windows of each (its first and last elements among them)
    check = None
    if lean and rank == 0:
        t0 = time.perf_counter()
        err, cnt = 0.0, 0
        for i in range(0, len(probs), max(1, len(probs) // 16)):
            p, h = probs[i], host[i]
            got = dev[i][4].cpu().to(torch.float64).numpy()
            kk = int(round(p.flops() / 2.0 / max(1, got.size)))
            e, c = oracle_err(1.0, h["A"].numpy(), p.labA, h["B"].numpy(), p.labB, 0.0, h["C"].numpy(),
                              p.labC, got, err_windows(got.size, kk, 0.25, seed=77 + i))
            err, cnt = max(err, e), cnt + c
        check = {"max_normalised_err_vs_oracle": err, "elements_checked": cnt,
                 "sample": "16 problems spread over the batch: first, last and 4 seeded windows of "
                           f"outputs each ({time.perf_counter() - t0:.1f} s of oracle time)"}
    if lean:
        plan.close()
        line = {"ms_per_step": round(ms, 4), "value": round(ws * flops / (ms * 1e-3) / 1e12, 5),
                "unit": "TFLOP/s", "steps": K, "warmup": warm, "total_flops": flops,
                "gpu_launches_per_step": int(per_step), "device_error": err_code, "autotune": tuned}
        line["roofline"] = batch_roofline(probs, dt, mode, kms, bkernel, traffic_for(bkernel, f"batch512_{mode}"))
        if check:
            line["oracle_check"] = check
        return line
    # end to end: inputs from pinned host memory, outputs back, every step
    pins = [tuple(torch.empty_strided(h[x].shape, h[x].stride(), dtype=dt).pin_memory().copy_(h[x])
                  for x in "ABC") for h in host]
    outs = [torch.empty_strided(h["C"].shape, h["C"].stride(), dtype=dt).pin_memory() for h in host]
    bi = sum(sum(t.numel() * t.element_size() for t in pp) for pp in pins)
    bo = sum(t.numel() * t.element_size() for t in outs)

    def e2e_step():
        for d, pp in zip(dev, pins):
            d[0].copy_(pp[0], non_blocking=True)
            d[2].copy_(pp[1], non_blocking=True)
            d[4].copy_(pp[2], non_blocking=True)
        plan.execute()
        for d, o in zip(dev, outs):
            o.copy_(d[4], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(max(1, K // 2)):
        e2e_step()
    f1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / max(1, K // 2), ws)
    line = {
        "metric": METRIC, "value": round(ws * flops / (ms * 1e-3) / 1e12, 5), "unit": "TFLOP/s",
        "n_gpus": ws, "steps": K, "warmup": warm, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if mode == "f64" else f"f32 data, {mode} products, f32 accumulate",
        "data": "synthetic (seeded uniform[-1,1]; random labels, ranks, extents 8..64, permuted dense layouts)",
        "config": {"workload": f"batch512: 512 independent contractions, d_P 1-3, ranks 2-6, extents 8..64, "
                               f"one CUDA-graph replay of a planned batch, mode={mode}",
                   "total_flops": flops, "autotune": tuned,
                   "l2": "inputs larger than L2 (%.2f GB)" % (bi / 1e9), "parallelism": f"replicas x{ws}"},
        "clocks": clk,
        "e2e": {"value": round(ws * flops / (e2e_ms * 1e-3) / 1e12, 5), "unit": "TFLOP/s",
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": int(per_step * K),
        "roofline": batch_roofline(probs, dt, mode, kms, bkernel, traffic_for(bkernel, f"batch512_{mode}")),
        "device_error": err_code,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        fl = 0.0
        i = 0
        while time.perf_counter() - t0 < 10.0 and i < len(probs):
            p, h = probs[i], host[i]
            c = np.array(h["C"].numpy(), copy=True)
            oracle.contract_(1.0, h["A"].numpy(), p.labA, h["B"].numpy(), p.labB, 0.0, c, p.labC,
                             mag=False)
            fl += p.flops()
            i += 1
        sec = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(fl / sec / 1e12, 8), "unit": "TFLOP/s",
                                "cores": __import__("oracle").num_threads(), "kind": "oracle",
                                "sample": f"the first {i} of 512 problems in full, {sec:.1f} s"}
    plan.close()
    return line


def run_calls(args, ws, rank, local, *, calls, inputs, outputs, flops, mode, desc, cfg_extra,
              hbm_bytes=None, cpu=None, checks=None):
    """Time one step = the tc_contract `calls` (tuples A, labA, B, labB, C, labC, alpha,
    beta) in order, with the same line as run_ours.  `inputs` / `outputs`: the
    device tensors a step reads from / returns to the host (for e2e).
    `hbm_bytes`: algorithmic DRAM bytes per step when the step is HBM-bound
    (roofline against the measured copy bandwidth), else the tensor/FP64 pipe
    is the denominator.  `cpu`: (spec, host arrays, index of the call) for the
    oracle baseline.  `checks`: (index of the call, host A, host B, host initial
    C) per output to compare with the oracle on sampled windows (lean lines).
    With args.lean the line holds only the timed numbers and the oracle check
    (no end-to-end leg, TTGT or CPU baseline)."""
    lean = getattr(args, "lean", False)
    warm, K = max(3, args.warmup), max(1, args.steps)
    C0 = [c[4].clone() for c in calls]
    works = [torch.empty(max(1, tc.workspace_size(c[0], c[1], c[2], c[3], c[4], c[5], mode=mode)),
                         dtype=torch.uint8, device="cuda") for c in calls]
    lib = L.lib()

    def step():
        for c, w in zip(calls, works):
            tc.contract(c[0], c[1], c[2], c[3], c[4], c[5], alpha=c[6], beta=c[7], mode=mode, workspace=w)

    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
           for _ in range(K)]
    for row in kev:
        for a, b in row:
            a.record()
            b.record()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.tc_launch_count()
    cev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(K)]
    e0.record()
    for i in range(K):
        for j, ((c, w), (ka, kb)) in enumerate(zip(zip(calls, works), kev[i])):
            cev[i][j].record()
            lib.tc_set_mainloop_events(L.c_vp(ka.cuda_event), L.c_vp(kb.cuda_event))
            tc.contract(c[0], c[1], c[2], c[3], c[4], c[5], alpha=c[6], beta=c[7], mode=mode, workspace=w)
        cev[i][-1].record()
    e1.record()
    torch.cuda.synchronize()
    launches = lib.tc_launch_count() - launches0
    call_ms = [round(float(np.mean([row[j].elapsed_time(row[j + 1]) for row in cev])), 4)
               for j in range(len(calls))]
    clk = clocks.stop()
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1) / K, ws)
    kms = max_over_ranks(float(np.mean([sum(a.elapsed_time(b) for a, b in row) for row in kev])), ws)
    if not lean:
        profiled_step(args, step)
    per_call = [round(float(np.mean([row[j][0].elapsed_time(row[j][1]) for row in kev])), 4)
                for j in range(len(calls))]
    err_code = tc.device_error()
    check = None
    if checks and rank == 0:
        for c, c0 in zip(calls, C0):
            c[4].copy_(c0)
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        check = {"per_output": []}
        for j, hA, hB, hC0 in checks:
            c = calls[j]
            got = c[4].cpu().to(torch.float64).numpy()
            kk = int(round(np.prod(hA.shape) * np.prod(hB.shape) / max(1, got.size))) if got.size else 1
            kk = int(round(np.sqrt(max(kk, 1))))
            e, n = oracle_err(c[6], hA, c[1], hB, c[3], c[7], hC0, c[5], got,
                              err_windows(got.size, kk, 1.0 / len(checks), seed=31 + j))
            check["per_output"].append({"output": c[5], "max_normalised_err_vs_oracle": e,
                                        "elements_checked": n})
        check["max_normalised_err_vs_oracle"] = max(x["max_normalised_err_vs_oracle"]
                                                     for x in check["per_output"])
        check["sample"] = ("per output: its first and last elements and 4 seeded windows "
                           f"({time.perf_counter() - t0:.1f} s of oracle time)")

    if lean:
        prods = 1 if mode == "f64" else (3 if mode == "bf16x3" else 6)
        line = {"ms_per_step": round(ms, 4), "value": round(ws * flops / (ms * 1e-3) / 1e12, 5),
                "unit": "TFLOP/s", "steps": K, "warmup": warm, "flops_per_step": flops,
                "gpu_launches": int(launches), "device_error": err_code}
        if hbm_bytes is not None:
            mp = measured_peaks()
            peak_v = mp.get("hbm_gbs", 6800.0)
            ach = hbm_bytes / (kms * 1e-3) / 1e9
            line["roofline"] = {"bound": "hbm", "achieved": round(ach, 3), "unit": "GB/s",
                                "peak": peak_v, "frac": round(ach / peak_v, 4),
                                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if mp else "fallback 6.8 TB/s",
                                "algorithmic": f"{hbm_bytes / 1e6:.1f} MB per step over {len(calls)} launches"}
        else:
            if mode == "f64":
                peak_v, src = fp64_peak_tflops(), "cuBLAS DGEMM 4096^3 measured in this run"
            else:
                mp = measured_peaks()
                peak_v = mp.get("bf16_tflops", 1900.0)
                src = "MEASURED_PEAKS.json bf16_tflops (burst)" if mp else "fallback 1.9 PFLOP/s bf16"
            ach = prods * flops / (kms * 1e-3) / 1e12
            line["roofline"] = {"bound": "tensor", "achieved": round(ach, 5), "unit": "TFLOP/s",
                                "peak": round(peak_v, 5), "frac": round(ach / peak_v, 4), "peak_source": src,
                                "algorithmic": f"{flops:.4g} flops per step"
                                               + (f" (x{prods} bf16 products)" if mode != "f64" else "")}
        forms = tc_forms(calls, mode)
        kname = kernel_name(mode, forms)
        if forms:
            line["forms"] = forms
        line["roofline"].update({"kernel": kname, "kernel_ms": round(kms, 4), "kernel_ms_per_call": per_call,
                                 "traffic": traffic_for(kname, getattr(args, "traffic_key", ""))})
        line["call_ms"] = call_ms
        if check:
            line["oracle_check"] = check
        return line

    # end to end through the public API: the step's inputs from pinned host
    # memory, its outputs back
    pins = [torch.empty_strided(t.shape, t.stride(), dtype=t.dtype).pin_memory().copy_(t.cpu())
            for t in inputs]
    outs = [torch.empty_strided(t.shape, t.stride(), dtype=t.dtype).pin_memory() for t in outputs]
    bi = sum(t.numel() * t.element_size() for t in pins)
    bo = sum(t.numel() * t.element_size() for t in outs)

    def e2e_step():
        for t, h in zip(inputs, pins):
            t.copy_(h, non_blocking=True)
        step()
        for t, o in zip(outputs, outs):
            o.copy_(t, non_blocking=True)

    # many gigabytes per step (the benchmark strings): fewer end-to-end steps
    ew, ek = (1, min(K, 3)) if bi + bo > 4e9 else (warm, K)
    for _ in range(ew):
        e2e_step()
    torch.cuda.synchronize()
    barrier(ws)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(ek):
        e2e_step()
    f1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / ek, ws)

    prods = 1 if mode == "f64" else (3 if mode == "bf16x3" else 6)
    forms = tc_forms(calls, mode)
    kname = kernel_name(mode, forms)
    if hbm_bytes is not None:
        mp = measured_peaks()
        peak_v = mp.get("hbm_gbs", 6800.0)
        peak_src = "MEASURED_PEAKS.json hbm_gbs" if mp else "fallback 6.8 TB/s"
        roof = {"bound": "hbm", "achieved": round(hbm_bytes / (kms * 1e-3) / 1e9, 3), "unit": "GB/s",
                "algorithmic": f"{hbm_bytes / 1e6:.1f} MB per step (each operand read once, each "
                               f"output written once) over {len(calls)} launches"}
    else:
        if mode == "f64":
            peak_v = fp64_peak_tflops()
            peak_src = "cuBLAS DGEMM 4096^3 measured in this run (no FP64 entry in MEASURED_PEAKS.json)"
        else:
            mp = measured_peaks()
            peak_v = mp.get("bf16_tflops", 1900.0)
            peak_src = "MEASURED_PEAKS.json bf16_tflops (burst)" if mp else "fallback 1.9 PFLOP/s bf16"
        roof = {"bound": "tensor", "achieved": round(prods * flops / (kms * 1e-3) / 1e12, 5),
                "unit": "TFLOP/s",
                "algorithmic": f"{flops:.4g} flops per step over {len(calls)} launches"
                               + (f" (x{prods} bf16 products)" if mode != "f64" else "")}
    roof.update({"kernel": kname, "peak": round(peak_v, 5), "frac": round(roof["achieved"] / peak_v, 4),
                 "peak_source": peak_src, "kernel_ms": round(kms, 4), "kernel_ms_per_call": per_call,
                 "traffic": None})
    cfg = {"workload": desc}
    cfg.update(cfg_extra)
    cfg["parallelism"] = f"replicas x{ws}"
    roof["call_ms"] = call_ms
    line = {
        "metric": METRIC, "value": round(ws * flops / (ms * 1e-3) / 1e12, 5), "unit": "TFLOP/s",
        "n_gpus": ws, "steps": K, "warmup": warm, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if mode == "f64" else f"f32 data, {mode} products, f32 accumulate",
        "data": "synthetic (seeded, layouts of the workload; see config)",
        "config": cfg, "clocks": clk,
        "e2e": {"value": round(ws * flops / (e2e_ms * 1e-3) / 1e12, 5), "unit": "TFLOP/s",
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": int(launches), "roofline": roof, "device_error": err_code,
    }
    if forms:
        line["forms"] = forms
    if not args.no_ttgt:
        for c, c0 in zip(calls, C0):
            c[4].copy_(c0)
        tt = ttgt_legs(calls, warm, K, flops, ws, ms, mode != "f64")
        tt["ours_workspace_bytes"] = int(sum(w.numel() for w in works))
        line["ttgt"] = tt
    if cpu is not None and rank == 0 and ws == 1 and not args.no_cpu_baseline:
        spec0, h0, ci = cpu
        for c, c0 in zip(calls, C0):
            c[4].copy_(c0)
        step()
        torch.cuda.synchronize()
        fl, sec, S, cores, cref, mag = oracle_sample(spec0, h0, seconds=12.0)
        got = calls[ci][4].cpu().to(torch.float64).numpy()
        # the oracle's first S elements: colexicographic over C's own dims
        g = got.ravel(order="F")[:S]
        r = cref.ravel(order="F")[:S]
        m = mag.ravel(order="F")[:S]
        err = float(np.max(np.abs(g - r) / np.maximum(m, 1e-300)))
        line["cpu_baseline"] = {"value": round(fl / sec / 1e12, 8), "unit": "TFLOP/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"first {S} output elements of {spec0.labC} <- "
                                          f"{spec0.labA}.{spec0.labB} (all k terms each), {sec:.1f} s "
                                          f"on {cores} host threads",
                                "max_normalised_err_gpu_vs_oracle": err}
    if check:
        line["oracle_check"] = check
    return line


def run_paper(args, ws, rank, local):
    """Section 9's randomly generated contractions of one matrix shape (square
    m = n = k, or rank-k m = n >> k): three seeded contractions, 1-3 dims per
    bundle, random label and storage orders; one step = the three tc_contract
    calls.  Effective lengths from the flops actually performed."""
    shape = W.PAPER_SHAPES[args.workload]
    mode = args.mode or "f64"
    dt = torch.float64 if mode == "f64" else torch.float32
    probs = W.paper_problems(args.workload)
    host = [W.make_random_inputs(p, seed=shape["seed"] * 10 + i, dtype=dt) for i, p in enumerate(probs)]
    calls = [(to_device(h["A"], dt), p.labA, to_device(h["B"], dt), p.labB, to_device(h["C"], dt),
              p.labC, 1.0, 0.0) for p, h in zip(probs, host)]
    flops = sum(p.flops() for p in probs)
    square = shape["m"] == shape["n"] == shape["k"]
    eff = [round(W.effective_square(p.flops()) if square
                 else W.effective_rank_k(p.flops(), shape["m"], shape["n"]), 1) for p in probs]
    desc = (f"{args.workload}: {len(probs)} random contractions shaped like m={shape['m']}, "
            f"n={shape['n']}, k={shape['k']} (1-3 dims per bundle, random label and storage "
            f"orders, seed {shape['seed']}): " + "; ".join(
                f"{p.labC} <- {p.labA}.{p.labB}" for p in probs) + f"; mode={mode}")
    extra = {"effective_lengths": eff,
             "extents": [{str(k): v for k, v in p.ext.items()} for p in probs],
             "l2": "operands larger than L2" if max(c[0].numel() * c[0].element_size() for c in calls)
                   > L2_BYTES else "operands smaller than L2"}
    p0 = probs[0]
    spec0 = W.Spec(args.workload, p0.labA, p0.labB, p0.labC, {str(k): v for k, v in p0.ext.items()},
                   dt, 1.0, 0.0)
    return run_calls(args, ws, rank, local, calls=calls,
                     inputs=[t for c in calls for t in (c[0], c[2], c[4])], outputs=[c[4] for c in calls],
                     flops=flops, mode=mode, desc=desc, cfg_extra=extra, cpu=(spec0, host[0], 0))


# The paper's BSMTC on one Haswell core for the benchmark strings (GFLOP/s,
# Section 9.3's benchmark figure, single-core panel), in the order of
# W.TCCG_STRINGS: context only -- the paper's extents are not known here, and
# the hardware is a CPU core.
PAPER_BSMTC_1CORE_GFLOPS = [3.67, 3.63, 2.32, 2.03, 6.77, 6.34, 17.25, 21.99, 20.68, 20.69, 17.33,
                            19.84, 27.52, 27.85, 23.32, 28.51, 27.85, 25.62, 36.45, 37.37, 42.57,
                            40.70, 41.75, 40.32]


def run_tccg(args, ws, rank, local):
    """The Tensor Contraction Benchmark's 24 contraction strings (Section 9.3)
    with synthetic extents (every index of a contraction the same extent, about
    2^34 flops each; column-major; uniform[-1,1], drawn on the device from a
    seed); one step = the 24 tc_contract calls.  Per string: our time, the
    TTGT form's time and the ratio, beside the paper's single-core BSMTC rate."""
    mode = args.mode or "f64"
    lean = getattr(args, "lean", False)
    dt = torch.float64 if mode == "f64" else torch.float32
    probs = W.tccg_problems()
    dev = [W.make_random_inputs_on(p, seed=2000 + i, dtype=dt, device="cuda") for i, p in enumerate(probs)]
    calls = [(d["A"], p.labA, d["B"], p.labB, d["C"], p.labC, 1.0, 0.0) for p, d in zip(probs, dev)]
    flops = sum(p.flops() for p in probs)
    desc = (f"tccg: the 24 contraction strings of the paper's Tensor Contraction Benchmark figure "
            f"(C-A-B), synthetic extents (one extent per contraction, e = round((2^33)^(1/L)) for "
            f"L indices: about 2^34 flops each), column-major, uniform[-1,1]; mode={mode}")
    extra = {"strings": W.TCCG_STRINGS, "extents": [p.ext[p.labC[0]] for p in probs],
             "l2": "operands larger than L2 in most strings", "mode": mode}
    host = lambda i: {k: v.cpu().double() for k, v in dev[i].items()}  # noqa: E731
    checks = None
    if lean:
        # every third string (eight of them, both ends of the figure included)
        checks = []
        for i in range(0, len(probs), 3):
            h = host(i)
            checks.append((i, h["A"].numpy(), h["B"].numpy(), np.zeros(tuple(dev[i]["C"].shape), order="F")))
    p0 = probs[0]
    spec0 = W.Spec("tccg", p0.labA, p0.labB, p0.labC, dict(p0.ext), dt, 1.0, 0.0)
    line = run_calls(args, ws, rank, local, calls=calls,
                     inputs=[t for c in calls for t in (c[0], c[2], c[4])], outputs=[c[4] for c in calls],
                     flops=flops, mode=mode, desc=desc, cfg_extra=extra,
                     cpu=None if lean else (spec0, host(0), 0), checks=checks)
    call_ms = line.get("call_ms") or line["roofline"].get("call_ms")
    kms = line["roofline"].get("kernel_ms_per_call") or call_ms
    tt = (line.get("ttgt") or {}).get("ms_per_problem")
    # each string's floor: its algorithmic bytes (A and B read once, C written
    # once) at the measured copy bandwidth, or its products at the pipe's peak
    mp = measured_peaks()
    hbm_peak = mp.get("hbm_gbs", 6800.0)
    es = 8 if mode == "f64" else 4
    if mode == "f64":
        pipe_peak, prods = fp64_peak_tflops(), 1
    else:
        pipe_peak, prods = mp.get("bf16_tflops", 1900.0), (3 if mode == "bf16x3" else 6)
    rows = []
    for i, (s_, p) in enumerate(zip(W.TCCG_STRINGS, probs)):
        nbytes = es * sum(int(np.prod([p.ext[x] for x in lab])) for lab in (p.labA, p.labB, p.labC))
        t_hbm = nbytes / (hbm_peak * 1e9) * 1e3
        t_pipe = prods * p.flops() / (pipe_peak * 1e12) * 1e3
        floor = max(t_hbm, t_pipe)
        r = {"string": s_, "extent": p.ext[p.labC[0]], "ms": call_ms[i], "kernel_ms": kms[i],
             "tflops": round(p.flops() / (call_ms[i] * 1e-3) / 1e12, 4),
             "bound": "hbm" if t_hbm >= t_pipe else "tensor", "floor_ms": round(floor, 4),
             "floor_over_kernel": round(floor / kms[i], 4),
             "paper_bsmtc_1core_gflops": PAPER_BSMTC_1CORE_GFLOPS[i]}
        if tt:
            r["ttgt_ms"] = tt[i]
            r["ttgt_time_over_ours"] = round(tt[i] / call_ms[i], 3)
        rows.append(r)
    line["per_string"] = rows
    # the line's roofline over all strings: bound by the larger of the summed
    # HBM and pipe floors (most strings are HBM-bound)
    r0 = line["roofline"]
    per = [(es * sum(int(np.prod([p.ext[x] for x in lab])) for lab in (p.labA, p.labB, p.labC)), p.flops())
           for p in probs]
    src = r0.get("peak_source") if r0.get("unit") == "TFLOP/s" else "MEASURED_PEAKS.json bf16_tflops (burst)"
    rr = mixed_roofline(per, sum(kms), pipe_peak, src, prods, r0.get("kernel"), r0.get("traffic"))
    rr["kernel_ms_per_call"] = r0.get("kernel_ms_per_call")
    line["roofline"] = rr
    return line


def run_grad(args, ws, rank, local):
    """The gradient workload forward and backward (autograd's three
    contractions): C = A.B, dA = dC . B over J, dB = A . dC over I, each a
    transposition-free tc_contract on the tensors' own layouts."""
    spec = W.SPECS["grad_f32"]
    mode = args.mode or spec.mode
    dt = spec.dtype
    seed = 1000 + list(W.SPECS).index(spec.name)
    host = W.make_inputs(spec, seed=seed)
    g = torch.Generator().manual_seed(seed + 7)
    shapeC = spec.shape(spec.labC)
    dC_h = W.colmajor(torch.randn(int(np.prod(shapeC)), generator=g, dtype=torch.float64)
                      .to(dt).to(torch.float64), shapeC)
    A, B, C = (to_device(host[x], dt) for x in "ABC")
    dC = to_device(dC_h, dt)
    dA = torch.empty_like(A)
    dB = torch.empty_like(B)
    calls = [(A, spec.labA, B, spec.labB, C, spec.labC, 1.0, 0.0),
             (dC, spec.labC, B, spec.labB, dA, spec.labA, 1.0, 0.0),
             (A, spec.labA, dC, spec.labC, dB, spec.labB, 1.0, 0.0)]
    flops = 3 * spec.flops()
    es = torch.tensor([], dtype=dt).element_size()
    nbytes = lambda t: t.numel() * es  # noqa: E731
    hbm = sum(nbytes(c[0]) + nbytes(c[2]) + nbytes(c[4]) for c in calls)
    desc = (f"grad_f32 forward + backward: {spec.labC} <- {spec.labA}.{spec.labB}, "
            f"d{spec.labA} <- d{spec.labC}.{spec.labB}, d{spec.labB} <- {spec.labA}.d{spec.labC}, extents "
            + ",".join(f"{k}={v}" for k, v in sorted(spec.ext.items()))
            + f", column-major, normal inputs, mode={mode}")
    extra = {"l2": f"inputs larger than L2 (A = {nbytes(A) / 1e6:.1f} MB > {L2_BYTES / 1e6:.0f} MB)",
             "m_n_k": [[16384, 128, 4096], [16384, 4096, 128], [4096, 128, 16384]], "mode": mode}
    zeros = lambda lab: np.zeros(spec.shape(lab), dtype=np.float64, order="F")  # noqa: E731
    checks = [(0, host["A"].numpy(), host["B"].numpy(), zeros(spec.labC)),
              (1, dC_h.numpy(), host["B"].numpy(), zeros(spec.labA)),
              (2, host["A"].numpy(), dC_h.numpy(), zeros(spec.labB))]
    return run_calls(args, ws, rank, local, calls=calls, inputs=[A, B, dC], outputs=[C, dA, dB],
                     flops=flops, mode=mode, desc=desc, cfg_extra=extra, hbm_bytes=hbm,
                     cpu=(spec, host, 0), checks=checks if getattr(args, "lean", False) else None)


def run_ours(args, ws, rank, local):
    if args.workload == "batch512":
        return run_batch(args, ws, rank, local)
    if args.workload == "tccg":
        return run_tccg(args, ws, rank, local)
    if args.workload in W.PAPER_SHAPES:
        return run_paper(args, ws, rank, local)
    if args.workload == "grad_f32":
        return run_grad(args, ws, rank, local)
    spec = W.SPECS[args.workload]
    lean = getattr(args, "lean", False)
    if args.mode:
        import dataclasses
        spec = dataclasses.replace(spec, mode=args.mode)
    warm = max(3, args.warmup)
    K = max(1, args.steps)
    seed = 1000 + list(W.SPECS).index(spec.name)
    host = W.make_inputs(spec, seed=seed)
    dt = spec.dtype
    dA, dB, dC = (to_device(host[x], dt) for x in "ABC")
    C0 = dC.clone()
    wsz = tc.workspace_size(dA, spec.labA, dB, spec.labB, dC, spec.labC, mode=spec.mode)
    work = torch.empty(max(1, wsz), dtype=torch.uint8, device="cuda")
    flops = spec.flops()
    lib = L.lib()

    def step():
        tc.contract(dA, spec.labA, dB, spec.labB, dC, spec.labC, alpha=spec.alpha, beta=spec.beta,
                    mode=spec.mode, workspace=work)

    for _ in range(warm):
        step()
    torch.cuda.synchronize()

    # device-resident timed region
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in kev:  # torch creates the CUDA event handles on first record
        a.record()
        b.record()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.tc_launch_count()
    e0.record()
    for i in range(K):
        lib.tc_set_mainloop_events(L.c_vp(kev[i][0].cuda_event), L.c_vp(kev[i][1].cuda_event))
        step()
    e1.record()
    torch.cuda.synchronize()
    launches = lib.tc_launch_count() - launches0
    clk = clocks.stop()
    barrier(ws)
    ms = e0.elapsed_time(e1) / K
    kms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
    ms_max = max_over_ranks(ms, ws)
    kms_max = max_over_ranks(kms, ws)
    if not lean:
        profiled_step(args, step)
    err_code = tc.device_error()
    if lean:
        prods = 1 if spec.mode == "f64" else (3 if spec.mode == "bf16x3" else 6)
        form = None if spec.mode == "f64" else tc.operand_form(dA, spec.labA, dB, spec.labB, dC,
                                                               spec.labC, spec.mode)
        kname = "k_f64" if spec.mode == "f64" else KERNELS[form]
        if spec.mode == "f64":
            peak_v, src = fp64_peak_tflops(), "cuBLAS DGEMM 4096^3 measured in this run"
        else:
            mp = measured_peaks()
            peak_v = mp.get("bf16_tflops", 1900.0)
            src = "MEASURED_PEAKS.json bf16_tflops (burst)" if mp else "fallback 1.9 PFLOP/s bf16"
        ach = prods * flops / (kms_max * 1e-3) / 1e12
        line = {"ms_per_step": round(ms_max, 4), "value": round(ws * flops / (ms_max * 1e-3) / 1e12, 5),
                "unit": "TFLOP/s", "steps": K, "warmup": warm, "mode": spec.mode,
                "gpu_launches": int(launches), "device_error": err_code,
                "roofline": {"bound": "tensor", "kernel": kname, "achieved": round(ach, 5),
                             "peak": round(peak_v, 5), "unit": "TFLOP/s", "frac": round(ach / peak_v, 4),
                             "peak_source": src, "kernel_ms": round(kms_max, 4),
                             "traffic": traffic_for(kname, f"{spec.name}_{spec.mode}") if spec.mode != "f64" else None,
                             "algorithmic": f"{flops:.4g} flops per launch"
                                            + (f" (x{prods} bf16 products)" if spec.mode != "f64" else "")}}
        if spec.mode != "f64":
            line["operand_access"] = form
        if rank == 0:
            dC.copy_(C0)
            step()
            torch.cuda.synchronize()
            got = dC.cpu().to(torch.float64).numpy()
            m_, n_, k_ = bundle_lengths(spec)
            t0 = time.perf_counter()
            e, cnt = oracle_err(spec.alpha, host["A"].numpy(), spec.labA, host["B"].numpy(), spec.labB,
                                spec.beta, host["C"].numpy(), spec.labC, got,
                                err_windows(got.size, k_, 1.0, seed=seed))
            line["oracle_check"] = {"max_normalised_err_vs_oracle": e, "elements_checked": cnt,
                                    "sample": "first and last elements and 4 seeded windows of the "
                                              f"output ({time.perf_counter() - t0:.1f} s of oracle time)"}
        return line

    # end-to-end through the public API with host buffers
    # pinned host copies keep the column-major strides of the host views
    hA = torch.empty_strided(host["A"].shape, host["A"].stride(), dtype=dt).pin_memory().copy_(host["A"])
    hB = torch.empty_strided(host["B"].shape, host["B"].stride(), dtype=dt).pin_memory().copy_(host["B"])
    hC = torch.empty_strided(host["C"].shape, host["C"].stride(), dtype=dt).pin_memory().copy_(host["C"])
    hOut = torch.empty_strided(hC.shape, hC.stride(), dtype=dt).pin_memory()
    bi = sum(host_bytes(spec))
    bo = host_bytes(spec)[2]

    def e2e_step():
        dA.copy_(hA, non_blocking=True)
        dB.copy_(hB, non_blocking=True)
        dC.copy_(hC, non_blocking=True)
        step()
        hOut.copy_(dC, non_blocking=True)

    for _ in range(warm):
        e2e_step()
    torch.cuda.synchronize()
    barrier(ws)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(K):
        e2e_step()
    f1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / K, ws)

    peak = fp64_peak_tflops() if spec.mode == "f64" else None
    if spec.mode == "f64":
        peak_v, peak_src = peak, "cuBLAS DGEMM 4096^3 measured in this run (no FP64 entry in MEASURED_PEAKS.json)"
        bound, unit, ach = "tensor", "TFLOP/s", flops / (kms_max * 1e-3) / 1e12
        kname = "k_f64"
    else:
        mp = measured_peaks()
        peak_v = mp.get("bf16_tflops", 1900.0)
        peak_src = "MEASURED_PEAKS.json bf16_tflops (burst)" if mp else "fallback 1.9 PFLOP/s bf16"
        prods = 3 if spec.mode == "bf16x3" else 6
        bound, unit, ach = "tensor", "TFLOP/s", prods * flops / (kms_max * 1e-3) / 1e12
        kname = KERNELS[tc.operand_form(dA, spec.labA, dB, spec.labB, dC, spec.labC, spec.mode)]
    value = ws * flops / (ms_max * 1e-3) / 1e12
    extra = {"l2": f"inputs larger than L2 (A = {host_bytes(spec)[0] / 1e6:.1f} MB > {L2_BYTES / 1e6:.0f} MB)",
             "parallelism": f"replicas x{ws}"}
    if spec.mode != "f64":
        form = tc.operand_form(dA, spec.labA, dB, spec.labB, dC, spec.labC, spec.mode)
        how = {"gather": "A and B gathered through their scatter vectors",
               "box": "A and B TMA boxes", "pair": "A and B TMA boxes on CTA pairs",
               "packed": "A and B packed once (k_pack), then streamed by bulk copies (k_tcp)"}
        extra["operand_access"] = f"{args.access}: {how[form]}"
    line = {
        "metric": METRIC, "value": round(value, 5), "unit": "TFLOP/s", "n_gpus": ws, "steps": K,
        "warmup": warm, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if spec.mode == "f64" else f"f32 data, {spec.mode} products, f32 accumulate",
        "data": "synthetic (seeded uniform[-1,1], column-major; shapes of the paper's CC-style contractions)",
        "config": workload_config(spec, extra),
        "clocks": clk,
        "e2e": {"value": round(ws * flops / (e2e_ms * 1e-3) / 1e12, 5), "unit": "TFLOP/s",
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": int(launches),
        "roofline": {"bound": bound, "kernel": kname, "achieved": round(ach, 5), "peak": round(peak_v, 5),
                     "unit": unit, "frac": round(ach / peak_v, 4), "peak_source": peak_src,
                     "kernel_ms": round(kms_max, 4),
                     "traffic": traffic_for(kname, spec.name if spec.mode == "f64" else f"{spec.name}_{spec.mode}"),
                     "algorithmic": f"{flops:.4g} flops per launch"
                                    + (f" (x{prods} bf16 products)" if spec.mode != "f64" else "")},
        "device_error": err_code,
    }

    # the TTGT form of the same step (cuBLAS GEMM between transposition copies)
    if not args.no_ttgt:
        dC.copy_(C0)
        tt = ttgt_legs([(dA, spec.labA, dB, spec.labB, dC, spec.labC, spec.alpha, spec.beta)],
                       warm, K, flops, ws, ms_max, spec.mode != "f64")
        tt["ours_workspace_bytes"] = int(wsz)
        line["ttgt"] = tt

    # CPU baseline: the oracle on a bounded sample, rank 0 at N = 1 only
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        dC.copy_(C0)
        step()
        torch.cuda.synchronize()
        got = dC.cpu().to(torch.float64).numpy()
        fl, sec, S, cores, cref, mag = oracle_sample(spec, host, seconds=12.0)
        sel = np.arange(S)
        g = got.ravel(order="F")[sel]
        r = cref.ravel(order="F")[sel]
        m = mag.ravel(order="F")[sel]
        err = float(np.max(np.abs(g - r) / np.maximum(m, 1e-300)))
        fro = float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300))
        line["cpu_baseline"] = {"value": round(fl / sec / 1e12, 8), "unit": "TFLOP/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"first {S} of {got.size} output elements (all k terms each), "
                                          f"{sec:.1f} s on {cores} host threads",
                                "max_normalised_err_gpu_vs_oracle": err,
                                "frobenius_rel_err_gpu_vs_oracle": fro}
    return line


# ---- the other configurations, on the default line --------------------------------------------

# normalised-error bars: FP64 path on FP64 data; on FP32 data the FP64 result
# is rounded once to FP32 (2^-24 of |C| <= the magnitude); BF16x3's derived
# bound (two bf16 pieces keep 16 significand bits); BF16x6 the stated 1e-5
TOL = {"f64": 1e-12, "f64_on_f32": 2.0 ** -24 + 1e-12, "bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24,
       "bf16x6": 1e-5}


def secondary_configs(args, ws, rank, local):
    """The precision form (spiky_f32 in BF16x3, BF16x6 and through the plain FP64
    path), the gradient workload forward + backward, and the 512-problem batch in
    both modes: fewer steps, the timed numbers, the roofline and an oracle
    check of sampled outputs each, without the end-to-end, TTGT and CPU legs."""
    import copy
    out = {}
    runs = [("spiky_f32_bf16x3", "spiky_f32", "bf16x3"), ("spiky_f32_bf16x6", "spiky_f32", "bf16x6"),
            ("spiky_f32_f64", "spiky_f32", "f64"), ("grad_f32_bf16x3", "grad_f32", "bf16x3"),
            ("batch512_bf16x3", "batch512", "bf16x3"), ("batch512_f64", "batch512", "f64"),
            ("tccg_bf16x3", "tccg", "bf16x3"), ("tccg_f64", "tccg", "f64")]
    # steps per entry: a timed region of about 0.1-0.5 s each (a few milliseconds would
    # measure the host's start-up of the clock sampler rather than the step)
    steps = {"spiky_f32_bf16x3": 200, "spiky_f32_bf16x6": 200, "spiky_f32_f64": 3,
             "grad_f32_bf16x3": 200, "batch512_bf16x3": 50, "batch512_f64": 3,
             "tccg_bf16x3": 10, "tccg_f64": 3}
    for key, wl, mode in runs:
        a = copy.copy(args)
        a.workload, a.mode, a.lean = wl, mode, True
        a.steps = steps[key]
        a.warmup = 3
        a.no_ttgt = a.no_cpu_baseline = True
        a.profile = False
        a.traffic_key = "grad_f32" if wl == "grad_f32" else wl
        t0 = time.perf_counter()
        try:
            r = run_ours(a, ws, rank, local)
        except Exception as exc:  # a failing secondary config must not hide the headline
            r = {"error": f"{type(exc).__name__}: {exc}"}
        r["wall_s"] = round(time.perf_counter() - t0, 1)
        chk = r.get("oracle_check")
        if chk is not None:
            tol = TOL["f64_on_f32" if mode == "f64" and wl in ("spiky_f32", "grad_f32") else mode]
            if mode != "f64" and wl == "tccg":
                tol = TOL[mode]
            chk["tolerance"] = tol
            chk["within_tolerance"] = chk["max_normalised_err_vs_oracle"] <= tol
        out[key] = r
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    f64 = out.get("spiky_f32_f64", {}).get("ms_per_step")
    for key in ("spiky_f32_bf16x3", "spiky_f32_bf16x6"):
        if f64 and out.get(key, {}).get("ms_per_step"):
            out[key]["speedup_over_f64_path"] = round(f64 / out[key]["ms_per_step"], 2)
    return out


# ---- reference arm: the CPU oracle as it stands ------------------------------------------------

def run_reference(args, ws, rank):
    if rank != 0:
        return
    spec = W.SPECS[args.workload]
    seed = 1000 + list(W.SPECS).index(spec.name)
    host = W.make_inputs(spec, seed=seed)
    warm, K = max(3, args.warmup), max(1, args.steps)
    per_step = max(0.5, min(4.0, 90.0 / (warm + K)))
    fl, sec, S, cores, _, _ = oracle_sample(spec, host, seconds=per_step)
    for _ in range(warm - 1):
        oracle_sample(spec, host, seconds=per_step, out_count=S)
    times = []
    for _ in range(K):
        fl, sec, _, _, _, _ = oracle_sample(spec, host, seconds=per_step, out_count=S)
        times.append(sec)
    t = float(np.mean(times))
    v = fl / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 8), "unit": "TFLOP/s", "n_gpus": ws,
            "steps": K, "warmup": warm, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(spec, {"sample": f"first {S} output elements per step"}),
            "cpu_baseline": {"value": round(v, 8), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {S} output elements of {spec.name} per step"},
            "e2e": {"value": round(v, 8), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        if not torch.cuda.is_available():
            raise SystemExit("bench.py --impl ours needs a GPU")
        tc.set_access(args.access)
        line = run_ours(args, ws, rank, local)
        if args.workload == "cc4x4_f64" and not args.no_configs and args.mode is None \
                and args.access == "auto":
            line["configs"] = secondary_configs(args, ws, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
