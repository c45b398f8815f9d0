#!/usr/bin/env python
"""Benchmark: D3M dual block LDL^T factor + solve on one GB300 (or N independent ones).

Workload (default): 8 x 8 x 1 domain grid, 112 interfaces, m = 512 dual unknowns per
interface (n = 57,344), nested-dissection order, M_i = G G^T - k^2 I + i tau I with k^2 = 2,
tau = 0.05, 8 right-hand sides, seeded synthetic data.

One step = d3m_factor (copy of K + persistent tile-task kernel) + d3m_solve (sweeps +
FP64 residual refinement to omega <= 1e-12) through the C ABI, inputs resident in HBM.
value = effective TFLOP/s = (algorithmic factor flops + solve flops x nrhs) / step time,
summed over ranks (each rank solves its own instance: weak scaling, no data collective).

Also reported: the plain FP64 GPU path on the same matrix (time-to-solution), the
end-to-end number with host buffers (H2D of K and B, D2H of X inside the timed region),
the roofline of the dominant kernel, clocks sampled during the timed region, and the CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "factor+solve time & TFLOP/s at 1e-9 rel err: mixed-prec vs FP64 block LDLᵀ"
FP64_PEAK_GFLOPS = 1250.0     # GB300 FP64 nominal (152 SMs x 2.07 GHz x ~4 flop/clk/SM)
# the residual's products issue on the FP32 pipe in double-float form: 60 FP32 instructions per
# complex multiply-add (8 flops) and right-hand side
RESID_PEAK_TFLOPS = 152 * 128 * 2.07e9 * 8 / 60 / 1e12


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="d3m", choices=["d3m", "reference"])
    ap.add_argument("--workload", default="grid6x6x6_m512")
    ap.add_argument("--precision", default="auto", choices=["auto", "bf16x3", "tf32", "simt32", "fp64"],
                    help="tile engine; auto: tf32 for a throughput-bound factorization, else bf16x3")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--report-modules", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--seg-group", type=int, default=0, help="source blocks per update task (0 = library default)")
    ap.add_argument("--graphs", type=int, default=0, help="1: replay the factorization and each refinement "
                    "step as CUDA graphs")
    return ap.parse_args()


def cross_rank_max(v: float, dist, device) -> float:
    """Largest v over the ranks (the step time a multi-rank line reports); v when dist is None."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ recorded DRAM traffic
# Per-launch DRAM bytes of a kernel come from an ncu capture (profiles/traffic_<workload>.txt,
# lines "<kernel>:<engine> <bytes per launch> <sha1 of the code of its source files>"); a number whose kernel
# sources have changed since the capture is not reported.
TRAFFIC_SOURCES = {"factor_kernel": ("factor_tc.cu", "device.cuh"), "residual": ("resid_tc.cu",),
                   "solve_sweep": ("gather_tc.cu", "solve.cu")}


def source_sha(kernel: str):
    """SHA-1 of the code of a kernel's source files: comments, blank lines and trailing spaces
    removed, so that an edit of the comments keeps a record valid and any change of code voids it."""
    import hashlib
    import re
    h = hashlib.sha1()
    for src in TRAFFIC_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2002_05026_gb300", "csrc", src)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        code = []
        for line in text.splitlines():
            # a // comment outside a string literal (the sources have no "//" inside strings)
            line = line.split("//", 1)[0].rstrip()
            if line:
                code.append(line)
        h.update("\n".join(code).encode())
    return h.hexdigest()


def recorded_traffic(workload: str, kernel: str, engine: str):
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if kernel not in TRAFFIC_SOURCES or not os.path.exists(path):
        return None
    sha = source_sha(kernel)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 3 and parts[0] == f"{kernel}:{engine}" and parts[2] == sha:
                return float(parts[1])
    return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle sample
def host_gemm_rate(m: int) -> float:
    """Flops/s of the host's complex128 m x m matrix product (the step that dominates the oracle's
    block factorization), used only to size the oracle sample."""
    import numpy as np
    a = np.ones((m, m), dtype=np.complex128)
    a @ a
    t0 = time.perf_counter()
    for _ in range(3):
        a @ a
    return 3 * 8.0 * m ** 3 / max(time.perf_counter() - t0, 1e-6)


class OracleSample:
    """The oracle (numpy FP64) right-looking block LDL^T of the first C block columns of a
    workload, in the oracle's own nested-dissection order, C chosen for about `seconds` of host
    work.  Only the domains adjacent to those C interfaces are generated: the factor of the first
    C columns depends on K's first C (permuted) columns alone, and those are exact; the trailing
    Schur updates they produce (timed as well) land in blocks that are left partial.  Nothing
    here loads the CUDA library."""

    def __init__(self, w: dict, seed: int, seconds: float):
        import numpy as np
        import oracle as O
        import synth
        nx, ny, nz, m = w["nx"], w["ny"], w["nz"], w["m"]
        self.m = m
        self.perm = O.nd_order(nx, ny, nz)
        colptr, rowidx = synth.lower_pattern(nx, ny, nz)
        N = colptr.size - 1
        self.N = N
        inv = np.empty(N, dtype=np.int64)
        inv[self.perm] = np.arange(N)
        keys = []
        for g in range(N):
            for e in range(colptr[g], colptr[g + 1]):
                i, j = int(inv[rowidx[e]]), int(inv[g])
                keys.append((max(i, j), min(i, j)))
        st, _ = O.block_symbolic(N, keys)

        def col_flops(k):
            s_ = len(st[k])
            return (4 / 3) * m ** 3 + s_ * 4 * m ** 3 + s_ * 4 * m ** 3 + s_ * (s_ - 1) / 2 * 8 * m ** 3

        cf = [col_flops(k) for k in range(N)]
        total = sum(cf)
        budget = host_gemm_rate(m) * seconds
        C, acc = 0, 0.0
        while C < N and acc + cf[C] <= budget:
            acc += cf[C]
            C += 1
        self.C = max(C, 1)
        self.flops = sum(cf[:self.C])
        self.share = self.flops / total
        doms = synth.interface_domains(nx, ny, nz, self.perm[:self.C])
        p = synth.make_problem(nx, ny, nz, m, w["k2"], w["tau"], seed, device="cpu", domains=doms)
        flat = p.blocks.numpy()
        Kb = {}
        for g in range(N):
            for e in range(colptr[g], colptr[g + 1]):
                f = int(rowidx[e])
                if min(inv[f], inv[g]) < self.C:
                    Kb[(f, g)] = flat[e * m * m:(e + 1) * m * m].reshape(m, m).T.copy()
        del p, flat
        self.Kp = O.permute_lower(Kb, self.perm)
        self.ndomains = len(doms)

    def run(self) -> float:
        import oracle as O
        t0 = time.perf_counter()
        O.block_ldlt(self.Kp, self.N, self.m, ncols=self.C)
        return time.perf_counter() - t0

    def describe(self, workload: str, dt: float) -> str:
        return (f"oracle (numpy FP64) right-looking block LDL^T of the first {self.C} of {self.N} block columns "
                f"({100 * self.share:.2f}% of the factor flops) of the {workload} matrix, {dt:.1f} s "
                f"(the {self.ndomains} domains adjacent to those columns generated)")


def make_workload(w, seed, device):
    import numpy as np
    import synth
    p = synth.make_problem(w["nx"], w["ny"], w["nz"], w["m"], w["k2"], w["tau"], seed, device=device)
    B = synth.rhs(seed + 1, p.n, w["nrhs"])
    return p, np.ascontiguousarray(B.T)      # (nrhs, n) = column-major (n, nrhs)


# ------------------------------------------------------------------ engine choice
# TF32 does two thirds of split-BF16x3's tensor-core work per product but its factor is less
# accurate (about 2^-11), so the refinement needs one more solve.  On a factorization large
# enough to keep every SM busy (throughput-bound, under the power cap) the cheaper products win;
# on a smaller one, bound by its critical path of diagonal tiles, they do not.  Measured on one
# GB300: 6x6x6 m=512 (1.8e14 factor flops, 32 RHS) 466 ms (tf32) vs 498 ms (bf16x3) per step;
# 8x8 m=512 (3.6e12 flops, 8 RHS) 25.7 vs 22.8 ms.  Both reach omega <= 1e-12.
AUTO_TF32_FLOPS = 5e13


def resolve_precision(args, colptr, rowidx, m, perm) -> str:
    if args.precision != "auto":
        return args.precision
    from paper_2002_05026_gb300 import d3m_analyze
    flops = d3m_analyze(colptr, rowidx, m=m, perm=perm)["factor_flops"]
    return "tf32" if flops >= AUTO_TF32_FLOPS else "bf16x3"


# ------------------------------------------------------------------ reference arm (the oracle)
def reference_arm(args, rank, world):
    """The oracle on the host cores, on a bounded sample of the workload; loads neither torch's
    CUDA nor the CUDA library (only `oracle` and `synth`)."""
    if rank != 0:
        return
    import synth
    w = synth.WORKLOADS[args.workload]
    per_step = min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup))
    smp = OracleSample(w, w["seed"], per_step)
    for _ in range(args.warmup):
        smp.run()
    times = [smp.run() for _ in range(args.steps)]
    vals = [smp.flops / t / 1e12 for t in times]
    value = sum(vals) / len(vals)
    cores = os.cpu_count()
    sample = smp.describe(args.workload, sum(times) / len(times))
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "grid": [w["nx"], w["ny"], w["nz"]], "m": w["m"],
                       "nrhs": w["nrhs"], "k2": w["k2"], "tau": w["tau"]},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.report_modules:
        # what this process loaded of the product: its Python package and any mapped libd3m.so
        maps = open("/proc/self/maps").read() if os.path.exists("/proc/self/maps") else ""
        line["product_modules"] = sorted(k for k in sys.modules if k.startswith("paper_2002_05026_gb300"))
        line["product_so_mapped"] = "libd3m.so" in maps
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ adjoint arm
ADJ_METRIC = "adjoint gradient evaluations: factor + refined solve + refined adjoint solve + dJ/deps"


def adjoint_arm(args, rank, world, local):
    """J = Re(c^T x), x = K(eps)^{-1} b on the 8x8 grid with m = 256 (64 domain parameters eps_i).
    One step = one gradient evaluation: factor K(eps), x = solve(b), Lambda = adjoint(c) (same
    factors, K^T = K), dJ/deps_i = Re(k2 sum_{u in I(i)} Lambda_u x_u).  Value = evaluations/s."""
    import numpy as np
    import torch
    import synth
    from paper_2002_05026_gb300 import D3M, d3m_order_grid_nd

    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    seed = w["seed"] + rank
    ndom = w["nx"] * w["ny"] * w["nz"]
    eps = synth.domain_eps(seed + 3, ndom)
    p = synth.make_problem(w["nx"], w["ny"], w["nz"], w["m"], w["k2"], w["tau"], seed, eps=eps, device="cuda")
    perm = d3m_order_grid_nd(w["nx"], w["ny"], w["nz"])
    b = torch.from_numpy(np.ascontiguousarray(synth.rhs(seed + 1, p.n, 1))).cuda()
    c = torch.from_numpy(np.ascontiguousarray(synth.sparse_adjoint_vector(seed + 2, p.n, p.m,
                                                                           support_block=int(perm[-1])))).cuda()
    args.precision = resolve_precision(args, p.colptr, p.rowidx, p.m, perm)
    s = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision=args.precision, max_nrhs=1)
    stream = torch.cuda.current_stream()

    def step():
        s.factor(p.blocks)
        x = s.solve(b)
        lam = s.adjoint(c)
        return s.grad_eps(lam, x, p.dom_if, w["k2"])     # host array; synchronizes the stream

    for _ in range(args.warmup):
        g = step()
    info0 = s.info()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g = step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    info = s.info()
    peaks, peak_kind = measured_peaks()
    fms = info["factor_kernel_ms_total"] / max(1, info["factor_kernel_calls"])
    roof = {"bound": "tensor", "achieved": info["factor_flops"] / (fms * 1e-3) / 1e12,
            "peak": peaks["bf16_tflops"] / 3.0, "unit": "TFLOP/s", "kernel": "factor_kernel",
            "kernel_ms": fms, "peak_source": "bf16_tflops/3 (burst)", "traffic": None, "peak_kind": peak_kind}
    if args.precision == "tf32":
        roof.update({"peak": peaks["bf16_tflops"] / 2.0, "peak_source": "bf16_tflops/2 (burst; tf32 dense rate)"})
    elif args.precision != "bf16x3":
        roof.update({"bound": "alu", "peak": FP64_PEAK_GFLOPS / 1e3 if args.precision == "fp64" else
                     152 * 2.07e9 * 256 / 1e12, "peak_source": "ALU nominal"})
    roof["frac"] = roof["achieved"] / roof["peak"]
    line = {"metric": ADJ_METRIC, "value": 1e3 / ms * world, "unit": "gradients/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16x3": "c64+bf16x3/fp64-refine", "tf32": "c64+tf32/fp64-refine", "fp64": "c128"}.get(
                args.precision, "c64/fp64-refine"), "data": "synthetic",
            "config": {"workload": args.workload, "grid": [w["nx"], w["ny"], w["nz"]], "m": w["m"], "n": p.n,
                       "parameters": ndom, "k2": w["k2"], "tau": w["tau"], "precision": args.precision},
            "roofline": roof,
            "accuracy": {"omega": info["omega"], "refine_solves_last_call": info["refine_iters"],
                         "max_abs_dJ_deps": float(np.max(np.abs(g)))},
            "clocks": clocks, "gpu_launches": info["kernel_launches"] - info0["kernel_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()


# ------------------------------------------------------------------ batched arm
BATCH_METRIC = "batched factor+solve throughput: uneven instances, mixed-prec + FP64 refinement"


def batch_arm(args, rank, world, local):
    """256 uneven instances (2-D grids 2x2..6x6, m in {64,128,256}, 4 RHS each) in one batched
    handle: one persistent factorization launch and graph-replayed refinement steps; the tile
    engine comes from the autotuner.  Value = instances factored and solved per second."""
    import numpy as np
    import torch
    import synth
    from paper_2002_05026_gb300 import D3M, D3MBatch, autotune, d3m_order_grid_nd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def allmax(v: float) -> float:
        return cross_rank_max(v, dist, "cuda")

    count, nrhs = 256, 4
    specs = synth.batch_instances(count, seed=20260105 + 100003 * rank)   # each rank its own batch
    probs = [synth.make_problem(w["nx"], w["ny"], w["nz"], w["m"], w["k2"], w["tau"], w["seed"], device="cuda")
             for w in specs]
    perms = [d3m_order_grid_nd(w["nx"], w["ny"], w["nz"]) for w in specs]
    inst = [(p.colptr, p.rowidx, p.m) for p in probs]
    K = torch.cat([p.blocks for p in probs])
    Bs = [synth.rhs(w["seed"] + 1, p.n, nrhs) for w, p in zip(specs, probs)]
    Bt = torch.from_numpy(np.ascontiguousarray(np.concatenate(Bs).T)).cuda()   # (nrhs, n) column-major
    n_tot = Bt.shape[1]
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    tune = autotune.tune_batch(inst, perms, K, Bt, nrhs)
    s = D3MBatch(inst, perms, precision=tune["precision"], max_nrhs=nrhs, graphs=True, task_cost=tune["task_cost"])
    lib = s._lib
    Xt = torch.empty_like(Bt)

    def step(Kp, Bp, Xp):
        rc = lib.d3m_factor(s.h, ctypes.c_void_p(Kp), sp)
        if rc:
            raise RuntimeError(s.last_error())
        rc = lib.d3m_solve(s.h, ctypes.c_void_p(Bp), ctypes.c_void_p(Xp), nrhs, sp)
        if rc:
            raise RuntimeError(f"solve rc={rc}: {s.last_error()}")

    for _ in range(args.warmup):
        step(K.data_ptr(), Bt.data_ptr(), Xt.data_ptr())
    info0 = s.info()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(K.data_ptr(), Bt.data_ptr(), Xt.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = allmax(e0.elapsed_time(e1) / args.steps)
    info = s.info()
    w_inst = s.instance_omega()
    launches = info["kernel_launches"] - info0["kernel_launches"]
    flops_step = info["factor_flops"] + info["solve_flops_per_rhs"] * nrhs
    value = count * world / (ms * 1e-3)
    peaks, peak_kind = measured_peaks()
    fms = info["factor_kernel_ms_total"] / max(1, info["factor_kernel_calls"])
    if tune["precision"] == "bf16x3":
        pk, bound, pname = peaks["bf16_tflops"] / 3.0, "tensor", "bf16_tflops/3 (burst)"
    else:
        pk, bound, pname = 152 * 2.07e9 * 256 / 1e12, "alu", "FP32 FMA 152 SMs x 128 x 2 x 2.07 GHz"
    ach = info["factor_flops"] / (fms * 1e-3) / 1e12
    roof = {"bound": bound, "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "traffic": None,
            "kernel": "factor graph (copy of K, ||K_i||, persistent factor kernel)", "kernel_ms": fms,
            "peak_source": pname, "peak_kind": peak_kind}

    # looping the plain FP64 path over the same instances, one handle each
    fp64 = None
    if not args.no_fp64:
        offs = np.concatenate([[0], np.cumsum([p.n for p in probs])])
        koffs = np.concatenate([[0], np.cumsum([p.blocks.numel() for p in probs])])
        hs = [D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision="fp64", max_nrhs=nrhs) for p, pm in zip(probs, perms)]
        Bi = [Bt[:, offs[i]:offs[i + 1]].contiguous() for i in range(count)]
        Xi = [torch.empty_like(b) for b in Bi]

        def loop64():
            for i, h in enumerate(hs):
                lib.d3m_factor(h.h, ctypes.c_void_p(K.data_ptr() + int(koffs[i]) * 16), sp)
                rc = lib.d3m_solve(h.h, ctypes.c_void_p(Bi[i].data_ptr()), ctypes.c_void_p(Xi[i].data_ptr()), nrhs, sp)
                if rc:
                    raise RuntimeError(h.last_error())

        loop64()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            loop64()
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = allmax(f0.elapsed_time(f1) / args.fp64_steps)
        X64 = torch.cat(Xi, dim=1)
        rel = 0.0
        for i in range(count):
            a, b = Xt[:, offs[i]:offs[i + 1]], X64[:, offs[i]:offs[i + 1]]
            rel = max(rel, (torch.linalg.norm(a - b, dim=1) / torch.linalg.norm(b, dim=1)).max().item())
        fp64 = {"ms_per_step": ms64, "value": count * world / (ms64 * 1e-3), "unit": "solves/s",
                "speedup_batched_vs_fp64_loop": ms64 / ms, "max_rel_diff_batched_vs_fp64": rel}
        for h in hs:
            h.close()

    e2e = None
    if not args.no_e2e:
        Kh = K.cpu().pin_memory()
        Bh = Bt.cpu().pin_memory()
        Xh = torch.empty_like(Bh).pin_memory()
        step(Kh.data_ptr(), Bh.data_ptr(), Xh.data_ptr())
        torch.cuda.synchronize()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            step(Kh.data_ptr(), Bh.data_ptr(), Xh.data_ptr())
        g1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = allmax(g0.elapsed_time(g1) / args.steps)
        e2e = {"value": count * world / (ems * 1e-3), "unit": "solves/s", "ms_per_step": ems,
               "h2d_bytes_per_step": int(Kh.numel() * 16 + Bh.numel() * 16),
               "d2h_bytes_per_step": int(Xh.numel() * 16)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        t0 = time.perf_counter()
        done = 0
        for w, p, B in zip(specs, probs, Bs):
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
            pm = O.nd_order(w["nx"], w["ny"], w["nz"])       # the oracle's own ordering
            blocks = p.blocks.cpu().numpy()
            Kb = O.lower_blocks(p.colptr, p.rowidx, blocks, p.m)
            F = O.block_ldlt(O.permute_lower(Kb, pm), p.nblk, p.m)
            F.perm = pm
            O.block_solve(F, B)
            done += 1
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle (numpy FP64) block LDL^T + solve of the first {done} of {count} instances, {dt:.1f} s"}

    if rank == 0:
        line = {"metric": BATCH_METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64+bf16x3/fp64-refine" if tune["precision"] == "bf16x3" else
                "c64/fp64-refine", "data": "synthetic",
                "config": {"workload": "batch256", "instances": count, "nrhs": nrhs, "n_total": int(n_tot),
                           "grids": "2-D, uniform over {2x2,3x3,4x4,6x6}", "m": "uniform over {64,128,256}",
                           "k2": "U(0.5,4)", "tau": "U(0.01,0.2)", "tile_engine": tune["precision"],
                           "autotune_ms": {k: v["ms"] for k, v in tune["timings"].items()}, "graphs": True,
                           "task_cost_ns": tune["task_cost"],
                           "l2": f"inputs larger than L2 (K is {K.numel() * 16 / 1e9:.2f} GB)"},
                "roofline": roof,
                "accuracy": {"omega_max_over_instances": float(np.max(w_inst)), "refine_solves": info["refine_iters"]},
                "fp64_loop": fp64, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": int(launches), "flops_per_step": flops_step,
                "effective_tflops": flops_step * world / (ms * 1e-3) / 1e12}
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ main arm
def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import numpy as np
    import torch
    import synth
    from paper_2002_05026_gb300 import D3M, build, d3m_order_grid_nd

    build.build()
    if args.workload == "batch256":
        batch_arm(args, rank, world, local)
        return
    if args.workload.startswith("adjoint"):
        adjoint_arm(args, rank, world, local)
        return
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def allmax(v: float) -> float:
        return cross_rank_max(v, dist, "cuda")

    w = synth.WORKLOADS[args.workload]
    seed = w["seed"] + rank
    dev_total = torch.cuda.mem_get_info()[1]
    mem_peak = [0]

    def mem_sample():
        # device-wide high-water mark: total - free at sampled points (cudaMemGetInfo)
        free, total = torch.cuda.mem_get_info()
        mem_peak[0] = max(mem_peak[0], total - free)

    p, Bnp = make_workload(w, seed, "cuda")
    nrhs = w["nrhs"]
    K = p.blocks                                            # device c128, lower blocks
    Bt = torch.from_numpy(Bnp).cuda()                       # (nrhs, n)
    Xt = torch.empty_like(Bt)
    perm = d3m_order_grid_nd(w["nx"], w["ny"], w["nz"])
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    args.precision = resolve_precision(args, p.colptr, p.rowidx, p.m, perm)
    s = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision=args.precision, max_nrhs=nrhs, graphs=bool(args.graphs),
            seg_group=args.seg_group)
    lib = s._lib
    mem_sample()

    def step(Kp, Bp, Xp):
        rc = lib.d3m_factor(s.h, ctypes.c_void_p(Kp), sp)
        if rc:
            raise RuntimeError(s.last_error())
        rc = lib.d3m_solve(s.h, ctypes.c_void_p(Bp), ctypes.c_void_p(Xp), nrhs, sp)
        if rc:
            raise RuntimeError(f"solve rc={rc}: {s.last_error()}")

    for _ in range(args.warmup):
        step(K.data_ptr(), Bt.data_ptr(), Xt.data_ptr())
    torch.cuda.synchronize()
    mem_sample()
    info0 = s.info()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(K.data_ptr(), Bt.data_ptr(), Xt.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = allmax(ms)
    info = s.info()
    flops_step = info["factor_flops"] + info["solve_flops_per_rhs"] * nrhs
    value = flops_step * world / (ms * 1e-3) / 1e12
    launches = info["kernel_launches"] - info0["kernel_launches"]
    X_mixed = Xt.clone()

    # ---------------------------------------------------------------- roofline of the dominant kernel
    # tensor-core kernels are scored against the BURST bf16 peak (the larger of the two measured
    # figures): a conservative denominator whatever the clocks were during the run
    peaks, peak_kind = measured_peaks()
    b = info["tile"]
    kern = []
    if info["factor_kernel_calls"]:
        fms = info["factor_kernel_ms_total"] / info["factor_kernel_calls"]
        if args.precision == "bf16x3":
            pk, unit, bound, pname = peaks["bf16_tflops"] / 3.0, "TFLOP/s", "tensor", \
                "bf16_tflops/3 (burst; split-BF16x3: 3 bf16 products per FP32-level product)"
        elif args.precision == "tf32":
            pk, unit, bound, pname = peaks["bf16_tflops"] / 2.0, "TFLOP/s", "tensor", \
                "bf16_tflops/2 (burst; tf32 dense rate = half the bf16 rate, nominal 1.1 vs 2.25 PFLOP/s)"
        elif args.precision == "fp64":
            pk, unit, bound, pname = FP64_PEAK_GFLOPS / 1e3, "TFLOP/s", "alu", "FP64 nominal 1.25 TFLOP/s"
        else:
            pk, unit, bound, pname = 152 * 2.07e9 * 256 / 1e12, "TFLOP/s", "alu", "FP32 FMA 152 SMs x 128 x 2 x 2.07 GHz"
        kern.append(("factor_kernel", info["factor_kernel_ms_total"],
                     {"bound": bound, "achieved": info["factor_flops"] / (fms * 1e-3) / 1e12, "peak": pk,
                      "unit": unit, "peak_source": pname, "kernel_ms": fms}))
    if info["residual_calls"]:
        rms = info["residual_ms_total"] / info["residual_calls"]
        kbytes = info["residual_bytes_fixed"] + info["residual_bytes_per_rhs"] * nrhs
        kern.append(("residual", info["residual_ms_total"],
                     {"bound": "hbm", "achieved": kbytes / (rms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                      "unit": "GB/s", "peak_source": "hbm_gbs (algorithmic bytes: K's stored lower blocks in "
                                                     "c128 + x, b and r per right-hand side)",
                      "kernel_ms": rms,
                      "fp64_accurate_tflops": info["residual_flops_per_rhs"] * nrhs / (rms * 1e-3) / 1e12}))
    if info["sweep_calls"]:
        sms = info["sweep_ms_total"] / info["sweep_calls"]
        esz = 16 if args.precision == "fp64" else 8
        lbytes = 2.0 * info["ntiles"] * b * b * esz
        kern.append(("solve_sweep", info["sweep_ms_total"],
                     {"bound": "hbm", "achieved": lbytes / (sms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                      "unit": "GB/s", "peak_source": "hbm_gbs", "kernel_ms": sms}))
    kern.sort(key=lambda t: -t[1])
    dom_name, _, roof = kern[0]
    roof = dict(roof)
    roof["kernel"] = dom_name
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = recorded_traffic(args.workload, dom_name, args.precision)
    roof["peak_kind"] = peak_kind
    breakdown = {k: {"ms_per_step": t / args.steps, **{kk: v for kk, v in r.items() if kk in ("achieved", "peak", "unit", "bound")}}
                 for k, t, r in kern}
    memory = {"handle_device_bytes": int(info["device_bytes"]),
              "torch_peak_allocated_bytes": int(torch.cuda.max_memory_allocated()),
              "device_used_high_water_bytes": int(mem_peak[0]), "device_total_bytes": int(dev_total),
              "how": "handle_device_bytes = every buffer the solver handle owns; device_used_high_water = max of "
                     "(total - free) from cudaMemGetInfo after create, after warm-up and after the timed steps"}

    # ---------------------------------------------------------------- end to end, host buffers
    e2e = None
    if not args.no_e2e:
        Kh = K.cpu().pin_memory()
        Bh = Bt.cpu().pin_memory()
        Xh = torch.empty_like(Bh).pin_memory()
        step(Kh.data_ptr(), Bh.data_ptr(), Xh.data_ptr())
        torch.cuda.synchronize()
        mem_sample()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            step(Kh.data_ptr(), Bh.data_ptr(), Xh.data_ptr())
        g1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = allmax(g0.elapsed_time(g1) / args.steps)
        e2e = {"value": flops_step * world / (ems * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ems,
               "h2d_bytes_per_step": int(Kh.numel() * 16 + Bh.numel() * 16),
               "d2h_bytes_per_step": int(Xh.numel() * 16)}
        del Kh
    memory["device_used_high_water_bytes"] = int(mem_peak[0])
    s.close()
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- plain FP64 GPU path
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        s64 = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision="fp64", max_nrhs=nrhs)
        X64 = torch.empty_like(Bt)

        def step64():
            rc = lib.d3m_factor(s64.h, ctypes.c_void_p(K.data_ptr()), sp)
            if rc:
                raise RuntimeError(s64.last_error())
            rc = lib.d3m_solve(s64.h, ctypes.c_void_p(Bt.data_ptr()), ctypes.c_void_p(X64.data_ptr()), nrhs, sp)
            if rc:
                raise RuntimeError(s64.last_error())

        # a factorization of more than 1e13 flops runs for minutes at FP64 rates: one timed run
        # without a warm-up run (first-launch overheads are below a millisecond)
        warm64 = info["factor_flops"] < 1e13
        if warm64:
            step64()
            torch.cuda.synchronize()
            s64.info()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            step64()
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = allmax(f0.elapsed_time(f1) / args.fp64_steps)
        i64 = s64.info()
        rel = (torch.linalg.norm(X_mixed - X64, dim=1) / torch.linalg.norm(X64, dim=1)).max().item()
        fk = i64["factor_kernel_ms_total"] / max(1, i64["factor_kernel_calls"])
        fp64 = {"ms_per_step": ms64, "tflops": flops_step / (ms64 * 1e-3) / 1e12,
                "speedup_mixed_vs_fp64": ms64 / ms, "factor_kernel_ms": fk, "warmup_run": warm64,
                "steps": args.fp64_steps, "handle_device_bytes": int(i64["device_bytes"]),
                "factor_roofline": {"bound": "alu", "achieved": i64["factor_flops"] / (fk * 1e-3) / 1e12,
                                    "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                                    "peak_source": "FP64 nominal 1.25 TFLOP/s (not measured)",
                                    "frac": i64["factor_flops"] / (fk * 1e-3) / 1e12 / (FP64_PEAK_GFLOPS / 1e3)},
                "max_rel_diff_mixed_vs_fp64": rel}
        s64.close()
        del X64

    # ---------------------------------------------------------------- CPU oracle sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = OracleSample(w, seed, args.cpu_seconds)
        dt = smp.run()
        cpu = {"value": smp.flops / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": smp.describe(args.workload, dt)}

    if rank == 0:
        dtype = {"bf16x3": "c64+bf16x3/fp64-refine", "tf32": "c64+tf32/fp64-refine", "fp64": "c128"}.get(
            args.precision, "c64/fp64-refine")
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": args.workload, "grid": [w["nx"], w["ny"], w["nz"]], "m": w["m"],
                           "n": p.n, "nrhs": nrhs, "k2": w["k2"], "tau": w["tau"], "precision": args.precision,
                           "cuda_graphs": bool(args.graphs), "seg_group": args.seg_group or "default",
                           "order": "nested dissection", "l2": "inputs larger than L2 (K is "
                           f"{K.numel() * 16 / 1e9:.2f} GB)"},
                "roofline": roof, "kernels": breakdown,
                "accuracy": {"omega": info["omega"], "omega_first_solve": info["omega_first"],
                             "refine_solves": info["refine_iters"]},
                "memory": memory,
                "fp64_path": fp64, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": int(launches),
                "flops_per_step": flops_step, "factor_flops": info["factor_flops"]}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
