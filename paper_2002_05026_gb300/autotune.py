"""Autotuner: picks the tile engine (tile shape and tensor-core or SIMT tiles) for a given mix
of instances by timing the real factor + refined solve on the device, and measures the task
durations of the chosen engine that the device scheduler's critical-path priority is built from.

Candidates (each a complete configuration of libd3m.so):
  * "bf16x3" - 128 x 128 tiles, Schur updates as split-BF16x3 tcgen05 products;
  * "simt32" - 64 x 64 tiles, complex FP32 SIMT products.
Small interfaces waste most of a 128-row tile (m = 64 fills a quarter of it), large ones run
far faster on the tensor cores, so the best choice depends on the batch's mix of m.  Each
candidate is timed with CUDA events on the caller's stream after one untimed warm-up call
(which also captures its CUDA graphs); the result is cached per batch signature, in memory
and optionally in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from .solver import D3MBatch

CANDIDATES = ("bf16x3", "simt32")
_memo: dict = {}


def signature(instances, nrhs: int) -> str:
    """Order-independent key of a batch: the multiset of (blocks, block sizes, stored blocks)."""
    items = []
    for colptr, rowidx, msz in instances:
        sizes = (int(msz),) if np.isscalar(msz) else tuple(int(v) for v in msz)
        items.append((len(colptr) - 1, sizes, int(len(rowidx))))
    items.sort()
    h = hashlib.sha1(repr((items, int(nrhs))).encode()).hexdigest()[:16]
    return h


def fit_task_costs(trace: np.ndarray) -> list:
    """Duration model cost = base + per_k * nk (ns) for the three task kinds of the factorization
    (update, diagonal final, off-diagonal final), least squares over the traced tasks
    (trace rows: start_ns, end_ns, sm, flags | tile << 8 | nk << 40, ...; a paired update task,
    flag 32, counts 2 nk tile products).  The paper weights its
    dual tasks with benchmarked GEMM, sytrf and triSolve times (Sec. II); here the benchmark is a
    traced factorization of the actual pattern."""
    ok = (trace[:, 0] > 0) & (trace[:, 1] >= trace[:, 0])
    t = trace[ok]
    dur = (t[:, 1] - t[:, 0]).astype(np.float64)
    flags = t[:, 3] & 0xFF
    nk = (t[:, 3] >> 40).astype(np.float64)
    nk = np.where(flags & 32, 2.0 * nk, nk)      # a paired update task does nk products for two tiles
    kind = np.where(flags & 4, 0, np.where(flags & 1, 1, 2))
    out = []
    for k in range(3):
        sel = kind == k
        if sel.sum() == 0:
            out += [0.0, 0.0]
            continue
        A = np.stack([np.ones(sel.sum()), nk[sel]], axis=1)
        if np.ptp(nk[sel]) == 0:
            coef = np.array([np.median(dur[sel]), 0.0])
        else:
            coef, *_ = np.linalg.lstsq(A, dur[sel], rcond=None)
        base, per = float(coef[0]), float(coef[1])
        # a model must stay positive over the tasks it covers
        base = max(base, 1.0)
        per = max(per, 0.0)
        out += [base, per]
    return out


def measure_task_costs(instances, perms, K, precision: str, batch: bool = True, stream=None) -> list:
    """Factor once with task tracing (after one untimed warm-up) and fit the duration model."""
    from .solver import D3M
    if batch:
        s = D3MBatch(instances, perms, precision=precision, debug_flags=2, stream=stream)
    else:
        colptr, rowidx, m = instances[0]
        s = D3M(colptr, rowidx, m=m, perm=perms[0] if perms else None, precision=precision, debug_flags=2,
                stream=stream)
    try:
        s.factor(K)
        s.factor(K)
        return fit_task_costs(s.trace())
    finally:
        s.close()


def _time_candidate(instances, perms, K, B, nrhs, precision, reps, stream):
    import torch
    s = D3MBatch(instances, perms, precision=precision, max_nrhs=nrhs, graphs=True, stream=stream)
    try:
        X = torch.empty_like(B)
        st = stream if stream is not None else torch.cuda.current_stream()

        def once():
            s.factor(K)
            s.solve(B.T, X=X, allow_not_converged=True)

        once()                                   # warm-up, graph capture
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            once()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        w = float(np.max(s.instance_omega()))
        return ms, w
    finally:
        s.close()


def tune_batch(instances, perms, K, B, nrhs: int, candidates=CANDIDATES, reps: int = 2, tol: float = 1e-12,
               cache_path: str | None = None, stream=None) -> dict:
    """Time every candidate on this batch (K: device lower blocks of all instances; B: device
    (nrhs, n) column-major right-hand sides) and return {"precision", "ms", "timings", "key"}.
    A candidate whose refinement does not reach `tol` is never chosen."""
    key = signature(instances, nrhs)
    if key in _memo:
        return _memo[key]
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            disk = json.load(f)
        if key in disk and disk[key].get("precision") in candidates:
            _memo[key] = disk[key]
            return disk[key]
    timings = {}
    for c in candidates:
        ms, w = _time_candidate(instances, perms, K, B, nrhs, c, reps, stream)
        timings[c] = {"ms": ms, "omega": w}
    ok = [c for c in candidates if timings[c]["omega"] <= tol]
    if not ok:
        raise RuntimeError(f"no candidate reached omega <= {tol}: {timings}")
    best = min(ok, key=lambda c: timings[c]["ms"])
    res = {"precision": best, "ms": timings[best]["ms"], "timings": timings, "key": key,
           "task_cost": measure_task_costs(instances, perms, K, best, batch=True, stream=stream)}
    _memo[key] = res
    if cache_path:
        disk = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                disk = json.load(f)
        disk[key] = res
        with open(cache_path, "w") as f:
            json.dump(disk, f, indent=1)
    return res
