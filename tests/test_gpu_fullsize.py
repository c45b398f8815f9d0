"""Parity at the full benchmark sizes, in the launch configuration bench.py times.

The oracle cannot factor these matrices in seconds, so the checks use what it can compute at
any size (Sec. I/II method; readings R7, R8, R14):
* the normwise backward error omega of the returned X, recomputed on the host in FP64 from the
  same K and B (oracle residual), must meet the 1e-12 target, and the device's own omega must
  agree with it;
* the mixed-precision solution must agree with the plain FP64 GPU path to 1e-9 (relative, per
  column), and the FP64 path's own omega must be at the FP64 rounding level;
* the 6 x 6 x 6 grid with m = 512 (n = 276,480, 32 right-hand sides, the largest single-GPU
  workload and the bench's default) gets the same two checks, for both tensor-core engines;
* batched: every one of the 256 uneven instances meets omega <= 1e-12 (oracle residual) and its
  solution agrees with a single-instance FP64 handle on a sample of instances.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2002_05026_gb300 import build
    build.build()
    return torch


def _fwd(X, Xr):
    return float(np.max(np.linalg.norm(X - Xr, axis=0) / np.linalg.norm(Xr, axis=0)))


def test_grid8x8_m512_full_size(torch_cuda):
    torch = torch_cuda
    from paper_2002_05026_gb300 import D3M, d3m_order_grid_nd
    w = synth.WORKLOADS["grid8x8_m512"]
    p = synth.make_problem(w["nx"], w["ny"], w["nz"], w["m"], w["k2"], w["tau"], w["seed"], device="cuda")
    perm = d3m_order_grid_nd(w["nx"], w["ny"], w["nz"])
    B = synth.rhs(w["seed"] + 1, p.n, w["nrhs"])
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    s = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision="bf16x3", max_nrhs=w["nrhs"])
    s.factor(p.blocks)
    X = s.solve(Bd).cpu().numpy()
    info = s.info()
    s.close()
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks.cpu().numpy(), p.m)
    om = O.omega(Kb, p.nblk, p.m, X, B)
    assert np.max(om) <= 1e-12, np.max(om)
    assert info["omega"] == pytest.approx(np.max(om), rel=0.05)
    s64 = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision="fp64", max_nrhs=w["nrhs"], fp64_omega=True)
    s64.factor(p.blocks)
    X64 = s64.solve(Bd).cpu().numpy()
    assert s64.info()["omega"] <= 1e-14
    s64.close()
    assert _fwd(X, X64) <= 1e-9


def test_grid6x6x6_m512_full_size(torch_cuda):
    """Both tensor-core engines (split-BF16x3 and TF32, the bench's choice at this size) against the
    oracle residual and the plain FP64 GPU path."""
    torch = torch_cuda
    from paper_2002_05026_gb300 import D3M, d3m_order_grid_nd
    w = synth.WORKLOADS["grid6x6x6_m512"]
    p = synth.make_problem(w["nx"], w["ny"], w["nz"], w["m"], w["k2"], w["tau"], w["seed"], device="cuda")
    perm = d3m_order_grid_nd(w["nx"], w["ny"], w["nz"])
    B = synth.rhs(w["seed"] + 1, p.n, w["nrhs"])
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Xs, infos = {}, {}
    for prec in ("bf16x3", "tf32"):
        s = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision=prec, max_nrhs=w["nrhs"])
        s.factor(p.blocks)
        Xs[prec] = s.solve(Bd).cpu().numpy()
        infos[prec] = s.info()
        s.close()
        torch.cuda.empty_cache()
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks.cpu().numpy(), p.m)
    for prec, X in Xs.items():
        om = O.omega(Kb, p.nblk, p.m, X, B)
        assert np.max(om) <= 1e-12, (prec, np.max(om))
        assert infos[prec]["omega"] == pytest.approx(np.max(om), rel=0.05, abs=5e-15), prec
    del Kb
    s64 = D3M(p.colptr, p.rowidx, m=p.m, perm=perm, precision="fp64", max_nrhs=w["nrhs"])
    s64.factor(p.blocks)
    X64 = s64.solve(Bd).cpu().numpy()
    s64.close()
    for prec, X in Xs.items():
        assert _fwd(X, X64) <= 1e-9, prec


def test_batch256_full_size(torch_cuda):
    torch = torch_cuda
    from paper_2002_05026_gb300 import D3M, D3MBatch, d3m_order_grid_nd
    specs = synth.batch_instances(256)
    probs = [synth.make_problem(q["nx"], q["ny"], q["nz"], q["m"], q["k2"], q["tau"], q["seed"], device="cuda")
             for q in specs]
    perms = [d3m_order_grid_nd(q["nx"], q["ny"], q["nz"]) for q in specs]
    Bs = [synth.rhs(q["seed"] + 1, p.n, 4) for q, p in zip(specs, probs)]
    K = torch.cat([p.blocks for p in probs])
    s = D3MBatch([(p.colptr, p.rowidx, p.m) for p in probs], perms, precision="bf16x3", max_nrhs=4, graphs=True)
    s.factor(K)
    X = s.solve(torch.from_numpy(np.ascontiguousarray(np.concatenate(Bs))).cuda()).cpu().numpy()
    w_dev = s.instance_omega()
    offs = s.offsets
    s.close()
    for i, p in enumerate(probs):
        Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks.cpu().numpy(), p.m)
        om = np.max(O.omega(Kb, p.nblk, p.m, X[offs[i]:offs[i + 1]], Bs[i]))
        assert om <= 1e-12, (i, om)
        # the device residual's floor is about 1e-15 of ||K|| ||x|| (several instances reach it)
        assert w_dev[i] == pytest.approx(om, rel=0.05, abs=5e-15), (i, w_dev[i], om)
    # sampled instances against a single-instance FP64 handle (includes the slowest-converging one)
    worst = int(np.argmax(w_dev))
    for i in sorted({0, 17, 100, 255, worst}):
        p = probs[i]
        one = D3M(p.colptr, p.rowidx, m=p.m, perm=perms[i], precision="fp64", max_nrhs=4)
        one.factor(p.blocks)
        X64 = one.solve(torch.from_numpy(np.ascontiguousarray(Bs[i])).cuda()).cpu().numpy()
        one.close()
        assert _fwd(X[offs[i]:offs[i + 1]], X64) <= 1e-9, i
