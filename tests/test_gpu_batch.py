"""Batched handles (d3m_create_batch): uneven instances in one block-diagonal system, one
persistent factorization launch and level-merged sweeps, checked instance by instance against
the FP64 oracle with the same bars as single systems."""
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


def _instances(specs):
    out = []
    for (g, m, k2, tau, seed) in specs:
        p = synth.make_problem(*g, m, k2, tau, seed)
        pm = O.nd_order(*g)
        Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, p.m)
        F = O.block_ldlt(O.permute_lower(Kb, pm), p.nblk, p.m)
        F.perm = pm
        out.append((p, pm, Kb, F))
    return out


SPECS = [((2, 2, 1), 64, 1.0, 0.1, 1), ((3, 3, 1), 16, 2.5, 0.05, 2), ((2, 2, 1), 100, 0.7, 0.15, 3),
         ((4, 4, 1), 32, 3.0, 0.02, 4), ((1, 2, 1), 128, 2.0, 0.05, 5), ((3, 2, 1), 200, 1.5, 0.1, 6)]


@pytest.mark.parametrize("precision", ["fp64", "bf16x3", "simt32"])
def test_batch_matches_oracle_per_instance(torch_cuda, precision):
    from paper_2002_05026_gb300 import D3MBatch
    inst = _instances(SPECS)
    s = D3MBatch([(p.colptr, p.rowidx, p.m) for p, _, _, _ in inst], perms=[pm for _, pm, _, _ in inst],
                 precision=precision, max_nrhs=4, fp64_omega=True)
    assert s.info()["instances"] == len(inst)
    K = np.concatenate([p.blocks for p, _, _, _ in inst])
    s.factor(torch_cuda.from_numpy(K).cuda())
    nrhs = 3
    Bs = [synth.rhs(50 + i, p.n, nrhs) for i, (p, _, _, _) in enumerate(inst)]
    X = s.solve(torch_cuda.from_numpy(np.ascontiguousarray(np.concatenate(Bs))).cuda()).cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-9
    w = s.instance_omega()
    for i, (p, pm, Kb, F) in enumerate(inst):
        Xi = X[s.offsets[i]:s.offsets[i + 1]]
        Xo = O.block_solve(F, Bs[i])
        err = np.max(np.linalg.norm(Xi - Xo, axis=0) / np.linalg.norm(Xo, axis=0))
        assert err <= tol, (i, err)
        wo = np.max(O.omega(Kb, p.nblk, p.m, Xi, Bs[i]))
        if precision != "fp64":
            assert wo <= 1e-12 and w[i] <= 1e-12, (i, wo, w[i])
        # the per-instance omega is the instance's own (its ||K_i||, |x_i|, |b_i|)
        if precision == "fp64":
            assert w[i] <= 1e-14 and wo <= 1e-14, (i, w[i], wo)      # FP64 rounding level
        else:
            assert w[i] == pytest.approx(wo, rel=0.02), (i, w[i], wo)
    info = s.info()
    assert info["status"] == 0
    assert info["factor_kernel_calls"] == 1          # one persistent launch for all instances


def test_batch_omega_is_per_instance(torch_cuda):
    # instance 1 scaled by 1e6: a global norm would hide instance 0's residual behind it
    from paper_2002_05026_gb300 import D3MBatch
    inst = _instances(SPECS[:2])
    K0 = inst[0][0].blocks
    K1 = inst[1][0].blocks * 1e6
    s = D3MBatch([(p.colptr, p.rowidx, p.m) for p, _, _, _ in inst], perms=[pm for _, pm, _, _ in inst],
                 precision="bf16x3", max_nrhs=2)
    s.factor(torch_cuda.from_numpy(np.concatenate([K0, K1])).cuda())
    B0 = synth.rhs(7, inst[0][0].n, 2)
    B1 = synth.rhs(8, inst[1][0].n, 2) * 1e6
    X = s.solve(torch_cuda.from_numpy(np.ascontiguousarray(np.concatenate([B0, B1]))).cuda()).cpu().numpy()
    X0 = X[:inst[0][0].n]
    Xo = O.block_solve(inst[0][3], B0)
    assert np.max(np.linalg.norm(X0 - Xo, axis=0) / np.linalg.norm(Xo, axis=0)) <= 1e-9
    w = s.instance_omega()
    assert np.all(w <= 1e-12)


def test_batch_equals_single_handles(torch_cuda):
    # FP64: the batched factors are the single-instance factors (same tile tasks, same order)
    from paper_2002_05026_gb300 import D3M, D3MBatch
    inst = _instances(SPECS[:3])
    s = D3MBatch([(p.colptr, p.rowidx, p.m) for p, _, _, _ in inst], perms=[pm for _, pm, _, _ in inst],
                 precision="fp64", max_nrhs=2)
    s.factor(torch_cuda.from_numpy(np.concatenate([p.blocks for p, _, _, _ in inst])).cuda())
    off = 0
    for i, (p, pm, Kb, F) in enumerate(inst):
        one = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision="fp64", max_nrhs=2)
        one.factor(torch_cuda.from_numpy(p.blocks).cuda())
        for (a, b) in list(F.L.keys())[:6]:
            La = s.factor_block(off + a, off + b, p.m, p.m)
            Lb = one.factor_block(a, b, p.m, p.m)
            assert np.array_equal(La, Lb), (i, a, b)
        off += p.nblk


def test_graph_replay_matches_stream_launches(torch_cuda):
    # graphs=1 replays captured launch sequences: same kernels, same inputs, same bits
    from paper_2002_05026_gb300 import D3MBatch
    inst = _instances(SPECS[:4])
    K = torch_cuda.from_numpy(np.concatenate([p.blocks for p, _, _, _ in inst])).cuda()
    B = np.concatenate([synth.rhs(60 + i, p.n, 3) for i, (p, _, _, _) in enumerate(inst)])
    Bd = torch_cuda.from_numpy(np.ascontiguousarray(B)).cuda()
    out, launches = [], []
    for graphs in (False, True):
        s = D3MBatch([(p.colptr, p.rowidx, p.m) for p, _, _, _ in inst], perms=[pm for _, pm, _, _ in inst],
                     precision="bf16x3", max_nrhs=3, graphs=graphs)
        l0 = s.info()["kernel_launches"]
        for _ in range(3):                       # first round captures, later rounds replay
            s.factor(K)
            X = s.solve(Bd).cpu().numpy()
        out.append(X)
        launches.append(s.info()["kernel_launches"] - l0)
        s.close()
    assert np.array_equal(out[0], out[1])
    assert launches[0] == launches[1]


def test_autotuner_picks_a_converging_engine(torch_cuda):
    from paper_2002_05026_gb300 import D3MBatch, autotune
    inst = _instances(SPECS[:3])
    K = torch_cuda.from_numpy(np.concatenate([p.blocks for p, _, _, _ in inst])).cuda()
    B = np.concatenate([synth.rhs(70 + i, p.n, 2) for i, (p, _, _, _) in enumerate(inst)])
    Bt = torch_cuda.from_numpy(np.ascontiguousarray(B.T)).cuda()
    spec = [(p.colptr, p.rowidx, p.m) for p, _, _, _ in inst]
    perms = [pm for _, pm, _, _ in inst]
    res = autotune.tune_batch(spec, perms, K, Bt, nrhs=2, reps=1)
    assert res["precision"] in autotune.CANDIDATES
    assert set(res["timings"]) == set(autotune.CANDIDATES)
    assert res["ms"] == min(v["ms"] for v in res["timings"].values() if v["omega"] <= 1e-12)
    assert autotune.tune_batch(spec, perms, K, Bt, nrhs=2) is res          # cached by signature
    # the measured task-duration model (ns): positive, and the update tasks' cost grows with
    # their tile products; the handle built with it still solves to the oracle's accuracy
    tc = res["task_cost"]
    assert len(tc) == 6 and all(v >= 0 for v in tc) and tc[0] > 0 and tc[2] > 0
    s = D3MBatch(spec, perms, precision=res["precision"], max_nrhs=2, task_cost=tc)
    s.factor(K)
    X = s.solve(Bt.T).cpu().numpy()
    for i, (p, pm, Kb, F) in enumerate(inst):
        Xi = X[int(s.offsets[i]):int(s.offsets[i + 1])]
        Bi = B[int(s.offsets[i]):int(s.offsets[i + 1])]
        Xo = O.block_solve(F, Bi)
        assert np.max(np.linalg.norm(Xi - Xo, axis=0) / np.linalg.norm(Xo, axis=0)) <= 1e-9


def test_measured_task_costs_single_handle(torch_cuda):
    # a traced factorization of the 4x4 m = 512 pattern gives the duration model: the update
    # tasks' cost per tile product and the diagonal tasks' cost are positive and of the order of
    # the tensor-core engine's tile times (microseconds); a handle built with the model factors
    # and solves to the oracle's accuracy
    from paper_2002_05026_gb300 import D3M, autotune
    g, m = (4, 4, 1), 512
    p = synth.make_problem(*g, m, 2.0, 0.05, 41)
    perm = O.nd_order(*g)
    K = torch_cuda.from_numpy(p.blocks).cuda()
    tc = autotune.measure_task_costs([(p.colptr, p.rowidx, m)], [perm], K, "bf16x3", batch=False)
    assert 100.0 < tc[1] < 1e6 and 100.0 < tc[2] < 1e7, tc
    s = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="bf16x3", max_nrhs=4, task_cost=tc)
    s.factor(K)
    B = synth.rhs(5, p.n, 2)
    X = s.solve(torch_cuda.from_numpy(np.ascontiguousarray(B)).cuda()).cpu().numpy()
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, m)
    assert np.max(O.omega(Kb, p.nblk, m, X, B)) <= 1e-12
