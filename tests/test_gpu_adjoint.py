"""Adjoint (hand-written backward that reuses the factors, K^T = K) against the oracle gradient
and central finite differences; J = Re(c^T x) with x = K(eps)^{-1} b."""
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


def _op(torch, g, m, k2, tau, seed, precision, perm):
    from paper_2002_05026_gb300.autograd import D3MOperator
    p0 = synth.make_problem(*g, m, k2, tau, seed, eps=np.zeros(g[0] * g[1] * g[2]))
    K0 = torch.from_numpy(p0.blocks).cuda()
    return p0, D3MOperator(p0.colptr, p0.rowidx, m, K0, p0.dom_if, k2, perm=perm, precision=precision)


def _oracle_grad(g, m, k2, tau, seed, eps, b, c, perm):
    p = synth.make_problem(*g, m, k2, tau, seed, eps=eps)
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, m)
    F = O.block_ldlt(O.permute_lower(Kb, perm), p.nblk, m)
    F.perm = perm
    x = O.block_solve(F, b)
    lam, geps, gb = O.adjoint_gradients(F, x, c, k2, p.dom_if, m)
    return p, Kb, x, lam, geps, gb


def _loss_and_grads(torch, op, eps, b, c):
    e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch.tensor(b, dtype=torch.complex128, device="cuda", requires_grad=True)
    x = op(e, bt)
    J = (torch.tensor(c, device="cuda") * x).sum().real
    J.backward()
    return J.item(), e.grad.cpu().numpy(), bt.grad.cpu().numpy(), x.detach().cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_grad_matches_oracle_small(torch_cuda, precision):
    g, m, k2, tau, seed = (3, 3, 1), 8, 2.0, 0.05, 31
    perm = O.nd_order(*g)
    p0, op = _op(torch_cuda, g, m, k2, tau, seed, precision, perm)
    eps = synth.domain_eps(17, 9)
    b = synth.rhs(3, p0.n, 1)
    c = synth.sparse_adjoint_vector(4, p0.n, m, support_block=int(perm[-1]))
    _, _, xo, lam, geps_o, gb_o = _oracle_grad(g, m, k2, tau, seed, eps, b, c, perm)
    J, geps, gb, x = _loss_and_grads(torch_cuda, op, eps, b, c)
    assert np.abs(J - np.real(c.T @ xo).item()) <= 1e-10 * abs(J)
    assert np.max(np.abs(geps - geps_o)) <= 1e-9 * np.max(np.abs(geps_o))
    assert np.max(np.abs(gb - gb_o)) <= 1e-9 * np.max(np.abs(gb_o))


def test_grad_central_differences(torch_cuda):
    g, m, k2, tau, seed = (3, 3, 1), 8, 2.0, 0.05, 32
    perm = O.nd_order(*g)
    p0, op = _op(torch_cuda, g, m, k2, tau, seed, "fp64", perm)
    eps = synth.domain_eps(18, 9)
    b = synth.rhs(5, p0.n, 1)
    c = synth.rhs(6, p0.n, 1)
    _, geps, gb, _ = _loss_and_grads(torch_cuda, op, eps, b, c)
    h = 1e-6
    tb = torch_cuda.tensor(b, device="cuda")
    tc = torch_cuda.tensor(c, device="cuda")

    def J(e, bb=tb):
        with torch_cuda.no_grad():
            return (tc * op(torch_cuda.tensor(e, device="cuda"), bb)).sum().real.item()

    for i in range(9):
        ep, em = eps.copy(), eps.copy()
        ep[i] += h
        em[i] -= h
        fd = (J(ep) - J(em)) / (2 * h)
        assert abs(fd - geps[i]) <= 1e-5 * np.max(np.abs(geps))
    for u in (0, 7, 30):
        for unit, comp in ((1.0, np.real), (1j, np.imag)):
            bp, bm = tb.clone(), tb.clone()
            bp[u] += h * unit
            bm[u] -= h * unit
            fd = (J(eps, bp) - J(eps, bm)) / (2 * h)
            assert abs(fd - comp(gb[u, 0])) <= 1e-5 * np.max(np.abs(gb))


def test_pattern_gradient(torch_cuda):
    g, m, k2, tau, seed = (2, 2, 1), 6, 1.0, 0.1, 33
    perm = O.nd_order(*g)
    p, Kb, x, lam, _, _ = _oracle_grad(g, m, k2, tau, seed, np.ones(4), synth.rhs(1, 24, 2), synth.rhs(2, 24, 2), perm)
    Go = O.pattern_gradient(Kb.keys(), m, lam, x)
    from paper_2002_05026_gb300 import D3M
    s = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="fp64")
    s.factor(torch_cuda.from_numpy(p.blocks).cuda())
    dK = s.grad_pattern(torch_cuda.from_numpy(lam).cuda(), torch_cuda.from_numpy(x).cuda(), p.blocks.size).cpu().numpy()
    got = O.lower_blocks(p.colptr, p.rowidx, dK, m)
    for k in Go:
        assert np.abs(got[k] - Go[k]).max() <= 1e-12 * np.abs(Go[k]).max()


def test_adjoint_workload_8x8_m256(torch_cuda):
    # 8x8x1 grid, m = 256, eps_i ~ U(1,4) (64 parameters), c ~ complex N(0,1) on the first
    # interface of the root separator; mixed precision vs the oracle gradient (<= 1e-9), and
    # central differences on four parameters with the FP64 path (<= 1e-5)
    w = synth.WORKLOADS["adjoint8x8_m256"]
    g, m, k2, tau, seed = (w["nx"], w["ny"], w["nz"]), w["m"], w["k2"], w["tau"], w["seed"]
    perm = O.nd_order(*g)
    eps = synth.domain_eps(seed, 64)
    p0, op = _op(torch_cuda, g, m, k2, tau, seed, "bf16x3", perm)
    b = synth.rhs(seed + 1, p0.n, 1)
    c = synth.sparse_adjoint_vector(seed + 2, p0.n, m, support_block=int(perm[-8]))
    _, _, xo, lam, geps_o, gb_o = _oracle_grad(g, m, k2, tau, seed, eps, b, c, perm)
    J, geps, gb, x = _loss_and_grads(torch_cuda, op, eps, b, c)
    assert np.max(np.abs(geps - geps_o)) <= 1e-9 * np.max(np.abs(geps_o))
    assert np.max(np.abs(gb - gb_o)) <= 1e-9 * np.max(np.abs(gb_o))
    _, op64 = _op(torch_cuda, g, m, k2, tau, seed, "fp64", perm)
    tb, tc = torch_cuda.tensor(b, device="cuda"), torch_cuda.tensor(c, device="cuda")
    h = 1e-6
    for i in (0, 9, 27, 63):
        ep, em = eps.copy(), eps.copy()
        ep[i] += h
        em[i] -= h
        with torch_cuda.no_grad():
            Jp = (tc * op64(torch_cuda.tensor(ep, device="cuda"), tb)).sum().real.item()
            Jm = (tc * op64(torch_cuda.tensor(em, device="cuda"), tb)).sum().real.item()
        assert abs((Jp - Jm) / (2 * h) - geps_o[i]) <= 1e-5 * np.max(np.abs(geps_o))
