"""torch.autograd front end: x = K(eps)^{-1} b with a hand-written adjoint that reuses the factors.

K(eps) = K0 - k^2 sum_i eps_i E_i, where K0 is the assembled dual matrix at eps = 0 and E_i is
the identity on the unknowns of the interfaces of domain i (every interface belongs to the two
domains it separates).  Forming K(eps) is a diagonal shift of K0 (input assembly, done with
torch); the factorization, the solves and the gradient contractions run in libd3m.so.

Backward, for a real loss with upstream gradient g = dL/dRe(x) + i dL/dIm(x) (PyTorch's
convention): lambda = K^{-1} conj(g) with the same factors (K^T = K, d3m_adjoint),
dL/db = conj(lambda), dL/deps_i = Re(k^2 sum_{u in I(i)} lambda_u x_u) (d3m_grad_eps).
"""
from __future__ import annotations

import numpy as np
import torch

from .solver import D3M


class D3MOperator:
    """Holds the pattern, K0, the domain -> interface lists and one library handle."""

    def __init__(self, colptr, rowidx, m: int, K0: torch.Tensor, dom_if, k2: float, perm=None,
                 precision: str = "bf16x3", max_nrhs: int = 32):
        self.m = int(m)
        self.k2 = float(k2)
        self.dom_if = [list(map(int, I)) for I in dom_if]
        self.K0 = K0
        self.handle = D3M(colptr, rowidx, m=m, perm=perm, precision=precision, max_nrhs=max_nrhs)
        nblk = len(colptr) - 1
        colptr = np.asarray(colptr)
        # flat positions of the diagonal entries of every diagonal block (block (f, f) is the
        # first block of column f; column-major m x m)
        diag_blk = colptr[:-1].astype(np.int64)
        u = np.arange(self.m, dtype=np.int64)
        pos = (diag_blk[:, None] * self.m * self.m + u[None, :] * (self.m + 1)).reshape(-1)
        self.diag_pos = torch.from_numpy(pos).to(K0.device)
        # interface -> its domains
        owners = [[] for _ in range(nblk)]
        for i, I in enumerate(self.dom_if):
            for f in I:
                owners[f].append(i)
        rows, cols = [], []
        for f, ds in enumerate(owners):
            for d in ds:
                rows.append(f)
                cols.append(d)
        A = torch.zeros(nblk, len(self.dom_if), dtype=torch.float64)
        A[rows, cols] = 1.0
        self.if_dom = A.to(K0.device)          # interface x domain incidence

    def assemble(self, eps: torch.Tensor) -> torch.Tensor:
        shift = -self.k2 * (self.if_dom @ eps.to(torch.float64))      # per interface
        K = self.K0.clone()
        K[self.diag_pos] += shift.repeat_interleave(self.m).to(K.dtype)
        return K

    def __call__(self, eps: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        return D3MSolveFn.apply(eps, b, self)


class D3MSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, b, op: D3MOperator):
        K = op.assemble(eps.detach())
        op.handle.factor(K)
        x = op.handle.solve(b.detach())
        ctx.op = op
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        op = ctx.op
        lam = op.handle.adjoint(torch.conj(gx).resolve_conj())        # K^T = K: same factors
        x2 = x if x.dim() == 2 else x.reshape(-1, 1)
        l2 = lam if lam.dim() == 2 else lam.reshape(-1, 1)
        geps = op.handle.grad_eps(l2, x2, op.dom_if, op.k2)
        grad_eps = torch.from_numpy(geps).to(x.device)
        return grad_eps, torch.conj(lam), None
