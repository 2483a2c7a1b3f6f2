"""torch.autograd wrapper of the solver: X = A^-1 B and log det A as
differentiable functions of A's stored lower values (and of B).

Forward: FP64 factorization of P A P^T (Section 4), the two triangular solves
and log det A = 2 sum_j log L_jj.  Backward: one more solve for G = A^-1 dl/dX
and the value gradient

    dl/dv_e = g_logdet * w_e * (A^-1)(i, j) - (G_i . X_j + G_j . X_i)   (i != j)
    dl/dv_e = g_logdet * (A^-1)(i, i)       -  G_i . X_i                (i == j)

with w_e = 2 because a stored off-diagonal value stands for both (i, j) and
(j, i).  A^-1 is needed only on the pattern of A, which lies inside the
pattern of L: it comes from the selected inverse (Takahashi's recurrences on
the supernodal factor), never from a dense inverse.  Every step runs in the
CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import Solver


def _colmajor(t: torch.Tensor) -> torch.Tensor:
    """A column-major (stride(0) == 1, leading dimension n) FP64 copy; always
    a new tensor, since the solver overwrites it."""
    if t.dim() == 1:
        t = t.unsqueeze(1)
    out = torch.empty((t.shape[1], t.shape[0]), dtype=torch.float64, device=t.device).t()
    out.copy_(t.detach())
    return out


class SPDSystem:
    """One sparsity pattern of A (lower CSC incl. the diagonal, sorted),
    analyzed once; its values may change between calls."""

    def __init__(self, colptr, rowidx, basis=None, **solver_options):
        self.solver = Solver(**solver_options).analyze(colptr, rowidx, basis)
        self.n = self.solver.n
        self.nnz = self.solver.nnz
        self._values = None      # values of the current factorization
        self._token = 0

    def _factor(self, values: torch.Tensor) -> int:
        v = values.detach().to(torch.float64).contiguous()
        if not v.is_cuda:
            raise ValueError("values must be a CUDA tensor")
        self.solver.factor(v, "fp64")
        self._values = v
        self._token += 1
        return self._token

    def solve_logdet(self, values: torch.Tensor, B: torch.Tensor):
        """(X, logdet) with X = A(values)^-1 B, differentiable in values and B."""
        return _SolveLogdet.apply(values, B, self)

    def solve(self, values: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
        return self.solve_logdet(values, B)[0]

    def logdet(self, values: torch.Tensor) -> torch.Tensor:
        B = torch.zeros((self.n, 0), dtype=torch.float64, device=values.device)
        return self.solve_logdet(values, B)[1]


class _SolveLogdet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, B, system: SPDSystem):
        squeeze = B.dim() == 1
        token = system._factor(values)
        s = system.solver
        X = _colmajor(B)
        if X.shape[1] > 0:
            s.solve(X, with_info=False)
        ld = torch.tensor(s.logdet(), dtype=torch.float64, device=values.device)
        ctx.system = system
        ctx.token = token
        ctx.squeeze = squeeze
        ctx.save_for_backward(values.detach(), X)
        Xo = X[:, 0] if squeeze else X
        return Xo, ld

    @staticmethod
    def backward(ctx, gX, gld):
        values, X = ctx.saved_tensors
        system: SPDSystem = ctx.system
        s = system.solver
        if system._token != ctx.token:      # another factorization happened since forward
            ctx.token = system._factor(values)
        g_logdet = float(gld) if gld is not None else 0.0
        ncols = X.shape[1]
        if gX is not None and ncols > 0:
            G = _colmajor(gX)
            s.solve(G, with_info=False)
        else:
            G = torch.zeros_like(X)
        gvals = s.value_gradient(g_logdet, X, G) if (ncols > 0 or g_logdet != 0.0) else None
        if gvals is None:
            gvals = torch.zeros(system.nnz, dtype=torch.float64, device=X.device)
        gB = None
        if ctx.needs_input_grad[1]:
            gB = G[:, 0] if ctx.squeeze else G
        return gvals.to(values.dtype), gB, None


def gp_negative_log_likelihood(system: SPDSystem, values: torch.Tensor, Y: torch.Tensor,
                               mean: bool = False) -> torch.Tensor:
    """1/2 sum_c y_c^T A^-1 y_c + (ncols / 2) log det A  (mean=True: divided by
    the number of columns); the Gaussian negative log-likelihood of the
    columns of Y up to the constant (n / 2) log 2 pi per column."""
    if Y.dim() == 1:
        Y = Y.unsqueeze(1)
    X, ld = system.solve_logdet(values, Y)
    m = Y.shape[1]
    loss = 0.5 * (Y.to(torch.float64) * X).sum() + 0.5 * m * ld
    return loss / m if mean else loss
