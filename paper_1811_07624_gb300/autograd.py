"""Differentiable reflector transforms on top of the plan API.

``apply(X, U, d, sign, mode)`` is a ``torch.autograd.Function``: the forward
runs the library's apply kernel, the backward its adjoint kernel
(``hh_backward``), which recomputes the chain's intermediate vectors from the
saved output (modes "W", "WT") or, for "SYM", from p = W^T (sigma .* x) and
the output kept by the forward (``hh_apply_sym_p``, ``hh_backward_sym_py``).
Gradients flow to X, to the reflector rows U (as given, unnormalised) and to
the spectrum d.
"""

from __future__ import annotations

import torch

from .api import Plan


def _check_generation(ctx):
    # The plan holds the reflector values of the forward pass only until it is
    # updated in place; a backward after that would use the new values.
    if ctx.plan.generation != ctx.generation:
        raise RuntimeError(
            "the reflector plan was updated after this forward pass; its backward would use "
            "the new reflector values (run backward before the next optimiser step, or use a "
            "new plan)")


class _ChainFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, U, d, plan, mode):
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.mode = mode
        # SYM keeps p = W^T (sigma .* x) and the output: the adjoint reads both
        # states instead of recomputing them (hh_apply_sym_p, hh_backward_sym_py)
        if mode == "SYM":
            Y, P = plan.apply_sym_p(X.contiguous())
            ctx.save_for_backward(P, Y)
        else:
            Y = plan.apply_mode(mode, X.contiguous())
            ctx.save_for_backward(Y)
        return Y

    @staticmethod
    def backward(ctx, gY):
        _check_generation(ctx)
        saved = ctx.saved_tensors
        need_x, need_u, need_d = ctx.needs_input_grad[:3]
        sym = ctx.mode == "SYM"
        gX, gU, gd = ctx.plan.backward(ctx.mode, None if sym else saved[0], gY.contiguous(),
                                       need_gX=need_x, need_gU=need_u, need_gd=need_d and sym,
                                       Y=saved[1] if sym else None, P=saved[0] if sym else None)
        return gX, gU, gd, None, None


def apply(X: torch.Tensor, U: torch.Tensor, d: torch.Tensor | None = None,
          sign: torch.Tensor | None = None, mode: str = "W") -> torch.Tensor:
    """Rows of X through sigma.*(W x) ("W"), W^T(sigma.*x) ("WT") or
    sigma.*W(d.*W^T(sigma.*x)) ("SYM"), W = H_1...H_h with H_k from row k of U."""
    plan = Plan(U.detach(), d=None if d is None else d.detach(), sign=sign)
    return _ChainFunction.apply(X, U, d, plan, mode)


class _MahalanobisFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, U, d, plan, ia, ib):
        out = plan.mahalanobis(X.contiguous(), ia, ib)
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.save_for_backward(X, ia, ib)
        return out

    @staticmethod
    def backward(ctx, gout):
        _check_generation(ctx)
        X, ia, ib = ctx.saved_tensors
        gU, gd = ctx.plan.mahalanobis_backward(X.contiguous(), ia, ib, gout.contiguous(),
                                               need_gU=ctx.needs_input_grad[1],
                                               need_gd=ctx.needs_input_grad[2])
        return None, gU, gd, None, None, None


def mahalanobis(X: torch.Tensor, ia: torch.Tensor, ib: torch.Tensor, U: torch.Tensor,
                d: torch.Tensor, sign: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable fast Mahalanobis distances of the row pairs (ia[p], ib[p]) of X,
    with gradients for U and d (§IV-C)."""
    plan = Plan(U.detach(), d=d.detach(), sign=sign)
    return _MahalanobisFunction.apply(X, U, d, plan, ia, ib)


class ReflectorTransform(torch.nn.Module):
    """h learnable reflector vectors (rows of ``U``) and an optional learnable
    spectrum ``d``; ``forward(X, mode)`` applies the chain to the rows of X.

    The module keeps one plan and refreshes it in place (``hh_update``, no
    allocation or host synchronisation) when its parameters have changed since
    the last forward, e.g. after an optimiser step."""

    def __init__(self, n: int, h: int, spectrum: bool = True, sign: torch.Tensor | None = None,
                 dtype=torch.float32, device="cuda", generator=None):
        super().__init__()
        U = torch.randn(h, n, dtype=dtype, device=device, generator=generator)
        self.U = torch.nn.Parameter(U)
        self.d = torch.nn.Parameter(torch.ones(n, dtype=dtype, device=device)) if spectrum else None
        self.register_buffer("sign", None if sign is None else sign.to(device=device, dtype=torch.int8))
        self._plan = None
        self._plan_key = None

    def plan(self) -> Plan:
        """The plan for the current parameter values."""
        U = self.U.detach()
        d = None if self.d is None else self.d.detach()
        key = (U.data_ptr(), U._version, None if d is None else (d.data_ptr(), d._version))
        if self._plan is None or self._plan.dtype != U.dtype:
            self._plan = Plan(U.contiguous(), d=d, sign=self.sign)
        elif key != self._plan_key:
            self._plan.update(U.contiguous(), d)
        self._plan_key = key
        return self._plan

    def forward(self, X: torch.Tensor, mode: str = "W") -> torch.Tensor:
        plan = self.plan()
        return _ChainFunction.apply(X, self.U, self.d if mode == "SYM" else None, plan, mode)
