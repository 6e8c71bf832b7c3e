"""Differentiable multi-step zero-beta MHD on the GPU library (torch.autograd.Function).

`simulate(grid, state, nsteps, ...)` advances (vr, vt, vp, br, bt, bp) by `nsteps` calls of
mhd_step. Backward runs mhd_adjoint_step in reverse. The forward pass keeps a checkpoint of the
state every `checkpoint_every` steps and records each step's dt and alpha_SI. The backward pass
recomputes the states inside a segment from its checkpoint with those dt and alpha_SI frozen, which
reproduces the forward trajectory exactly, and then applies the adjoint steps backwards. That is
the map the adjoint differentiates: dt, alpha_SI, alpha_nu and the upwind directions held at
their forward values (all arithmetic stays in the CUDA library; this module only orders the calls
and holds the checkpoints).
"""
from __future__ import annotations

import torch

from . import (MHD_ERR_NOCONV, MHD_OK, make_fields, make_params, mhd_adjoint_step, mhd_step)

KEYS = ("vr", "vt", "vp", "br", "bt", "bp")


def _fields(t):
    return make_fields(t["br"], t["bt"], t["bp"], t["vr"], t["vt"], t["vp"])


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grid, prm_kw, nsteps, every, *tensors):
        state = {k: t.detach().clone() for k, t in zip(KEYS, tensors)}
        f = _fields(state)
        kwf = {k: v for k, v in prm_kw.items() if k != "adj_tol"}
        ckpts, dts, alphas = [], [], []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append({k: v.clone() for k, v in state.items()})
            st, info = mhd_step(grid, make_params(**kwf), f)
            if st not in (MHD_OK, MHD_ERR_NOCONV):
                raise RuntimeError(f"mhd_step failed with status {st}")
            dts.append(info["dt"])
            alphas.append(info["alpha_si"])
        ctx.grid, ctx.prm_kw, ctx.nsteps, ctx.every = grid, prm_kw, nsteps, every
        ctx.ckpts, ctx.dts, ctx.alphas = ckpts, dts, alphas
        ctx.adj_tol = prm_kw.get("adj_tol", prm_kw.get("tol", 1e-9))
        return tuple(state[k] for k in KEYS)

    @staticmethod
    def backward(ctx, *grads):
        grid, kw = ctx.grid, dict(ctx.prm_kw)
        kw.pop("adj_tol", None)
        lam = {k: (g.contiguous() if g is not None else torch.zeros_like(c)) for k, g, c in
               zip(KEYS, grads, (ctx.ckpts[0][k] for k in KEYS))}
        out = {k: torch.empty_like(v) for k, v in lam.items()}
        nseg = len(ctx.ckpts)
        for s in reversed(range(nseg)):
            n0 = s * ctx.every
            n1 = min(ctx.nsteps, n0 + ctx.every)
            # recompute the segment's states with the recorded dt and alpha_SI
            states = [{k: v.clone() for k, v in ctx.ckpts[s].items()}]
            for n in range(n0, n1 - 1):
                cur = {k: v.clone() for k, v in states[-1].items()}
                p = make_params(**dict(kw, dt_fixed=ctx.dts[n], alpha_si_fixed=ctx.alphas[n]))
                mhd_step(grid, p, _fields(cur))
                states.append(cur)
            for n in reversed(range(n0, n1)):
                p = make_params(**dict(kw, alpha_si_fixed=ctx.alphas[n], tol=ctx.adj_tol))
                st = mhd_adjoint_step(grid, p, _fields(states[n - n0]), ctx.dts[n], _fields(lam), _fields(out))
                if st not in (MHD_OK, MHD_ERR_NOCONV):
                    raise RuntimeError(f"mhd_adjoint_step failed with status {st}")
                lam, out = out, lam
        return (None, None, None, None) + tuple(lam[k] for k in KEYS)


def simulate(grid, state: dict, nsteps: int, checkpoint_every: int = 5, **params):
    """Advance `state` (dict of float64 CUDA tensors vr, vt, vp, br, bt, bp) by `nsteps` steps.
    Differentiable with respect to every input tensor. `params` go to make_params (nu, eta, cfl,
    tol, ...); `adj_tol` sets the PCG tolerance of the adjoint solves (default: tol)."""
    outs = _Steps.apply(grid, params, nsteps, checkpoint_every, *[state[k] for k in KEYS])
    return dict(zip(KEYS, outs))
