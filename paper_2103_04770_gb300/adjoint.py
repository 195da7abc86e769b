"""Differentiable final homogenised stress: a torch.autograd.Function whose
backward is the library's hand-written reverse sweep over the converged
increments (rve_adjoint_forward / rve_adjoint_backward of the C ABI)."""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B

PARAM_KEYS = ("sigma_y", "H", "eps_C", "eps_R")


def _phase_dicts(cfg, params):
    out = []
    for q, d in enumerate(cfg.params):
        e = dict(d)
        for k, key in enumerate(PARAM_KEYS):
            e[key] = float(params[q, k])
        out.append(e)
    return out


def _ell_table(cfg, ell_own):
    ell = np.array(cfg.ell, dtype=np.float64, copy=True)
    for j in range(ell.shape[0]):
        ell[j] *= float(ell_own[j]) / float(np.max(cfg.ell[j]))
    return ell


class FinalStress(torch.autograd.Function):
    """J = <sigma_N>_11 after the whole load path of ``cfg`` (FP64), as a
    function of the per-phase parameters [n_phases, 4] (sigma_y, H, eps_C,
    eps_R; kappa_C, kappa_R for cracking phases), the own-phase length of
    every non-local variable [J] (its row of the length table scales with
    it) and the per-voxel modulus factor [V].  The forward pass keeps a
    checkpoint every ``checkpoint_every`` increments; the backward pass
    re-solves each segment from its checkpoint and runs the adjoint."""

    @staticmethod
    def forward(ctx, params, ell_own, stiff, cfg, checkpoint_every=5, options=None):
        p = params.detach().cpu().double().numpy()
        e = ell_own.detach().cpu().double().numpy()
        s = stiff.detach().cpu().double().numpy()
        J = int(np.asarray(cfg.ell).shape[0])
        h = B.rve_create(len(cfg.n), cfg.n, cfg.L, B.RVE_FP64, J)
        try:
            if options is not None:
                B.rve_set_options(h, options)
            B.rve_set_phases(h, cfg.phase, _phase_dicts(cfg, p), _ell_table(cfg, e))
            B.rve_set_load_path(h, cfg.strain_ctrl, cfg.target)
            B.rve_set_stiffness_field(h, s)
            val = B.rve_adjoint_forward(h, checkpoint_every)
        except Exception:
            B.rve_free(h)
            raise
        ctx.h = h
        ctx.dims = (p.shape[0], J, s.size)
        ctx.dev = params.device
        ctx.info = None
        return torch.tensor(val, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, gJ):
        h = ctx.h
        try:
            gp, ge, gs, info = B.rve_adjoint_backward(h, float(gJ), *ctx.dims)
        finally:
            B.rve_free(h)
            ctx.h = None
        FinalStress.last_info = info
        dev = ctx.dev
        return (torch.as_tensor(gp, device=dev), torch.as_tensor(ge, device=dev),
                torch.as_tensor(gs, device=dev), None, None, None)


def final_stress(cfg, params=None, ell_own=None, stiff=None, checkpoint_every=5, options=None):
    """Convenience wrapper: tensors default to the values in ``cfg``."""
    if params is None:
        params = torch.tensor([[d[k] for k in PARAM_KEYS] for d in cfg.params], dtype=torch.float64)
    if ell_own is None:
        ell_own = torch.tensor(np.max(np.asarray(cfg.ell), axis=1), dtype=torch.float64)
    if stiff is None:
        stiff = torch.ones(int(np.prod(cfg.n)), dtype=torch.float64)
    return FinalStress.apply(params, ell_own, stiff, cfg, checkpoint_every, options)
