"""torch.autograd adjoints of the coupling-step operators.

Every forward and backward runs in libifem's CUDA kernels through the C ABI;
these classes only wire them into torch's autograd graph.

* ``SpreadFn``: f = S*(F) in the density form, f_J = (n/L)^3 sum_k phi_Jk F_k.
  Its transpose is (n/L)^3 times interpolation: dL/dF_k = (n/L)^3 sum_J phi_Jk g_J.
* ``InterpFn``: v = S(u), v_k = sum_J phi_Jk u_J. Its transpose is spreading in
  the literal force form: dL/du_J = sum_k phi_Jk g_k.
* ``ElasticForceFn``: F = F_el(x) = -dE/dx (Eq. FEM / FEM_Membrane without
  bending). Its Jacobian is -H with H the (symmetric) Hessian of E, so
  dL/dx = -H g, computed by ``ifem_force_hvp``.

Node positions enter S and S* through the kernel weights; gradients with
respect to x through the weights are not propagated by SpreadFn / InterpFn
(None is returned), as the coupling step treats the stencil as fixed within
a step.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ifem as I


def _node_box_scale(coupler) -> torch.Tensor:
    """(n_b/L_b)^3 of each node's box, as a (1, N) tensor of the coupler's dtype."""
    wl = coupler.wl
    s = np.concatenate([np.full(wl.templates[i.tmpl].n_nodes, (wl.boxes[i.box].n / wl.boxes[i.box].L) ** 3)
                        for i in wl.instances]) if wl.instances else np.zeros(0)
    return torch.as_tensor(s, dtype=coupler.dtype, device=coupler.device)[None, :]


class SpreadFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, x, coupler):
        f = coupler.zeros_grid()
        I.ifem_spread(coupler.ctx, coupler.batch, coupler.grid, x.contiguous(), F.contiguous(), f,
                      I.IFEM_SPREAD_DENSITY)
        ctx.coupler = coupler
        ctx.save_for_backward(x)
        return f

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        cp = ctx.coupler
        v = cp.empty_nodes()
        I.ifem_interpolate(cp.ctx, cp.batch, cp.grid, g.contiguous(), x.contiguous(), v)
        return v * _node_box_scale(cp), None, None


class InterpFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, x, coupler):
        v = coupler.empty_nodes()
        I.ifem_interpolate(coupler.ctx, coupler.batch, coupler.grid, u.contiguous(), x.contiguous(), v)
        ctx.coupler = coupler
        ctx.save_for_backward(x)
        return v

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        cp = ctx.coupler
        gu = cp.zeros_grid()
        I.ifem_spread(cp.ctx, cp.batch, cp.grid, x.contiguous(), g.contiguous(), gu, I.IFEM_SPREAD_FORCE)
        return gu, None, None


class ElasticForceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, coupler):
        if any(t.kind == "membrane" and t.kb != 0.0 for t in coupler.wl.templates):
            raise ValueError("ElasticForceFn: the Hessian-vector product covers the elastic energy only; "
                             "use templates without bending")
        F = coupler.empty_nodes()
        I.ifem_compute_forces(coupler.ctx, coupler.batch, x.contiguous(), F)
        ctx.coupler = coupler
        ctx.save_for_backward(x)
        return F

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        cp = ctx.coupler
        Hg = cp.empty_nodes()
        I.ifem_force_hvp(cp.ctx, cp.batch, x.contiguous(), g.contiguous(), Hg)
        return -Hg, None


def spread(F, x, coupler):
    return SpreadFn.apply(F, x, coupler)


def interpolate(u, x, coupler):
    return InterpFn.apply(u, x, coupler)


def elastic_forces(x, coupler):
    return ElasticForceFn.apply(x, coupler)
