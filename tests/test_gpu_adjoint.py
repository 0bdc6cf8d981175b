"""Adjoint pair and Hessian-vector product through torch.autograd (FP64 GPU).

interp is the transpose of spread (<interp u, F> = h^3 <u, spread F>), the
autograd backward passes match central finite differences of the forward
maps at eps = 1e-6, and the backward of the element forces (-H g, from
ifem_force_hvp) matches central differences of F and the oracle's HVP.
"""
import dataclasses

import numpy as np
import pytest

import ifem_workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _coupler(wl, precision=1):
    from paper_1807_08219_gb300 import ifem as I
    return I.Coupler(wl, precision=precision)


@pytest.mark.parametrize("kernel", [0, 1])
def test_adjoint_identity_on_gpu(kernel):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    wl = W.make("C3")
    cp = I.Coupler(wl, precision=I.IFEM_FP64, kernel=kernel)
    try:
        rng = np.random.default_rng(0)
        x = cp.nodes_to_device(wl.x_local_all())
        F = cp.nodes_to_device(rng.standard_normal((wl.n_nodes, 3)))
        u = cp.grid_to_device([rng.standard_normal((3, b.n, b.n, b.n)) for b in wl.boxes])
        f, v = cp.zeros_grid(), cp.empty_nodes()
        I.ifem_spread(cp.ctx, cp.batch, cp.grid, x, F, f)
        I.ifem_interpolate(cp.ctx, cp.batch, cp.grid, u, x, v)
        h3 = (wl.boxes[0].L / wl.boxes[0].n) ** 3
        lhs = float((v * F).sum())
        rhs = h3 * float((u * f).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12)
    finally:
        cp.close()


def test_spread_and_interp_backward_vs_fd():
    import torch
    from paper_1807_08219_gb300 import autograd as A
    wl = W.make("C1")
    cp = _coupler(wl)
    try:
        rng = np.random.default_rng(1)
        x = cp.nodes_to_device(wl.x_local_all())
        F = cp.nodes_to_device(rng.standard_normal((wl.n_nodes, 3))).requires_grad_(True)
        wgrid = cp.grid_to_device([rng.standard_normal((3, b.n, b.n, b.n)) for b in wl.boxes])
        L = (A.spread(F, x, cp) * wgrid).sum()
        L.backward()
        dF = cp.nodes_to_device(rng.standard_normal((wl.n_nodes, 3)))
        eps = 1e-6
        with torch.no_grad():
            Lp = (A.spread(F + eps * dF, x, cp) * wgrid).sum()
            Lm = (A.spread(F - eps * dF, x, cp) * wgrid).sum()
        fd = float((Lp - Lm) / (2 * eps))
        assert float((F.grad * dF).sum()) == pytest.approx(fd, rel=1e-7)

        u = wgrid.clone().requires_grad_(True)
        gv = cp.nodes_to_device(rng.standard_normal((wl.n_nodes, 3)))
        Lv = (A.interpolate(u, x, cp) * gv).sum()
        Lv.backward()
        du = cp.grid_to_device([rng.standard_normal((3, b.n, b.n, b.n)) for b in wl.boxes])
        with torch.no_grad():
            fd = float((((A.interpolate(u + eps * du, x, cp) - A.interpolate(u - eps * du, x, cp)) * gv).sum())
                       / (2 * eps))
        assert float((u.grad * du).sum()) == pytest.approx(fd, rel=1e-7)
    finally:
        cp.close()


@pytest.mark.parametrize("case", ["C3", "C1-skalak", "C2-elastic"])
def test_elastic_force_backward_vs_fd_and_oracle(case):
    import torch
    from paper_1807_08219_gb300 import autograd as A
    if case == "C3":
        wl = W.make("C3")
    elif case == "C1-skalak":
        wl = W.make("C1", law="skalak")
    else:
        w2 = W.make("C2")
        wl = dataclasses.replace(w2, templates=[dataclasses.replace(t, kb=0.0) for t in w2.templates])
    cp = _coupler(wl)
    try:
        rng = np.random.default_rng(2)
        xl = wl.x_local_all()
        x = cp.nodes_to_device(xl).requires_grad_(True)
        g = cp.nodes_to_device(rng.standard_normal((wl.n_nodes, 3)))
        (A.elastic_forces(x, cp) * g).sum().backward()
        grad = cp.nodes_to_host(x.grad)
        # oracle: d/dx <g, F(x)> = -H g
        tm = wl.templates[0]
        gh = cp.nodes_to_host(g)
        if tm.kind == "membrane":
            Hg = O.membrane_hvp(tm.law, tm.mu, tm.C, tm.elems, tm.X, xl, gh)
        else:
            Hg = O.tet_hvp(tm.lam, tm.mu, tm.elems, tm.X, xl, gh)
        assert np.linalg.norm(grad + Hg) <= 1e-10 * np.linalg.norm(Hg)
        # central finite differences of <g, F(x + e dx)> at eps = 1e-6
        dx = rng.standard_normal((wl.n_nodes, 3)) * np.abs(xl).max() * 1e-2
        eps = 1e-6
        with torch.no_grad():
            dxd = cp.nodes_to_device(dx)
            Lp = float((A.elastic_forces(x + eps * dxd, cp) * g).sum())
            Lm = float((A.elastic_forces(x - eps * dxd, cp) * g).sum())
        fd = (Lp - Lm) / (2 * eps)
        assert float(np.sum(grad * dx)) == pytest.approx(fd, rel=1e-6)
    finally:
        cp.close()


def test_elastic_force_rejects_bending():
    from paper_1807_08219_gb300 import autograd as A
    wl = W.make("C2")
    cp = _coupler(wl)
    try:
        x = cp.nodes_to_device(wl.x_local_all())
        with pytest.raises(ValueError):
            A.elastic_forces(x, cp)
    finally:
        cp.close()
