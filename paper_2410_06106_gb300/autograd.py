"""Differentiable forms built on the library's kernels.

- `project(img, geom, sel)`: the projector (Eq. 4) as a torch.autograd.Function
  whose backward is the matched backprojection kernel, and `backproject` the
  other way round.
- `unrolled_admm(...)`: K iterations of the unquantized decentralized ADMM
  (Algorithm 4 with Algorithms 2 and 3, complete message graph: every node's
  view of x is the concatenation of the owners' segments), differentiable
  with respect to the penalty rho and the sinogram, with one activation
  checkpoint per iteration. eta1 and eta2 are held fixed.

Every array operation of the iteration runs in libtomo kernels (projector,
backprojector, linear combinations, FP64 dots); torch only gathers each
node's sinogram rows, slices and concatenates row bands, and does the scalar
arithmetic of the coefficients on the host (rho is a CPU float64 scalar
tensor).
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint as ckpt

from . import api


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, geom, sel):
        ctx.geom, ctx.sel = geom, sel
        return geom.project(img.contiguous(), sel)

    @staticmethod
    def backward(ctx, g):
        return ctx.geom.backproject(g.contiguous(), ctx.sel), None, None


class _Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sino, geom, sel):
        ctx.geom, ctx.sel = geom, sel
        return geom.backproject(sino.contiguous(), sel)

    @staticmethod
    def backward(ctx, g):
        return ctx.geom.project(g.contiguous(), ctx.sel), None, None


class _Residual(torch.autograd.Function):
    """r = P_sel u - d"""

    @staticmethod
    def forward(ctx, u, d, geom, sel):
        ctx.geom, ctx.sel = geom, sel
        return geom.project(u.contiguous(), sel, subtract=d.contiguous())

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gu = ctx.geom.backproject(g, ctx.sel) if ctx.needs_input_grad[0] else None
        gd = api.lincomb([g], [-1.0]) if ctx.needs_input_grad[1] else None
        return gu, gd, None, None


class _LinComb(torch.autograd.Function):
    """out = sum_j c[j] x_j; c is a CPU float64 vector (differentiable)"""

    @staticmethod
    def forward(ctx, c, *xs):
        xs = [x.contiguous() for x in xs]
        ctx.save_for_backward(*xs)
        ctx.c = [float(v) for v in c.detach().tolist()]
        return api.lincomb(xs, ctx.c)

    @staticmethod
    def backward(ctx, g):
        xs = ctx.saved_tensors
        g = g.contiguous()
        gx = [api.lincomb([g], [cj]) if ctx.needs_input_grad[1 + j] else None for j, cj in enumerate(ctx.c)]
        gc = None
        if ctx.needs_input_grad[0]:
            gc = torch.stack([api.dot(g, x).cpu() for x in xs])
        return (gc, *gx)


def project(img, geom, sel=None):
    return _Project.apply(img, geom, sel)


def backproject(sino, geom, sel=None):
    return _Backproject.apply(sino, geom, sel)


def _lincomb(coefs, *xs):
    return _LinComb.apply(torch.stack([torch.as_tensor(c, dtype=torch.float64) for c in coefs]), *xs)


def admm_iteration(u, lam, xt, rho, d_nodes, geom, node_sel, seg_rows, eta1, eta2, E1, E2):
    """One unquantized dADMM iteration on a complete graph.

    u, lam: lists of M [N, N] tensors; xt: [N, N] (the owners' segments);
    rho: CPU float64 scalar tensor; d_nodes[m]: [A_m, B] data of node m.
    Returns (u', lam', x')."""
    M = len(u)
    x = xt  # complete graph, no quantizer: every node's view is conc of the segments
    u_new = []
    for m in range(M):
        um = u[m]
        e1 = float(eta1[m])
        # Algorithm 2: u <- u - eta1 (P^T (P u - d) + rho (u - x) + lambda)
        cu = (1.0 - e1 * rho, -e1, e1 * rho, -e1)
        for _ in range(E1):
            r = _Residual.apply(um, d_nodes[m], geom, node_sel[m])
            g = _Backproject.apply(r, geom, node_sel[m])
            um = _lincomb(cu, um, g, x, lam[m])
        u_new.append(um)
    # Algorithm 3, E2 GD steps in closed form: a x + (1 - a)(u + lambda / rho), a = (1 - eta2 rho)^E2
    a = (1.0 - eta2 * rho) ** E2
    segs = []
    for m in range(M):
        r0, r1 = int(seg_rows[m]), int(seg_rows[m + 1])
        segs.append(_lincomb((a, 1.0 - a, (1.0 - a) / rho), xt[r0:r1], u_new[m][r0:r1], lam[m][r0:r1]))
    x_new = torch.cat(segs, dim=0)
    # Eq. 18
    lam_new = [_lincomb((1.0, rho, -rho), lam[m], u_new[m], x_new) for m in range(M)]
    return u_new, lam_new, x_new


def unrolled_admm(sino, geom, node_sel, seg_rows, rho, eta1, eta2=0.2, E1=10, E2=10, iters=10,
                  checkpoint=True):
    """x after `iters` iterations of unquantized dADMM from zero.

    sino: [A, B] CUDA float32 (may require grad); node_sel: list of M int32
    angle-index arrays; seg_rows: M+1 row boundaries; rho: float or CPU
    float64 scalar tensor (may require grad); eta1: M steps (fixed)."""
    if not isinstance(rho, torch.Tensor):
        rho = torch.tensor(float(rho), dtype=torch.float64)
    M, N = len(node_sel), geom.N
    dev = sino.device
    for sel in node_sel:  # every operator call below then runs without device allocation
        geom.plan(sel, 1)
    d_nodes = [sino.index_select(0, torch.as_tensor(sel, dtype=torch.long, device=dev)) for sel in node_sel]
    u = [torch.zeros(N, N, device=dev, dtype=sino.dtype) for _ in range(M)]
    lam = [torch.zeros(N, N, device=dev, dtype=sino.dtype) for _ in range(M)]
    xt = torch.zeros(N, N, device=dev, dtype=sino.dtype)

    def step(rho_, *flat):
        uu, ll, x_ = list(flat[:M]), list(flat[M:2 * M]), flat[2 * M]
        dn = list(flat[2 * M + 1:])
        un, ln, xn = admm_iteration(uu, ll, x_, rho_, dn, geom, node_sel, seg_rows, eta1, eta2, E1, E2)
        return (*un, *ln, xn)

    for _ in range(iters):
        args = (rho, *u, *lam, xt, *d_nodes)
        out = ckpt.checkpoint(step, *args, use_reentrant=False) if checkpoint else step(*args)
        u, lam, xt = list(out[:M]), list(out[M:2 * M]), out[2 * M]
    return xt
