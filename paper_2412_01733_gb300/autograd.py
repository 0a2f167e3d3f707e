"""Gradients through K leapfrog steps of the tree force (not in the paper).

``TreeLeapfrog.apply(x0, v0, m, ws, K, tau, ckpt)`` runs K kick-drift-kick steps
(Eqs. 2-5) with tree forces on the GPU and returns (x_K, v_K, W_K), W_K =
1/2 sum m_i phi_i at x_K.  Its backward pass differentiates the discrete map
with the tree structure of every force evaluation held fixed (key order,
cells, walk groups and interaction lists of the primal trajectory; the cell
moments follow x and m).

Memory: the forward pass keeps (x, v, a) every ``ckpt`` steps; the backward
pass recomputes each segment from its checkpoint, then walks it in reverse,
rebuilding the tree (with interaction lists) at every state and calling the
library's reverse leapfrog step.  All arithmetic runs in libtreegb kernels
(the cotangents of W included: tree_energy_vjp); this module only orders the
calls.
"""
from __future__ import annotations

import torch

from . import treegb


class TreeLeapfrog(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, ws: "treegb.Workspace", K: int, tau: float, ckpt: int = 4):
        K, ckpt = int(K), max(1, int(ckpt))
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        md = m.detach().contiguous()
        a, phi = ws.accel(x, md)
        ckpts = {0: (x.clone(), v.clone(), a.clone())}
        for s in range(K):
            ws.leapfrog_step(x, v, md, a, tau, phi=phi)
            if (s + 1) % ckpt == 0 and s + 1 < K:
                ckpts[s + 1] = (x.clone(), v.clone(), a.clone())
        W = ws.diagnostics(x, v, md, phi)[1].clone()
        ctx.ws, ctx.K, ctx.tau, ctx.ckpt, ctx.ckpts = ws, K, float(tau), ckpt, ckpts
        ctx.save_for_backward(md, phi.clone())
        return x, v, W

    @staticmethod
    def backward(ctx, gx, gv, gW):
        ws, K, tau, ckpt, ckpts = ctx.ws, ctx.K, ctx.tau, ctx.ckpt, ctx.ckpts
        m, phiK = ctx.saved_tensors
        dt = m.dtype
        xb = gx.detach().to(dt).clone().contiguous() if gx is not None else torch.zeros_like(ckpts[0][0])
        vb = gv.detach().to(dt).clone().contiguous() if gv is not None else torch.zeros_like(ckpts[0][0])
        ab = torch.zeros_like(xb)
        mb = torch.zeros_like(m)
        pb = None
        if gW is not None:
            # phi_bar = gW m / 2 and m_bar += gW phi / 2, the VJP of W = 1/2 sum m phi
            pb = ws.energy_vjp(m, phiK, gW.detach().to(torch.float64).reshape(1).contiguous(), m_bar=mb)
        starts = sorted(ckpts)
        for si in range(len(starts) - 1, -1, -1):
            s0 = starts[si]
            s1 = starts[si + 1] if si + 1 < len(starts) else K
            x, v, a = (t.clone() for t in ckpts[s0])
            xs = [x.clone()]
            for _ in range(s0, s1):
                ws.leapfrog_step(x, v, m, a, tau)
                xs.append(x.clone())
            for n in range(s1 - 1, s0 - 1, -1):
                xn1 = xs[n + 1 - s0]
                ws.build(xn1)
                ws.moments(xn1, m)
                ws.forces(lists_only=True)
                ws.leapfrog_adjoint_step(xb, vb, ab, mb, tau, phi_bar=pb if n + 1 == K else None)
        # a_0 = F(x_0)
        x0 = ckpts[0][0]
        ws.build(x0)
        ws.moments(x0, m)
        ws.forces(lists_only=True)
        ws.forces_adjoint(ab, pb if K == 0 else None, xb, mb)
        return xb, vb, mb, None, None, None, None


def tree_leapfrog(x0, v0, m, ws, K, tau, ckpt=4):
    """Functional form of TreeLeapfrog.apply."""
    return TreeLeapfrog.apply(x0, v0, m, ws, K, tau, ckpt)
