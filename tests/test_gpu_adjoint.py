"""GPU adjoint (tree_forces_adjoint, leapfrog_adjoint_step, TreeLeapfrog)
against the FP64 oracle adjoint on identical trees (the oracle adjoint is
pinned by finite differences and autograd in test_oracle_adjoint.py)."""
import numpy as np
import pytest
import torch

from paper_2412_01733_gb300 import inputs

pytestmark = pytest.mark.gpu


def _tg():
    from paper_2412_01733_gb300 import build, treegb
    build.build()
    return treegb


def _np(t):
    return t.detach().double().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 2e-4)])
@pytest.mark.parametrize("quad,theta,gs", [(True, 0.7, 32), (False, 0.5, 64)])
def test_force_vjp_parity(orc, precision, tol, quad, theta, gs):
    tg = _tg()
    n = 6000
    dt = torch.float64 if precision == "f64" else torch.float32
    x, v, m = inputs.plummer(n, 41)
    m = m * (0.5 + torch.rand(n, generator=torch.Generator().manual_seed(1), dtype=torch.float64))
    xg, mg = x.to("cuda", dt).contiguous(), m.to("cuda", dt).contiguous()
    p = dict(eps=0.05, theta=theta, order=2 if quad else 0, leaf_cap=8, group_size=gs, precision=precision)
    ws = tg.Workspace(n, **p)
    ws.build(xg); ws.moments(xg, mg); ws.forces(emit_lists=True)
    g = torch.Generator().manual_seed(2)
    ab = torch.randn((3, n), generator=g, dtype=torch.float64)
    pb = torch.randn(n, generator=g, dtype=torch.float64)
    xb, mb = ws.forces_adjoint(ab.to("cuda", dt).contiguous(), pb.to("cuda", dt).contiguous())
    torch.cuda.synchronize()
    assert ws.status() == 0
    r = orc.tree_forces(_np(xg), _np(mg), eps=0.05, theta=theta, lcap=8, gs=gs, quad=quad)
    xo, mo = orc.tree_forces_vjp(r, _np(xg), _np(mg), _np(ab.to(dt)), _np(pb.to(dt)), eps=0.05, quad=quad)
    assert _rel(_np(xb), xo) <= tol, _rel(_np(xb), xo)
    assert _rel(_np(mb), mo) <= tol, _rel(_np(mb), mo)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-9), ("f32", 5e-4)])
def test_tree_leapfrog_gradient_parity(orc, precision, tol):
    """Loss = sum |x_i^K|^2 over the first 256 particles + W_K through K = 6
    steps with checkpoints every 4, against the oracle's reverse sweep."""
    tg = _tg()
    from paper_2412_01733_gb300.autograd import TreeLeapfrog
    n, K, tau, nsel = 4000, 6, 0.01, 256
    dt = torch.float64 if precision == "f64" else torch.float32
    x, v, m = inputs.plummer(n, 43)
    xg = x.to("cuda", dt).contiguous().requires_grad_(True)
    vg = v.to("cuda", dt).contiguous().requires_grad_(True)
    mg = m.to("cuda", dt).contiguous().requires_grad_(True)
    ws = tg.Workspace(n, eps=0.01, theta=0.7, order=2, leaf_cap=16, group_size=32, precision=precision)
    xK, vK, WK = TreeLeapfrog.apply(xg, vg, mg, ws, K, tau, 4)
    loss = (xK[:, :nsel].double() ** 2).sum() + WK
    loss.backward()
    torch.cuda.synchronize()
    assert ws.status() == 0
    kw = dict(eps=0.01, theta=0.7, lcap=16, gs=32, quad=True)
    xs, vs, as_, ps, rs = orc.kdk_forward(_np(xg), _np(vg), _np(mg), tau, K, **kw)
    mo = _np(mg)
    xbK = np.zeros_like(xs[-1]); xbK[:, :nsel] = 2 * xs[-1][:, :nsel]
    gx, gv, gm = orc.kdk_adjoint(xs, mo, tau, rs, xbK, np.zeros_like(xbK), 0.5 * mo, eps=0.01, quad=True)
    gm = gm + 0.5 * ps[-1]
    assert abs(loss.item() - ((xs[-1][:, :nsel] ** 2).sum() + 0.5 * (mo * ps[-1]).sum())) <= 1e-5 * abs(loss.item())
    assert _rel(_np(xg.grad), gx) <= tol, _rel(_np(xg.grad), gx)
    assert _rel(_np(vg.grad), gv) <= tol, _rel(_np(vg.grad), gv)
    assert _rel(_np(mg.grad), gm) <= tol, _rel(_np(mg.grad), gm)


def test_tree_leapfrog_fd_unfrozen():
    """The adjoint config in miniature (Plummer, eps = 0.01, theta = 0.7, 16
    steps, checkpoints every 4, FP64): central FD (h = 1e-6) of the full GPU
    map, tree rebuilt every step, on 32 coordinates (mass steps relative, 1e-4).
    A perturbation that moves a particle across a cell boundary changes the
    structure and the map jumps.  Every coordinate whose difference quotient
    misses the frozen-structure gradient (1e-5 plus the finite-difference
    round-off) must be one whose +h or -h run changed the structure of some
    step (key order, nodes, walk groups or interaction counts); the fraction of
    such coordinates is reported, and at least 24 of 32 must match."""
    tg = _tg()
    from paper_2412_01733_gb300.autograd import TreeLeapfrog
    n, K, tau, nsel = 8192, 16, 0.01, 1024
    x, v, m = inputs.plummer(n, 47)
    xg = x.cuda().contiguous().requires_grad_(True)
    vg = v.cuda().contiguous().requires_grad_(True)
    mg = m.cuda().contiguous().requires_grad_(True)
    ws = tg.Workspace(n, eps=0.01, theta=0.7, order=2, leaf_cap=16, group_size=32, precision="f64")
    xK, vK, WK = TreeLeapfrog.apply(xg, vg, mg, ws, K, tau, 4)
    loss = (xK[:, :nsel] ** 2).sum() + WK
    loss.backward()
    weights = torch.arange(1, n + 1, dtype=torch.int64, device="cuda")

    def structure():
        inf = ws.info()
        perm = ws.export_tree()["perm"].long()
        gf = ws.export_groups()
        return (inf["n_nodes"], inf["n_groups"], inf["pp_pairs"], inf["pc_pairs"],
                int((perm * weights).sum()), int(gf.sum()))

    def L(xx, vv, mm):
        xx, vv = xx.clone(), vv.clone()
        a, phi = ws.accel(xx, mm)
        sig = [structure()]
        for _ in range(K):
            ws.leapfrog_step(xx, vv, mm, a, tau, phi=phi)
            sig.append(structure())
        return ((xx[:, :nsel] ** 2).sum() + ws.diagnostics(xx, vv, mm, phi)[1]).item(), sig

    rng = np.random.default_rng(3)
    ok = changed = 0
    x0, v0, m0 = xg.detach(), vg.detach(), mg.detach()
    L0, sig0 = L(x0, v0, m0)
    assert abs(L0 - loss.item()) <= 1e-12 * abs(L0)
    mism = []
    for k in range(32):
        which, d, i = k % 3, int(rng.integers(0, 3)), int(rng.integers(0, n))
        if which == 2:
            h = 1e-4 * m0[i].item()
            mp = m0.clone(); mp[i] += h; mn = m0.clone(); mn[i] -= h
            (Lp, sp), (Ln, sn) = L(x0, v0, mp), L(x0, v0, mn)
            g = mg.grad[i].item()
        else:
            h = 1e-6
            base = x0 if which == 0 else v0
            bp = base.clone(); bp[d, i] += h; bn = base.clone(); bn[d, i] -= h
            (Lp, sp), (Ln, sn) = (L(bp, v0, m0), L(bn, v0, m0)) if which == 0 else (L(x0, bp, m0), L(x0, bn, m0))
            g = (xg.grad if which == 0 else vg.grad)[d, i].item()
        fd = (Lp - Ln) / (2 * h)
        # central-difference round-off: a few ulps of the loss divided by 2h
        noise = 20 * 2.2e-16 * abs(L0) / (2 * h)
        good = abs(fd - g) <= 1e-5 * abs(g) + noise
        ch = sp != sig0 or sn != sig0
        ok += good
        changed += ch
        if not good:
            mism.append((k, ch))
    print(f"FD unfrozen: {ok}/32 match, {changed}/32 perturbations changed the structure, "
          f"mismatches {mism}")
    assert all(ch for _, ch in mism), mism     # every mismatch is a structure change
    assert ok >= 24, ok
