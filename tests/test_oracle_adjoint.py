"""Pins of the oracle's adjoint: the VJP of the tree force and the reverse
leapfrog sweep, with the tree structure held fixed per force evaluation.

Checked against central finite differences of the frozen-structure forward
map (an independent route to the same derivative) and, at theta = 0 where the
tree is the direct sum of Eq. 1, against torch autograd of a direct-sum
leapfrog written in plain torch ops."""
import numpy as np
import pytest
import torch

from paper_2412_01733_gb300 import inputs

KW = dict(G=1.0, eps=0.05)


def _setup(n, seed, theta, quad=True, lcap=8, gs=16):
    x, v, m = inputs.plummer(n, seed)
    x, v, m = x.numpy(), v.numpy(), m.numpy()
    m = m * (0.5 + np.random.default_rng(seed).random(n))   # unequal masses
    return x, v, m, dict(theta=theta, lcap=lcap, gs=gs, quad=quad, **KW)


@pytest.mark.parametrize("theta,quad", [(0.7, True), (0.5, False), (1.0, True)])
def test_force_vjp_matches_frozen_fd(orc, theta, quad):
    n = 500
    x, v, m, kw = _setup(n, 3, theta, quad)
    r = orc.tree_forces(x, m, **kw)
    rng = np.random.default_rng(7)
    ab = rng.standard_normal((3, n)); pb = rng.standard_normal(n)
    xb, mb = orc.tree_forces_vjp(r, x, m, ab, pb, quad=quad, **KW)

    def J(xx, mm):
        a, phi = orc.tree_forces_frozen(r, xx, mm, quad=quad, **KW)
        return (a * ab).sum() + (phi * pb).sum()

    h = 1e-6
    for trial in range(3):
        dx = rng.standard_normal((3, n)); dm = rng.standard_normal(n) * m
        fd_x = (J(x + h * dx, m) - J(x - h * dx, m)) / (2 * h)
        fd_m = (J(x, m + h * dm) - J(x, m - h * dm)) / (2 * h)
        assert abs(fd_x - (xb * dx).sum()) <= 1e-6 * abs(fd_x), (fd_x, (xb * dx).sum())
        assert abs(fd_m - (mb * dm).sum()) <= 1e-6 * abs(fd_m), (fd_m, (mb * dm).sum())


def _loss_and_grad_oracle(orc, x, v, m, kw, tau, K, nsel):
    xs, vs, as_, ps, rs = orc.kdk_forward(x, v, m, tau, K, **kw)
    xK, phiK = xs[-1], ps[-1]
    L = (xK[:, :nsel] ** 2).sum() + 0.5 * (m * phiK).sum()
    xbK = np.zeros_like(xK); xbK[:, :nsel] = 2 * xK[:, :nsel]
    gx, gv, gm = orc.kdk_adjoint(xs, m, tau, rs, xbK, np.zeros_like(xK), 0.5 * m,
                                 G=kw["G"], eps=kw["eps"], quad=kw["quad"])
    gm = gm + 0.5 * phiK
    return L, gx, gv, gm, rs


def test_leapfrog_adjoint_matches_frozen_fd(orc):
    """Loss = sum of |x_i^K|^2 over the first particles + W(x^K); gradient with
    respect to x_0, v_0 and m on 32 random coordinates, central FD with h = 1e-6
    for positions and velocities and a relative step 1e-4 for masses."""
    n, K, tau, nsel = 400, 4, 0.01, 50
    x, v, m, kw = _setup(n, 11, 0.7)
    L, gx, gv, gm, rs = _loss_and_grad_oracle(orc, x, v, m, kw, tau, K, nsel)

    def loss(xx, vv, mm):
        xK, vK, phiK = orc.kdk_frozen(xx, vv, mm, tau, rs, G=kw["G"], eps=kw["eps"], quad=True)
        return (xK[:, :nsel] ** 2).sum() + 0.5 * (mm * phiK).sum()

    rng = np.random.default_rng(5)
    h = 1e-6
    for k in range(32):
        which = k % 3
        d, i = rng.integers(0, 3), rng.integers(0, n)
        xx, vv, mm = x.copy(), v.copy(), m.copy()
        if which == 0:
            xp = x.copy(); xp[d, i] += h; xm = x.copy(); xm[d, i] -= h
            fd = (loss(xp, v, m) - loss(xm, v, m)) / (2 * h); g = gx[d, i]
        elif which == 1:
            vp = v.copy(); vp[d, i] += h; vm = v.copy(); vm[d, i] -= h
            fd = (loss(x, vp, m) - loss(x, vm, m)) / (2 * h); g = gv[d, i]
        else:
            # masses are O(1/n): a relative step keeps round-off of the O(100) loss small
            hm = 1e-4 * m[i]
            mp = m.copy(); mp[i] += hm; mmn = m.copy(); mmn[i] -= hm
            fd = (loss(x, v, mp) - loss(x, v, mmn)) / (2 * hm); g = gm[i]
        assert abs(fd - g) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gx).max()), (which, d, i, fd, g)


def test_leapfrog_adjoint_theta0_equals_autograd(orc):
    """At theta = 0 the tree force is the direct sum (Eq. 1); the adjoint must
    equal torch autograd of a direct-sum leapfrog in FP64."""
    n, K, tau, nsel = 120, 3, 0.02, 30
    x, v, m, kw = _setup(n, 17, 0.0)
    L, gx, gv, gm, _ = _loss_and_grad_oracle(orc, x, v, m, kw, tau, K, nsel)
    G, eps = kw["G"], kw["eps"]
    X = torch.tensor(x, requires_grad=True); V = torch.tensor(v, requires_grad=True)
    Mt = torch.tensor(m, requires_grad=True)
    eye = torch.eye(n, dtype=torch.float64)

    def acc(xx):
        d = xx[:, None, :] - xx[:, :, None]            # d[:, i, j] = x_j - x_i
        r2 = (d * d).sum(0) + eps * eps
        w = (1 - eye) * G * Mt[None, :] * r2 ** -1.5
        a = (d * w[None]).sum(2)
        phi = -((1 - eye) * G * Mt[None, :] * r2 ** -0.5).sum(1)
        return a, phi

    xx, vv = X, V
    a, phi = acc(xx)
    for _ in range(K):
        vv = vv + 0.5 * tau * a
        xx = xx + tau * vv
        a, phi = acc(xx)
        vv = vv + 0.5 * tau * a
    Lt = (xx[:, :nsel] ** 2).sum() + 0.5 * (Mt * phi).sum()
    Lt.backward()
    assert abs(Lt.item() - L) <= 1e-12 * abs(L)
    np.testing.assert_allclose(gx, X.grad.numpy(), rtol=0, atol=1e-10 * np.abs(X.grad.numpy()).max())
    np.testing.assert_allclose(gv, V.grad.numpy(), rtol=0, atol=1e-10 * np.abs(V.grad.numpy()).max())
    np.testing.assert_allclose(gm, Mt.grad.numpy(), rtol=0, atol=1e-10 * np.abs(Mt.grad.numpy()).max())
