"""Pins of the oracle's direct sum (Eq. 1) to closed forms and invariants."""
import math

import numpy as np
import pytest

from paper_2412_01733_gb300 import inputs


def test_two_body_closed_form(orc):
    # m = (1, 2) at (0,0,0) and (3,4,0): separation 5.
    x = np.array([[0.0, 3.0], [0.0, 4.0], [0.0, 0.0]])
    m = np.array([1.0, 2.0])
    a, phi = orc.direct(x, m, G=1.0, eps=0.0)
    np.testing.assert_allclose(a[:, 0], [2 * 3 / 125, 2 * 4 / 125, 0.0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(a[:, 1], [-3 / 125, -4 / 125, 0.0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(phi, [-2 / 5, -1 / 5], rtol=1e-15)
    # softened: r_s^2 = 25 + eps^2
    a, phi = orc.direct(x, m, G=2.0, eps=1.0)
    s3 = 26.0 ** 1.5
    np.testing.assert_allclose(a[:, 0], [2 * 2 * 3 / s3, 2 * 2 * 4 / s3, 0.0], rtol=1e-14)
    np.testing.assert_allclose(phi[1], -2.0 * 1.0 / math.sqrt(26.0), rtol=1e-15)


def test_self_term_excluded(orc):
    x = np.zeros((3, 1)); m = np.ones(1)
    a, phi = orc.direct(x, m, eps=0.1)
    assert np.all(a == 0) and phi[0] == 0


def test_zero_net_force(orc):
    x, v, m = inputs.plummer(600, 11)
    x = x.numpy(); m = (m * torch_rand_masses(600)).numpy()
    a, _ = orc.direct(x, m, eps=0.01)
    s = np.abs((m * a).sum(axis=1))
    assert np.all(s <= 1e-12 * np.abs(m * a).sum(axis=1))


def torch_rand_masses(n):
    import torch
    g = torch.Generator().manual_seed(5)
    return 0.5 + torch.rand(n, generator=g, dtype=torch.float64)


def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    th = np.arccos(1 - 2 * i / n)
    ph = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])


@pytest.mark.parametrize("p", [(0.3, 0.1, 0.2), (0.5, -0.2, 0.1), (2.0, 0.5, -1.0), (0.0, 0.0, 3.0)])
def test_shell_theorem(orc, p):
    """Uniform shell of mass 1, radius 1: no force inside, point mass outside."""
    ns = 4000
    x = np.concatenate([_fibonacci_sphere(ns), np.array(p)[:, None]], axis=1)
    m = np.concatenate([np.full(ns, 1.0 / ns), [0.0]])
    a, phi = orc.direct(x, m, targets=[ns])
    p = np.array(p); r = np.linalg.norm(p)
    if r < 1:
        assert np.linalg.norm(a[:, 0]) < 1e-5
        assert abs(phi[0] + 1.0) < 1e-5
    else:
        np.testing.assert_allclose(a[:, 0], -p / r ** 3, atol=1e-5 / r ** 2)
        assert abs(phi[0] + 1.0 / r) < 1e-5


def test_plummer_profile(orc):
    """Binned radial acceleration of a sampled Plummer sphere follows the
    shell theorem, -G M(<r) / r^2 with M(<r) the sampled enclosed mass, and
    the binned potential follows -G M / sqrt(r^2 + a^2) (M = 1, a = 1)."""
    n = 16384
    x, _, m = inputs.plummer(n, 3)
    x = x.numpy(); m = m.numpy()
    a, phi = orc.direct(x, m, eps=0.005)
    r = np.linalg.norm(x, axis=0)
    ar = (a * x).sum(axis=0) / r
    order = np.argsort(r)
    menc = np.empty_like(r)
    menc[order] = np.cumsum(m[order]) - m[order]
    edges = np.array([0.3, 0.5, 0.7, 1.0, 1.4, 2.0, 3.0, 5.0])
    for lo_, hi_ in zip(edges[:-1], edges[1:]):
        sel = (r >= lo_) & (r < hi_)
        assert sel.sum() > 500
        rc = r[sel]
        rel = np.mean(ar[sel]) / np.mean(-menc[sel] / rc ** 2) - 1.0
        assert abs(rel) < 0.01, (lo_, hi_, rel)
        relp = np.mean(phi[sel]) / np.mean(-1.0 / np.sqrt(rc ** 2 + 1)) - 1.0
        assert abs(relp) < 0.01, (lo_, hi_, relp)
