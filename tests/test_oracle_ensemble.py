"""Pins of the oracle's ensemble definition: independent systems, each
treated as if alone, with no forces between systems."""
import numpy as np

from paper_2412_01733_gb300 import inputs


def _ens(B=4, seed=5):
    x, v, m, off = inputs.ensemble(B, seed, nmin=40, nmax=400)
    return x.numpy(), v.numpy(), m.numpy(), off


def test_theta0_is_blockwise_direct_sum(orc):
    """At theta = 0 every system's tree force is its own direct sum (Eq. 1);
    particles of other systems contribute nothing."""
    x, v, m, off = _ens()
    a, phi, rs = orc.ensemble_tree_forces(x, m, off, eps=0.01, theta=0.0, lcap=4, gs=16)
    for b0, b1 in zip(off[:-1], off[1:]):
        ad, pd = orc.direct(x[:, b0:b1], m[b0:b1], eps=0.01)
        np.testing.assert_allclose(a[:, b0:b1], ad, rtol=0, atol=1e-12 * np.abs(ad).max())
        np.testing.assert_allclose(phi[b0:b1], pd, rtol=0, atol=1e-12 * np.abs(pd).max())
    # the whole set as one system would feel the other clusters (they overlap in space)
    ad_all, _ = orc.direct(x, m, eps=0.01)
    assert np.abs(ad_all - a).max() > 1e-3 * np.abs(a).max()


def test_single_system_and_identical_copies(orc):
    x, v, m, off = _ens(B=1)
    a1, p1, _ = orc.ensemble_tree_forces(x, m, off, eps=0.01, theta=0.7)
    r = orc.tree_forces(x, m, eps=0.01, theta=0.7)
    assert np.array_equal(a1, r.a) and np.array_equal(p1, r.phi)
    n = m.shape[0]
    x2, m2 = np.concatenate([x, x], 1), np.concatenate([m, m])
    a2, p2, rs = orc.ensemble_tree_forces(x2, m2, [0, n, 2 * n], eps=0.01, theta=0.7)
    assert np.array_equal(a2[:, :n], r.a) and np.array_equal(a2[:, n:], r.a)
    assert np.array_equal(rs[0].key, rs[1].key) and np.array_equal(rs[0].pc_list, rs[1].pc_list)
