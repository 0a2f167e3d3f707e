"""Pins of the oracle's kick-drift-kick leapfrog (Eqs. 2-5)."""
import math

import numpy as np

from paper_2412_01733_gb300 import inputs


def _direct_accel(orc, m, eps):
    return lambda x: orc.direct(x, m, eps=eps)


def test_circular_orbit_period(orc):
    eps = 0.1
    x, v, m, om = inputs.two_body_circular(0.3, 0.7, 1.0, eps)
    x, v, m = x.numpy(), v.numpy(), m.numpy()
    T = 2 * math.pi / om
    nst = 4000
    xe, ve, a, phi = orc.kdk(x, v, m, T / nst, nst, _direct_accel(orc, m, eps))
    assert np.abs(xe - x).max() < 1e-5
    d0 = orc.diagnostics(x, v, m, orc.direct(x, m, eps=eps)[1])
    d1 = orc.diagnostics(xe, ve, m, phi)
    assert abs(d1["etot"] - d0["etot"]) < 1e-8 * abs(d0["etot"])


def test_time_reversibility(orc):
    x, v, m = inputs.plummer(64, 31)
    x, v, m = x.numpy(), v.numpy(), m.numpy()
    acc = _direct_accel(orc, m, 0.05)
    x1, v1, a1, p1 = orc.kdk(x, v, m, 0.01, 50, acc)
    x2, v2, _, _ = orc.kdk(x1, -v1, m, 0.01, 50, acc, a0=(a1, p1))
    assert np.abs(x2 - x).max() < 1e-12
    assert np.abs(-v2 - v).max() < 1e-12


def test_energy_error_scales_as_tau_squared(orc):
    x, v, m = inputs.plummer(48, 37)
    x, v, m = x.numpy(), v.numpy(), m.numpy()
    acc = _direct_accel(orc, m, 0.1)
    e0 = orc.diagnostics(x, v, m, acc(x)[1])["etot"]
    errs = []
    for tau in (0.02, 0.01, 0.005):
        nst = int(round(1.0 / tau))
        xe, ve, _, phi = orc.kdk(x, v, m, tau, nst, acc)
        errs.append(abs(orc.diagnostics(xe, ve, m, phi)["etot"] - e0))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs


def test_momentum_conserved_with_direct_forces(orc):
    x, v, m = inputs.plummer(100, 41)
    x, v, m = x.numpy(), v.numpy(), m.numpy()
    xe, ve, _, _ = orc.kdk(x, v, m, 0.01, 20, _direct_accel(orc, m, 0.02))
    P0 = (m * v).sum(axis=1); P1 = (m * ve).sum(axis=1)
    assert np.abs(P1 - P0).max() < 1e-14
