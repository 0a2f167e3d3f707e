"""Seeded synthetic particle sets (initial conditions).

This module only draws inputs.  It holds none of the force, tree or integrator
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper runs a galactic stellar disc whose equilibrium recipe it does not
give (Sec. 2).  The stand-ins are:

* ``plummer``  -- a Plummer sphere sampled with the Aarseth-Henon-Wielen (1974)
  method: radius from the inverted cumulative mass, speed by von Neumann
  rejection from g(q) = q^2 (1 - q^2)^(7/2), isotropic directions.
* ``galaxy``   -- exponential disc (sech^2 vertical profile) + Hernquist bulge
  + NFW-like halo hard-truncated at r_t, all components truncated at r_t,
  equal particle mass within a component, disc on circular orbits plus a
  fractional isotropic dispersion, bulge and halo isotropic with the
  dispersion of the isotropic Jeans equation in the spherical total mass.
* ``cluster_sizes`` -- ensemble sizes N_c = floor(exp(U(ln nmin, ln nmax))).

Random numbers come from a ``torch.Generator`` on the requested device, so a
given (seed, device) pair is reproducible; CPU and CUDA generators give
different streams.  Tests that compare two implementations draw once and
hand the same arrays to both.

Arrays are returned as ``x`` (3, N), ``v`` (3, N), ``m`` (N) -- structure of
arrays, the layout of the C-ABI.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DEFAULT_SEED = 20241202


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _uniform(g, n, device, lo=0.0, hi=1.0):
    return lo + (hi - lo) * torch.rand(n, generator=g, device=device, dtype=torch.float64)


def _isotropic(g, n, device):
    """Unit vectors uniform on the sphere, shape (3, n)."""
    cth = _uniform(g, n, device, -1.0, 1.0)
    ph = _uniform(g, n, device, 0.0, 2.0 * math.pi)
    sth = torch.sqrt(torch.clamp(1.0 - cth * cth, min=0.0))
    return torch.stack((sth * torch.cos(ph), sth * torch.sin(ph), cth))


def _interp(u, xp, fp):
    """Piecewise-linear interpolation of the table (xp ascending, fp) at u."""
    i = torch.searchsorted(xp, u).clamp(1, xp.numel() - 1)
    x0, x1 = xp[i - 1], xp[i]
    f0, f1 = fp[i - 1], fp[i]
    w = torch.where(x1 > x0, (u - x0) / (x1 - x0), torch.zeros_like(u))
    return f0 + w * (f1 - f0)


def _com_frame(x, v, m):
    mt = m.sum()
    x = x - (x * m).sum(dim=1, keepdim=True) / mt
    v = v - (v * m).sum(dim=1, keepdim=True) / mt
    return x, v


def plummer(n: int, seed: int = DEFAULT_SEED, *, a: float = 1.0, M: float = 1.0,
            G: float = 1.0, xmax: float = 0.999, device="cpu",
            dtype=torch.float64, com: bool = True):
    """Plummer sphere of n equal-mass particles (x, v, m).

    Radii: cumulative mass fraction X ~ U(0, xmax), r = a / sqrt(X^(-2/3) - 1).
    Speeds: q ~ g(q) = q^2 (1-q^2)^(7/2) by rejection, v = q sqrt(2 G M / a)
    (1 + r^2/a^2)^(-1/4).
    """
    n = int(n)
    g = _gen(seed, device)
    X = _uniform(g, n, device, 0.0, xmax)
    r = a / torch.sqrt(torch.pow(X, -2.0 / 3.0) - 1.0)
    x = r * _isotropic(g, n, device)
    # speed fraction q by rejection sampling (envelope 0.1 > max g = 0.0920)
    q = torch.empty(0, dtype=torch.float64, device=device)
    while q.numel() < n:
        k = int(2.2 * (n - q.numel())) + 64
        qq = _uniform(g, k, device)
        yy = _uniform(g, k, device, 0.0, 0.1)
        acc = yy < qq * qq * torch.pow(1.0 - qq * qq, 3.5)
        q = torch.cat((q, qq[acc]))
    q = q[:n]
    speed = q * math.sqrt(2.0 * G * M / a) * torch.pow(1.0 + (r / a) ** 2, -0.25)
    v = speed * _isotropic(g, n, device)
    m = torch.full((n,), M / max(n, 1), dtype=torch.float64, device=device)
    if com and n > 0:
        x, v = _com_frame(x, v, m)
    return x.to(dtype), v.to(dtype), m.to(dtype)


def galaxy(n: int, seed: int = DEFAULT_SEED, *, f_disk=0.6, f_bulge=0.1, Rd=1.0,
           z0=0.1, a_b=0.2, rs=5.0, rt=50.0, M=1.0, G=1.0, sigma_frac=0.1,
           device="cpu", dtype=torch.float64, shuffle: bool = True, return_component: bool = False):
    """Galaxy-like model: exponential disc + Hernquist bulge + truncated NFW halo.

    Component masses f_disk M, f_bulge M, (1 - f_disk - f_bulge) M; particle
    counts in the same proportions, so particle masses are equal within a
    component.  Output order is a random permutation of the particles.
    return_component: also return each particle's component (int8: 0 disc,
    1 bulge, 2 halo), in the same order.
    """
    n = int(n)
    g = _gen(seed, device)
    f_halo = 1.0 - f_disk - f_bulge
    n_d = int(round(f_disk * n))
    n_b = int(round(f_bulge * n))
    n_h = n - n_d - n_b
    f64 = dict(dtype=torch.float64, device=device)

    # --- inverse-CDF tables (numpy, float64, small) ---------------------
    Rg = np.linspace(0.0, min(40.0 * Rd, rt), 8193)
    FR = 1.0 - (1.0 + Rg / Rd) * np.exp(-Rg / Rd)
    FR /= FR[-1]
    ub_max = (rt / (rt + a_b)) ** 2
    def m_nfw(x):
        return np.log1p(x) - x / (1.0 + x)
    rg = np.concatenate(([0.0], np.geomspace(1e-6 * rs, rt, 8192)))
    Fh = m_nfw(rg / rs) / m_nfw(rt / rs)

    def m_tot(r):
        """Spherical enclosed mass used for the velocity model."""
        r = np.asarray(r, dtype=np.float64)
        Rc = np.minimum(r, Rg[-1])
        md = f_disk * M * np.interp(Rc, Rg, FR)
        mb = f_bulge * M * np.minimum(1.0, (r / (r + a_b)) ** 2 / ub_max)
        mh = f_halo * M * np.minimum(1.0, m_nfw(np.minimum(r, rt) / rs) / m_nfw(rt / rs))
        return md + mb + mh

    # isotropic Jeans dispersion on a log grid, sigma^2 = (1/rho) int_r^rt rho G M / r'^2
    jr = np.geomspace(1e-5, rt, 4096)
    gM = G * m_tot(jr) / jr ** 2

    def jeans(rho):
        f = rho * gM
        seg = 0.5 * (f[1:] + f[:-1]) * np.diff(jr)
        tail = np.concatenate((np.cumsum(seg[::-1])[::-1], [0.0]))
        return np.sqrt(np.maximum(tail / rho, 0.0))

    sig_b = jeans(a_b / (jr * (jr + a_b) ** 3))
    sig_h = jeans(1.0 / ((jr / rs) * (1.0 + jr / rs) ** 2))

    T = lambda a: torch.as_tensor(a, **f64)
    Rg_t, FR_t, rg_t, Fh_t, jr_t = T(Rg), T(FR), T(rg), T(Fh), T(jr)
    sig_b_t, sig_h_t = T(sig_b), T(sig_h)
    # circular speed table on the same grid as the dispersions
    vc_t = T(np.sqrt(G * m_tot(jr) / jr))

    # --- disc -------------------------------------------------------------
    R = _interp(_uniform(g, n_d, device), FR_t, Rg_t)
    ph = _uniform(g, n_d, device, 0.0, 2.0 * math.pi)
    uz = _uniform(g, n_d, device, 1e-12, 1.0 - 1e-12)
    z = z0 * torch.atanh(2.0 * uz - 1.0)
    xd = torch.stack((R * torch.cos(ph), R * torch.sin(ph), z))
    vc = _interp(torch.clamp(R, min=jr[0]), jr_t, vc_t)
    vd = torch.stack((-vc * torch.sin(ph), vc * torch.cos(ph), torch.zeros_like(vc)))
    vd = vd + sigma_frac * vc * torch.randn((3, n_d), generator=g, **f64)

    # --- bulge --------------------------------------------------------------
    su = torch.sqrt(_uniform(g, n_b, device, 0.0, ub_max))
    rb = a_b * su / (1.0 - su)
    xb = rb * _isotropic(g, n_b, device)
    sb = _interp(torch.clamp(rb, min=jr[0]), jr_t, sig_b_t)
    vb = sb * torch.randn((3, n_b), generator=g, **f64)

    # --- halo ---------------------------------------------------------------
    rh = _interp(_uniform(g, n_h, device), Fh_t, rg_t)
    xh = rh * _isotropic(g, n_h, device)
    sh = _interp(torch.clamp(rh, min=jr[0]), jr_t, sig_h_t)
    vh = sh * torch.randn((3, n_h), generator=g, **f64)

    x = torch.cat((xd, xb, xh), dim=1)
    v = torch.cat((vd, vb, vh), dim=1)
    m = torch.cat((torch.full((n_d,), f_disk * M / max(n_d, 1), **f64),
                   torch.full((n_b,), f_bulge * M / max(n_b, 1), **f64),
                   torch.full((n_h,), f_halo * M / max(n_h, 1), **f64)))
    comp = torch.cat((torch.zeros(n_d, dtype=torch.int8, device=device),
                      torch.ones(n_b, dtype=torch.int8, device=device),
                      torch.full((n_h,), 2, dtype=torch.int8, device=device)))
    if shuffle and n > 1:
        p = torch.randperm(n, generator=g, device=device)
        x, v, m, comp = x[:, p], v[:, p], m[p], comp[p]
    if return_component:
        return x.to(dtype), v.to(dtype), m.to(dtype), comp
    return x.to(dtype), v.to(dtype), m.to(dtype)


def cluster_sizes(B: int, seed: int = DEFAULT_SEED, nmin: int = 1024, nmax: int = 65536):
    """Ensemble sizes N_c = floor(exp(U(ln nmin, ln nmax))), c = 0..B-1 (numpy ints)."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=B))).astype(np.int64)


def ensemble(B: int, seed: int = DEFAULT_SEED, *, nmin=1024, nmax=65536, device="cpu",
             dtype=torch.float64, **kw):
    """B independent Plummer clusters, concatenated; returns (x, v, m, offsets[B+1])."""
    sizes = cluster_sizes(B, seed, nmin, nmax)
    xs, vs, ms = [], [], []
    for c, nc in enumerate(sizes):
        x, v, m = plummer(int(nc), seed + 1 + c, device=device, dtype=dtype, **kw)
        xs.append(x); vs.append(v); ms.append(m)
    off = np.concatenate(([0], np.cumsum(sizes))).astype(np.int64)
    return torch.cat(xs, 1), torch.cat(vs, 1), torch.cat(ms), off


def two_body_circular(m1=0.5, m2=0.5, d=1.0, eps=0.0, G=1.0, dtype=torch.float64):
    """Two bodies on a circular orbit about their common centre of mass.

    With softening the relative acceleration is G (m1+m2) d / (d^2+eps^2)^(3/2),
    so omega^2 = G (m1+m2) / (d^2+eps^2)^(3/2).
    """
    M = m1 + m2
    om = math.sqrt(G * M / (d * d + eps * eps) ** 1.5)
    r1, r2 = d * m2 / M, d * m1 / M
    x = torch.tensor([[-r1, r2], [0.0, 0.0], [0.0, 0.0]], dtype=torch.float64)
    v = torch.tensor([[0.0, 0.0], [-om * r1, om * r2], [0.0, 0.0]], dtype=torch.float64)
    m = torch.tensor([m1, m2], dtype=torch.float64)
    return x.to(dtype), v.to(dtype), m.to(dtype), om
