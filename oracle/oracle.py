"""FP64 CPU oracle of the TreeCode method -- Python side.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the library.  It shares no code
with the CUDA path.

The heavy loops are plain C (oracle.c, loaded through ctypes); the leapfrog
integrator (Eqs. 2-5) and the diagnostics are plain numpy here.

Canonical tree (the paper's Sec. 2 octree with the readings listed in each
oracle.c function): box -> keys -> (key, index) order -> breadth-first octree
with leaf capacity lcap -> cell moments -> group lists with the opening angle
theta -> cell expansion + PP forces.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import build as _build

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.orc_direct.argtypes = [i64, _D, _D, dbl, dbl, i64, _I64, _D, _D]
        L.orc_box.argtypes = [i64, _D, _D, _I32]
        L.orc_box.restype = ctypes.c_int
        L.orc_keys.argtypes = [i64, _D, _D, i32, _U32, _U64]
        L.orc_sort.argtypes = [i64, _U64, _I64]
        L.orc_octree.argtypes = [i64, _U64, i32, i64, _I32, _U32, _I64, _I64, _I64, _I32]
        L.orc_octree.restype = i64
        L.orc_moments.argtypes = [i64, _I64, _I64, _D, _I64, i64, _D, _D, _D, _D, _D]
        L.orc_groups.argtypes = [i64, _U64, i64, _I32, _I64, _I64, _I32, i32, i32, i64, _I64]
        L.orc_groups.restype = i64
        L.orc_lists.argtypes = [i64, _U32, i64, _I64, i64, _I64, dbl, i64, _I32, _U32, _I64, _I32,
                                _I64, _I64, _I64, _I64]
        L.orc_tree_forces.argtypes = [i64, _D, _D, _I64, i64, _I64, i64, _I64, i64, _D, _D, _D, _I64, _I64,
                                      _I64, _I64, _I64, _I64, dbl, dbl, i32, _D, _D]
        L.orc_tree_forces_vjp.argtypes = [i64, _D, _D, _I64, i64, _I64, i64, _D, _D, _D, _I64, _I64,
                                          _I64, _I64, _I64, _I64, dbl, dbl, i32, _D, _D, _D, _D]
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


# --------------------------------------------------------------------------- #
# Eq. 1
def direct(x, m, G=1.0, eps=0.0, targets=None):
    """Direct PP sum (Eq. 1) for the given target indices (default: all).

    Returns a (3, nt) and phi (nt), FP64.
    """
    x = _f64(x); m = _f64(m)
    n = m.shape[0]
    tgt = np.arange(n, dtype=np.int64) if targets is None else \
        np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
    nt = tgt.shape[0]
    a = np.zeros((3, nt)); phi = np.zeros(nt)
    lib().orc_direct(n, _p(x, _D), _p(m, _D), float(G), float(eps), nt, _p(tgt, _I64),
                     _p(a, _D), _p(phi, _D))
    return a, phi


# --------------------------------------------------------------------------- #
# Canonical tree
def box(x):
    x = _f64(x)
    lo = np.zeros(3); k = ctypes.c_int32(0)
    rc = lib().orc_box(x.shape[1], _p(x, _D), _p(lo, _D), ctypes.byref(k))
    if rc == -1:
        raise ValueError("non-finite coordinate")
    if rc == -2:
        raise ValueError("empty particle set")
    return lo, int(k.value)


def keys(x, lo, k):
    x = _f64(x); lo = _f64(lo)
    n = x.shape[1]
    q = np.zeros((3, n), dtype=np.uint32); key = np.zeros(n, dtype=np.uint64)
    lib().orc_keys(n, _p(x, _D), _p(lo, _D), int(k), _p(q, _U32), _p(key, _U64))
    return q, key


def sort(key):
    key = np.ascontiguousarray(key, dtype=np.uint64)
    perm = np.zeros(key.shape[0], dtype=np.int64)
    lib().orc_sort(key.shape[0], _p(key, _U64), _p(perm, _I64))
    return perm


@dataclasses.dataclass
class Octree:
    level: np.ndarray     # (nn,) int32
    corner: np.ndarray    # (3, nn) uint32
    first: np.ndarray     # (nn,) int64, sorted index of the first member
    count: np.ndarray     # (nn,) int64
    child: np.ndarray     # (nn,) int64, first child or -1
    nchild: np.ndarray    # (nn,) int32

    @property
    def nn(self):
        return self.level.shape[0]


def octree(skey, lcap):
    skey = np.ascontiguousarray(skey, dtype=np.uint64)
    n = skey.shape[0]
    cap = 0 if n > (1 << 22) else max(64, 2 * n)   # large n: count first, then fill exact arrays
    while True:
        lv = np.zeros(cap, np.int32); co = np.zeros((3, cap), np.uint32)
        fi = np.zeros(cap, np.int64); cn = np.zeros(cap, np.int64)
        ch = np.zeros(cap, np.int64); nc = np.zeros(cap, np.int32)
        nn = lib().orc_octree(n, _p(skey, _U64), int(lcap), cap, _p(lv, _I32), _p(co, _U32),
                              _p(fi, _I64), _p(cn, _I64), _p(ch, _I64), _p(nc, _I32))
        if nn <= cap:
            return Octree(lv[:nn].copy(), np.ascontiguousarray(co[:, :nn]), fi[:nn].copy(),
                          cn[:nn].copy(), ch[:nn].copy(), nc[:nn].copy())
        cap = int(nn)


def cell_centre(tree: Octree, lo, k):
    """Geometric centre lo + (corner + s/2) 2^(k-21) of every cell, (3, nn)."""
    s = np.ldexp(1.0, 21 - tree.level.astype(np.int64))
    u = np.ldexp(1.0, int(k) - 21)
    return np.asarray(lo, np.float64)[:, None] + (tree.corner.astype(np.float64) + 0.5 * s) * u


def moments(tree: Octree, perm, x, m, lo, k):
    """Cell moments (orc_moments).  The members of a cell are sorted positions first..first+count,
    i.e. particles perm[first..]; they are passed in sorted order (the same particles, summed in the
    same order) so the sums read memory contiguously."""
    x = _f64(x); m = _f64(m)
    nn = tree.nn
    cen = np.ascontiguousarray(cell_centre(tree, lo, k))
    M = np.zeros(nn); R = np.zeros((3, nn)); Q = np.zeros((6, nn))
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    xs = np.ascontiguousarray(x[:, perm]); ms = np.ascontiguousarray(m[perm])
    ident = np.arange(perm.shape[0], dtype=np.int64)
    lib().orc_moments(nn, _p(tree.first, _I64), _p(tree.count, _I64), _p(cen, _D),
                      _p(ident, _I64), ms.shape[0], _p(xs, _D), _p(ms, _D),
                      _p(M, _D), _p(R, _D), _p(Q, _D))
    return M, R, Q


def groups(skey, tree: Octree, gs, delta=3, cmax=None):
    """First sorted index of every walk group, plus n at the end (orc_groups).
    cmax defaults to 128 gs when delta > 0 and to 0 (no cell-size cut) for plain chunks."""
    skey = np.ascontiguousarray(skey, dtype=np.uint64)
    n = skey.shape[0]
    if cmax is None:
        cmax = 128 * int(gs) if delta > 0 else 0
    gf = np.zeros(n + 1, np.int64)
    ng = lib().orc_groups(n, _p(skey, _U64), tree.nn, _p(tree.level, _I32), _p(tree.first, _I64),
                          _p(tree.count, _I64), _p(tree.nchild, _I32), int(gs), int(delta), cmax, _p(gf, _I64))
    return gf[: ng + 1].copy()


def lists(qs, gfirst, theta, tree: Octree, gsel=None):
    """CSR interaction lists per group: (pc_off, pc_list, pp_off, pp_list).  gsel: walk only these
    groups (CSR entry k = group gsel[k]); default all groups in order."""
    qs = np.ascontiguousarray(qs, dtype=np.uint32)
    gfirst = np.ascontiguousarray(gfirst, dtype=np.int64)
    n = qs.shape[1]
    ng = gfirst.shape[0] - 1
    gsel = None if gsel is None else np.ascontiguousarray(gsel, dtype=np.int64)
    nsel = ng if gsel is None else gsel.shape[0]
    pc_off = np.zeros(nsel + 1, np.int64); pp_off = np.zeros(nsel + 1, np.int64)
    args = (n, _p(qs, _U32), ng, _p(gfirst, _I64), nsel, _p(gsel, _I64), float(theta), tree.nn,
            _p(tree.level, _I32), _p(tree.corner, _U32), _p(tree.child, _I64), _p(tree.nchild, _I32))
    lib().orc_lists(*args, _p(pc_off, _I64), _p(pp_off, _I64), None, None)
    pc = np.zeros(max(1, pc_off[-1]), np.int64); pp = np.zeros(max(1, pp_off[-1]), np.int64)
    lib().orc_lists(*args, _p(pc_off, _I64), _p(pp_off, _I64), _p(pc, _I64), _p(pp, _I64))
    return pc_off, pc[:pc_off[-1]], pp_off, pp[:pp_off[-1]]


@dataclasses.dataclass
class TreeResult:
    lo: np.ndarray
    k: int
    q: np.ndarray         # (3, n) uint32, original order
    key: np.ndarray       # (n,) uint64, original order
    perm: np.ndarray      # sorted position -> original index
    tree: Octree
    M: np.ndarray
    R: np.ndarray
    Q: np.ndarray
    gfirst: np.ndarray    # walk groups: first sorted index of each, then n
    gsel: np.ndarray      # groups whose lists and forces were evaluated (None: all)
    pc_off: np.ndarray
    pc_list: np.ndarray
    pp_off: np.ndarray
    pp_list: np.ndarray
    a: np.ndarray         # (3, n) original order
    phi: np.ndarray       # (n,)


def tree_forces(x, m, *, G=1.0, eps=0.0, theta=0.7, lcap=16, gs=32, quad=True, delta=3, cmax=None,
                want_forces=True, groups_sel=None, timings=None):
    """Whole canonical tree pipeline; returns every intermediate and a, phi.

    groups_sel: walk groups (indices into the canonical groups) whose lists and forces are evaluated;
    default all.  The box, keys, order, octree, moments and groups always cover every particle;
    a and phi are zero outside the selected groups' particles.  timings: a dict that receives the
    wall time of each stage."""
    import time
    T = timings if timings is not None else {}
    t = time.perf_counter()

    def lap(name):
        nonlocal t
        now = time.perf_counter()
        T[name] = now - t
        t = now

    x = _f64(x); m = _f64(m)
    n = m.shape[0]
    lo, k = box(x); lap("box")
    q, key = keys(x, lo, k); lap("keys")
    perm = sort(key); lap("sort")
    skey = key[perm]
    tr = octree(skey, lcap); lap("octree")
    M, R, Q = moments(tr, perm, x, m, lo, k); lap("moments")
    gf = groups(skey, tr, gs, delta, cmax); lap("groups")
    del skey
    qs = np.ascontiguousarray(q[:, perm])
    gsel = None if groups_sel is None else np.ascontiguousarray(groups_sel, dtype=np.int64)
    pc_off, pc, pp_off, pp = lists(qs, gf, theta, tr, gsel); lap("lists")
    del qs
    a = np.zeros((3, n)); phi = np.zeros(n)
    if want_forces:
        lib().orc_tree_forces(n, _p(x, _D), _p(m, _D), _p(perm, _I64), gf.shape[0] - 1, _p(gf, _I64),
                              0 if gsel is None else gsel.shape[0], _p(gsel, _I64), tr.nn,
                              _p(M, _D), _p(R, _D), _p(Q, _D), _p(tr.first, _I64),
                              _p(tr.count, _I64), _p(pc_off, _I64), _p(pc, _I64),
                              _p(pp_off, _I64), _p(pp, _I64), float(G), float(eps),
                              1 if quad else 0, _p(a, _D), _p(phi, _D))
    lap("forces")
    return TreeResult(lo, k, q, key, perm, tr, M, R, Q, gf, gsel, pc_off, pc, pp_off, pp, a, phi)


def tree_accel(x, m, **kw):
    r = tree_forces(x, m, **kw)
    return r.a, r.phi


# --------------------------------------------------------------------------- #
# Ensembles (not in the paper): independent systems, system b = particles
# [offsets[b], offsets[b+1]).  By definition each is treated exactly as if it
# were alone -- its own box, keys, tree, groups and lists -- and systems exert
# no force on one another.
def ensemble_tree_forces(x, m, offsets, **kw):
    """tree_forces of every system alone; returns (a, phi) in the caller's order
    and the list of per-system TreeResults."""
    x = _f64(x); m = _f64(m)
    n = m.shape[0]
    offsets = [int(o) for o in offsets]
    assert offsets[0] == 0 and offsets[-1] == n and all(b > a for a, b in zip(offsets, offsets[1:]))
    a = np.zeros((3, n)); phi = np.zeros(n); rs = []
    for b0, b1 in zip(offsets[:-1], offsets[1:]):
        r = tree_forces(x[:, b0:b1], m[b0:b1], **kw)
        a[:, b0:b1] = r.a; phi[b0:b1] = r.phi
        rs.append(r)
    return a, phi, rs


def ensemble_accel(x, m, offsets, **kw):
    a, phi, _ = ensemble_tree_forces(x, m, offsets, **kw)
    return a, phi


# --------------------------------------------------------------------------- #
# Eqs. 2-5: kick-drift-kick leapfrog, a^0 computed once before the first step.
def kdk(x, v, m, tau, nsteps, accel, a0=None):
    """Run nsteps of Eqs. 2-5.  accel(x) -> (a, phi).  Returns x, v, a, phi."""
    x = _f64(x).copy(); v = _f64(v).copy()
    if a0 is None:
        a, phi = accel(x)
    else:
        a, phi = a0
    for _ in range(int(nsteps)):
        v = v + 0.5 * tau * a          # Eq. 2
        x = x + tau * v                # Eq. 3
        a, phi = accel(x)              # Eq. 4
        v = v + 0.5 * tau * a          # Eq. 5
    return x, v, a, phi


def diagnostics(x, v, m, phi):
    """E_kin = 1/2 sum m v^2, W = 1/2 sum m phi, P = sum m v, L = sum m x cross v."""
    x = _f64(x); v = _f64(v); m = _f64(m); phi = _f64(phi)
    ek = 0.5 * float(np.sum(m * np.sum(v * v, axis=0)))
    w = 0.5 * float(np.sum(m * phi))
    P = np.sum(m * v, axis=1)
    L = np.sum(m * np.cross(x.T, v.T).T, axis=1)
    return dict(ekin=ek, epot=w, etot=ek + w, P=P, L=L)


# --------------------------------------------------------------------------- #
# Adjoint of the tree force and of the leapfrog with the tree structure held
# fixed per force evaluation (order, cells, groups, lists from the primal
# state; moments recomputed from the perturbed positions and masses).
def tree_forces_frozen(r: TreeResult, x, m, *, G=1.0, eps=0.0, quad=True):
    """Forces of (x, m) through the structure of r: moments recomputed, lists reused."""
    x = _f64(x); m = _f64(m)
    n = m.shape[0]
    M, R, Q = moments(r.tree, r.perm, x, m, r.lo, r.k)
    a = np.zeros((3, n)); phi = np.zeros(n)
    gf, tr = r.gfirst, r.tree
    lib().orc_tree_forces(n, _p(x, _D), _p(m, _D), _p(r.perm, _I64), gf.shape[0] - 1, _p(gf, _I64), 0, None,
                          tr.nn, _p(M, _D), _p(R, _D), _p(Q, _D), _p(tr.first, _I64), _p(tr.count, _I64),
                          _p(r.pc_off, _I64), _p(r.pc_list, _I64), _p(r.pp_off, _I64), _p(r.pp_list, _I64),
                          float(G), float(eps), 1 if quad else 0, _p(a, _D), _p(phi, _D))
    return a, phi


def tree_forces_vjp(r: TreeResult, x, m, abar, phibar=None, *, G=1.0, eps=0.0, quad=True):
    """(xbar, mbar) = VJP of (a, phi) = tree_forces_frozen(r, x, m) with cotangents (abar, phibar)."""
    x = _f64(x); m = _f64(m); abar = _f64(abar)
    phibar = None if phibar is None else _f64(phibar)
    n = m.shape[0]
    M, R, Q = moments(r.tree, r.perm, x, m, r.lo, r.k)
    xbar = np.zeros((3, n)); mbar = np.zeros(n)
    gf, tr = r.gfirst, r.tree
    lib().orc_tree_forces_vjp(n, _p(x, _D), _p(m, _D), _p(r.perm, _I64), gf.shape[0] - 1, _p(gf, _I64), tr.nn,
                              _p(M, _D), _p(R, _D), _p(Q, _D), _p(tr.first, _I64), _p(tr.count, _I64),
                              _p(r.pc_off, _I64), _p(r.pc_list, _I64), _p(r.pp_off, _I64), _p(r.pp_list, _I64),
                              float(G), float(eps), 1 if quad else 0, _p(abar, _D), _p(phibar, _D),
                              _p(xbar, _D), _p(mbar, _D))
    return xbar, mbar


def kdk_forward(x, v, m, tau, nsteps, **tree_kw):
    """Eqs. 2-5 with tree forces; returns the states x_n, v_n, a_n, phi_n (n = 0..K) and the
    structure used at every x_n (the primal trajectory of the adjoint)."""
    x = _f64(x).copy(); v = _f64(v).copy(); m = _f64(m)
    r = tree_forces(x, m, **tree_kw)
    xs, vs, as_, ps, rs = [x], [v], [r.a], [r.phi], [r]
    for _ in range(int(nsteps)):
        vh = vs[-1] + 0.5 * tau * as_[-1]
        xn = xs[-1] + tau * vh
        r = tree_forces(xn, m, **tree_kw)
        vs.append(vh + 0.5 * tau * r.a); xs.append(xn); as_.append(r.a); ps.append(r.phi); rs.append(r)
    return xs, vs, as_, ps, rs


def kdk_frozen(x, v, m, tau, structures, *, G=1.0, eps=0.0, quad=True):
    """The same K steps with every force evaluated through the given structures (for finite
    differences of the frozen-structure map).  Returns x_K, v_K, phi_K."""
    x = _f64(x).copy(); v = _f64(v).copy(); m = _f64(m)
    a, phi = tree_forces_frozen(structures[0], x, m, G=G, eps=eps, quad=quad)
    for r in structures[1:]:
        v = v + 0.5 * tau * a
        x = x + tau * v
        a, phi = tree_forces_frozen(r, x, m, G=G, eps=eps, quad=quad)
        v = v + 0.5 * tau * a
    return x, v, phi


def kdk_adjoint(xs, m, tau, structures, xbar_K, vbar_K, phibar_K=None, *, G=1.0, eps=0.0, quad=True):
    """Reverse sweep of Eqs. 2-5 through frozen structures.  Given cotangents of x_K, v_K and of the
    final potentials phi_K, returns (xbar_0, vbar_0, mbar).  Step n maps (x_n, v_n, a_n) to
    (x_{n+1}, v_{n+1}, a_{n+1}): v' = v_n + tau/2 a_n, x_{n+1} = x_n + tau v', a_{n+1} = F(x_{n+1}),
    v_{n+1} = v' + tau/2 a_{n+1}; a_0 = F(x_0)."""
    m = _f64(m)
    K = len(xs) - 1
    h = 0.5 * tau
    xb = _f64(xbar_K).copy(); vb = _f64(vbar_K).copy(); mb = np.zeros_like(m)
    ab = np.zeros_like(xb)             # cotangent of a_{n+1}
    pb = None if phibar_K is None else _f64(phibar_K)
    for nstep in range(K - 1, -1, -1):
        ab = ab + h * vb                                   # v_{n+1} = v' + h a_{n+1}
        dx, dm = tree_forces_vjp(structures[nstep + 1], xs[nstep + 1], m, ab,
                                 pb if nstep == K - 1 else None, G=G, eps=eps, quad=quad)
        xb = xb + dx; mb = mb + dm
        vb = vb + tau * xb                                  # x_{n+1} = x_n + tau v'
        ab = h * vb                                         # v' = v_n + h a_n
    dx, dm = tree_forces_vjp(structures[0], xs[0], m, ab, pb if K == 0 else None, G=G, eps=eps, quad=quad)
    xb = xb + dx; mb = mb + dm
    return xb, vb, mb
