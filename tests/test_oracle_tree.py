"""Pins of the oracle's canonical tree (Sec. 2 octree, theta criterion, cell
expansion) to hand-derived values, brute force and mathematical invariants."""
import math
import os

import numpy as np
import pytest

from paper_2412_01733_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- box / keys
@pytest.mark.parametrize("ext,k", [(1.0, 1), (0.75, 0), (0.5, 0), (0.3, -1), (0.0, 0),
                                   (3.0, 2), (4.0, 3), (0.2500001, -1), (0.25, -1)])
def test_box_power_of_two(orc, ext, k):
    x = np.array([[1.5, 1.5 + ext], [-2.0, -2.0], [7.0, 7.0]])
    lo, kk = orc.box(x)
    np.testing.assert_array_equal(lo, [1.5, -2.0, 7.0])
    assert kk == k
    L = 2.0 ** kk
    assert L > ext and (ext == 0 or L / 2 <= ext)


def test_box_rejects_nonfinite(orc):
    with pytest.raises(ValueError):
        orc.box(np.array([[0.0, np.nan], [0.0, 0.0], [0.0, 0.0]]))


def test_keys_hand_derived(orc):
    tab = np.loadtxt(os.path.join(GOLDEN, "morton_keys.txt"), dtype=np.uint64)
    q = tab[:, :3].astype(np.float64).T
    # an anchor at the origin and one at the far corner fix lo = 0 and k = 0
    u = 2.0 ** -21
    x = np.concatenate([np.zeros((3, 1)), np.full((3, 1), (2 ** 21 - 1) * u), q * u], axis=1)
    lo, k = orc.box(x)
    assert k == 0 and np.all(lo == 0)
    qq, key = orc.keys(x, lo, k)
    np.testing.assert_array_equal(qq[:, 2:], q.astype(np.uint32))
    np.testing.assert_array_equal(key[2:], tab[:, 3])


def test_key_octant_digit(orc):
    """The top octant digit of a particle in the upper-x half is >= 4, etc."""
    x = np.array([[0.0, 0.99, 0.1, 0.1], [0.0, 0.99, 0.9, 0.1], [0.0, 0.99, 0.1, 0.9]])
    lo, k = orc.box(x)
    q, key = orc.keys(x, lo, k)
    top = key >> np.uint64(60)
    np.testing.assert_array_equal(top, [0, 7, 2, 1])


def test_sort_ties_by_index(orc):
    key = np.array([5, 3, 5, 3, 0, 5], dtype=np.uint64)
    np.testing.assert_array_equal(orc.sort(key), [4, 1, 3, 0, 2, 5])


# ---------------------------------------------------------------- octree
def _brute_octree(q, lcap):
    """Independent recursive geometric subdivision of the 2^21 grid.

    Returns {(level, cx, cy, cz): sorted member tuple} and the set of internal
    node keys.  Members are original indices.
    """
    nodes, internal = {}, set()

    def rec(level, c, members):
        nodes[(level,) + tuple(c)] = tuple(sorted(members))
        if len(members) > lcap and level < 21:
            internal.add((level,) + tuple(c))
            h = 1 << (21 - level - 1)
            for ox in (0, 1):
                for oy in (0, 1):
                    for oz in (0, 1):
                        cc = (c[0] + ox * h, c[1] + oy * h, c[2] + oz * h)
                        sub = [i for i in members
                               if all(cc[d] <= q[d, i] < cc[d] + h for d in range(3))]
                        if sub:
                            rec(level + 1, cc, sub)

    rec(0, (0, 0, 0), list(range(q.shape[1])))
    return nodes, internal


@pytest.mark.parametrize("n,lcap,seed,clump", [(64, 1, 1, False), (64, 4, 2, False),
                                               (50, 16, 3, False), (40, 2, 4, True),
                                               (33, 1, 5, True), (1, 1, 6, False)])
def test_octree_brute_force(orc, n, lcap, seed, clump):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((3, n))
    if clump:  # coincident and nearly coincident particles reach depth 21
        x[:, : n // 3] = x[:, :1]
        x[:, n // 3: n // 2] = x[:, :1] + 1e-9
    lo, k = orc.box(x)
    q, key = orc.keys(x, lo, k)
    perm = orc.sort(key)
    t = orc.octree(key[perm], lcap)
    want, internal = _brute_octree(q, lcap)
    got = {}
    for c in range(t.nn):
        members = tuple(sorted(perm[t.first[c]: t.first[c] + t.count[c]].tolist()))
        got[(int(t.level[c]),) + tuple(int(v) for v in t.corner[:, c])] = members
        assert (t.nchild[c] > 0) == ((int(t.level[c]),) + tuple(int(v) for v in t.corner[:, c]) in internal)
    assert got == want
    # breadth-first numbering: levels non-decreasing, first indices ascending within a level,
    # children contiguous and in octant order
    assert np.all(np.diff(t.level) >= 0)
    for lv in np.unique(t.level):
        f = t.first[t.level == lv]
        assert np.all(np.diff(f) > 0)
    for c in range(t.nn):
        if t.nchild[c]:
            ch = np.arange(t.child[c], t.child[c] + t.nchild[c])
            assert np.all(t.level[ch] == t.level[c] + 1)
            assert t.first[ch[0]] == t.first[c]
            assert t.count[ch].sum() == t.count[c]


# ---------------------------------------------------------------- moments
def test_moments_two_particles(orc):
    x = np.array([[0.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    m = np.array([1.0, 3.0])
    lo, k = orc.box(x)
    q, key = orc.keys(x, lo, k)
    perm = orc.sort(key)
    t = orc.octree(key[perm], 1)
    M, R, Q = orc.moments(t, perm, x, m, lo, k)
    assert M[0] == 4.0
    np.testing.assert_allclose(R[:, 0], [0.75, 0, 0], rtol=1e-15)
    # y = (-0.75, 0.25) along x: Qxx = sum 2 m y^2 = 1.5, Qyy = Qzz = -0.75
    np.testing.assert_allclose(Q[:, 0], [1.5, -0.75, -0.75, 0, 0, 0], rtol=1e-15, atol=1e-15)


def test_moments_parallel_axis(orc):
    """Each internal cell's (M, R, Q) equals its children's combined with the
    parallel-axis theorem of the traceless quadrupole; the oracle computes
    every cell from its members, so this is an independent relation."""
    x, _, m = inputs.plummer(3000, 7)
    x = x.numpy(); m = m.numpy() * (1 + np.arange(3000) % 3)
    lo, k = orc.box(x)
    q, key = orc.keys(x, lo, k)
    perm = orc.sort(key)
    t = orc.octree(key[perm], 8)
    M, R, Q = orc.moments(t, perm, x, m, lo, k)
    np.testing.assert_allclose(Q[0] + Q[1] + Q[2], 0, atol=1e-12 * np.abs(Q[:3]).max())
    for c in np.nonzero(t.nchild)[0][:200]:
        ch = np.arange(t.child[c], t.child[c] + t.nchild[c])
        Mc = M[ch].sum()
        Rc = (M[ch] * R[:, ch]).sum(axis=1) / Mc
        d = R[:, ch] - Rc[:, None]
        d2 = (d * d).sum(axis=0)
        shift = np.stack([3 * d[0] * d[0] - d2, 3 * d[1] * d[1] - d2, 3 * d[2] * d[2] - d2,
                          3 * d[0] * d[1], 3 * d[0] * d[2], 3 * d[1] * d[2]])
        Qc = (Q[:, ch] + M[ch] * shift).sum(axis=1)
        scale = M[c] * (2.0 ** (k - t.level[c])) ** 2
        assert abs(Mc - M[c]) <= 1e-12 * M[c]
        np.testing.assert_allclose(Rc, R[:, c], atol=1e-13 * 2.0 ** k)
        np.testing.assert_allclose(Qc, Q[:, c], atol=1e-12 * scale)


# ---------------------------------------------------------------- lists
def _check_lists(orc, x, theta, gs, lcap, delta=3):
    lo, k = orc.box(x)
    q, key = orc.keys(x, lo, k)
    perm = orc.sort(key)
    t = orc.octree(key[perm], lcap)
    qs = q[:, perm]
    gf = orc.groups(key[perm], t, gs, delta)
    pc_off, pc, pp_off, pp = orc.lists(qs, gf, theta, t)
    n = x.shape[1]
    ng = len(gf) - 1
    parent = np.full(t.nn, -1)
    for c in range(t.nn):
        if t.nchild[c]:
            parent[t.child[c]: t.child[c] + t.nchild[c]] = c
    th2 = theta * theta
    for g in range(ng):
        s0, s1 = gf[g], gf[g + 1]
        glo = qs[:, s0:s1].min(axis=1).astype(np.int64)
        ghi = qs[:, s0:s1].max(axis=1).astype(np.int64) + 1

        def accepted(c):
            s = 1 << (21 - int(t.level[c]))
            cc = t.corner[:, c].astype(np.int64)
            gap = np.maximum(0, np.maximum(cc - ghi, glo - (cc + s)))
            return float(s * s) < th2 * float((gap * gap).sum())

        P = pc[pc_off[g]: pc_off[g + 1]]; L = pp[pp_off[g]: pp_off[g + 1]]
        assert np.all(np.diff(P) > 0) and np.all(np.diff(L) > 0)
        cover = np.zeros(n, dtype=np.int64)
        for c in P:
            assert accepted(c)
            cover[t.first[c]: t.first[c] + t.count[c]] += 1
        for c in L:
            assert t.nchild[c] == 0 and not accepted(c)
            cover[t.first[c]: t.first[c] + t.count[c]] += 1
        # every particle is counted exactly once: the lists partition the system
        assert np.all(cover == 1)
        # every ancestor of a listed node was opened, i.e. not accepted
        for c in np.concatenate([P, L]):
            p = parent[c]
            while p >= 0:
                assert not accepted(p)
                p = parent[p]
    return pc_off, pp_off


@pytest.mark.parametrize("theta,gs,lcap,delta", [(0.7, 32, 16, 3), (1.0, 16, 4, 2), (0.4, 64, 1, 1),
                                                (0.0, 32, 8, 2), (0.7, 32, 16, 0)])
def test_lists_partition_and_criterion(orc, theta, gs, lcap, delta):
    x, _, _ = inputs.plummer(700, 13)
    pc_off, pp_off = _check_lists(orc, x.numpy(), theta, gs, lcap, delta)
    if theta == 0.0:
        assert pc_off[-1] == 0


def _octal_digits(key):
    """The 21 octal digits of a 63-bit key, most significant first."""
    return [(int(key) >> (3 * (20 - i))) & 7 for i in range(21)]


@pytest.mark.parametrize("kind,n,gs,lcap,delta,cmax", [("plummer", 3000, 32, 16, 3, 4096), ("galaxy", 4000, 32, 8, 2, 256),
                                                       ("galaxy", 2000, 64, 4, 1, 0), ("plummer", 1000, 16, 1, 3, 64),
                                                       ("plummer", 500, 32, 16, 0, 0), ("plummer", 3000, 32, 16, 0, 128)])
def test_groups_rule(orc, kind, n, gs, lcap, delta, cmax):
    """Walk groups: chunks of gs in key order, cut between neighbours that do
    not share the cell delta levels above the finer of their leaves, or whose
    smallest common cell holds more than cmax particles.  Checked by counting
    shared octal digits directly, with leaf levels from a scan of the leaves and
    cell populations from counting equal key prefixes, and through the two
    bounds the rule implies."""
    x, _, _ = (inputs.plummer if kind == "plummer" else inputs.galaxy)(n, 29)
    x = x.numpy()
    lo, k = orc.box(x)
    q, key = orc.keys(x, lo, k)
    perm = orc.sort(key)
    sk = key[perm]
    t = orc.octree(sk, lcap)
    gf = orc.groups(sk, t, gs, delta, cmax)
    leaf_level = np.full(n, -1)
    for c in np.nonzero(t.nchild == 0)[0]:
        leaf_level[t.first[c]: t.first[c] + t.count[c]] = t.level[c]
    assert np.all(leaf_level >= 0)
    digits = [_octal_digits(v) for v in sk]
    prefixes = [tuple(dd) for dd in digits]

    def population(i, lvl):
        return sum(1 for p in prefixes if p[:lvl] == prefixes[i][:lvl])

    want = [0]
    for i in range(1, n):
        shared = 21
        for j in range(21):
            if digits[i][j] != digits[i - 1][j]:
                shared = j
                break
        cut = i % gs == 0 or (delta > 0 and shared < max(leaf_level[i], leaf_level[i - 1]) - delta)
        if not cut and cmax > 0 and population(i, shared) > cmax:
            cut = True
        if cut:
            want.append(i)
    np.testing.assert_array_equal(gf, want + [n])
    sizes = np.diff(gf)
    assert sizes.min() >= 1 and sizes.max() <= gs
    if delta == 0 and cmax == 0:
        assert len(gf) - 1 == (n + gs - 1) // gs
    qs = q[:, perm]
    for g in range(len(gf) - 1):
        a, b = gf[g], gf[g + 1]
        if delta > 0:
            lvl = max(0, leaf_level[a:b].min() - delta)
            cell = (qs[:, a:b] >> (21 - lvl))
            assert np.all(cell == cell[:, :1]), (g, lvl)     # fits one cell of that level
        if cmax > 0 and b - a > 1:
            common = min(next((j for j in range(21) if digits[a][j] != digits[b - 1][j]), 21), 21)
            assert population(a, common) <= cmax              # its smallest cell is small


# ---------------------------------------------------------------- forces
def test_theta_zero_equals_direct(orc):
    x, _, m = inputs.plummer(2048, 17)
    x = x.numpy(); m = m.numpy()
    r = orc.tree_forces(x, m, eps=0.01, theta=0.0, lcap=8, gs=32, quad=True)
    a, phi = orc.direct(x, m, eps=0.01)
    err = np.linalg.norm(r.a - a, axis=0) / np.linalg.norm(a, axis=0)
    assert err.max() < 1e-12
    assert np.abs(r.phi - phi).max() < 1e-12 * np.abs(phi).max()


def _single_cell_case(orc, D, quad, direction):
    """A 40-particle clump of side 1 at the origin acting on one massless
    particle at distance D, through the clump's own cell expansion."""
    rng = np.random.default_rng(21)
    xc = rng.uniform(-0.5, 0.5, (3, 40))
    mc = rng.uniform(0.5, 1.5, 40)
    tgt = D * np.asarray(direction, float) / np.linalg.norm(direction)
    x = np.ascontiguousarray(np.concatenate([xc, tgt[:, None]], axis=1))
    m = np.concatenate([mc, [0.0]])
    n = 41
    perm = np.arange(n, dtype=np.int64)
    first = np.array([0, 40], np.int64); count = np.array([40, 1], np.int64)
    tree = orc.Octree(np.zeros(2, np.int32), np.zeros((3, 2), np.uint32), first, count,
                      np.array([-1, -1], np.int64), np.zeros(2, np.int32))
    M, R, Q = orc.moments(tree, perm, x, m, np.zeros(3), 0)
    # group 0 = the clump (PP with itself), group 1 = the target (PC with cell 0)
    gf = np.array([0, 40, 41], np.int64)
    pc_off = np.array([0, 0, 1], np.int64); pc = np.array([0], np.int64)
    pp_off = np.array([0, 1, 1], np.int64); pp = np.array([0], np.int64)
    a = np.zeros((3, n)); phi = np.zeros(n)
    P = orc._p
    orc.lib().orc_tree_forces(n, P(x, orc._D), P(m, orc._D), P(perm, orc._I64), 2, P(gf, orc._I64), 0, None, 2,
                              P(M, orc._D), P(R, orc._D), P(Q, orc._D), P(first, orc._I64),
                              P(count, orc._I64), P(pc_off, orc._I64), P(pc, orc._I64),
                              P(pp_off, orc._I64), P(pp, orc._I64), 1.0, 0.0,
                              1 if quad else 0, P(a, orc._D), P(phi, orc._D))
    ad, phid = orc.direct(x, m, targets=[40])
    return (np.linalg.norm(a[:, 40] - ad[:, 0]) / np.linalg.norm(ad[:, 0]),
            abs(phi[40] - phid[0]) / abs(phid[0]))


@pytest.mark.parametrize("direction", [(1, 0.3, -0.2), (-0.4, 1, 0.7), (0.1, -0.2, -1)])
def test_multipole_convergence_order(orc, direction):
    """Monopole error falls as (b/D)^2, quadrupole error as (b/D)^3: pins the
    sign and every coefficient of the quadrupole terms of the expansion."""
    Ds = [8.0, 16.0, 32.0, 64.0]
    em = [_single_cell_case(orc, D, False, direction) for D in Ds]
    eq = [_single_cell_case(orc, D, True, direction) for D in Ds]
    for i in range(len(Ds) - 1):
        rm = em[i][0] / em[i + 1][0]
        rq = eq[i][0] / eq[i + 1][0]
        assert 3.0 < rm < 5.5, (Ds[i], rm)      # acceleration, (b/D)^2
        assert 6.0 < rq < 11.0, (Ds[i], rq)     # acceleration, (b/D)^3
        assert eq[i][0] < em[i][0] and eq[i][1] < em[i][1]
    # potential: relative error falls by (64/8)^2 = 64 for the monopole and by
    # about (64/8)^3 = 512 with the quadrupole (a scalar, so its error can
    # change sign between two distances; compare the ends of the range)
    assert 40.0 < em[0][1] / em[-1][1] < 100.0
    assert eq[0][1] / eq[-1][1] > 200.0


def test_error_falls_with_theta(orc):
    x, _, m = inputs.plummer(4096, 23)
    x = x.numpy(); m = m.numpy()
    a, _ = orc.direct(x, m, eps=0.01)
    med = []
    for th in (1.0, 0.7, 0.5, 0.3):
        r = orc.tree_forces(x, m, eps=0.01, theta=th, lcap=16, gs=32, quad=True)
        e = np.linalg.norm(r.a - a, axis=0) / np.linalg.norm(a, axis=0)
        med.append(np.median(e))
    assert all(med[i] > med[i + 1] for i in range(3)), med
    rm = orc.tree_forces(x, m, eps=0.01, theta=0.7, quad=False)
    em = np.median(np.linalg.norm(rm.a - a, axis=0) / np.linalg.norm(a, axis=0))
    assert med[1] < em


def test_plain_config_force_error(orc):
    """Plummer N = 16384, eps = 0.01, theta = 0.7, monopole, leaf <= 16: median
    relative force error against the direct sum below 1e-3."""
    x, _, m = inputs.plummer(16384, 20241202)
    x = x.numpy(); m = m.numpy()
    r = orc.tree_forces(x, m, eps=0.01, theta=0.7, lcap=16, gs=32, quad=False)
    a, phi = orc.direct(x, m, eps=0.01)
    e = np.linalg.norm(r.a - a, axis=0) / np.linalg.norm(a, axis=0)
    assert np.median(e) < 1e-3
    assert np.median(np.abs(r.phi - phi) / np.abs(phi)) < 1e-3


def test_group_selection_equals_full_walk(orc):
    """Lists and forces of a selection of walk groups (any order) are those of the
    full walk for the same groups, bit for bit; other particles are untouched."""
    x, _, m = inputs.galaxy(6000, 31)
    x = x.numpy(); m = m.numpy()
    kw = dict(eps=0.02, theta=0.7, lcap=16, gs=32, quad=True)
    full = orc.tree_forces(x, m, **kw)
    ng = len(full.gfirst) - 1
    sel = np.random.default_rng(5).permutation(ng)[: ng // 5]
    part = orc.tree_forces(x, m, groups_sel=sel, **kw)
    np.testing.assert_array_equal(part.gfirst, full.gfirst)
    touched = np.zeros(x.shape[1], bool)
    for k, g in enumerate(sel):
        np.testing.assert_array_equal(part.pc_list[part.pc_off[k]: part.pc_off[k + 1]],
                                      full.pc_list[full.pc_off[g]: full.pc_off[g + 1]])
        np.testing.assert_array_equal(part.pp_list[part.pp_off[k]: part.pp_off[k + 1]],
                                      full.pp_list[full.pp_off[g]: full.pp_off[g + 1]])
        touched[full.perm[full.gfirst[g]: full.gfirst[g + 1]]] = True
    np.testing.assert_array_equal(part.a[:, touched], full.a[:, touched])
    np.testing.assert_array_equal(part.phi[touched], full.phi[touched])
    assert np.all(part.a[:, ~touched] == 0) and np.all(part.phi[~touched] == 0)


def test_sort_matches_stable_library_sort(orc):
    """(key, original index) order equals a stable library sort of the keys."""
    key = np.random.default_rng(8).integers(0, 50, 20000).astype(np.uint64)
    np.testing.assert_array_equal(orc.sort(key), np.argsort(key, kind="stable"))
