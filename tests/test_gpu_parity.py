"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bit-exact: keys, sort permutation, node arrays and interaction lists (as sets
per group) under the canonical tree definition.  Floating point: moments to
FP64 rounding; FP32 forces to median relative error <= 1e-5 and max <= 1e-4
against the oracle on the identical tree; the FP64 walk to 1e-11.
"""
import numpy as np
import pytest
import torch

from paper_2412_01733_gb300 import inputs

pytestmark = pytest.mark.gpu


def _tg():
    from paper_2412_01733_gb300 import build, treegb
    build.build()
    return treegb


def _to_gpu(x, m, dtype):
    return x.to("cuda", dtype).contiguous(), m.to("cuda", dtype).contiguous()


def _np64(t):
    return t.detach().double().cpu().numpy()


def _run(x, m, *, precision="f32", emit=True, **p):
    tg = _tg()
    dt = torch.float64 if precision == "f64" else torch.float32
    xg, mg = _to_gpu(x, m, dt)
    n = xg.shape[1]
    ws = tg.Workspace(max(n, 1), precision=precision, **p)
    ws.build(xg)
    ws.moments(xg, mg)
    a, phi = ws.forces(emit_lists=emit)
    torch.cuda.synchronize()
    return ws, xg, mg, a, phi


def _rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.maximum(np.linalg.norm(ref, axis=0), 1e-300)


def _segment_sorted(off, vals):
    """Entries of each CSR segment in ascending order (segments kept in place)."""
    off = np.asarray(off, np.int64)
    g = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    key = (g << 32) | np.asarray(vals, np.int64)
    return np.sort(key) & 0xffffffff


def _check_structure(orc, ws, xg, mg, ref, gs):
    ex = ws.export_tree()
    n = xg.shape[1]
    np.testing.assert_array_equal(ex["keys"].cpu().numpy().astype(np.uint64), ref.key[ref.perm])
    np.testing.assert_array_equal(ex["perm"].cpu().numpy().astype(np.int64), ref.perm)
    t = ref.tree
    assert ex["info"]["n_nodes"] == t.nn
    np.testing.assert_array_equal(ex["level"].cpu().numpy(), t.level)
    np.testing.assert_array_equal(ex["corner"].cpu().numpy().astype(np.uint32), t.corner)
    np.testing.assert_array_equal(ex["first"].cpu().numpy(), t.first)
    np.testing.assert_array_equal(ex["count"].cpu().numpy(), t.count)
    np.testing.assert_array_equal(ex["child"].cpu().numpy(), t.child)
    np.testing.assert_array_equal(ex["nchild"].cpu().numpy(), t.nchild)
    assert ex["info"]["box_k"] == ref.k
    np.testing.assert_array_equal(np.array(ex["info"]["box_lo"]), ref.lo)
    # moments (FP64 on both sides, different summation order)
    M, R, Q = (_np64(v) for v in ws.export_moments())
    side = np.ldexp(1.0, ref.k - t.level.astype(np.int64))
    np.testing.assert_allclose(M, ref.M, rtol=1e-12, atol=0)
    assert np.all(np.abs(R - ref.R) <= 1e-12 * np.ldexp(1.0, ref.k))
    assert np.all(np.abs(Q - ref.Q) <= 1e-10 * (np.abs(ref.M) * side * side + 1e-300))
    # walk groups
    np.testing.assert_array_equal(ws.export_groups().cpu().numpy(), ref.gfirst)
    # lists, as sets per group
    pc_off, pc, pp_off, pp = (v.cpu().numpy() for v in ws.export_lists())
    np.testing.assert_array_equal(pc_off, ref.pc_off)
    np.testing.assert_array_equal(pp_off, ref.pp_off)
    np.testing.assert_array_equal(_segment_sorted(pc_off, pc), ref.pc_list)
    np.testing.assert_array_equal(_segment_sorted(pp_off, pp), ref.pp_list)


CASES = [
    # (name, generator, n, params)
    ("plummer16k_mono", "plummer", 16384, dict(eps=0.01, theta=0.7, order=0, leaf_cap=16, group_size=32)),
    ("plummer50001_quad_g64", "plummer", 50001, dict(eps=0.005, theta=0.5, order=2, leaf_cap=8, group_size=64)),
    ("galaxy30k_quad", "galaxy", 30000, dict(eps=0.02, theta=0.7, order=2, leaf_cap=16, group_size=32)),
    ("plummer3k_lcap1_g16", "plummer", 3001, dict(eps=0.01, theta=1.0, order=2, leaf_cap=1, group_size=16)),
    ("galaxy20k_chunks", "galaxy", 20000, dict(eps=0.02, theta=0.7, order=2, leaf_cap=16, group_size=32,
                                               group_split=0)),
    ("galaxy20k_split1_g64", "galaxy", 20011, dict(eps=0.02, theta=0.6, order=2, leaf_cap=8, group_size=64,
                                                   group_split=1)),
]


def _gen(kind, n, seed=20241202):
    if kind == "plummer":
        x, _, m = inputs.plummer(n, seed)
    else:
        x, _, m = inputs.galaxy(n, seed)
    return x, m


@pytest.mark.parametrize("name,kind,n,p", CASES, ids=[c[0] for c in CASES])
def test_fp32_parity(orc, name, kind, n, p):
    x, m = _gen(kind, n)
    ws, xg, mg, a, phi = _run(x, m, **p)
    assert ws.status() == 0
    ref = orc.tree_forces(_np64(xg), _np64(mg), eps=p["eps"], theta=p["theta"], lcap=p["leaf_cap"],
                          gs=p["group_size"], quad=p["order"] == 2, delta=p.get("group_split", 3))
    _check_structure(orc, ws, xg, mg, ref, p["group_size"])
    e = _rel_err(_np64(a), ref.a)
    assert np.median(e) <= 1e-5, np.median(e)
    assert e.max() <= 1e-4, (e.max(), int(np.argmax(e)))
    ep = np.abs(_np64(phi) - ref.phi) / np.abs(ref.phi)
    assert np.median(ep) <= 1e-5 and ep.max() <= 1e-4
    inf = ws.info()
    # interaction counts agree with the oracle's lists
    sizes = np.diff(ref.gfirst)
    assert inf["pc_pairs"] == int((sizes * np.diff(ref.pc_off)).sum())
    leaf_pp = np.zeros(len(ref.pp_off) - 1, np.int64)
    np.add.at(leaf_pp, np.repeat(np.arange(len(leaf_pp)), np.diff(ref.pp_off)), ref.tree.count[ref.pp_list])
    assert inf["pp_pairs"] == int((sizes * leaf_pp).sum())


@pytest.mark.parametrize("name,kind,n,p", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_fp64_parity(orc, name, kind, n, p):
    x, m = _gen(kind, n)
    ws, xg, mg, a, phi = _run(x, m, precision="f64", **p)
    assert ws.status() == 0
    ref = orc.tree_forces(_np64(xg), _np64(mg), eps=p["eps"], theta=p["theta"], lcap=p["leaf_cap"],
                          gs=p["group_size"], quad=p["order"] == 2, delta=p.get("group_split", 3))
    _check_structure(orc, ws, xg, mg, ref, p["group_size"])
    e = _rel_err(_np64(a), ref.a)
    assert e.max() <= 1e-11, e.max()
    assert np.max(np.abs(_np64(phi) - ref.phi) / np.abs(ref.phi)) <= 1e-11


def test_sparse_potential_far_below_self_term(orc):
    """Particles far apart compared with eps: |phi_i| is below 1e-4 of m_i/eps,
    so the self pair must be left out, not added and subtracted in FP32
    (that would cost ~1e-3 relative)."""
    g = torch.Generator().manual_seed(9)
    n = 200
    x = torch.rand((3, n), generator=g, dtype=torch.float64) * 1e5
    m = torch.full((n,), 1.0 / n, dtype=torch.float64)
    p = dict(eps=0.01, theta=0.7, order=2, leaf_cap=4, group_size=32)
    ws, xg, mg, a, phi = _run(x, m, **p)
    assert ws.status() == 0
    ref = orc.tree_forces(_np64(xg), _np64(mg), eps=0.01, theta=0.7, lcap=4, gs=32, quad=True)
    assert np.abs(ref.phi).max() < 1e-4 * (1.0 / n) / 0.01
    ep = np.abs(_np64(phi) - ref.phi) / np.abs(ref.phi)
    assert np.median(ep) <= 1e-5 and ep.max() <= 1e-4, (np.median(ep), ep.max())
    e = _rel_err(_np64(a), ref.a)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4


def test_kahan_off_still_within_tolerance(orc):
    x, m = _gen("plummer", 20000)
    p = dict(eps=0.01, theta=0.6, order=2, leaf_cap=16, group_size=32)
    ws, xg, mg, a, phi = _run(x, m, emit=False, kahan=0, **p)
    ref = orc.tree_forces(_np64(xg), _np64(mg), eps=0.01, theta=0.6, lcap=16, gs=32, quad=True)
    e = _rel_err(_np64(a), ref.a)
    assert np.median(e) <= 1e-5


def test_far_cell_forms_agree(orc):
    """The FP32 walk evaluates full far-cell tiles with the quadrupole term's
    r^-5 taken out of the acceleration when the tree's cube is at most 2^24 on a
    side, and with the full form otherwise.  Scaling positions and eps by a power
    of two leaves the tree unchanged and scales every FP32 operation exactly; the
    scale here puts the cube at 2^25, past that limit but with r^-5 still within
    a few binades of the normal range (>= 20 bits).  a * s^2 and phi * s of the
    scaled run (full form) must match the unscaled run (r^-5 form) to FP32
    rounding, and the scaled run must match the oracle."""
    x, m = _gen("galaxy", 40000)
    p = dict(theta=0.7, order=2, leaf_cap=16, group_size=32)
    ws1, xg1, mg1, a1, phi1 = _run(x, m, emit=False, eps=0.02, **p)
    k = ws1.info()["box_k"]
    assert k <= 24
    s = 2.0 ** (25 - k)
    ws2, xg2, mg2, a2, phi2 = _run(x * s, m, emit=False, eps=0.02 * s, **p)
    assert ws1.status() == 0 and ws2.status() == 0 and ws2.info()["box_k"] == 25
    np.testing.assert_array_equal(ws1.export_tree()["perm"].cpu().numpy(), ws2.export_tree()["perm"].cpu().numpy())
    e = _rel_err(_np64(a2) * s * s, _np64(a1))
    assert np.median(e) <= 1e-6 and e.max() <= 1e-4, (np.median(e), e.max())
    ep = np.abs(_np64(phi2) * s - _np64(phi1)) / np.abs(_np64(phi1))
    assert np.median(ep) <= 1e-6 and ep.max() <= 1e-4, (np.median(ep), ep.max())
    ref = orc.tree_forces(_np64(xg2), _np64(mg2), eps=0.02 * s, theta=0.7, lcap=16, gs=32, quad=True)
    e2 = _rel_err(_np64(a2), ref.a)
    assert np.median(e2) <= 1e-5 and e2.max() <= 1e-4, (np.median(e2), e2.max())


def test_keys_exact_near_cell_boundaries(orc):
    """FP32 coordinates are quantised in FP32 arithmetic where that provably
    gives the FP64 definition's cell and in FP64 otherwise.  Points on cell
    boundaries, one or two ulps either side of them, tiny coordinates 2^-60 or
    more below the box corner's magnitude (where the FP64 subtraction rounds)
    and zeros must get the oracle's keys bit for bit."""
    rng = np.random.default_rng(5)
    k, lo = 4, -8.0
    unit = 2.0 ** (k - 21)
    g = (lo + rng.integers(0, 2 ** 21, size=(3, 4000)) * unit).astype(np.float32)
    up, down = np.nextafter(g, np.float32(np.inf)), np.nextafter(g, np.float32(-np.inf))
    up2 = np.nextafter(up, np.float32(np.inf))
    tiny = (rng.uniform(-1.0, 1.0, size=(3, 2000)) * 10.0 ** rng.integers(-30, -18, size=(3, 2000))).astype(np.float32)
    x = np.concatenate([np.full((3, 1), lo, np.float32), g, up, down, up2, tiny, np.zeros((3, 50), np.float32)], axis=1)
    x = np.clip(x, np.float32(lo), np.float32(7.5))
    m = np.full(x.shape[1], 1.0 / x.shape[1])
    ws, xg, mg, a, phi = _run(torch.from_numpy(x.astype(np.float64)), torch.from_numpy(m), emit=False, eps=0.01,
                              theta=0.7, order=2, leaf_cap=16, group_size=32)
    assert ws.status() == 0 and ws.info()["box_k"] == k
    x64 = _np64(xg)
    blo, bk = orc.box(x64)
    assert bk == k and np.all(blo == lo)
    _, key = orc.keys(x64, blo, bk)
    perm = orc.sort(key)
    ex = ws.export_tree()
    np.testing.assert_array_equal(ex["keys"].cpu().numpy().astype(np.uint64), key[perm])
    np.testing.assert_array_equal(ex["perm"].cpu().numpy().astype(np.int64), perm)


def test_theta_zero_equals_direct_sum(orc):
    x, m = _gen("plummer", 4000)
    ws, xg, mg, a, phi = _run(x, m, eps=0.01, theta=0.0, order=2, leaf_cap=16, group_size=32)
    ad, phid = orc.direct(_np64(xg), _np64(mg), eps=0.01)
    e = _rel_err(_np64(a), ad)
    assert np.median(e) <= 1e-6 and e.max() <= 1e-4
    # the GPU direct-sum reference agrees as well
    tg = _tg()
    tgt = torch.arange(0, 4000, 7)
    a2, p2 = ws.direct(xg, mg, tgt, precision="f32")
    e2 = _rel_err(_np64(a2), ad[:, tgt.numpy()])
    assert e2.max() <= 1e-5
    a3, p3 = ws.direct(xg.double(), mg.double(), tgt, precision="f64")
    assert _rel_err(_np64(a3), ad[:, tgt.numpy()]).max() <= 1e-12


# ------------------------------------------------------------------ edge cases
def _edge(orc, x, m, p, exact_structure=True):
    x = torch.as_tensor(x, dtype=torch.float64)
    m = torch.as_tensor(m, dtype=torch.float64)
    ws, xg, mg, a, phi = _run(x, m, **p)
    assert ws.status() == 0
    ref = orc.tree_forces(_np64(xg), _np64(mg), eps=p["eps"], theta=p["theta"], lcap=p["leaf_cap"],
                          gs=p["group_size"], quad=p["order"] == 2)
    if exact_structure:
        _check_structure(orc, ws, xg, mg, ref, p["group_size"])
    scale = np.abs(ref.a).max() + 1e-30
    assert np.abs(_np64(a) - ref.a).max() <= 1e-5 * scale
    return ws, a, phi, ref


P0 = dict(eps=0.01, theta=0.7, order=2, leaf_cap=4, group_size=32)


def test_single_particle(orc):
    ws, a, phi, ref = _edge(orc, [[0.3], [0.1], [-0.2]], [2.0], P0)
    assert torch.all(a == 0) and torch.all(phi == 0)


def test_two_particles(orc):
    _edge(orc, [[0.0, 1.0], [0.0, 0.5], [0.0, 0.0]], [1.0, 3.0], P0)


@pytest.mark.parametrize("n", [5, 31, 33, 63, 65, 4097])
def test_ragged_sizes(orc, n):
    x, m = _gen("plummer", n, seed=n)
    _edge(orc, x, m, dict(P0, group_size=32 if n % 2 else 64))


def test_coincident_particles_depth21(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 400))
    x[:, :100] = x[:, :1]                      # 100 coincident: a depth-21 leaf of 100 (> 16)
    x[:, 100:130] = x[:, :1] + 1e-7            # nearly coincident
    m = rng.uniform(0.5, 1.5, 400) / 400
    _edge(orc, x, m, dict(P0, leaf_cap=2))


def test_planar_and_collinear(orc):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 3000)); x[2] = 0.0
    _edge(orc, x, np.full(3000, 1 / 3000), P0)
    y = np.zeros((3, 500)); y[0] = np.linspace(-1, 1, 500)
    _edge(orc, y, np.full(500, 1 / 500), P0)


def test_all_at_one_point(orc):
    x = np.full((3, 40), 0.25)
    m = np.full(40, 0.025)
    ws, a, phi, ref = _edge(orc, x, m, P0)
    assert ws.info()["box_k"] == 0
    assert torch.all(a == 0)


def test_unsoftened(orc):
    x, m = _gen("plummer", 3000, seed=9)
    _edge(orc, x, m, dict(P0, eps=0.0))


def test_empty_input():
    tg = _tg()
    ws = tg.Workspace(10)
    x = torch.empty((3, 0), device="cuda")
    m = torch.empty((0,), device="cuda")
    a, phi = ws.accel(x, m)
    assert a.shape == (3, 0)
    assert ws.status() == 0


def test_nonfinite_reported():
    tg = _tg()
    x, m = _gen("plummer", 1000)
    xg, mg = _to_gpu(x, m, torch.float32)
    xg[1, 17] = float("nan")
    ws = tg.Workspace(1000)
    ws.accel(xg, mg)
    st = ws.status()
    assert st & tg.DEV_NONFINITE
    assert ws.status() == 0  # cleared


def test_capacity_and_argument_errors():
    tg = _tg()
    ws = tg.Workspace(100)
    x = torch.zeros((3, 200), device="cuda")
    with pytest.raises(tg.TreeError) as e:
        ws.build(x)
    assert e.value.code == tg.TREE_ERR_CAPACITY
    with pytest.raises(tg.TreeError) as e:
        ws2 = tg.Workspace(100)
        ws2.forces(torch.zeros((3, 0), device="cuda"))
    assert e.value.code in (tg.TREE_ERR_STATE,)


def test_node_capacity_degrades_gracefully(orc):
    """A node array too small for the tree turns deep cells into large
    leaves: the status says so and the forces are still right."""
    tg = _tg()
    x, m = _gen("plummer", 20000)
    xg, mg = _to_gpu(x, m, torch.float32)
    ws = tg.Workspace(20000, eps=0.01, theta=0.6, leaf_cap=4, node_cap=3000)
    a, phi = ws.accel(xg, mg)
    st = ws.status()
    assert st == tg.DEV_NODES
    ad, _ = orc.direct(_np64(xg), _np64(mg), eps=0.01, targets=np.arange(0, 20000, 97))
    e = _rel_err(_np64(a)[:, ::97], ad)
    assert np.median(e) < 1e-3


def test_stack_overflow_reported():
    tg = _tg()
    x, m = _gen("plummer", 30000)
    xg, mg = _to_gpu(x, m, torch.float32)
    ws = tg.Workspace(30000, eps=0.001, theta=0.15, leaf_cap=1, stack_depth=256)
    ws.accel(xg, mg)
    st = ws.status()
    inf = ws.info()
    assert (st & tg.DEV_STACK) or inf["max_stack"] <= 256


# ------------------------------------------------------------------ leapfrog
def test_leapfrog_plain_config(orc):
    """Plummer N = 16384, eps = 0.01, theta = 0.7, monopole, leaf <= 16: one force
    evaluation + 10 KDK steps (tau = 0.01) against the FP64 oracle; energy and
    momentum diagnostics in FP64."""
    tg = _tg()
    n, tau, steps = 16384, 0.01, 10
    x, v, m = inputs.plummer(n, 20241202)
    p = dict(eps=0.01, theta=0.7, order=0, leaf_cap=16, group_size=32)
    xg, vg, mg = (t.to("cuda", torch.float32).contiguous() for t in (x, v, m))
    ws = tg.Workspace(n, **p)
    a, phi = ws.accel(xg, mg)
    d0 = ws.diagnostics(xg, vg, mg, phi).cpu().numpy()
    x64, v64, m64 = _np64(xg), _np64(vg), _np64(mg)
    acc = lambda xx: orc.tree_accel(xx, m64, eps=0.01, theta=0.7, lcap=16, gs=32, quad=False)
    a0 = acc(x64)
    for _ in range(steps):
        ws.leapfrog_step(xg, vg, mg, a, tau, phi=phi)
    torch.cuda.synchronize()
    assert ws.status() == 0
    xo, vo, ao, po = orc.kdk(x64, v64, m64, tau, steps, acc, a0=a0)
    assert np.abs(_np64(xg) - xo).max() < 2e-5
    assert np.abs(_np64(vg) - vo).max() < 2e-4
    d1 = ws.diagnostics(xg, vg, mg, phi).cpu().numpy()
    do = orc.diagnostics(xo, vo, m64, po)
    assert abs(d1[0] - do["ekin"]) < 1e-5 * abs(do["ekin"])
    assert abs(d1[1] - do["epot"]) < 1e-5 * abs(do["epot"])
    e0 = d0[0] + d0[1]
    assert abs((d1[0] + d1[1]) - e0) < 1e-3 * abs(e0)
    np.testing.assert_allclose(d1[2:5], do["P"], atol=1e-5)
    np.testing.assert_allclose(d1[5:8], do["L"], atol=1e-5)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_leapfrog_forces_equal_standalone_evaluation(precision):
    """The leapfrog's force pass reads the packed (x, y, z, m) copy written by its
    kick-drift pass; a separate tree_build + tree_moments + tree_forces on the
    drifted positions reads the caller's arrays.  Same tree, same sums: the
    accelerations and potentials must agree bit for bit."""
    tg = _tg()
    n, tau = 20011, 0.005
    x, v, m = inputs.galaxy(n, 7)
    dt = torch.float64 if precision == "f64" else torch.float32
    xg, vg, mg = (t.to("cuda", dt).contiguous() for t in (x, v, m))
    p = dict(eps=0.02, theta=0.6, order=2, leaf_cap=16, group_size=32, precision=precision)
    with tg.Workspace(n, **p) as ws, tg.Workspace(n, **p) as w2:
        a, phi = ws.accel(xg, mg)
        ws.leapfrog_step(xg, vg, mg, a, tau, phi=phi)
        a2, phi2 = w2.accel(xg, mg)
        torch.cuda.synchronize()
        assert ws.status() == 0 and w2.status() == 0
        assert torch.equal(a, a2)
        assert torch.equal(phi, phi2)


def test_diagnostics_match_oracle(orc):
    tg = _tg()
    x, v, m = inputs.plummer(5000, 2)
    xg, vg, mg = (t.to("cuda", torch.float64).contiguous() for t in (x, v, m))
    ws = tg.Workspace(5000, precision="f64")
    phi = torch.linspace(-1, -0.1, 5000, device="cuda", dtype=torch.float64)
    d = ws.diagnostics(xg, vg, mg, phi).cpu().numpy()
    do = orc.diagnostics(_np64(xg), _np64(vg), _np64(mg), _np64(phi))
    np.testing.assert_allclose(d[0], do["ekin"], rtol=1e-13)
    np.testing.assert_allclose(d[1], do["epot"], rtol=1e-13)
    np.testing.assert_allclose(d[2:5], do["P"], atol=1e-15)
    np.testing.assert_allclose(d[5:8], do["L"], atol=1e-14)


def test_export_lists_groups_matches_full_export():
    """tree_export_lists_groups gives, for any selection of groups (any order,
    repeats allowed), exactly the segments of the full list export."""
    tg = _tg()
    x, m = _gen("galaxy", 30000)
    ws, xg, mg, a, phi = _run(x, m, eps=0.02, theta=0.7, order=2, leaf_cap=16, group_size=32)
    pc_off, pc, pp_off, pp = (v.cpu().numpy() for v in ws.export_lists())
    ng = len(pc_off) - 1
    sel = [ng - 1, 0, 17, 17, ng // 2, 3]
    so, spc, po, spp = ws.export_lists_groups(sel)
    spc, spp = spc.cpu().numpy(), spp.cpu().numpy()
    for k, g in enumerate(sel):
        np.testing.assert_array_equal(spc[so[k]: so[k + 1]], pc[pc_off[g]: pc_off[g + 1]])
        np.testing.assert_array_equal(spp[po[k]: po[k + 1]], pp[pp_off[g]: pp_off[g + 1]])
    with pytest.raises(tg.TreeError) as e:
        ws.export_lists_groups([ng])
    assert e.value.code == tg.TREE_ERR_ARG


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_state_step_equals_device_step(precision, pinned):
    """leapfrog_step_host (state in host memory, copies up inside the call, x
    copied back under the walk; v, a, phi written by the walk into mapped
    page-locked arrays, or copied back after it from pageable ones) gives
    exactly the device-resident step: the same kernels on the same data."""
    tg = _tg()
    n, tau = 20011, 0.005
    x, v, m = inputs.galaxy(n, 5)
    dt = torch.float64 if precision == "f64" else torch.float32
    xg, vg, mg = (t.to("cuda", dt).contiguous() for t in (x, v, m))
    p = dict(eps=0.02, theta=0.6, order=2, leaf_cap=16, group_size=32, precision=precision)
    with tg.Workspace(n, **p) as wd, tg.Workspace(n, **p) as wh:
        a, phi = wd.accel(xg, mg)
        host = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
        xh, vh, mh, ah = (host(t.cpu()) for t in (xg, vg, mg, a))
        ph = host(torch.empty(n, dtype=dt))
        dh = host(torch.empty(8, dtype=torch.float64))
        diag = torch.empty(8, dtype=torch.float64, device="cuda")
        for _ in range(3):
            wd.leapfrog_step(xg, vg, mg, a, tau, phi=phi)
            wd.diagnostics(xg, vg, mg, phi, out=diag)
            wh.leapfrog_step_host(xh, vh, mh, ah, tau, phi=ph, diag=dh)
        torch.cuda.synchronize()
        assert wd.status() == 0 and wh.status() == 0
        for dev_t, host_t in ((xg, xh), (vg, vh), (a, ah), (phi, ph), (diag, dh)):
            assert torch.equal(dev_t.cpu(), host_t)


def test_fp32_peak_probe():
    """The FP32 FMA peak the roofline is reported against: positive, below the
    unit-count bound (152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s,
    with a small margin for clock reporting), packed at least as fast as scalar
    within a few percent."""
    tg = _tg()
    scalar, packed = tg.fp32_peak()
    assert 10.0 < scalar < 82.0 and 10.0 < packed < 82.0, (scalar, packed)
    assert packed > 0.9 * scalar
