"""Ensembles on the GPU: independent systems in one build (tree_set_segments).

Each system must come out exactly as if it were alone: the batched build's
keys, permutation, box, nodes, walk groups and interaction lists restricted to
a system equal (bit for bit, after renumbering the nodes) those of a
workspace holding that system alone, and its FP32 forces, leapfrog states and
per-system diagnostics agree with the lone run -- bit-identical where the
arithmetic is the same, to FP64 rounding for the reductions -- and with the
FP64 oracle of each system (median relative error <= 1e-5, max <= 1e-4).  Also: a captured CUDA
graph of a step replays the eager steps bit for bit; the autotuner returns
the fastest valid candidate.
"""
import numpy as np
import pytest
import torch

from paper_2412_01733_gb300 import inputs

pytestmark = pytest.mark.gpu

P = dict(eps=0.01, theta=0.6, order=2, leaf_cap=8, group_size=32)


def _tg():
    from paper_2412_01733_gb300 import build, treegb
    build.build()
    return treegb


def _np64(t):
    return t.detach().double().cpu().numpy()


def _mixed_ensemble(seed=11):
    """Systems of very different sizes, centres and scales (incl. 1 and 2 particles)."""
    sizes = [1, 2, 17, 33, 700, 4101, 9000]
    xs, vs, ms = [], [], []
    for b, nb in enumerate(sizes):
        if b % 2:
            x, v, m = inputs.plummer(nb, seed + b)
        else:
            x, v, m = inputs.galaxy(nb, seed + b)
        scale = [0.1, 1.0, 10.0][b % 3]
        shift = torch.tensor([3.0 * b, -1.0 * b, 0.5 * b], dtype=torch.float64)[:, None]
        xs.append(x * scale + shift); vs.append(v); ms.append(m)
    off = np.concatenate(([0], np.cumsum(sizes))).astype(np.int64)
    return torch.cat(xs, 1), torch.cat(vs, 1), torch.cat(ms), off


def _run(tg, x, m, off=None, **p):
    n = x.shape[1]
    ws = tg.Workspace(n, **p)
    if off is not None:
        ws.set_segments(off)
    ws.build(x); ws.moments(x, m)
    a, phi = ws.forces(emit_lists=True)
    torch.cuda.synchronize()
    assert ws.status() == 0
    return ws, a, phi


def _check_system(ex, groups, lists, b0, b1, exa, groupsa, listsa):
    """Batched structure restricted to sorted range [b0, b1) vs the lone build."""
    np.testing.assert_array_equal(ex["keys"][b0:b1].cpu().numpy(), exa["keys"].cpu().numpy())
    np.testing.assert_array_equal(ex["perm"][b0:b1].cpu().numpy() - b0, exa["perm"].cpu().numpy())
    first = ex["first"].cpu().numpy().astype(np.int64)
    sel = np.nonzero((first >= b0) & (first < b1))[0]          # this system's nodes, batched numbering
    nn = exa["info"]["n_nodes"]
    assert sel.size == nn
    for f in ("level", "count", "nchild"):
        np.testing.assert_array_equal(ex[f].cpu().numpy()[sel], exa[f].cpu().numpy())
    np.testing.assert_array_equal(ex["corner"].cpu().numpy()[:, sel], exa["corner"].cpu().numpy())
    np.testing.assert_array_equal(first[sel] - b0, exa["first"].cpu().numpy())
    ch, cha = ex["child"].cpu().numpy()[sel], exa["child"].cpu().numpy()
    np.testing.assert_array_equal(ch[cha < 0], -1)
    np.testing.assert_array_equal(ch[cha >= 0], sel[cha[cha >= 0]])
    # walk groups and lists (in walk order: the relative order of cells is preserved)
    inv = np.full(first.size, -1, np.int64)
    inv[sel] = np.arange(nn)
    gf = groups.cpu().numpy()
    gsel = np.nonzero((gf[:-1] >= b0) & (gf[:-1] < b1))[0]
    np.testing.assert_array_equal(gf[gsel] - b0, groupsa.cpu().numpy()[:-1])
    for (off, lst), (offa, lsta) in zip(((lists[0], lists[1]), (lists[2], lists[3])),
                                        ((listsa[0], listsa[1]), (listsa[2], listsa[3]))):
        off, lst, offa, lsta = (t.cpu().numpy() for t in (off, lst, offa, lsta))
        for k, g in enumerate(gsel):
            mine = inv[lst[off[g]:off[g + 1]]]
            np.testing.assert_array_equal(mine, lsta[offa[k]:offa[k + 1]])


def test_ensemble_equals_each_system_alone(orc):
    tg = _tg()
    x, v, m, off = _mixed_ensemble()
    xg, mg = x.float().cuda().contiguous(), m.float().cuda().contiguous()
    ws, a, phi = _run(tg, xg, mg, off, **P)
    assert ws.info()["n_segments"] == len(off) - 1
    ex = ws.export_tree()
    groups = ws.export_groups()
    lists = ws.export_lists()
    lo, k = ws.export_boxes()
    for b, (b0, b1) in enumerate(zip(off[:-1], off[1:])):
        xb, mb = xg[:, b0:b1].contiguous(), mg[b0:b1].contiguous()
        wa, aa, pa = _run(tg, xb, mb, **P)
        _check_system(ex, groups, lists, b0, b1, wa.export_tree(), wa.export_groups(), wa.export_lists())
        ia = wa.info()
        assert int(k[b]) == ia["box_k"] and lo[b].tolist() == ia["box_lo"]
        assert torch.equal(a[:, b0:b1], aa) and torch.equal(phi[b0:b1], pa)
        # the FP64 oracle of this system alone
        ref = orc.tree_forces(_np64(xb), _np64(mb), eps=P["eps"], theta=P["theta"], lcap=P["leaf_cap"],
                              gs=P["group_size"], quad=True)
        assert int(k[b]) == ref.k and np.array_equal(lo[b].numpy(), ref.lo)
        nb = b1 - b0
        if nb == 1:
            assert float(a[:, b0].abs().max()) == 0.0
            assert abs(float(phi[b0])) <= 1e-6 * float(mb[0]) / P["eps"]
            continue
        e = np.linalg.norm(_np64(aa) - ref.a, axis=0) / np.linalg.norm(ref.a, axis=0)
        assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (b, np.median(e), e.max())
        ep = np.abs(_np64(pa) - ref.phi) / np.abs(ref.phi)
        assert np.median(ep) <= 1e-5 and ep.max() <= 1e-4


def test_ensemble_mixed_far_cell_forms():
    """The FP32 walk chooses its far-cell form per segment (the r^-5 form only
    where the segment's cube is at most 2^24 on a side): an ensemble holding a
    system with a small cube and the same system scaled past 2^24 gives each
    system the forces it gets alone, bit for bit."""
    tg = _tg()
    x, _, m = inputs.galaxy(3000, 21)
    w1 = tg.Workspace(3000, **P)
    w1.build(x.float().cuda().contiguous())
    s = 2.0 ** (25 - w1.info()["box_k"])
    x2 = torch.cat([x, x * s], 1)
    m2 = torch.cat([m, m])
    off = np.array([0, 3000, 6000], np.int64)
    xe, me = x2.float().cuda().contiguous(), m2.float().cuda().contiguous()
    ws, a, phi = _run(tg, xe, me, off, **P)
    _, kb = ws.export_boxes()
    assert int(kb[0]) <= 24 and int(kb[1]) == 25
    for b0, b1 in ((0, 3000), (3000, 6000)):
        wa, aa, pa = _run(tg, xe[:, b0:b1].contiguous(), me[b0:b1].contiguous(), **P)
        assert torch.equal(a[:, b0:b1], aa) and torch.equal(phi[b0:b1], pa)


def test_ensemble_leapfrog_and_diagnostics_equal_alone():
    tg = _tg()
    x, v, m, off = _mixed_ensemble(seed=23)
    xg, vg, mg = (t.float().cuda().contiguous() for t in (x, v, m))
    tau, K = 0.002, 3
    ws = tg.Workspace(xg.shape[1], **P)
    ws.set_segments(off)
    xb, vb = xg.clone(), vg.clone()
    a, phi = ws.accel(xb, mg)
    for _ in range(K):
        ws.leapfrog_step(xb, vb, mg, a, tau, phi=phi)
    d = ws.diagnostics_segments(xb, vb, mg, phi).cpu().numpy()
    assert ws.status() == 0
    for b, (b0, b1) in enumerate(zip(off[:-1], off[1:])):
        wa = tg.Workspace(b1 - b0, **P)
        xa, va, ma = xg[:, b0:b1].clone(), vg[:, b0:b1].clone(), mg[b0:b1].contiguous()
        aa, pa = wa.accel(xa, ma)
        for _ in range(K):
            wa.leapfrog_step(xa, va, ma, aa, tau, phi=pa)
        assert torch.equal(xb[:, b0:b1], xa) and torch.equal(vb[:, b0:b1], va)
        assert torch.equal(a[:, b0:b1], aa) and torch.equal(phi[b0:b1], pa)
        da = wa.diagnostics(xa, va, ma, pa).cpu().numpy()
        # FP32 products summed in runs of 32, runs in FP64: the runs differ between the two reductions
        mv = float((ma.double() * va.double().norm(dim=0)).sum())
        mxv = float((ma.double() * xa.double().norm(dim=0) * va.double().norm(dim=0)).sum())
        mp = float((ma.double() * pa.double().abs()).sum())
        assert abs(d[b, 0] - da[0]) <= 1e-5 * abs(da[0]) + 1e-12
        assert abs(d[b, 1] - da[1]) <= 1e-5 * mp + 1e-12
        assert np.all(np.abs(d[b, 2:5] - da[2:5]) <= 1e-5 * mv + 1e-12)
        assert np.all(np.abs(d[b, 5:8] - da[5:8]) <= 1e-5 * mxv + 1e-12)


@pytest.mark.parametrize("segmented", [False, True])
def test_graph_replay_equals_eager_steps(segmented):
    tg = _tg()
    x, v, m, off = _mixed_ensemble(seed=31)
    xg, vg, mg = (t.float().cuda().contiguous() for t in (x, v, m))
    tau, K = 0.002, 4
    ws = tg.Workspace(xg.shape[1], **P)
    we = tg.Workspace(xg.shape[1], **P)
    if segmented:
        ws.set_segments(off); we.set_segments(off)
    xa, va = xg.clone(), vg.clone()
    a, phi = ws.accel(xa, mg)
    xe, ve = xg.clone(), vg.clone()
    ae, pe = we.accel(xe, mg)
    diag = torch.zeros(8, dtype=torch.float64, device="cuda")
    l0 = ws.launches()
    ws.graph_capture(xa, va, mg, a, tau, phi=phi, diag=diag)
    assert ws.launches() == l0          # capturing runs nothing
    for _ in range(K):
        ws.graph_launch()
        we.leapfrog_step(xe, ve, mg, ae, tau, phi=pe)
    de = we.diagnostics(xe, ve, mg, pe)
    torch.cuda.synchronize()
    assert ws.status() == 0 and we.status() == 0
    assert torch.equal(xa, xe) and torch.equal(va, ve) and torch.equal(a, ae) and torch.equal(phi, pe)
    assert torch.equal(diag, de)
    assert ws.launches() > l0
    # the workspace holds the tree of the last replayed step
    assert ws.info()["n_groups"] == we.info()["n_groups"]


def test_autotune_picks_fastest_valid():
    tg = _tg()
    x, v, m, off = inputs.ensemble(16, 5, nmin=512, nmax=8192, device="cuda", dtype=torch.float32)
    best, table = tg.autotune(x.contiguous(), m.contiguous(), offsets=off, reps=2, **P)
    assert len(table) == 18
    ms = np.array([r[3] for r in table])
    err = np.array([r[4] for r in table])
    assert np.isfinite(ms).any()
    # every candidate meets the default bound (median error <= 1e-3) at theta = 0.6
    assert np.all(err[np.isfinite(ms)] <= 1e-3) and np.all(err > 0)
    i = int(np.nanargmin(np.where(np.isfinite(ms), ms, np.inf)))
    assert (best.leaf_cap, best.group_size, best.stack_depth) == tuple(int(t) for t in table[i][:3])
    assert best.theta == P["theta"] and best.eps == P["eps"]


def test_autotune_error_bound_excludes_fastest():
    """With a bound just below the error of the fastest candidate, the tuner must
    return a slower candidate that meets it: the fastest one among those whose
    median force error against the FP64 direct sum is within the bound."""
    tg = _tg()
    x, v, m, off = inputs.ensemble(16, 5, nmin=512, nmax=8192, device="cuda", dtype=torch.float32)
    x, m = x.contiguous(), m.contiguous()
    _, free = tg.autotune(x, m, offsets=off, reps=2, max_err=None, **P)
    ms = np.array([r[3] for r in free]); err = np.array([r[4] for r in free])
    i0 = int(np.argmin(ms))
    assert np.isfinite(ms[i0])
    bound = 0.999 * err[i0]
    assert (err <= bound).any(), "some candidate is more accurate than the fastest one"
    best, tab = tg.autotune(x, m, offsets=off, reps=2, max_err=bound, **P)
    ms2 = np.array([r[3] for r in tab]); err2 = np.array([r[4] for r in tab])
    np.testing.assert_array_equal(err2, err)             # the error column does not depend on timing
    assert not np.isfinite(ms2[err2 > bound]).any()      # every candidate above the bound is rejected
    j = [tuple(int(t) for t in r[:3]) for r in tab].index((best.leaf_cap, best.group_size, best.stack_depth))
    assert err2[j] <= bound and ms2[j] == np.min(ms2[np.isfinite(ms2)])
    assert tuple(int(t) for t in tab[j][:3]) != tuple(int(t) for t in free[i0][:3])
    # a bound below every candidate's error leaves none
    with pytest.raises(tg.TreeError) as e:
        tg.autotune(x, m, offsets=off, reps=1, max_err=0.5 * err.min(), **P)
    assert e.value.code == tg.TREE_ERR_DEVICE


def test_ensemble_adjoint_equals_alone():
    tg = _tg()
    x, v, m, off = _mixed_ensemble(seed=41)
    xg, mg = x.cuda().contiguous(), m.cuda().contiguous()
    p = dict(P, precision="f64")
    ws, a, phi = _run(tg, xg, mg, off, **p)
    g = torch.Generator().manual_seed(3)
    ab = torch.randn(xg.shape, generator=g, dtype=torch.float64).cuda()
    pb = torch.randn(mg.shape, generator=g, dtype=torch.float64).cuda()
    xb, mb = ws.forces_adjoint(ab, pb)
    for b0, b1 in zip(off[:-1], off[1:]):
        wa, aa, pa = _run(tg, xg[:, b0:b1].contiguous(), mg[b0:b1].contiguous(), **p)
        xa, ma = wa.forces_adjoint(ab[:, b0:b1].contiguous(), pb[b0:b1].contiguous())
        sx = float(xa.abs().max()) + 1e-300
        sm = float(ma.abs().max()) + 1e-300
        assert float((xb[:, b0:b1] - xa).abs().max()) <= 1e-12 * sx
        assert float((mb[b0:b1] - ma).abs().max()) <= 1e-12 * sm


def test_segment_argument_errors():
    tg = _tg()
    ws = tg.Workspace(100, **P)
    for bad in ([0, 10, 10, 20], [1, 10, 20], [0, 50, 101]):
        with pytest.raises(tg.TreeError):
            ws.set_segments(bad)
    ws.set_segments([0, 40, 100])
    x = torch.zeros((3, 99), dtype=torch.float32, device="cuda")
    with pytest.raises(tg.TreeError):
        ws.build(x)
    ws.set_segments(None)
    assert ws.segments() == 1


def test_ensemble_full_size_sampled(orc):
    """512 Plummer clusters, N_c = floor(exp U(ln 1024, ln 65536)), the ensemble
    benchmark's launch configuration: sampled systems equal their lone runs bit
    for bit, the smallest also the FP64 oracle."""
    tg = _tg()
    x, v, m, off = inputs.ensemble(512, 20241202, device="cuda", dtype=torch.float32)
    x, m = x.contiguous(), m.contiguous()
    p = dict(eps=0.01, theta=0.6, order=2, leaf_cap=16, group_size=32)
    ws = tg.Workspace(x.shape[1], **p)
    ws.set_segments(off)
    a, phi = ws.accel(x, m)
    torch.cuda.synchronize()
    assert ws.status() == 0
    sizes = np.diff(off)
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 7, 300})
    for b in pick:
        b0, b1 = int(off[b]), int(off[b + 1])
        xb, mb = x[:, b0:b1].contiguous(), m[b0:b1].contiguous()
        wa = tg.Workspace(b1 - b0, **p)
        aa, pa = wa.accel(xb, mb)
        assert torch.equal(a[:, b0:b1], aa) and torch.equal(phi[b0:b1], pa)
        if b == int(np.argmin(sizes)):
            ref = orc.tree_forces(_np64(xb), _np64(mb), eps=0.01, theta=0.6, lcap=16, gs=32, quad=True)
            e = np.linalg.norm(_np64(aa) - ref.a, axis=0) / np.linalg.norm(ref.a, axis=0)
            assert np.median(e) <= 1e-5 and e.max() <= 1e-4


def test_ensemble_fp64_equals_each_system_alone():
    """The FP64 plain walk with systems: bit-identical to each system alone."""
    tg = _tg()
    x, v, m, off = _mixed_ensemble(seed=53)
    xg, mg = x.cuda().contiguous(), m.cuda().contiguous()
    p = dict(P, precision="f64")
    ws, a, phi = _run(tg, xg, mg, off, **p)
    for b0, b1 in zip(off[:-1], off[1:]):
        wa, aa, pa = _run(tg, xg[:, b0:b1].contiguous(), mg[b0:b1].contiguous(), **p)
        assert torch.equal(a[:, b0:b1], aa) and torch.equal(phi[b0:b1], pa)


def test_many_systems_two_segment_passes():
    """300 systems (> 256: the system index takes two sort passes), sizes 1..40."""
    tg = _tg()
    sizes = np.random.default_rng(7).integers(1, 41, size=300)
    xs, ms = [], []
    for b, nb in enumerate(sizes):
        x, _, m = inputs.plummer(int(nb), 100 + b)
        xs.append(x * (0.5 + (b % 5))); ms.append(m)
    off = np.concatenate(([0], np.cumsum(sizes))).astype(np.int64)
    xg, mg = torch.cat(xs, 1).float().cuda().contiguous(), torch.cat(ms).float().cuda().contiguous()
    ws, a, phi = _run(tg, xg, mg, off, **P)
    ex = ws.export_tree()
    perm = ex["perm"].cpu().numpy()
    # every system's particles stay in its own sorted range
    for b0, b1 in zip(off[:-1], off[1:]):
        assert perm[b0:b1].min() >= b0 and perm[b0:b1].max() < b1
    for b in (0, 150, 299):
        b0, b1 = int(off[b]), int(off[b + 1])
        wa, aa, pa = _run(tg, xg[:, b0:b1].contiguous(), mg[b0:b1].contiguous(), **P)
        assert torch.equal(a[:, b0:b1], aa) and torch.equal(phi[b0:b1], pa)
