"""The allocation-free direct sum (tree_direct_forces_noalloc).

Some callers cannot allocate device memory (their own pool owns the GPU, or
they may only use the buffers they are handed), so they cannot create a
workspace.  This entry point gives them the direct summation of Eq. 1 using
a fixed scratch array inside the library.  It must agree with the workspace
version, call after call (the scratch array is shared and reused).

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2412_01733_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2412_01733_gb300 import build, treegb
    build.build()
    return treegb


def _noalloc(tg, x, m, targets, precision, G, eps):
    nt = targets.numel()
    a = torch.empty((3, nt), dtype=torch.float64, device="cuda")
    phi = torch.empty((nt,), dtype=torch.float64, device="cuda")
    dt = tg.F64 if precision == "f64" else tg.F32
    code = tg.lib().tree_direct_forces_noalloc(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr()), x.shape[1], dt, float(G), float(eps),
        ctypes.c_void_p(targets.data_ptr()), nt, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == tg.TREE_OK, tg.status_string(code)
    return a, phi


@pytest.mark.parametrize("precision,rtol,rtol_orc", [("f32", 1e-6, 1e-5), ("f64", 1e-12, 1e-12)])
def test_noalloc_matches_workspace_direct(orc, precision, rtol, rtol_orc):
    tg = _lib()
    dt = torch.float64 if precision == "f64" else torch.float32
    n = 30000
    x, _, m = inputs.plummer(n, 17)
    x = x.to("cuda", dt).contiguous()
    m = m.to("cuda", dt).contiguous()
    G, eps = 1.3, 0.01
    ws = tg.Workspace(n, precision=precision, G=G, eps=eps)
    gen = torch.Generator().manual_seed(3)
    for call in range(2):  # two calls in a row share and reuse the scratch array
        nt = (4096, 1500)[call]
        tgt = torch.randint(0, n, (nt,), generator=gen).to("cuda")
        a0, p0 = ws.direct(x, m, tgt, precision=precision)
        a1, p1 = _noalloc(tg, x, m, tgt, precision, G, eps)
        torch.cuda.synchronize()
        ea = ((a1 - a0).norm(dim=0) / a0.norm(dim=0)).max().item()
        ep = ((p1 - p0).abs() / p0.abs()).max().item()
        assert ea <= rtol and ep <= rtol, (call, ea, ep)
        # and the FP64 oracle's direct sum of Eq. 1 on the same inputs (first 300 targets)
        t3 = tgt[:300].cpu().numpy()
        ao, po = orc.direct(x.double().cpu().numpy(), m.double().cpu().numpy(), G=G, eps=eps, targets=t3)
        a1n, p1n = a1[:, :300].cpu().numpy(), p1[:300].cpu().numpy()
        eo = (np.linalg.norm(a1n - ao, axis=0) / np.linalg.norm(ao, axis=0)).max()
        epo = (np.abs(p1n - po) / np.abs(po)).max()
        assert eo <= rtol_orc and epo <= rtol_orc, (call, eo, epo)


def test_noalloc_rejects_too_many_targets():
    tg = _lib()
    x = torch.zeros((3, 10), device="cuda")
    m = torch.ones(10, device="cuda")
    nt = tg.lib().tree_direct_forces_noalloc  # noqa: F841  (symbol present)
    tgt = torch.zeros(4097, dtype=torch.int64, device="cuda")
    out = torch.empty((3, 4097), dtype=torch.float64, device="cuda")
    code = tg.lib().tree_direct_forces_noalloc(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr()), 10, tg.F32, 1.0, 0.01,
        ctypes.c_void_p(tgt.data_ptr()), 4097, ctypes.c_void_p(out.data_ptr()), None, None)
    assert code == tg.TREE_ERR_CAPACITY


def test_noalloc_target_out_of_range_gives_nan():
    """A target index outside [0, n) reads nothing and yields NaN for that
    target only."""
    tg = _lib()
    x, _, m = inputs.plummer(500, 4)
    x = x.to("cuda", torch.float32).contiguous()
    m = m.to("cuda", torch.float32).contiguous()
    tgt = torch.tensor([-1, 500, 3, 1 << 40], dtype=torch.int64, device="cuda")
    a, phi = _noalloc(tg, x, m, tgt, "f32", 1.0, 0.01)
    torch.cuda.synchronize()
    bad = torch.tensor([True, True, False, True], device="cuda")
    assert torch.isnan(a[:, bad]).all() and torch.isnan(phi[bad]).all()
    assert torch.isfinite(a[:, 2]).all() and torch.isfinite(phi[2])
