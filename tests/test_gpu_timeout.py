"""Bounded device-side waits (failure detection without a GPU fault).

Every decoupled look-back of the build gives up after a limit of clock cycles.
A test injection makes one tile of one onesweep pass keep its look-back words
unpublished, so the tiles after it run into a short limit: the call must
return, report TREE_DEV_TIMEOUT, leave the tree empty (the later kernels of the
build return without work), and the next call, with the injection off, must
give exactly the results of an undisturbed workspace.  No wait is unbounded,
and every write of the disturbed pass stays in bounds (an unpublished prefix
is read as zero, so positions never exceed the true ones).
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


@pytest.mark.parametrize("sort_pass,tile", [(0, 0), (3, 5), (7, 11)])
def test_sort_lookback_timeout_reported_then_recovered(sort_pass, tile):
    tg = _tg()
    n = 50000                       # 13 sort tiles of 4096 keys per pass
    x, _, m = inputs.plummer(n, 3)
    xg, mg = x.to("cuda", torch.float32).contiguous(), m.to("cuda", torch.float32).contiguous()
    p = dict(eps=0.01, theta=0.7, order=2, leaf_cap=16, group_size=32)
    with tg.Workspace(n, **p) as ref, tg.Workspace(n, **p) as ws:
        a_ref, phi_ref = ref.accel(xg, mg)
        assert ref.status() == 0
        ws.set_waits(wait_cycles=200_000, withhold=(sort_pass, tile))
        ws.accel(xg, mg)
        st = ws.status()
        assert st & tg.DEV_TIMEOUT, st
        inf = ws.info()
        assert inf["n_nodes"] == 0 and inf["n_groups"] == 0     # nothing after the wait ran
        ws.set_waits(wait_cycles=2_000_000_000, withhold=None)
        a, phi = ws.accel(xg, mg)
        assert ws.status() == 0
        assert torch.equal(a, a_ref) and torch.equal(phi, phi_ref)


def test_withheld_last_tile_needs_no_wait():
    """Nobody waits for the last tile of a pass: withholding its words changes nothing."""
    tg = _tg()
    n = 50000
    x, _, m = inputs.plummer(n, 3)
    xg, mg = x.to("cuda", torch.float32).contiguous(), m.to("cuda", torch.float32).contiguous()
    with tg.Workspace(n) as ref, tg.Workspace(n) as ws:
        a_ref, _ = ref.accel(xg, mg)
        ws.set_waits(wait_cycles=200_000, withhold=(2, (n + 4095) // 4096 - 1))
        a, _ = ws.accel(xg, mg)
        assert ws.status() == 0
        assert torch.equal(a, a_ref)


def test_set_waits_argument_checks():
    tg = _tg()
    with tg.Workspace(100) as ws:
        for bad in (dict(wait_cycles=-1), dict(withhold=(10, 0)), dict(withhold=(0, 1 << 33))):
            with pytest.raises(tg.TreeError) as e:
                ws.set_waits(**bad)
            assert e.value.code == tg.TREE_ERR_ARG
