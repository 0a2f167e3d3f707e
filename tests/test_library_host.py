"""Host-side checks of the C-ABI library: it loads, exports every entry point
that include/treegb.h declares, and its host-only logic (the integer form of
the opening criterion, argument checks) is right.  No GPU work is issued."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "treegb.h")


@pytest.fixture(scope="module")
def tg():
    from paper_2412_01733_gb300 import build, treegb
    build.build()
    treegb.lib()
    return treegb


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:tree|leapfrog)_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(tg):
    names = _declared()
    assert "tree_build" in names and "leapfrog_step" in names and "tree_forces" in names
    L = tg.lib()
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(names) == set(tg._SIGNATURES), set(names) ^ set(tg._SIGNATURES)


def test_version_and_status_strings(tg):
    assert tg.version().startswith("treegb")
    assert tg.status_string(0) == "ok"
    assert "argument" in tg.status_string(1)


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.6, 0.7, 1.0, 1.3, 0.123456789])
def test_mac_table_matches_criterion(tg, theta):
    """d2 >= D_l  <=>  s_l^2 < fl(theta^2 d2) for every level and many d2."""
    D = tg.mac_table(theta)
    th2 = theta * theta
    rng = np.random.default_rng(1)
    for lvl in range(22):
        s2 = float((1 << (21 - lvl)) ** 2)
        if theta == 0:
            assert D[lvl] == 2 ** 63 - 1
            continue
        cand = [D[lvl] - 1, D[lvl], D[lvl] + 1, int(s2 / th2), int(s2 / th2) + 1]
        cand += [int(v) for v in rng.integers(0, 3 * 4 ** 21, 50)]
        for d2 in cand:
            if d2 < 0 or d2 >= 2 ** 53:
                continue
            assert (d2 >= D[lvl]) == (s2 < th2 * float(d2)), (lvl, d2)


def test_invalid_params_rejected_without_gpu(tg):
    for bad in (dict(eps=-1.0), dict(theta=-0.1), dict(leaf_cap=0), dict(leaf_cap=17),
                dict(group_size=48), dict(order=1), dict(stack_depth=8), dict(precision=5),
                dict(theta=float("nan"))):
        p = tg.default_params(**bad)
        h = ctypes.c_void_p()
        assert tg.lib().tree_workspace_create(100, ctypes.byref(p), ctypes.byref(h)) == tg.TREE_ERR_ARG
        assert not h.value
    p = tg.default_params()
    h = ctypes.c_void_p()
    assert tg.lib().tree_workspace_create(-1, ctypes.byref(p), ctypes.byref(h)) == tg.TREE_ERR_ARG


def test_null_workspace_rejected(tg):
    L = tg.lib()
    assert L.tree_build(None, None, 10, 0, None) == tg.TREE_ERR_ARG
    assert L.tree_forces(None, None, None, 0, None) == tg.TREE_ERR_ARG
    assert L.leapfrog_step(None, None, None, None, None, None, 0.1, 10, None) == tg.TREE_ERR_ARG


def test_defaults(tg):
    p = tg.default_params()
    assert (p.G, p.eps, p.theta, p.order, p.leaf_cap, p.group_size) == (1.0, 0.01, 0.7, 2, 16, 32)
