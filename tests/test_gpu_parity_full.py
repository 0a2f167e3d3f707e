"""Parity with the FP64 oracle at the size of the theta-sweep workload:
Plummer N = 1,048,576 (2^20), eps = 0.005, theta = 0.7, quadrupole cells,
leaf <= 16, groups of 32 -- deep enough that the sort runs hundreds of tiles
per pass, the tree reaches its full depth and the dense-cell group cut fires.

Bit-exact: sorted keys, permutation, every node array, walk groups and the
interaction lists of every group (as sets).  Floating point: FP64 moments to
rounding; FP32 forces against the oracle on the identical tree to median
relative error <= 1e-5 and max <= 1e-4 (acceleration and potential).
"""
import numpy as np
import pytest

from paper_2412_01733_gb300 import inputs
from test_gpu_parity import _check_structure, _np64, _rel_err, _run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,p", [
    ("plummer", dict(eps=0.005, theta=0.7, order=2, leaf_cap=16, group_size=32)),
    ("galaxy", dict(eps=0.02, theta=0.7, order=2, leaf_cap=16, group_size=32, group_split=0)),
], ids=["plummer_2e20", "galaxy_2e20_chunks"])
def test_fp32_parity_2e20(orc, kind, p):
    n = 1 << 20
    x, _, m = (inputs.plummer if kind == "plummer" else inputs.galaxy)(n, 20241202)
    ws, xg, mg, a, phi = _run(x, m, **p)
    assert ws.status() == 0
    ref = orc.tree_forces(_np64(xg), _np64(mg), eps=p["eps"], theta=p["theta"], lcap=p["leaf_cap"],
                          gs=p["group_size"], quad=True, delta=p.get("group_split", 3))
    inf = ws.info()
    assert inf["depth"] >= 10 and inf["n_groups"] >= n // 32
    _check_structure(orc, ws, xg, mg, ref, p["group_size"])
    e = _rel_err(_np64(a), ref.a)
    assert np.median(e) <= 1e-5, np.median(e)
    assert e.max() <= 1e-4, (e.max(), int(np.argmax(e)))
    ep = np.abs(_np64(phi) - ref.phi) / np.abs(ref.phi)
    assert np.median(ep) <= 1e-5 and ep.max() <= 1e-4, (np.median(ep), ep.max())
    sizes = np.diff(ref.gfirst)
    assert inf["pc_pairs"] == int((sizes * np.diff(ref.pc_off)).sum())
    leaf_pp = np.zeros(len(ref.pp_off) - 1, np.int64)
    np.add.at(leaf_pp, np.repeat(np.arange(len(leaf_pp)), np.diff(ref.pp_off)), ref.tree.count[ref.pp_list])
    assert inf["pp_pairs"] == int((sizes * leaf_pp).sum())
