"""Launch-geometry tuning of local moving: in frozen-state mode the result
must not depend on the grid caps, and the autotuner must install valid caps
that leave results unchanged."""
import numpy as np
import pytest

import oracle
from paper_2402_11454_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsp():
    from paper_2402_11454_gb300 import build
    build.build()
    from paper_2402_11454_gb300 import gsp as g
    return g


@pytest.fixture()
def restore(gsp):
    saved = gsp.get_tuning()
    yield
    gsp.set_tuning(**saved)


CAPS = [dict(groups_blocks_per_sm=1, w512_blocks_per_sm=1, block_blocks_per_sm=1, hub_blocks_per_sm=1),
        dict(groups_blocks_per_sm=16, w512_blocks_per_sm=6, block_blocks_per_sm=8, hub_blocks_per_sm=16),
        dict(groups_blocks_per_sm=3, w512_blocks_per_sm=32, block_blocks_per_sm=2, hub_blocks_per_sm=7)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_result_independent_of_caps(gsp, restore, precision):
    off, tgt, w = gsp.gen_rmat(15, 16, seed=2)  # has every degree class, hubs included
    C0, q0, st0 = gsp.louvain(off, tgt, w, precision=precision)
    for caps in CAPS:
        gsp.set_tuning(**caps)
        C, q, st = gsp.louvain(off, tgt, w, precision=precision)
        assert st["iterations"] == st0["iterations"]
        assert (C == C0).all() and q == q0


def test_autotune_installs_valid_caps(gsp, restore):
    off, tgt, w = gsp.gen_rmat(16, 16, seed=2)
    C0, q0, _ = gsp.louvain(off, tgt, w, precision="fp64")
    caps, ms_before, ms_after = gsp.autotune(off, tgt, w)
    assert caps == gsp.get_tuning()
    assert all(1 <= v <= 32 for v in caps.values())
    assert 0 < ms_after <= ms_before
    C, q, _ = gsp.louvain(off, tgt, w, precision="fp64")
    assert (C == C0).all() and q == q0


def test_autotune_rejects_edgeless_graph(gsp, restore):
    import torch
    from paper_2402_11454_gb300._lib import GspError
    off = torch.zeros(5, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(0, dtype=torch.int32, device="cuda")
    w = torch.zeros(0, dtype=torch.float32, device="cuda")
    before = gsp.get_tuning()
    with pytest.raises(GspError):
        gsp.autotune(off, tgt, w)
    assert gsp.get_tuning() == before


def test_fp64_result_with_caps_equals_oracle(gsp, restore):
    off, tgt, w = graphgen.rmat(12, 16, seed=2)
    import torch
    d = (torch.from_numpy(off.astype(np.int64)).cuda(), torch.from_numpy(tgt.astype(np.int32)).cuda(),
         torch.from_numpy(w).cuda())
    gsp.set_tuning(**CAPS[2])
    C, q, st = gsp.louvain(*d, precision="fp64")
    Co, ost = oracle.louvain(oracle.Graph(off, tgt, w.astype(np.float64)), oracle.LouvainOptions(sync=True))
    assert np.array_equal(C.cpu().numpy().astype(np.uint32), Co)
