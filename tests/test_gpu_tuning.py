"""Launch-geometry tuning of local moving: in frozen-state mode the result
must not depend on the grid caps or on the degree boundaries between the
kernels, and the autotuner must install valid settings that leave results
unchanged."""
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


CAPS = [dict(groups_blocks_per_sm=1, w512_blocks_per_sm=1, block_blocks_per_sm=1, hub_blocks_per_sm=1,
             persist_max_vertices=0),
        dict(groups_blocks_per_sm=16, w512_blocks_per_sm=6, block_blocks_per_sm=8, hub_blocks_per_sm=16),
        dict(groups_blocks_per_sm=3, w512_blocks_per_sm=32, block_blocks_per_sm=2, hub_blocks_per_sm=7),
        # class boundaries moved: every class hands its upper half to the next kernel
        dict(groups_blocks_per_sm=8, w512_blocks_per_sm=3, block_blocks_per_sm=4, hub_blocks_per_sm=4,
             group_max_degree=64, warp_max_degree=256, block_max_degree=1024, big_max_degree=4096),
        dict(group_max_degree=128, warp_max_degree=512, block_max_degree=2048, big_max_degree=2049)]


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
    assert all(1 <= v <= 32 for k, v in caps.items() if k.endswith("_per_sm"))
    assert 33 <= caps["group_max_degree"] < caps["warp_max_degree"] < caps["block_max_degree"] < caps["big_max_degree"]
    assert 0 < ms_after <= ms_before
    C, q, _ = gsp.louvain(off, tgt, w, precision="fp64")
    assert (C == C0).all() and q == q0


def test_autotune_batched_installs_valid_caps(gsp, restore):
    # a batch of planted graphs of mixed sizes, one of them edgeless, tuned
    # through the batched call: the settings are valid and leave every
    # graph's result unchanged
    rng = np.random.default_rng(7)
    n_g = [int(x) for x in rng.integers(64, 4096, size=48)] + [8]
    k_g = [int(rng.integers(4, 16)) for _ in n_g[:-1]] + [4]
    e_g = [n * int(rng.integers(4, 24)) // 2 for n in n_g[:-1]] + [0]
    off, tgt, w = gsp.gen_planted_batch(n_g, k_g, e_g, [0.8] * len(n_g), list(range(1, len(n_g) + 1)))
    gvo = np.concatenate([[0], np.cumsum(n_g)]).astype(np.uint64)
    C0, q0, st0 = gsp.louvain_batched(gvo, off, tgt, w, precision="fp64")
    caps, ms_before, ms_after = gsp.autotune(off, tgt, w, graph_vertex_offsets=gvo, precision="fp64")
    assert caps == gsp.get_tuning()
    assert all(1 <= v <= 32 for k, v in caps.items() if k.endswith("_per_sm"))
    assert 33 <= caps["group_max_degree"] < caps["warp_max_degree"] < caps["block_max_degree"] < caps["big_max_degree"]
    assert 0 < ms_after <= ms_before
    C, q, st = gsp.louvain_batched(gvo, off, tgt, w, precision="fp64")
    assert st["iterations"] == st0["iterations"]
    assert (C == C0).all() and (q == q0).all()


def test_autotune_batched_rejects_bad_offsets(gsp, restore):
    from paper_2402_11454_gb300._lib import GspError
    off, tgt, w = gsp.gen_planted_batch([100, 100], [4, 4], [400, 400], [0.8, 0.8], [1, 2])
    before = gsp.get_tuning()
    for gvo in ([0, 100, 150], [0, 120, 100, 200], [1, 200]):
        with pytest.raises(GspError):
            gsp.autotune(off, tgt, w, graph_vertex_offsets=np.asarray(gvo, dtype=np.uint64))
    import torch
    params = torch.zeros(gsp.mlp_param_count(), dtype=torch.float32, device="cuda")
    with pytest.raises(GspError):  # batches support flag pruning only
        gsp.autotune(off, tgt, w, graph_vertex_offsets=np.asarray([0, 100, 200], dtype=np.uint64),
                     prune="learned", mlp_params=params)
    assert gsp.get_tuning() == before


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


# mixed precision sums float32 values in shared-memory atomic order: exact for
# the planted graph's unit weights, not for the grid's weights in [1, 10)
@pytest.mark.parametrize("name,precision", [("planted", "fp64"), ("planted", "mixed"), ("grid", "fp64")])
def test_persistent_sweep_equals_per_wave_launches(gsp, restore, name, precision):
    """Graphs without hubs sweep in one cooperative launch; the per-wave
    launches must give the same result (and, in FP64, the oracle's)."""
    import torch
    if name == "planted":
        off, tgt, w = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
    else:
        off, tgt, w = graphgen.grid(60, 70, seed=3)
    d = (torch.from_numpy(off.astype(np.int64)).cuda(), torch.from_numpy(tgt.astype(np.int32)).cuda(),
         torch.from_numpy(w).cuda())
    gsp.set_tuning(persist_max_vertices=1 << 20)
    C1, q1, st1 = gsp.louvain(*d, precision=precision)
    gsp.set_tuning(persist_max_vertices=0)
    C0, q0, st0 = gsp.louvain(*d, precision=precision)
    assert st1["iterations"] == st0["iterations"]
    assert torch.equal(C0, C1) and q0 == q1
    if precision == "fp64":
        Co, _ = oracle.louvain(oracle.Graph(off, tgt, w.astype(np.float64)), oracle.LouvainOptions(sync=True))
        assert np.array_equal(C1.cpu().numpy().astype(np.uint32), Co)


def test_persistent_sweep_in_batches(gsp, restore):
    """The batched driver uses the persistent sweep on its small passes: the
    result must not change when it is disabled."""
    import torch
    voff, eoff, off, tgt, w = graphgen.batch(num_graphs=12, nmax=3000, seed=4)
    d = (torch.from_numpy(off.astype(np.int64)).cuda(), torch.from_numpy(tgt.astype(np.int32)).cuda(),
         torch.from_numpy(w).cuda())
    gsp.set_tuning(persist_max_vertices=1 << 20)
    C1, q1, _ = gsp.louvain_batched(voff, *d, precision="fp64")
    gsp.set_tuning(persist_max_vertices=0)
    C0, q0, _ = gsp.louvain_batched(voff, *d, precision="fp64")
    assert torch.equal(C0, C1) and torch.equal(q0, q1)
