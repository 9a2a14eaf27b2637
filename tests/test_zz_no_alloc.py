"""gsp_modularity_static: modularity for callers that cannot allocate device
memory (graph capture, fixed memory pools).  Called through the C ABI, it must
return what gsp_modularity returns for the same inputs, on consecutive calls
(the shared scratch array keeps the previous call's contents, which each call
must clear).  Collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2402_11454_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2402_11454_gb300 import build
    build.build()
    from paper_2402_11454_gb300 import _lib
    return _lib.load()


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def _q(fn, off, tgt, w, wt, C):
    q = ctypes.c_double()
    st = fn(ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(tgt.data_ptr()), ctypes.c_void_p(w.data_ptr()), wt,
            off.numel() - 1, tgt.numel(), ctypes.c_void_p(C.data_ptr()), ctypes.byref(q), None)
    return st, q.value


@pytest.mark.parametrize("weighted", [False, True])
def test_static_modularity_matches_workspace_version(lib, weighted):
    if weighted:
        off, tgt, w = graphgen.grid(120, 150, seed=3)
        wt, wd = 1, np.float64  # float64 weights path
    else:
        off, tgt, w = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
        wt, wd = 0, np.float32
    n = len(off) - 1
    d_off, d_tgt, d_w = _dev(off, np.int64), _dev(tgt, np.int32), _dev(w, wd)
    rng = np.random.default_rng(4)
    memberships = [np.arange(n) % 64, rng.integers(0, n // 7, n)]
    for C in memberships:
        d_C = _dev(C, np.int32)
        st_ref, q_ref = _q(lib.gsp_modularity, d_off, d_tgt, d_w, wt, d_C)
        assert st_ref == 0
        for _ in range(2):  # consecutive calls share the scratch array
            st, q = _q(lib.gsp_modularity_static, d_off, d_tgt, d_w, wt, d_C)
            assert st == 0, lib.gsp_last_error()
            assert q == pytest.approx(q_ref, rel=1e-12, abs=1e-15)


def test_static_modularity_rejects_oversized_graph(lib):
    n = (1 << 20) + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(1, dtype=torch.int32, device="cuda")
    w = torch.ones(1, dtype=torch.float32, device="cuda")
    C = torch.zeros(n, dtype=torch.int32, device="cuda")
    q = ctypes.c_double()
    st = lib.gsp_modularity_static(ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(tgt.data_ptr()),
                                   ctypes.c_void_p(w.data_ptr()), 0, n, 0, ctypes.c_void_p(C.data_ptr()),
                                   ctypes.byref(q), None)
    assert st == -5
    assert b"static scratch limit" in lib.gsp_last_error()
