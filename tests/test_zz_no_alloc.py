"""gsp_modularity_static: modularity for callers that cannot allocate device
memory (an embedder whose device memory belongs to a fixed pool, a process
that must not grow after start-up).  Called through the C ABI it must return
what gsp_modularity returns for the same inputs, on consecutive calls (the
shared scratch array keeps the previous call's contents, which each call
must clear), and it must allocate nothing: the library's workspace and the
device's free memory stay as they were, also when it is the first call a
fresh process makes.  Collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2402_11454_gb300 import graphgen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
        torch.cuda.synchronize()
        reserved = lib.gsp_workspace_reserved()
        for _ in range(2):  # consecutive calls share the scratch array
            st, q = _q(lib.gsp_modularity_static, d_off, d_tgt, d_w, wt, d_C)
            assert st == 0, lib.gsp_last_error()
            assert q == pytest.approx(q_ref, rel=1e-12, abs=1e-15)
        assert lib.gsp_workspace_reserved() == reserved


_FRESH = r"""
import ctypes, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2402_11454_gb300 import graphgen, _lib
off, tgt, w = graphgen.planted(n=10000, k=64, mean_degree=16, p_intra=0.8, seed=1)
d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
     (off.astype(np.int64), tgt.astype(np.int32), w, (np.arange(len(off) - 1) % 64).astype(np.int32))]
torch.cuda.synchronize()
lib = _lib.load()
def call():
    q = ctypes.c_double()
    st = lib.gsp_modularity_static(*[ctypes.c_void_p(t.data_ptr()) for t in d[:3]], 0, len(off) - 1, len(tgt),
                                   ctypes.c_void_p(d[3].data_ptr()), ctypes.byref(q), None)
    assert st == 0, lib.gsp_last_error()
    return q.value
first = call()  # the library's first call in this process (loads its kernels)
free0 = torch.cuda.mem_get_info()[0]
qs = [call(), call()]
torch.cuda.synchronize()
print(json.dumps({"q": [first] + qs, "reserved": lib.gsp_workspace_reserved(), "free_before": free0,
                  "free_after": torch.cuda.mem_get_info()[0]}))
"""


def test_static_modularity_allocates_nothing_in_a_fresh_process(lib):
    """As the first library call of a new process, and on the calls after
    it, the entry point leaves the internal workspace empty and the device's
    free memory unchanged."""
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["reserved"] == 0
    assert d["free_after"] == d["free_before"]
    assert d["q"][1] == pytest.approx(d["q"][0], rel=1e-12) and d["q"][2] == pytest.approx(d["q"][0], rel=1e-12)


def test_static_modularity_rejects_bad_ids(lib):
    off, tgt, w = graphgen.planted(n=2000, k=16, mean_degree=8, p_intra=0.8, seed=1)
    d_off, d_w = _dev(off, np.int64), _dev(w, np.float32)
    bad_tgt = tgt.astype(np.int64).copy()
    bad_tgt[5] = len(off) + 3  # a target id beyond n
    st, _ = _q(lib.gsp_modularity_static, d_off, _dev(bad_tgt, np.int32), d_w, 0,
               _dev(np.zeros(len(off) - 1), np.int32))
    assert st == -1 and b"targets out of range" in lib.gsp_last_error()
    C = np.zeros(len(off) - 1, dtype=np.int64)
    C[7] = len(off) + 1  # a membership id beyond n
    st, _ = _q(lib.gsp_modularity_static, d_off, _dev(tgt, np.int32), d_w, 0, _dev(C, np.int32))
    assert st == -1 and b"membership" in lib.gsp_last_error()


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
