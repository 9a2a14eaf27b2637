"""The C ABI library loads on a machine without a GPU, exports every entry
point include/gsp.h declares, and rejects invalid arguments on the host
before any device work.  CPU only."""
import ctypes
import os
import re

import pytest

from paper_2402_11454_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    from paper_2402_11454_gb300 import _lib
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsp_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_declares_every_symbol():
    from paper_2402_11454_gb300 import _lib
    assert set(declared_symbols()) == set(_lib._SIGS)


def test_default_opts_and_strings(lib):
    from paper_2402_11454_gb300._lib import GspOpts
    o = GspOpts()
    lib.gsp_default_opts(ctypes.byref(o))
    assert (o.max_passes, o.max_iterations, o.tolerance, o.tolerance_drop,
            o.aggregation_tolerance) == (10, 20, 1e-2, 10.0, 0.8)
    assert o.split == 2 and o.split_when == 0 and o.move == 1 and o.waves == 0 and o.precision == 0
    assert o.wave_repeats == 3
    assert o.prune == 0 and o.full_sweep_every == 4 and abs(o.prune_threshold - 0.5) < 1e-7
    assert lib.gsp_status_string(-1) == b"invalid argument"
    assert lib.gsp_mlp_param_count() == 32 * 6 + 32 + 32 * 32 + 32 + 32 + 1


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2402_11454_gb300._lib import GspOpts
    # n = 0
    assert lib.gsp_louvain(None, None, None, 0, 0, None, None, None, None) == -1
    assert b"membership" in lib.gsp_last_error() or b"n must" in lib.gsp_last_error()
    o = GspOpts()
    lib.gsp_default_opts(ctypes.byref(o))
    o.max_passes = 0
    assert lib.gsp_louvain(None, None, None, 5, 0, ctypes.byref(o), None, None, None) == -1
    assert b"max_passes" in lib.gsp_last_error()
    lib.gsp_default_opts(ctypes.byref(o))
    o.split = 9
    assert lib.gsp_louvain(None, None, None, 5, 0, ctypes.byref(o), None, None, None) == -1
    assert lib.gsp_split(None, None, 0, 0, None, 3, None, None, None) == -1
    assert lib.gsp_renumber(0, None, None, None, None) == -1
    assert lib.gsp_gen_rmat(0, 16, 1, 2, 3, 0, None, None) == -1


def test_tuning_roundtrip_and_validation(lib):
    """Grid caps and class boundaries are host state: get/set work without a
    GPU and out-of-range values are rejected."""
    from paper_2402_11454_gb300._lib import GspTuning
    t = GspTuning()
    assert lib.gsp_get_tuning(ctypes.byref(t)) == 0
    assert (t.groups_blocks_per_sm, t.w512_blocks_per_sm, t.block_blocks_per_sm, t.hub_blocks_per_sm) == (8, 3, 4, 4)
    assert t.persist_max_vertices == 0
    assert (t.group_max_degree, t.warp_max_degree, t.block_max_degree, t.big_max_degree) == (128, 512, 2048, 8192)
    new = GspTuning(6, 2, 5, 8, 0, 64, 256, 2048, 4096)
    assert lib.gsp_set_tuning(ctypes.byref(new)) == 0
    got = GspTuning()
    lib.gsp_get_tuning(ctypes.byref(got))
    assert (got.groups_blocks_per_sm, got.w512_blocks_per_sm, got.block_blocks_per_sm, got.hub_blocks_per_sm,
            got.persist_max_vertices) == (6, 2, 5, 8, 0)
    assert (got.group_max_degree, got.warp_max_degree, got.block_max_degree, got.big_max_degree) == (64, 256, 2048, 4096)
    d = (128, 512, 2048, 8192)
    for bad in (GspTuning(0, 3, 4, 4, 0, *d), GspTuning(8, 33, 4, 4, 0, *d), GspTuning(8, 3, -1, 4, 0, *d),
                GspTuning(8, 3, 4, 4, 0, 256, 512, 2048, 8192),    # group table holds 128 edges at most
                GspTuning(8, 3, 4, 4, 0, 128, 1024, 2048, 8192),   # warp table: 512
                GspTuning(8, 3, 4, 4, 0, 128, 512, 512, 8192),     # boundaries must rise
                GspTuning(8, 3, 4, 4, 0, 128, 512, 2048, 16384)):  # big table: 8192
        assert lib.gsp_set_tuning(ctypes.byref(bad)) == -1
    assert lib.gsp_get_tuning(None) == -1
    assert lib.gsp_set_tuning(ctypes.byref(t)) == 0  # restore the defaults


def test_struct_layout_matches_the_header(tmp_path):
    """The ctypes mirrors of gsp_opts, gsp_stats and gsp_tuning have the
    sizes and field offsets a C compiler gives the header's structs."""
    from paper_2402_11454_gb300 import _lib
    import subprocess
    structs = {"gsp_opts": _lib.GspOpts, "gsp_stats": _lib.GspStats, "gsp_tuning": _lib.GspTuning,
               "gsp_device_graph": _lib.GspDeviceGraph}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsp.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, cls in structs.items():
        assert int(out["%s size" % cname]) == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert int(out["%s.%s" % (cname, f[0])]) == getattr(cls, f[0]).offset, (cname, f[0])


def test_new_defaults(lib):
    from paper_2402_11454_gb300._lib import GspOpts
    o = GspOpts()
    lib.gsp_default_opts(ctypes.byref(o))
    assert o.wave_repeats == 3 and o.count_disconnected == 0 and not o.workspace and o.workspace_bytes == 0
    assert lib.gsp_status_string(-6) == b"graph not symmetric"
    o.wave_repeats = 0
    assert lib.gsp_louvain(None, None, None, 5, 0, ctypes.byref(o), None, None, None) == -1
    assert b"wave_repeats" in lib.gsp_last_error()
    assert lib.gsp_workspace_reserved() >= 0


def test_batch_offsets_rejected_on_host(lib):
    """Batched calls and batched tuning check the graphs' vertex offsets (host
    array) before any device work."""
    import numpy as np
    from paper_2402_11454_gb300._lib import GspOpts, GspTuning
    o = GspOpts()
    lib.gsp_default_opts(ctypes.byref(o))
    t = GspTuning()
    for gvo, what in (([0, 4, 9], b"run from 0 to n"), ([1, 10], b"run from 0 to n"),
                      ([0, 6, 4, 10], b"must not decrease")):
        a = np.asarray(gvo, dtype=np.uint64)
        p = a.ctypes.data_as(ctypes.c_void_p)
        G = len(gvo) - 1
        assert lib.gsp_louvain_batched(G, p, None, None, None, 10, 0, ctypes.byref(o), None, None, None) == -1
        assert what in lib.gsp_last_error()
        assert lib.gsp_autotune_batched(G, p, None, None, None, 10, 0, ctypes.byref(o), ctypes.byref(t),
                                        None, None) == -1
        assert what in lib.gsp_last_error()
    assert lib.gsp_autotune_batched(0, None, None, None, None, 10, 0, None, None, None, None) == -1
