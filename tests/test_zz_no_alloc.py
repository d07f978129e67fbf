"""The allocation-free entry point hf_run_device_noalloc, for callers that
cannot allocate device memory when they run a chunk (inside a CUDA stream
capture, in a framework that owns every device allocation, in a real-time
loop).  The caller allocates the inputs and outputs beforehand; the entry
point itself allocates nothing and keeps its scratch in one static device
array.  Its results must equal those of hf_run_device, on two calls in a row
(the second call sees the first call's leftovers in the shared array), and
those of the FP64 oracle; a call allocates no device memory; a run that
overflows the array's FP64-recheck list still gives the oracle's results.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth
from synth import analyses
from tests.parity import assert_reco

pytestmark = pytest.mark.gpu


def _desc(an):
    from paper_2211_14346_gb300 import analysis_desc
    return analysis_desc(an)


def test_noalloc_matches_run_device_twice():
    import torch
    from paper_2211_14346_gb300 import build, Engine, DeviceColumns, DeviceResults, _lib, CUDA_STREAM_LEGACY
    build.build()
    lib = _lib.load()
    an = analyses.config2()
    cols = synth.gen_semilep(20000, 77)
    dc = DeviceColumns(cols)
    with Engine(0) as eng:
        aid = eng.define(an)
        ref = eng.run_device(aid, dc, V=16, seed=1002, first_event_id=5000).numpy()
    d, keep = _desc(an)
    cs = dc.struct()
    stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
    for call in range(2):
        out = DeviceResults(cols.n_events, len(an["cuts"]), an["hist"][0])
        rs = out.struct()
        st = lib.hf_run_device_noalloc(C.byref(d), C.byref(cs), cols.n_events, 5000, 1002, 16, C.byref(rs),
                                       C.c_void_p(stream))
        assert st == _lib.HF_OK, lib.hf_last_error(None)
        g = out.numpy()
        assert np.array_equal(g["cutflow"], ref["cutflow"]), (call, g["cutflow"], ref["cutflow"])
        assert np.array_equal(g["hist"], ref["hist"]), call
        assert np.array_equal(g["mask"], ref["mask"]), call
        assert np.array_equal(g["n_surv"], ref["n_surv"]), call
        assert_reco(g["reco"], ref["reco"], what="noalloc call %d" % call)


def test_noalloc_rejects_oversized_chunk():
    from paper_2211_14346_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    d, keep = _desc(analyses.config2())
    cs = _lib.hf_columns()
    st = lib.hf_run_device_noalloc(C.byref(d), C.byref(cs), (1 << 20) + 1, 0, 0, 1, None, None)
    assert st == _lib.HF_EINVAL
    assert b"HF_NOALLOC_MAX_EVENTS" in lib.hf_last_error(None)


def _noalloc(lib, an, dc, n, *, V, seed, first=0, out=None):
    import torch
    from paper_2211_14346_gb300 import DeviceResults, _lib, CUDA_STREAM_LEGACY
    d, keep = _desc(an)
    cs = dc.struct()
    if out is None:
        out = DeviceResults(n, len(an["cuts"]), an["hist"][0])
    rs = out.struct()
    stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
    st = lib.hf_run_device_noalloc(C.byref(d), C.byref(cs), n, first, seed, V, C.byref(rs), C.c_void_p(stream))
    assert st == _lib.HF_OK, lib.hf_last_error(None)
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_oracle_and_allocates_nothing(orc):
    """Two calls in a row against the oracle; after the first call (which
    looks up the array's address and loads the kernels), a call leaves the
    device's free memory unchanged."""
    import torch
    from paper_2211_14346_gb300 import build, DeviceColumns, DeviceResults, _lib
    from tests.parity import assert_parity
    build.build()
    lib = _lib.load()
    an = analyses.config2()
    cols = synth.gen_semilep(3000, 78)
    dc = DeviceColumns(cols)
    o = orc.run(an, cols, seed=1002, V=16, first_event_id=777)
    outs = [DeviceResults(cols.n_events, len(an["cuts"]), an["hist"][0]) for _ in range(3)]
    torch.cuda.synchronize()
    for call in range(3):
        free0 = torch.cuda.mem_get_info()[0]
        out = _noalloc(lib, an, dc, cols.n_events, V=16, seed=1002, first=777, out=outs[call])
        free1 = torch.cuda.mem_get_info()[0]
        if call > 0:
            assert free1 == free0, (call, free0, free1)
        assert_parity(out.numpy(), o, what="noalloc call %d" % call)


def test_noalloc_recheck_list_overflow_matches_oracle():
    """Dilepton events x 64 variations with more units to re-evaluate in FP64
    than the array's 65,536-entry recheck list holds: the units beyond it are
    evaluated inside the stage-2 kernels, and the results are still the
    oracle's (whole chunk, oracle in spawned processes)."""
    from paper_2211_14346_gb300 import build, DeviceColumns, _lib
    from tests import oracle_pool
    from tests.parity import assert_parity
    build.build()
    lib = _lib.load()
    an = analyses.config3()
    cols = synth.gen_dilep(160000, 79)
    out = _noalloc(lib, an, DeviceColumns(cols), cols.n_events, V=64, seed=1003)
    g = out.numpy()
    assert g["recheck_count"] > 65536, g["recheck_count"]
    o = oracle_pool.run(an, cols, seed=1003, V=64)
    assert_parity(g, o, model="dilep", what="noalloc recheck overflow")
