"""rt_rir_static, the histogram step that allocates no device memory.

Some callers cannot allocate device memory while they run, for instance a
real-time auralisation loop that re-bins image sources for a moving
listener under an audio deadline.  rt_rir_static serves them from a fixed
static scratch array.  These tests call it through the C ABI and check it
against rt_rir (which allocates) on two calls in a row.  The file is
collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402

TOL_RIR = 1e-4      # relative L2, as for every histogram comparison
P = ctypes.c_void_p


def _static(isrc, n_rcv, fs, n_bins, out):
    v = isrc.view
    stream = torch.cuda.current_stream().cuda_stream
    st = rt.lib().rt_rir_static(P(v.time), P(v.rcv), P(v.energy), int(v.n), int(n_rcv), float(fs), int(n_bins),
                                P(out.data_ptr()), P(stream))
    torch.cuda.synchronize()
    return st


def _case(sc, duration):
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    isrc = rt.rt_trace(tree, **rt.scene_args(sc))
    ref = rt.rt_rir(isrc, sc.fs, duration=duration).data.clone()
    return isrc, ref


def test_static_histograms_match_rt_rir_on_two_calls():
    cases = [(scenes.theatre(n_rays=200_000), 1.0), (scenes.shoebox(n_rays=50_000, n_bounces=40), 0.5)]
    # while these calls run, any allocation through the library's allocator fails
    prepared = [(sc, dur) + _case(sc, dur) for sc, dur in cases]
    rt.rt_set_allocator(lambda nbytes, stream, ctx: None, lambda p, s, c: None)
    try:
        for sc, dur, isrc, ref in prepared:
            n_rcv = len(sc.rcv_center)
            n_bins = int(math.ceil(dur * sc.fs))
            out = torch.full((n_rcv, 8, n_bins), float("nan"), dtype=torch.float32, device="cuda")
            assert _static(isrc, n_rcv, sc.fs, n_bins, out) == rt.RT_OK, rt.rt_last_error()
            assert isrc.n > 0 and torch.isfinite(out).all()
            err = float(torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double()))
            assert err < TOL_RIR, err
    finally:
        rt.rt_set_allocator(None, None)


def test_static_histograms_reject_sizes_beyond_the_limit():
    sc = scenes.shoebox(n_rays=2000, n_bounces=5)
    isrc, _ = _case(sc, 0.2)
    v = isrc.view
    out = torch.zeros((1, 8, 100), dtype=torch.float32, device="cuda")
    st = rt.lib().rt_rir_static(P(v.time), P(v.rcv), P(v.energy), rt.RT_RIR_STATIC_MAX_SOURCES + 1, 1,
                                float(sc.fs), 100, P(out.data_ptr()), None)
    assert st == rt.RT_ERR_INVALID_ARG
    assert "static scratch limit" in rt.rt_last_error()
