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


def _expected_launches(n, n_rcv, n_bins):
    """Kernels of one rt_rir_static call: bin keys, the radix sort's digit
    count and one scatter per 8 key bits, the FP64 bin sums."""
    if n == 0:
        return 0
    bits = max(int(n_rcv * n_bins).bit_length(), 1)
    return 3 + (bits + 7) // 8 if n > 1 else 2


def test_static_histograms_match_rt_rir_on_two_calls():
    cases = [(scenes.theatre(n_rays=200_000), 1.0), (scenes.shoebox(n_rays=50_000, n_bounces=40), 0.5)]
    prepared = [(sc, dur) + _case(sc, dur) for sc, dur in cases]
    outs = []
    for sc, dur, isrc, ref in prepared:
        n_rcv = len(sc.rcv_center)
        n_bins = int(math.ceil(dur * sc.fs))
        outs.append(torch.full((n_rcv, 8, n_bins), float("nan"), dtype=torch.float32, device="cuda"))
    # the first call on the device looks up the static array (and may load
    # the library's device code): done here, before the checked calls
    assert _static(prepared[1][2], 1, prepared[1][0].fs, 8, outs[1][:, :, :8].contiguous()) == rt.RT_OK
    torch.cuda.synchronize()
    # while the checked calls run, any allocation through the library's
    # allocator fails, device free memory must not drop, and the library
    # launches exactly the kernels of the binning step
    rt.rt_set_allocator(lambda nbytes, stream, ctx: None, lambda p, s, c: None)
    try:
        for rnd in range(2):
            launches0 = rt.rt_launch_count()
            want = 0
            for (sc, dur, isrc, ref), out in zip(prepared, outs):
                n_rcv = len(sc.rcv_center)
                n_bins = int(math.ceil(dur * sc.fs))
                out.fill_(float("nan"))
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info()[0]
                assert _static(isrc, n_rcv, sc.fs, n_bins, out) == rt.RT_OK, rt.rt_last_error()
                assert torch.cuda.mem_get_info()[0] >= free0, "device free memory dropped during the call"
                want += _expected_launches(isrc.n, n_rcv, n_bins)
                assert isrc.n > 0 and torch.isfinite(out).all()
                err = float(torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double()))
                assert err < TOL_RIR, (rnd, err)
            assert rt.rt_launch_count() - launches0 == want
    finally:
        rt.rt_set_allocator(None, None)


def test_static_histograms_through_the_binding():
    """rt.rt_rir_static with and without a caller-supplied output, and a
    wrong output rejected before any launch."""
    sc = scenes.shoebox(n_rays=20_000, n_bounces=30)
    isrc, ref = _case(sc, 0.5)
    a = rt.rt_rir_static(isrc, sc.fs, 0.5)
    out = torch.empty_like(ref)
    b = rt.rt_rir_static(isrc, sc.fs, 0.5, out=out)
    assert b is out
    for h in (a, b):
        err = float(torch.linalg.norm((h - ref).double()) / torch.linalg.norm(ref.double()))
        assert err < TOL_RIR, err
    launches0 = rt.rt_launch_count()
    for bad in (torch.empty_like(ref)[:, :, :-1], torch.empty_like(ref, dtype=torch.float64), ref.cpu(),
                torch.empty((ref.shape[2], 8, 1), device="cuda").transpose(0, 2)):
        with pytest.raises(ValueError):
            rt.rt_rir_static(isrc, sc.fs, 0.5, out=bad)
    assert rt.rt_launch_count() == launches0


def test_static_histograms_reject_sizes_beyond_the_limit():
    sc = scenes.shoebox(n_rays=2000, n_bounces=5)
    isrc, _ = _case(sc, 0.2)
    v = isrc.view
    out = torch.zeros((1, 8, 100), dtype=torch.float32, device="cuda")
    st = rt.lib().rt_rir_static(P(v.time), P(v.rcv), P(v.energy), rt.RT_RIR_STATIC_MAX_SOURCES + 1, 1,
                                float(sc.fs), 100, P(out.data_ptr()), None)
    assert st == rt.RT_ERR_INVALID_ARG
    assert "static scratch limit" in rt.rt_last_error()
