"""Room-acoustic parameters and pressure synthesis (CUDA) against the FP64
reference of oracle/post.py, on synthetic histograms and on traced rooms."""
import math

import numpy as np
import pytest

import oracle
import scenes
from oracle import post

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402


def _same(got, ref, rtol):
    """Equal NaN / inf pattern, finite values within rtol (absolute near zero)."""
    assert np.array_equal(np.isnan(got), np.isnan(ref)) and np.array_equal(np.isinf(got), np.isinf(ref))
    m = np.isfinite(ref)
    assert np.allclose(got[m], ref[m], rtol=rtol, atol=rtol * 1e-3), np.abs(got[m] - ref[m]).max()


def test_room_parameters_synthetic():
    fs, n = 48_000.0, 96_000
    g = np.random.default_rng(1)
    H = np.zeros((3, 8, n), np.float32)
    t = np.arange(n) / fs
    for k in range(3):
        for f in range(8):
            rate = g.uniform(3, 60)
            b0 = int(g.integers(0, 3000))
            e = np.exp(-rate * (t - b0 / fs)) * (t >= b0 / fs) * g.uniform(0.5, 1.5, n)
            e[b0] += g.uniform(1, 20)                            # a direct sound
            H[k, f] = e * 1e-3
    H[2, 5] = 0.0                                                # an empty band
    H[2, 6] = 0.0
    H[2, 6, 777] = 1.0                                           # a single arrival
    got = rt.rt_room_parameters(torch.as_tensor(H, device="cuda"), fs)
    ref = post.room_parameters(H.astype(np.float64), fs)
    _same(got, ref, 1e-9)


def test_room_parameters_of_a_traced_shoebox():
    sc = scenes.shoebox(n_rays=20_000, n_bounces=60, alpha=0.2)
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    isrc = rt.rt_trace(tree, **rt.scene_args(sc))
    resp = rt.rt_rir(isrc, 8000.0, duration=1.0)
    H = resp.data
    got = rt.rt_room_parameters(H, 8000.0)
    ref = post.room_parameters(H.cpu().numpy().astype(np.float64), 8000.0)
    _same(got, ref, 1e-9)
    assert np.isfinite(got[0, :, 0]).all()                       # EDT defined in every band


@pytest.mark.parametrize("n_taps,n_out", [(1023, 24_000), (3, 4_000), (4095, 2_000)])
def test_pressure_rir_matches_reference(n_taps, n_out):
    sc = scenes.shoebox(n_rays=20_000, n_bounces=30, alpha=0.15)
    sc.rcv_center = np.concatenate([sc.rcv_center, [[3.0, 5.0, 1.2]]]).astype(np.float32)
    sc.rcv_radius = np.concatenate([sc.rcv_radius, [0.6]]).astype(np.float32)
    sc.rcv_source = np.array([0, 0], np.int32)
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    isrc = rt.rt_trace(tree, **rt.scene_args(sc))
    fs = 16_000.0
    got = rt.rt_pressure_rir(isrc, fs, n_out, n_taps).cpu().numpy().astype(np.float64)
    rcv, tim, en = (x.cpu().numpy() for x in (isrc.rcv, isrc.time, isrc.energy))
    ref = post.pressure_rir(rcv, tim, en, isrc.n_rcv, fs, n_out, n_taps)
    assert got.shape == (2, n_out) and np.abs(ref).max() > 0
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-6 * scale, np.abs(got - ref).max() / scale
    # arrivals beyond n_out + D contribute nothing; every sample is written
    assert np.isfinite(got).all()


def test_pressure_rir_rejects_bad_arguments():
    sc = scenes.shoebox(n_rays=1000, n_bounces=3)
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    isrc = rt.rt_trace(tree, **rt.scene_args(sc))
    for kw in (dict(n_taps=4), dict(n_taps=1), dict(n_out=0)):
        a = dict(n_out=100, n_taps=5)
        a.update(kw)
        with pytest.raises(rt.RtError):
            rt.rt_pressure_rir(isrc, 8000.0, a["n_out"], a["n_taps"], out=torch.empty((1, 100), device="cuda"))
