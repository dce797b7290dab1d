"""Surrogate-tail mode through the C ABI: its inputs, prediction and gate
against the FP64 reference (oracle/surrogate.py, oracle/mlp.py,
oracle/prior.py), the fallback to full tracing, checkpoints, and the gain of
the trained networks over the method without them (the early trace joined
to the tail probe at the same cost, the specular prior alone, Eyring's
exponential)."""
import struct

import numpy as np
import pytest

import scenes
from oracle import mlp as OM
from oracle import prior as OP
from oracle import surrogate as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402
from paper_1811_05784_gb300 import surrogate as S  # noqa: E402
from paper_1811_05784_gb300.train_surrogate import errors, eyring_tail  # noqa: E402

C = S.C_SOUND


def test_checkpoint_resume_is_exact():
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(512, 64, generator=g).cuda()
    t = torch.tanh(x[:, :32] * 0.7).repeat(1, 2).cuda()
    a = rt.MLP(64, 64, 64, seed=1)
    a.set_weight_decay(1e-4)
    for k in range(20):
        a.train_step(x[k * 16:(k + 1) * 16 + 64], t[k * 16:(k + 1) * 16 + 64], lr=1e-3, want_loss=False)
    w, m, v, step = a.copy(0), a.copy(2), a.copy(3), a.step
    b = rt.MLP(64, 64, 64, seed=99)
    b.copy(0, w, to_device=True)
    b.copy(2, m, to_device=True)
    b.copy(3, v, to_device=True)
    b.step = step
    b.set_weight_decay(1e-4)
    for net in (a, b):
        net.train_step(x[:128], t[:128], lr=1e-3, want_loss=False)
    assert np.array_equal(a.copy(0), b.copy(0)) and a.step == b.step == 21


def _np(t):
    return t.cpu().numpy().astype(np.float64)


def test_inputs_match_the_reference():
    """Descriptors from the mesh, the prior, the features and the base curve
    of 24 rooms (shoeboxes and L-rooms) against the FP64 reference fed with
    the same traced histograms."""
    rooms = [scenes.surrogate_room(s) for s in range(7000, 7024)]
    d = S.inputs(rooms, rooms_per_launch=10)
    desc = _np(d["desc"])
    for k, sc in enumerate(rooms):
        ref = OS.descriptors(sc.vertices, sc.tris, sc.material_id, np.asarray(sc.alpha, np.float32), sc.meta["V"],
                             float(sc.rcv_radius[0]), np.asarray(sc.beta, np.float64), C)
        assert np.abs(desc[k] - ref).max() < 2e-6, (k, np.abs(desc[k] - ref).max())
    # prior: the descriptors' rates and level through the FP64 prior
    rates = np.maximum(10.0 ** desc[:, 13:37] - 1e-6, 0.0)
    level = np.pi * 10.0 ** (2 * desc[:, 45]) * C / 100.0 / 10.0 ** desc[:, 0]
    e = OP.tail_prior(rates.astype(np.float32).astype(np.float64), desc[:, 37:45],
                      level.astype(np.float32).astype(np.float64), 64, np.float64(np.float32(0.05)),
                      np.float64(np.float32(0.01)), 195)
    prior_ref = OS.tail_edc_db(e)
    assert np.abs(_np(d["prior_db"]) - prior_ref).max() < 2e-3
    X, base = OS.features(desc, _np(d["early"]), _np(d["probe"]), _np(d["prior_db"]))
    assert np.abs(_np(d["X"]) - X).max() < 1e-4
    assert np.abs(_np(d["base_db"]) - base).max() < 1e-4
    # the reference traces' tail curves
    env, tail_db = S.reference(rooms[:6], full_rays=65_536)
    assert np.abs(_np(tail_db) - OS.tail_edc_db(_np(env)[:, :, OS.FIRST_TAIL:])).max() < 1e-4
    assert np.allclose(_np(rt.rt_surrogate_envelope(d["early"][:6].contiguous(), d["probe"][:6].contiguous(),
                                                    False)),
                       OS.envelope(_np(d["early"][:6]), _np(d["probe"][:6]), False), rtol=1e-6, atol=1e-30)


def _parse_model(data: bytes):
    """Networks and statistics of an rt_surrogate_save buffer (layout of roomrays.h)."""
    magic = data[:8]
    n_nets, n_in, n_h, n_out, residual, n_hist = struct.unpack_from("<6i", data, 8)
    join_db, probe_db = struct.unpack_from("<2f", data, 32)
    assert magic.startswith(b"RTSUR01") and residual == 1
    o = 96
    st = np.frombuffer(data, np.float32, 2 * 951 + 2 * 1560 + 2 * 47, o).astype(np.float64)
    o += 4 * len(st) + 12 * n_hist
    stats = dict(xm=st[:951], xs=st[951:1902], ym=st[1902:3462], ys=st[3462:5022], lo=st[5022:5069],
                 hi=st[5069:5116])
    sizes = [(n_h, n_in), (n_h,), (n_h, n_h), (n_h,), (n_out, n_h), (n_out,)]
    nets = []
    for _ in range(n_nets):
        p = []
        for b, sh in enumerate(sizes):
            cnt = int(np.prod(sh))
            if b % 2 == 0:
                raw = np.frombuffer(data, np.uint16, cnt, o).astype(np.uint32) << 16
                p.append(raw.view(np.float32).astype(np.float64).reshape(sh))
                o += 2 * cnt
            else:
                p.append(np.frombuffer(data, np.float32, cnt, o).astype(np.float64))
                o += 4 * cnt
        nets.append(p)
    assert o == len(data)
    return nets, stats, join_db, probe_db


@pytest.fixture(scope="module")
def small_model():
    """4096 training rooms (targets: 65k-ray full traces), 2 members."""
    stream = torch.cuda.Stream()
    ws = rt.Workspace()
    parts = {}
    with torch.cuda.stream(stream):
        seeds = np.arange(2000, 2000 + 4096)
        for k in range(0, len(seeds), 128):
            rooms = [scenes.surrogate_room(int(s)) for s in seeds[k:k + 128]]
            d = S.inputs(rooms, stream=stream, workspace=ws)
            _, d["tail_db"] = S.reference(rooms, d["trees"], full_rays=65_536, stream=stream, workspace=ws)
            for key in ("desc", "early", "probe", "prior_db", "base_db", "X", "tail_db"):
                parts.setdefault(key, []).append(d[key])
        data = {k: torch.cat(v).contiguous() for k, v in parts.items()}
        model = S.train(data, n_nets=2, steps=1500, batch=512, stream=stream)
    torch.cuda.synchronize()
    return model, stream, ws


def test_prediction_and_gate_match_the_reference(small_model):
    """The ensemble's decay curves against the FP64 networks (BF16-rounded
    operands as the tensor cores read them) and the FP64 post-processing;
    the gate's gaps against the FP64 gate on the same curves."""
    model, stream, ws = small_model
    nets, st, join_db, probe_db = _parse_model(model.to_bytes())
    info = model.info()
    assert info["n_nets"] == 2 and 3.0 <= info["join_db"] < 60 and 3.0 <= info["probe_db"] < 60
    rooms = [scenes.surrogate_room(s) for s in range(8000, 8016)]
    with torch.cuda.stream(stream):
        d = S.inputs(rooms, stream=stream, workspace=ws)
        pred = model.predict(d["X"], d["base_db"], stream=stream)
        ok, gaps = model.gate(d["desc"], d["X"], pred, d["prior_db"], stream=stream)
    torch.cuda.synchronize()
    X = _np(d["X"])
    xn = np.zeros((len(X), 960))
    xn[:, :951] = (X - st["xm"]) / st["xs"]
    xn = xn.astype(np.float32).astype(np.float64)
    Y = [OM.forward(p, xn, bf16=True)[0] for p in nets]
    ref = OS.predict(Y, st["ym"], st["ys"], _np(d["base_db"]))
    assert np.abs(_np(pred) - ref).max() < 0.05, np.abs(_np(pred) - ref).max()
    inside, join, probe = OS.gate_gaps(_np(d["desc"]), X, _np(pred), _np(d["prior_db"]), st["lo"], st["hi"])
    assert np.allclose(gaps[:, 0], join, atol=1e-3) and np.allclose(gaps[:, 1], probe, atol=1e-3)
    clear = (np.abs(join - join_db) > 1e-3) & (np.abs(probe - probe_db) > 1e-3)
    want = inside & (join <= join_db) & (probe <= probe_db)
    assert np.array_equal(ok[clear], want[clear])


def test_fallback_outside_the_training_range_and_checkpoints(small_model, tmp_path):
    model, stream, ws = small_model
    inside = [scenes.surrogate_room(s) for s in range(5_000_000, 5_000_012)]
    outside = scenes.surrogate_room(5_000_100, v_min=400_000.0, v_max=500_000.0)   # far larger than trained
    with torch.cuda.stream(stream):
        env, fell_back = S.respond(inside + [outside], model, full_rays=131_072, stream=stream, workspace=ws)
        full, _ = S.reference([outside], full_rays=131_072, stream=stream, workspace=ws)
    torch.cuda.synchronize()
    assert fell_back[-1]
    # the fallback is the full trace itself (FP64 bin sums in each batch's own order)
    assert torch.allclose(env[-1], full[0], rtol=1e-6, atol=0)
    assert (~fell_back[:-1]).sum() >= 9                 # tolerances are the training rooms' 99th percentiles
    # a saved and reloaded model predicts the same
    path = tmp_path / "sur.rtsur"
    model.save(str(path))
    again = rt.SurrogateModel.load(str(path))
    with torch.cuda.stream(stream):
        d = S.inputs(inside[:4], stream=stream, workspace=ws)
        a = model.predict(d["X"], d["base_db"], stream=stream)
        b = again.predict(d["X"], d["base_db"], stream=stream)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert again.info()["join_db"] == model.info()["join_db"] and again.info()["n_nets"] == 2
    with pytest.raises(rt.RtError):
        rt.SurrogateModel.from_bytes(model.to_bytes()[:-4])


def test_network_beats_the_method_without_it(small_model):
    """On 64 held-out rooms judged against 262k-ray full traces the networks'
    T30 and EDT errors are below those of the early trace joined to the
    probe's own tail (same rays traced), of the prior alone and of Eyring."""
    model, stream, ws = small_model
    rooms = [scenes.surrogate_room(int(s)) for s in range(3_000_000, 3_000_064)]
    with torch.cuda.stream(stream):
        d = S.inputs(rooms, stream=stream, workspace=ws)
        ref, _ = S.reference(rooms, d["trees"], full_rays=262_144, stream=stream, workspace=ws)
        pred = model.predict(d["X"], d["base_db"], stream=stream)
        env = {"net": rt.rt_surrogate_envelope(d["early"], pred, True, stream),
               "probe": rt.rt_surrogate_envelope(d["early"], d["probe"], False, stream),
               "prior": rt.rt_surrogate_envelope(d["early"], d["prior_db"], True, stream)}
        ey = torch.tensor(eyring_tail(_np(d["desc"]), _np(d["early"])), dtype=torch.float32, device="cuda")
        env["eyring"] = rt.rt_surrogate_envelope(d["early"], ey.contiguous(), False, stream)
        ref_t = S.decay_times(ref, stream)
        mean = {k: {m: float(np.nanmean(e)) for m, e in errors(S.decay_times(v, stream), ref_t).items()}
                for k, v in env.items()}
    print("errors", mean)
    net = mean.pop("net")
    for name, w in mean.items():
        assert net["T30"] < w["T30"], (name, net, w)
    assert net["EDT"] < mean["prior"]["EDT"] and net["EDT"] < mean["eyring"]["EDT"]
    assert net["EDT"] < 1.15 * mean["probe"]["EDT"]
