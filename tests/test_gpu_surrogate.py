"""Surrogate-tail mode: checkpoint / resume of the GPU training, the gate with
its fallback to full tracing, and the gain of the trained networks over the
method without them (the early trace joined to the tail probe at the same
cost, the specular prior alone, Eyring's exponential)."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402
from paper_1811_05784_gb300 import surrogate as S  # noqa: E402
from paper_1811_05784_gb300.train_surrogate import errors  # noqa: E402

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


@pytest.fixture(scope="module")
def small_surrogate():
    """4096 training rooms (targets: 65k-ray full traces), 2 members."""
    stream = torch.cuda.Stream()
    ws = rt.Workspace()
    seeds = np.arange(2000, 2000 + 4096)
    desc, E, Pr, T = [], [], [], []
    with torch.cuda.stream(stream):
        for k in range(0, len(seeds), 32):
            rooms = [scenes.surrogate_room(int(s)) for s in seeds[k:k + 32]]
            sh = S.short_traces(rooms, stream=stream, workspace=ws)
            f, _ = S.full_histograms(rooms, 65_536, stream=stream, workspace=ws, trees=sh["trees"])
            desc.append(sh["desc"])
            E.append(sh["early"])
            Pr.append(sh["probe"])
            T.append(S._np(f)[:, :, S.FIRST_TAIL:])
        desc, E, Pr, T = (np.concatenate(x) for x in (desc, E, Pr, T))
        prior = S.tail_prior_edc_db(desc, stream=stream)
        sur = S.Surrogate.fit(S.features(desc, E, Pr, prior), S.tail_edc_db(T), desc, S.base_db(Pr, prior), prior,
                              n_nets=2, steps=1500, batch=512, stream=stream)
    return sur, stream, ws


def test_gate_falls_back_outside_the_training_range(small_surrogate, tmp_path):
    sur, stream, ws = small_surrogate
    inside = [scenes.surrogate_room(s) for s in range(5_000_000, 5_000_012)]
    outside = scenes.surrogate_room(5_000_100, v_min=400_000.0, v_max=500_000.0)   # far larger than trained
    with torch.cuda.stream(stream):
        env, fell_back = S.respond(inside + [outside], sur, full_rays=131_072, stream=stream, workspace=ws)
        full, _ = S.full_histograms([outside], 131_072, stream=stream, workspace=ws)
    assert fell_back[-1] and not sur.in_range(S.descriptors(outside)[None])[0]
    assert np.allclose(env[-1], S._np(full)[0])          # the fallback is the full trace itself
    assert (~fell_back[:-1]).sum() >= 9                   # tolerances are the training rooms' 99th percentiles
    inside = inside[int(np.argmin(fell_back[:-1]))]
    # a saved and reloaded surrogate predicts the same
    path = tmp_path / "sur.npz"
    sur.save(str(path))
    again = S.Surrogate.load(str(path), stream=stream)
    with torch.cuda.stream(stream):
        sh = S.short_traces([inside], stream=stream, workspace=ws)
        a = sur.predict_db(sh["X"], sh["base"], stream=stream)
        b = again.predict_db(sh["X"], sh["base"], stream=stream)
    assert np.array_equal(a, b) and again.join_db == sur.join_db and again.probe_db == sur.probe_db
    assert len(again.nets) == len(sur.nets) == 2


def test_network_beats_the_method_without_it(small_surrogate):
    """On 64 held-out rooms judged against 262k-ray full traces the networks'
    T30 and EDT errors are below those of the early trace joined to the
    probe's own tail (same rays traced), of the prior alone and of Eyring."""
    sur, stream, ws = small_surrogate
    rooms = [scenes.surrogate_room(int(s)) for s in range(3_000_000, 3_000_064)]
    with torch.cuda.stream(stream):
        sh, ref = [], []
        for k in range(0, 64, 32):
            sh.append(S.short_traces(rooms[k:k + 32], stream=stream, workspace=ws))
            f, _ = S.full_histograms(rooms[k:k + 32], 262_144, stream=stream, workspace=ws, trees=sh[-1]["trees"])
            ref.append(S._np(f))
        cat = lambda key: np.concatenate([x[key] for x in sh])
        X, early, probe, prior, base, desc = (cat(k) for k in ("X", "early", "probe", "prior", "base", "desc"))
        ref = np.concatenate(ref)
        pred = sur.predict_db(X, base, stream=stream)
    mean = lambda env: {m: float(np.nanmean(e)) for m, e in errors(env, ref).items()}
    net = mean(S.combine(early, S.edc_to_energy(pred)))
    without = {"probe": mean(S.combine(early, probe)), "prior": mean(S.combine(early, S.edc_to_energy(prior))),
               "eyring": mean(S.combine(early, S.eyring_tail_energy(desc, X)))}
    print("network", net, "without", without)
    for name, w in without.items():
        assert net["T30"] < w["T30"], (name, net, w)
    assert net["EDT"] < without["prior"]["EDT"] and net["EDT"] < without["eyring"]["EDT"]
    assert net["EDT"] < 1.15 * without["probe"]["EDT"]
