"""Train and judge the learned late-reverberation tail.

    python -m paper_1811_05784_gb300.train_surrogate --out DIR [--train-rooms 20000] [--test-rooms 500]

1. data: seeded rooms (scenes.surrogate_room), traced in batched launches by
   rt_surrogate_inputs (64k-ray 0-50 ms trace, 16k-ray 2 s tail probe,
   descriptors, prior, features, base curve) and rt_surrogate_reference
   (--target-rays full traces to 2 s: the targets);
2. training: rt_surrogate_train (BF16 tensor-core networks, AdamW);
3. judging on held-out rooms against full 1M-ray traces (rt_surrogate_reference):
   per-band EDT and T30 (rt_room_parameters on 10 ms envelopes) of the
   surrogate response (rt_rir_surrogate: traced 0-50 ms + predicted tail,
   full tracing where the gate fails; that cost is charged), and of the
   method without the network: the early trace joined to the probe's own
   tail (same rays), to the prior alone, and to Eyring's exponential;
   a defined reference value with an undefined estimate counts as a 100 %
   error (and is counted);
4. RIRs/s of the surrogate pipeline versus plain full tracing, same GPU.
Writes DIR/surrogate_report.json and the model (--model-out, default
DIR/surrogate_tail.rtsur, rt_surrogate_save format).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402

from . import rt  # noqa: E402
from . import surrogate as S  # noqa: E402

TEST_SEED0 = 1_000_000
KEYS = ("desc", "early", "probe", "prior_db", "base_db", "X")


def make_rooms(seeds):
    return [scenes.surrogate_room(int(s)) for s in seeds]


def dataset(seeds, early_rays, probe_rays, target_rays, per_batch, stream, ws, log=print):
    """Host arrays of every input of the rooms plus their target tail curves."""
    import torch
    parts = {k: [] for k in KEYS + ("tail_db",)}
    t0 = time.perf_counter()
    for k in range(0, len(seeds), per_batch):
        rooms = make_rooms(seeds[k:k + per_batch])
        d = S.inputs(rooms, early_rays=early_rays, probe_rays=probe_rays, stream=stream, workspace=ws)
        _, tail_db = S.reference(rooms, d["trees"], full_rays=target_rays, stream=stream, workspace=ws)
        for key in KEYS:
            parts[key].append(d[key].cpu().numpy())
        parts["tail_db"].append(tail_db.cpu().numpy())
        if (k // per_batch) % 50 == 0:
            log(f"  rooms {k + len(rooms)}/{len(seeds)}  {time.perf_counter() - t0:.1f} s")
    torch.cuda.synchronize()
    return {k: np.concatenate(v) for k, v in parts.items()}, time.perf_counter() - t0


def eyring_tail(desc, early):
    """Judging baseline, the method without the network in statistical form:
    an exponential tail at Eyring's rate c S (-ln(1 - alpha_f)) / (4 V) per
    band (+ air), joined to the traced 40-50 ms energy.  [n][8][195] per-bin energy."""
    V, Sa = 10 ** desc[:, 0], 10 ** desc[:, 1]
    a = np.clip(desc[:, 2:10], 1e-6, 0.999)
    rate = S.C_SOUND * Sa[:, None] * (-np.log(1 - a)) / (4 * V[:, None]) + desc[:, 37:45]
    e45 = early[:, :, 40:50].sum(-1)
    t = (np.arange(5, 200) + 0.5) / S.TAIL_FS
    return e45[:, :, None] * np.exp(-rate[:, :, None] * (t[None, None, :] - 0.045))


def errors(est, ref):
    """Relative EDT / T30 errors [n][8] of (EDT, T30) pairs; a defined
    reference with an undefined estimate is a 100 % error; an undefined
    reference leaves NaN (excluded, counted)."""
    out = {}
    for k, name in enumerate(("EDT", "T30")):
        a, b = est[k], ref[k]
        e = np.abs(a - b) / b
        e = np.where(np.isfinite(b) & ~np.isfinite(a), 1.0, e)
        out[name] = e
    return out


def summary(err, mask=None):
    res = {}
    for name, e in err.items():
        e = e if mask is None else e[mask]
        res[name] = {"mean_rel_error": float(np.nanmean(e)), "median_rel_error": float(np.nanmedian(e)),
                     "per_band_mean": [float(np.nanmean(e[:, f])) for f in range(8)],
                     "worst_band_mean": float(np.nanmax(np.nanmean(e, axis=0))),
                     "estimate_undefined": int(np.sum(e == 1.0)), "reference_undefined": int(np.isnan(e).sum())}
    return res


def judge(model, seeds, early_rays, probe_rays, ref_rays, per_batch, stream, ws, log=print):
    """Held-out rooms: surrogate vs plain full tracing (errors, RIRs/s)."""
    out = {k: [] for k in ("sur", "ref", "probe", "prior", "eyring", "fallback", "kind")}
    t_sur = t_plain = 0.0
    for k in range(0, len(seeds), per_batch):
        rooms = make_rooms(seeds[k:k + per_batch])
        (env, fb), dt_s = S.timed(lambda: S.respond(rooms, model, full_rays=ref_rays, early_rays=early_rays,
                                                    probe_rays=probe_rays, stream=stream, workspace=ws))
        (ref, _), dt_p = S.timed(lambda: S.reference(rooms, full_rays=ref_rays, stream=stream, workspace=ws))
        t_sur += dt_s
        t_plain += dt_p
        d = S.inputs(rooms, early_rays=early_rays, probe_rays=probe_rays, stream=stream, workspace=ws)
        out["sur"].append(S.decay_times(env, stream))
        out["ref"].append(S.decay_times(ref, stream))
        out["probe"].append(S.decay_times(rt.rt_surrogate_envelope(d["early"], d["probe"], False, stream), stream))
        out["prior"].append(S.decay_times(rt.rt_surrogate_envelope(d["early"], d["prior_db"], True, stream), stream))
        import torch
        ey = torch.tensor(eyring_tail(d["desc"].cpu().numpy().astype(np.float64),
                                      d["early"].cpu().numpy().astype(np.float64)), dtype=torch.float32,
                          device="cuda").contiguous()
        out["eyring"].append(S.decay_times(rt.rt_surrogate_envelope(d["early"], ey, False, stream), stream))
        out["fallback"].append(fb)
        out["kind"].append(np.array([r.meta["kind"] == "shoebox" for r in rooms]))
    cat = lambda key: tuple(np.concatenate([x[i] for x in out[key]]) for i in range(2))
    ref = cat("ref")
    box = np.concatenate(out["kind"])
    fb = np.concatenate(out["fallback"])
    judged = {"rooms": int(len(box)), "fallback_rooms": int(fb.sum()), "rirs_per_s_surrogate": len(box) / t_sur,
              "rirs_per_s_plain": len(box) / t_plain, "speedup": t_plain / t_sur}
    for name in ("sur", "probe", "prior", "eyring"):
        err = errors(cat(name), ref)
        judged[name] = {"all": summary(err), "shoebox": summary(err, box), "lroom": summary(err, ~box)}
    judged["sur_gated_rooms_only"] = summary(errors(cat("sur"), ref), ~fb)
    return judged


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train-rooms", type=int, default=20_000)
    ap.add_argument("--test-rooms", type=int, default=500)
    ap.add_argument("--early-rays", type=int, default=S.EARLY_RAYS)
    ap.add_argument("--probe-rays", type=int, default=S.PROBE_RAYS)
    ap.add_argument("--target-rays", type=int, default=262_144)
    ap.add_argument("--ref-rays", type=int, default=1_000_000)
    ap.add_argument("--per-batch", type=int, default=64)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nets", type=int, default=4, help="ensemble members")
    ap.add_argument("--data", default=None, help="cache of the traced data set (.npz; reused when present)")
    ap.add_argument("--model-out", default=None, help="model path (default: DIR/surrogate_tail.rtsur)")
    a = ap.parse_args(argv)
    import torch
    os.makedirs(a.out, exist_ok=True)
    stream = torch.cuda.Stream()
    ws = rt.Workspace()
    report = {"config": vars(a)}
    log = lambda m: print(m, flush=True)
    with torch.cuda.stream(stream):
        if a.data and os.path.exists(a.data):
            host = dict(np.load(a.data))
        else:
            log(f"tracing {a.train_rooms} training rooms")
            host, dt = dataset(np.arange(a.train_rooms), a.early_rays, a.probe_rays, a.target_rays, a.per_batch,
                               stream, ws, log)
            report["data"] = {"rooms": a.train_rooms, "seconds": dt}
            if a.data:
                np.savez(a.data, **host)
        dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous() for k, v in host.items()}
        log("training")
        model, dt = S.timed(lambda: S.train(dev, n_nets=a.nets, steps=a.steps, batch=a.batch, lr=a.lr, stream=stream))
        info = model.info()
        report["training"] = {"seconds": dt, "join_db": info["join_db"], "probe_db": info["probe_db"],
                              "validation_loss": info["history"].tolist()}
        model.save(a.model_out or os.path.join(a.out, "surrogate_tail.rtsur"))
        log(f"judging on {a.test_rooms} held-out rooms")
        report["judged"] = judge(model, np.arange(TEST_SEED0, TEST_SEED0 + a.test_rooms), a.early_rays,
                                 a.probe_rays, a.ref_rays, 16, stream, ws, log)
    with open(os.path.join(a.out, "surrogate_report.json"), "w") as fh:
        json.dump(report, fh, indent=1)
    j = report["judged"]
    line = {"speedup": j["speedup"], "rirs_per_s_surrogate": j["rirs_per_s_surrogate"],
            "rirs_per_s_plain": j["rirs_per_s_plain"], "fallback_rooms": j["fallback_rooms"],
            "join_db": info["join_db"], "probe_db": info["probe_db"]}
    for name in ("sur", "probe", "prior", "eyring"):
        for m in ("T30", "EDT"):
            line[f"{m}_{name}"] = round(j[name]["all"][m]["mean_rel_error"], 4)
            line[f"{m}_{name}_worst_band"] = round(j[name]["all"][m]["worst_band_mean"], 4)
    log(json.dumps(line))
    return report


if __name__ == "__main__":
    main()
