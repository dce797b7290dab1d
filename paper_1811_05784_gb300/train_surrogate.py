"""Train and judge the learned late-reverberation tail.

    python -m paper_1811_05784_gb300.train_surrogate --out DIR [--train-rooms 20000] [--test-rooms 500]

1. data: seeded rooms (scenes.surrogate_room), each traced in batched
   launches: a short trace (64k rays, 50 ms, 1 ms bins) and a tail probe
   (16k rays, 2 s, 10 ms bins) for the network input, and a full trace
   (--target-rays, 2 s, 10 ms bins) for the target;
2. training on the GPU (rt_mlp: BF16 tensor-core forward / backward, AdamW),
   the network predicting the correction to the specular tail prior;
3. judging on held-out rooms against full 1M-ray traces: per-band EDT and T30
   of the surrogate response (traced 0-50 ms + predicted tail) versus the
   full trace; the same for the method without the network: the early trace
   joined to the probe's tail (same cost), the prior alone, Eyring's
   exponential and the early decay continued; rooms failing the gate fall
   back to the full trace (its cost is charged);
4. RIRs/s of the surrogate pipeline versus plain full tracing, same GPU.
Writes DIR/surrogate_report.json and the checkpoint (--model-out, default
DIR/surrogate_model.npz); the traced data set goes to --data-dir (default DIR).
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


def make_rooms(seeds):
    return [scenes.surrogate_room(int(s)) for s in seeds]


def dataset(seeds, early_rays, probe_rays, target_rays, per_batch, stream, ws, log=print):
    """descriptors [n][47], early energies [n][8][50], probe and target tail
    energies [n][8][195]."""
    desc, E, Pr, T = [], [], [], []
    queries, t0 = 0, time.perf_counter()
    for k in range(0, len(seeds), per_batch):
        rooms = make_rooms(seeds[k:k + per_batch])
        sh = S.short_traces(rooms, early_rays, probe_rays, stream=stream, workspace=ws)
        f, q = S.full_histograms(rooms, target_rays, stream=stream, workspace=ws, trees=sh["trees"])
        desc.append(sh["desc"])
        E.append(sh["early"])
        Pr.append(sh["probe"])
        T.append(S._np(f)[:, :, S.FIRST_TAIL:])
        queries += sh["queries"] + q
        if (k // per_batch) % 100 == 0:
            log(f"  rooms {k + len(rooms)}/{len(seeds)}  {time.perf_counter() - t0:.1f} s  {queries:.3e} queries")
    return (np.concatenate(desc), np.concatenate(E), np.concatenate(Pr), np.concatenate(T), queries,
            time.perf_counter() - t0)


def errors(env, ref):
    """relative EDT / T30 errors per room and band (NaN where undefined)."""
    out = {}
    for name, fn in (("EDT", S.edt), ("T30", S.t30)):
        a, b = fn(env), fn(ref)
        out[name] = np.abs(a - b) / b
    return out


def summary(err, mask=None):
    res = {}
    for name, e in err.items():
        e = e if mask is None else e[mask]
        per_band = [float(np.nanmean(e[:, f])) for f in range(8)]
        res[name] = {"mean_rel_error": float(np.nanmean(e)), "median_rel_error": float(np.nanmedian(e)),
                     "per_band_mean": per_band, "defined": int(np.isfinite(e).sum())}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train-rooms", type=int, default=20_000)
    ap.add_argument("--test-rooms", type=int, default=500)
    ap.add_argument("--early-rays", type=int, default=65_536)
    ap.add_argument("--probe-rays", type=int, default=S.PROBE_RAYS)
    ap.add_argument("--target-rays", type=int, default=131_072)
    ap.add_argument("--ref-rays", type=int, default=1_000_000)
    ap.add_argument("--per-batch", type=int, default=16)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nets", type=int, default=4, help="ensemble members")
    ap.add_argument("--reuse-data", action="store_true")
    ap.add_argument("--data-dir", default=None, help="where the traced data set is cached (default: --out)")
    ap.add_argument("--model-out", default=None, help="checkpoint path (default: DIR/surrogate_model.npz)")
    a = ap.parse_args(argv)
    import torch
    os.makedirs(a.out, exist_ok=True)
    stream = torch.cuda.Stream()
    ws = rt.Workspace()
    report = {"config": vars(a)}
    log = lambda m: print(m, flush=True)
    os.makedirs(a.data_dir or a.out, exist_ok=True)
    data_path = os.path.join(a.data_dir or a.out, "surrogate_data.npz")
    with torch.cuda.stream(stream):
        if a.reuse_data and os.path.exists(data_path):
            d = np.load(data_path)
            desc, E, Pr, T = d["desc"], d["early"], d["probe"], d["tail"]
        else:
            log(f"tracing {a.train_rooms} training rooms")
            desc, E, Pr, T, q, dt = dataset(np.arange(a.train_rooms), a.early_rays, a.probe_rays, a.target_rays,
                                            a.per_batch, stream, ws, log)
            np.savez(data_path, desc=desc, early=E, probe=Pr, tail=T)
            report["data"] = {"rooms": a.train_rooms, "queries": q, "seconds": dt}
        prior = S.tail_prior_edc_db(desc, stream=stream)
        base = S.base_db(Pr, prior)
        X, Y = S.features(desc, E, Pr, prior), S.tail_edc_db(T)
        log("training")
        t0 = time.perf_counter()
        sur = S.Surrogate.fit(X, Y, desc, base, prior, n_nets=a.nets, steps=a.steps, batch=a.batch, lr=a.lr,
                              stream=stream)
        torch.cuda.synchronize()
        report["training"] = {"seconds": time.perf_counter() - t0, "validation_loss": sur.history,
                              "join_db": sur.join_db, "probe_db": sur.probe_db}
        sur.save(a.model_out or os.path.join(a.out, "surrogate_model.npz"))
        # fit on training rooms (their 10 ms response rebuilt from the stored energies)
        k = np.random.default_rng(2).choice(len(X), min(256, len(X)), replace=False)
        ref_tr = np.concatenate([E[k].reshape(len(k), 8, S.FIRST_TAIL, -1).sum(-1), T[k]], axis=2)
        env_tr = S.combine(E[k], S.edc_to_energy(sur.predict_db(X[k], base[k], stream=stream)))
        report["training"]["fit_on_training_rooms"] = summary(errors(env_tr, ref_tr))
        f = report["training"]["fit_on_training_rooms"]
        log(f"  training rooms: T30 {f['T30']['mean_rel_error']:.4f} EDT {f['EDT']['mean_rel_error']:.4f} (mean)")

        # -- held-out rooms -----------------------------------------------------
        log(f"judging on {a.test_rooms} held-out rooms")
        seeds = np.arange(TEST_SEED0, TEST_SEED0 + a.test_rooms)
        out = {k: [] for k in ("sur", "ref", "probe", "prior", "eyring", "extra", "gate", "outside", "kind")}
        t_sur = t_plain = 0.0
        n_fallback = 0
        for k in range(0, len(seeds), a.per_batch):
            rooms = make_rooms(seeds[k:k + a.per_batch])

            def surrogate_pipeline():
                sh = S.short_traces(rooms, a.early_rays, a.probe_rays, stream=stream, workspace=ws)
                pred = sur.predict_db(sh["X"], sh["base"], stream=stream)
                return sh, pred, sur.gate(sh["desc"], sh["X"], pred, sh["prior"])

            (sh, pred, ok), dt_s = S.timed(surrogate_pipeline)

            def plain_pipeline():
                trees = [rt.rt_build_tree(r.vertices, r.tris, r.material_id, r.surface_id, stream=stream)
                         for r in rooms]
                return S.full_histograms(rooms, a.ref_rays, stream=stream, workspace=ws, trees=trees)

            (f, _), dt_p = S.timed(plain_pipeline)
            t_sur += dt_s
            t_plain += dt_p
            env = S.combine(sh["early"], S.edc_to_energy(pred))
            ref = S._np(f)
            bad = ~ok          # fallback: rooms failing the gate take the full trace (its cost is charged)
            if bad.any():
                env[bad] = ref[bad]
                n_fallback += int(bad.sum())
                t_sur += dt_p * bad.sum() / len(rooms)
            e, Xb, d = sh["early"], sh["X"], sh["desc"]
            out["sur"].append(env)
            out["ref"].append(ref)
            out["probe"].append(S.combine(e, sh["probe"]))
            out["prior"].append(S.combine(e, S.edc_to_energy(sh["prior"])))
            out["eyring"].append(S.combine(e, S.eyring_tail_energy(d, Xb)))
            out["extra"].append(S.combine(e, 10 ** (S.extrapolated_tail_db(Xb) / 10.0)))
            out["gate"].append(ok)
            out["outside"].append(~sur.in_range(d))
            out["kind"].append(np.array([r.meta["kind"] == "shoebox" for r in rooms]))
        o = {k: np.concatenate(v) for k, v in out.items()}
        ref, box = o["ref"], o["kind"]
        judged = {"rooms": int(len(ref)), "fallback_rooms": n_fallback, "outside_training_range": int(o["outside"].sum()),
                  "rirs_per_s_surrogate": len(ref) / t_sur, "rirs_per_s_plain": len(ref) / t_plain,
                  "speedup": t_plain / t_sur}
        for name in ("sur", "probe", "prior", "eyring", "extra"):
            err = errors(o[name], ref)
            judged[name] = {"all": summary(err), "shoebox": summary(err, box), "lroom": summary(err, ~box)}
        judged["sur_gated_rooms_only"] = summary(errors(o["sur"], ref), o["gate"])
        report["judged"] = judged
    path = os.path.join(a.out, "surrogate_report.json")
    with open(path, "w") as fh:
        json.dump(report, fh, indent=1)
    j = report["judged"]
    line = {"speedup": j["speedup"], "rirs_per_s_surrogate": j["rirs_per_s_surrogate"],
            "rirs_per_s_plain": j["rirs_per_s_plain"], "fallback_rooms": j["fallback_rooms"]}
    for name in ("sur", "probe", "prior", "eyring", "extra"):
        for m in ("T30", "EDT"):
            line[f"{m}_{name}"] = round(j[name]["all"][m]["mean_rel_error"], 4)
    log(json.dumps(line))
    return report


if __name__ == "__main__":
    main()
