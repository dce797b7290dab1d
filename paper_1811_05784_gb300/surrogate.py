"""Learned late-reverberation tail on top of the traced early response.

A room is described by log10 volume, log10 surface area, its 8-band
area-weighted mean absorption, and - because a specular room with uneven
absorption decays at rates set by how the absorption is split between its
wall orientations - the share of its surface facing each axis, the 8-band
energy-decay rate that each axis group of walls contributes and the 8-band air
decay rate; plus the 8-band energy histogram of its first 50 ms (1 ms bins)
from a short trace, the receiver radius and how much of its bounding box the
room fills.  A 3-layer MLP (libroomrays' rt_mlp: BF16 tensor-core kernels,
FP32 accumulation, AdamW) predicts the 8-band energy decay from 50 ms to 2 s
in 10 ms bins: the energy still to arrive after each bin start
(backward-integrated, in dB), from which the tail's energy per bin follows by
differences.  It predicts the correction to a specular tail prior: the
direction mean of exp(-R(d) t) at the per-axis rates, at the diffuse level of
the measurement sphere (libroomrays' rt_tail_prior).  Rooms whose descriptors
leave the training range, or whose predicted tail does not join the traced
early response, fall back to full tracing.

Tracing, histograms, the prior and the network run in libroomrays; this
module orchestrates the calls, sums the mesh descriptors, converts between
energies and decay curves in dB and holds the normalisation statistics.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import rt

C_SOUND = 343.2
EARLY_S, EARLY_FS = 0.05, 1000.0          # 50 ms in 1 ms bins
TAIL_FS, DURATION = 100.0, 2.0            # 10 ms bins up to 2 s
N_EARLY = int(round(EARLY_S * EARLY_FS))  # 50
N_TAIL_BINS = int(round(DURATION * TAIL_FS))       # 200
FIRST_TAIL = int(round(EARLY_S * TAIL_FS))         # 5: tail starts at 50 ms
N_TAIL = N_TAIL_BINS - FIRST_TAIL                  # 195
# descriptor layout
D_BASIC = slice(0, 10)        # log10 V, log10 S, 8 area-weighted mean absorption coefficients
D_AXIS_SHARE = slice(10, 13)  # log10 of the share of S whose normal is closest to x, y, z
D_AXIS_RATE = slice(13, 37)   # log10 energy-decay rate (1/s) of each axis group, [axis][band]
D_AIR = slice(37, 45)         # air energy-decay rate c * beta (1/s) per band
D_RADIUS = 45                 # log10 of the measurement sphere's radius (m)
D_FILL = 46                   # log10 of V over the volume of the mesh's bounding box
N_DESC = 47
PROBE_BINS = np.r_[np.arange(0, 30), np.arange(30, N_TAIL, 5)]   # every bin up to 350 ms, then every 50 ms
N_PROBE = len(PROBE_BINS)                          # 63 per band
X_EARLY = slice(N_DESC, N_DESC + 8 * N_EARLY)      # 10 log10 early bins [8][50]
X_PROBE = slice(X_EARLY.stop, X_EARLY.stop + 8 * N_PROBE)   # probe minus prior, target form [8][63]
N_FEAT = X_PROBE.stop                              # 951
BASE_PROBE_BINS = 20    # the base curve follows the probe for the first 200 ms of the tail
BASIC_COLS = np.r_[np.arange(0, 10), np.arange(X_EARLY.start, X_EARLY.stop)]  # descriptors and early bins only
N_HIDDEN, N_OUT_RAW, N_OUT = 512, 8 * N_TAIL, 1568
FLOOR = 1e-30
FLOOR_IN = 1e-10        # -100 dB floor of the early-histogram features
REL_FLOOR_DB = 50.0     # the target decay is clamped this far below its start
PROBE_RAYS = 16_384     # rays of the short full-length trace that the network and the gate read


def _pad32(n: int) -> int:
    return (n + 31) // 32 * 32


N_IN = _pad32(N_FEAT)   # 960


def descriptors(scene) -> np.ndarray:
    """[log10 V, log10 S, alpha_mean[8], log10 share[3], log10 rate[3][8],
    air rate[8], log10 r, log10 (V / bounding-box volume)] of a one-receiver room.

    Each triangle is assigned to the axis its normal is closest to.  The
    decay rate of axis group k in band f is c A_k a_kf / (2 V), with A_k the
    group's area and a_kf its area-weighted -ln(1 - alpha): a ray of
    direction d loses energy at c sum_k |d_k| A_k a_k / (2 V) in a box (it
    meets the two walls normal to k every 2 V / (A_k c |d_k|) seconds), and
    the directional mean (|d_k| = 1/2) is Eyring's rate."""
    tri = scene.vertices[scene.tris]
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    area = 0.5 * np.linalg.norm(nrm, axis=1)
    S = float(area.sum())
    V = float(scene.meta["V"])
    alpha = scene.alpha[scene.material_id].astype(np.float64)
    a_mean = (area[:, None] * alpha).sum(0) / S
    loss = -np.log(np.clip(1.0 - alpha, 1e-6, 1.0))
    axis = np.argmax(np.abs(nrm), axis=1)
    share, rate = np.zeros(3), np.zeros((3, 8))
    for k in range(3):
        m = axis == k
        share[k] = area[m].sum() / S
        rate[k] = C_SOUND * (area[m, None] * loss[m]).sum(0) / (2.0 * V)
    air = C_SOUND * np.asarray(scene.beta, np.float64).reshape(8)
    ext = scene.vertices.max(0) - scene.vertices.min(0)
    fill = V / float(np.prod(ext))
    r = float(scene.rcv_radius[0])
    return np.concatenate([[math.log10(V), math.log10(S)], a_mean, np.log10(share + 1e-6),
                           np.log10(rate.reshape(-1) + 1e-6), air, [math.log10(r), math.log10(fill)]]
                          ).astype(np.float64)


PRIOR_NODES = 64


def tail_prior_edc_db(desc: np.ndarray, stream=None) -> np.ndarray:
    """Specular tail prior [n][8 * 195] in the form of tail_edc_db: libroomrays'
    rt_tail_prior with the per-axis and air rates of the descriptors and the
    diffuse level pi r^2 c dt / V (a sphere of radius r meets n / N = pi r^2 /
    (4 pi d^2) of the rays of an image source at distance d, and image sources
    at distance d arrive at 4 pi d^2 c dt / V per bin), then backward-integrated."""
    import torch
    rates = np.maximum(10.0 ** desc[:, D_AXIS_RATE] - 1e-6, 0.0).reshape(-1, 3, 8)
    air = desc[:, D_AIR]
    r = 10.0 ** desc[:, D_RADIUS]
    level = math.pi * r * r * C_SOUND / TAIL_FS / 10.0 ** desc[:, 0]
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    e = rt.rt_tail_prior(dev(rates), dev(air), dev(level), PRIOR_NODES, EARLY_S, 1.0 / TAIL_FS, N_TAIL,
                         stream=stream)
    return tail_edc_db(_np(e))


def _room(tree, sc):
    return dict(tree=tree, sources=sc.sources, rcv_center=sc.rcv_center, rcv_radius=sc.rcv_radius,
                rcv_source=sc.rcv_source, band_absorption=sc.alpha)


def trace_histograms(scene_list, n_rays, max_distance, n_bounces, fs, duration, stream=None, workspace=None,
                     trees=None):
    """Trace rooms in one batched launch and bin their responses: returns a CUDA
    tensor [n_rooms][8][bins] (one receiver per room) and the query count."""
    if trees is None:
        trees = [rt.rt_build_tree(s.vertices, s.tris, s.material_id, s.surface_id, stream=stream) for s in scene_list]
    rooms = [_room(t, s) for t, s in zip(trees, scene_list)]
    beta = scene_list[0].beta
    if any(not np.array_equal(s.beta, beta) for s in scene_list):
        raise ValueError("trace_histograms: the rooms of one batch share one air absorption")
    isrc = rt.rt_trace_batch(rooms, n_rays, n_bounces, max_distance=max_distance, air_beta=beta, c=C_SOUND,
                             tail_rays=rt.RT_TAIL_AUTOTUNE, stream=stream, workspace=workspace)
    resp = rt.rt_rir(isrc, fs, duration=duration, stream=stream)
    return resp.data.clone(), isrc.queries


def early_histograms(scene_list, n_rays=65_536, stream=None, workspace=None, trees=None):
    """0-50 ms in 1 ms bins from a short trace (rays stop after 50 ms of path)."""
    return trace_histograms(scene_list, n_rays, EARLY_S * C_SOUND, 64, EARLY_FS, EARLY_S, stream, workspace, trees)


def full_histograms(scene_list, n_rays, n_bounces=768, stream=None, workspace=None, trees=None):
    """0-2 s in 10 ms bins from a full trace (rays stop after 2 s of path)."""
    return trace_histograms(scene_list, n_rays, DURATION * C_SOUND, n_bounces, TAIL_FS, DURATION, stream,
                            workspace, trees)


def _np(x):
    return x.detach().cpu().numpy().astype(np.float64) if hasattr(x, "detach") else np.asarray(x, np.float64)


def probe_histograms(scene_list, n_rays=PROBE_RAYS, stream=None, workspace=None, trees=None):
    """The tail probe: a full-length (2 s) trace with few rays, 10 ms bins."""
    return full_histograms(scene_list, n_rays, stream=stream, workspace=workspace, trees=trees)


def features(desc: np.ndarray, early, probe_tail, prior_db: np.ndarray) -> np.ndarray:
    """Raw network input [n][951]: descriptors, 10 log10 of the early bins, and
    the probe's tail decay minus the prior's in target form (edc_to_targets)
    at PROBE_BINS."""
    n = len(desc)
    e = _np(early).reshape(n, -1)
    d = edc_to_targets(tail_edc_db(_np(probe_tail).reshape(n, 8, -1)[:, :, -N_TAIL:])) - edc_to_targets(prior_db)
    d = d.reshape(n, 8, N_TAIL)[:, :, PROBE_BINS].reshape(n, -1)
    return np.concatenate([desc, 10.0 * np.log10(e + FLOOR_IN), d], axis=1)


def base_db(probe_tail, prior_db: np.ndarray) -> np.ndarray:
    """The curve the network corrects [n][8 * 195] (tail_edc_db form): the
    probe's level and its decay over the first BASE_PROBE_BINS bins, where few
    rays already sum to a steady decay curve, then the prior's decay, joined
    without a step."""
    n = len(prior_db)
    a = edc_to_targets(tail_edc_db(_np(probe_tail).reshape(n, 8, -1)[:, :, -N_TAIL:])).reshape(n, 8, N_TAIL)
    b = edc_to_targets(prior_db).reshape(n, 8, N_TAIL)
    k = BASE_PROBE_BINS
    out = np.concatenate([a[:, :, :k], b[:, :, k:] - b[:, :, k - 1:k] + a[:, :, k - 1:k]], axis=2)
    out[:, :, 1:] = np.maximum(out[:, :, 1:], -REL_FLOOR_DB)
    return targets_to_edc_db(out.reshape(n, -1))


def loss_weights() -> np.ndarray:
    """Share of each output in the training loss [8 * 195]: the level at
    50 ms (x9) and the first 300 ms of the decay (x4), which decide the early
    decay time, weigh more than the late bins."""
    w = np.ones((8, N_TAIL))
    w[:, 0] = 9.0
    w[:, 1:30] = 4.0
    return w.reshape(-1)


def tail_edc_db(tail_energy) -> np.ndarray:
    """Energy decay of the tail [n][8 * 195]: 10 log10 of the energy arriving
    from each 10 ms bin start (50 ms ... 1.99 s) up to 2 s."""
    t = _np(tail_energy).reshape(-1, 8, N_TAIL)
    edc = np.cumsum(t[:, :, ::-1], axis=-1)[:, :, ::-1]
    return (10.0 * np.log10(edc + FLOOR)).reshape(len(t), -1)


def edc_to_targets(edc_db: np.ndarray) -> np.ndarray:
    """Network target [n][8 * 195] from a tail decay curve: per band the level
    at 50 ms, then the decay relative to it, clamped at -REL_FLOOR_DB (energy
    that far down changes no decay time, and float underflow of the traced
    energies makes it noise)."""
    d = edc_db.reshape(-1, 8, N_TAIL)
    rel = np.maximum(d - d[:, :, :1], -REL_FLOOR_DB)
    return np.concatenate([d[:, :, :1], rel[:, :, 1:]], axis=2).reshape(len(d), -1)


def targets_to_edc_db(y: np.ndarray) -> np.ndarray:
    """Inverse of edc_to_targets (up to the clamp)."""
    d = y.reshape(-1, 8, N_TAIL)
    rel = np.minimum(np.maximum(d[:, :, 1:], -REL_FLOOR_DB), 0.0)
    return np.concatenate([d[:, :, :1], d[:, :, :1] + rel], axis=2).reshape(len(d), -1)


def edc_to_energy(edc_db: np.ndarray) -> np.ndarray:
    """Per-bin tail energy [n][8][195] from a (predicted) decay curve; the
    curve is made non-increasing first."""
    e = 10.0 ** (edc_db.reshape(-1, 8, N_TAIL) / 10.0)
    e = np.minimum.accumulate(e, axis=-1)
    nxt = np.concatenate([e[:, :, 1:], np.zeros_like(e[:, :, :1])], axis=-1)
    return np.maximum(e - nxt, 0.0)


# ----------------------------------------------------------------------------
# decay metrics (ISO 3382-style, from 10 ms energy bins)
# ----------------------------------------------------------------------------
def schroeder_db(env: np.ndarray) -> np.ndarray:
    """Backward-integrated decay in dB re its start; env [..., bins]."""
    e = np.cumsum(env[..., ::-1], axis=-1)[..., ::-1]
    with np.errstate(divide="ignore", invalid="ignore"):
        return 10.0 * np.log10(e / e[..., :1])


def decay_time(env: np.ndarray, fs: float, lo_db: float, hi_db: float) -> np.ndarray:
    """60 dB decay time from a least-squares line through the Schroeder curve
    between lo_db and hi_db; NaN where the curve does not reach hi_db."""
    c = schroeder_db(env)
    t = np.arange(env.shape[-1]) / fs
    out = np.full(env.shape[:-1], np.nan)
    flat_c = c.reshape(-1, c.shape[-1])
    flat_o = out.reshape(-1)
    for k in range(flat_c.shape[0]):
        m = (flat_c[k] <= lo_db) & (flat_c[k] >= hi_db)
        if m.sum() >= 3 and flat_c[k].min() <= hi_db:
            A = np.stack([t[m], np.ones(m.sum())], 1)
            slope = np.linalg.lstsq(A, flat_c[k][m], rcond=None)[0][0]
            flat_o[k] = -60.0 / slope if slope < 0 else np.nan
    return out


def edt(env, fs=TAIL_FS):
    return decay_time(env, fs, 0.0, -10.0)


def t30(env, fs=TAIL_FS):
    return decay_time(env, fs, -5.0, -35.0)


def combine(early, tail_energy) -> np.ndarray:
    """Energy envelope [n][8][200] in 10 ms bins: traced 0-50 ms (1 ms bins
    summed by ten) followed by the predicted 50 ms - 2 s."""
    e = early.detach().cpu().numpy().astype(np.float64) if hasattr(early, "detach") else np.asarray(early)
    e10 = e.reshape(e.shape[0], 8, FIRST_TAIL, -1).sum(-1)
    return np.concatenate([e10, tail_energy.reshape(e.shape[0], 8, N_TAIL)], axis=2)


# ----------------------------------------------------------------------------
@dataclass
class Surrogate:
    """The trained tail networks (an ensemble averaged in target form) with
    their input columns, normalisation, training range and gate tolerances."""
    nets: list                  # rt.MLP members
    cols: np.ndarray            # columns of the raw features (features()) that the networks read
    x_mean: np.ndarray
    x_std: np.ndarray
    y_mean: np.ndarray
    y_std: np.ndarray
    desc_lo: np.ndarray
    desc_hi: np.ndarray
    join_db: float = 9.0        # allowed jump between traced 40-50 ms and predicted 50-60 ms
    probe_db: float = 9.0       # allowed distance between the predicted and the probe's decay
    residual: bool = True       # the networks predict the correction to the base curve
    history: list = field(default_factory=list)   # per member: (step, validation loss)

    @property
    def n_in(self) -> int:
        return _pad32(len(self.cols))

    @staticmethod
    def fit(X: np.ndarray, edc_db: np.ndarray, desc: np.ndarray, base: np.ndarray, prior: np.ndarray, cols=None,
            residual=True, n_nets=4, steps=6000, batch=1024, lr=1e-3, seed=0, stream=None, log_every=250,
            weight_decay=1e-4, input_noise=0.1, val_frac=0.05, out_weight=None):
        """Train n_nets networks on the GPU (rt_mlp) to map features X
        [n][951] (or the columns `cols` of them) to the tail decay edc_db
        [n][8 * 195]; with `residual` they learn the difference to `base`
        (base_db) in target form.  A val_frac share of the rooms is held out;
        each member keeps its weights of lowest validation loss.  Gaussian
        noise of input_noise standard deviations is added to the normalised
        inputs of every training batch; out_weight [8 * 195] scales each
        output's share of the loss (default loss_weights()).  The gate
        tolerances are then set to the 99th percentile of what the ensemble
        shows on its training rooms (`prior`: tail_prior_edc_db)."""
        import torch
        cols = np.arange(N_FEAT) if cols is None else np.asarray(cols)
        Y = edc_to_targets(edc_db)
        if residual:
            Y = Y - edc_to_targets(base)
        g = np.random.default_rng(seed)
        perm = g.permutation(len(X))
        n_val = max(1, int(val_frac * len(X)))
        vi, ti = perm[:n_val], perm[n_val:]
        Xc = X[:, cols]
        x_mean, x_std = Xc[ti].mean(0), Xc[ti].std(0) + 1e-6
        y_mean, y_std = Y[ti].mean(0), Y[ti].std(0) + 1e-6
        w = loss_weights() if out_weight is None else np.asarray(out_weight, np.float64)
        y_std = y_std / np.sqrt(w)         # a target scaled by sqrt(w) weighs w in the squared error
        n_in = _pad32(len(cols))
        s = Surrogate([], cols, x_mean, x_std, y_mean, y_std, desc[ti].min(0), desc[ti].max(0), residual=residual)
        xd = torch.tensor(s._norm_x(X[ti]), dtype=torch.float32, device="cuda")
        yd = torch.tensor(s._norm_y(Y[ti]), dtype=torch.float32, device="cuda")
        xv = torch.tensor(s._norm_x(X[vi]), dtype=torch.float32, device="cuda")
        yv = torch.tensor(s._norm_y(Y[vi]), dtype=torch.float32, device="cuda")
        noise_mask = torch.zeros(n_in, device="cuda")
        noise_mask[:len(cols)] = input_noise
        n = len(ti)
        for m in range(n_nets):
            net = rt.MLP(n_in, N_HIDDEN, N_OUT, seed=seed + m, stream=stream)
            net.set_weight_decay(weight_decay)
            gm = np.random.default_rng([seed, m])
            gen = torch.Generator(device="cuda").manual_seed(seed * 1000 + m)
            best, best_w, hist = math.inf, None, []
            for step in range(steps):
                idx = torch.as_tensor(gm.integers(0, n, batch), device="cuda")
                xb = xd[idx]
                if input_noise > 0:
                    xb = xb + torch.randn(xb.shape, device="cuda", generator=gen) * noise_mask
                lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / steps))   # cosine schedule
                net.train_step(xb, yd[idx], max(lr_t, 1e-6), stream=stream, want_loss=False)
                if (step + 1) % log_every == 0 or step == steps - 1:
                    yp = net.forward(xv, stream=stream)
                    vloss = float(((yp[:, :N_OUT_RAW] - yv[:, :N_OUT_RAW]) ** 2).mean())
                    hist.append((step + 1, vloss))
                    if vloss < best:
                        best, best_w = vloss, net.copy(0)
            if best_w is not None:
                net.copy(0, best_w, to_device=True)
            s.nets.append(net)
            s.history.append(hist)
        k = np.random.default_rng([seed, 99]).choice(ti, min(4096, len(ti)), replace=False)
        pred = s.predict_db(X[k], base[k], stream=stream)
        s.join_db = float(max(3.0, np.percentile(s.join_gap(X[k], pred), 99.0)))
        s.probe_db = float(max(3.0, np.percentile(s.probe_gap(X[k], pred, prior[k]), 99.0)))
        return s

    def join_gap(self, X: np.ndarray, pred_db: np.ndarray) -> np.ndarray:
        """Largest over bands of |predicted 50-60 ms - traced 40-50 ms| (dB)."""
        early = 10 ** (X[:, X_EARLY].reshape(len(X), 8, N_EARLY) / 10.0)
        traced = 10 * np.log10(early[:, :, 40:50].sum(-1) + FLOOR_IN)
        pred0 = 10 * np.log10(edc_to_energy(pred_db)[:, :, 0] + FLOOR_IN)
        return np.abs(pred0 - traced).max(1)

    def probe_gap(self, X: np.ndarray, pred_db: np.ndarray, prior: np.ndarray) -> np.ndarray:
        """Largest over bands of the RMS (dB, target form, at PROBE_BINS)
        between the predicted decay and the probe's."""
        n = len(X)
        pred = (edc_to_targets(pred_db) - edc_to_targets(prior)).reshape(n, 8, N_TAIL)[:, :, PROBE_BINS]
        probe = X[:, X_PROBE].reshape(n, 8, N_PROBE)
        return np.sqrt(((pred - probe) ** 2).mean(-1)).max(1)

    def _norm_x(self, X):
        Xn = (X[:, self.cols] - self.x_mean) / self.x_std
        out = np.zeros((len(X), self.n_in), np.float32)
        out[:, :len(self.cols)] = Xn
        return out

    def _norm_y(self, Y):
        Yn = (Y - self.y_mean) / self.y_std
        out = np.zeros((len(Y), N_OUT), np.float32)
        out[:, :N_OUT_RAW] = Yn
        return out

    def predict_db(self, X: np.ndarray, base: np.ndarray, stream=None) -> np.ndarray:
        """Predicted tail decay curve [n][8 * 195] in dB (see tail_edc_db):
        the members' mean correction added to `base`."""
        import torch
        xd = torch.tensor(self._norm_x(X), device="cuda")
        y = sum(net.forward(xd, stream=stream)[:, :N_OUT_RAW] for net in self.nets) / len(self.nets)
        y = y.cpu().numpy().astype(np.float64) * self.y_std + self.y_mean
        if self.residual:
            y = y + edc_to_targets(base)
        return targets_to_edc_db(y)

    def gate(self, desc: np.ndarray, X: np.ndarray, pred_db: np.ndarray, prior: np.ndarray) -> np.ndarray:
        """True where the surrogate may be used: descriptors inside the
        training range (2 % margin), the predicted 50-60 ms level within
        join_db of the traced 40-50 ms level in every band, and the predicted
        decay within probe_db of the probe's."""
        return (self.in_range(desc) & (self.join_gap(X, pred_db) <= self.join_db) &
                (self.probe_gap(X, pred_db, prior) <= self.probe_db))

    def in_range(self, desc: np.ndarray) -> np.ndarray:
        span = self.desc_hi - self.desc_lo
        return np.all((desc >= self.desc_lo - 0.02 * span) & (desc <= self.desc_hi + 0.02 * span), axis=1)

    def save(self, path):
        np.savez(path, w=np.stack([n.copy(0) for n in self.nets]), m=np.stack([n.copy(2) for n in self.nets]),
                 v=np.stack([n.copy(3) for n in self.nets]), step=np.array([n.step for n in self.nets]),
                 cols=self.cols, x_mean=self.x_mean, x_std=self.x_std, y_mean=self.y_mean, y_std=self.y_std,
                 desc_lo=self.desc_lo, desc_hi=self.desc_hi, join_db=self.join_db, probe_db=self.probe_db,
                 residual=self.residual, history=np.array(self.history, float))

    @staticmethod
    def load(path, stream=None):
        d = np.load(path)
        cols = d["cols"]
        nets = []
        for k in range(len(d["w"])):
            net = rt.MLP(_pad32(len(cols)), N_HIDDEN, N_OUT, seed=0, stream=stream)
            net.copy(0, d["w"][k], to_device=True)
            net.copy(2, d["m"][k], to_device=True)
            net.copy(3, d["v"][k], to_device=True)
            net.step = int(d["step"][k])
            nets.append(net)
        s = Surrogate(nets, cols, d["x_mean"], d["x_std"], d["y_mean"], d["y_std"], d["desc_lo"], d["desc_hi"],
                      float(d["join_db"]), float(d["probe_db"]), bool(d["residual"]))
        s.history = [[tuple(x) for x in h] for h in d["history"]]
        return s


def short_traces(scene_list, early_rays=65_536, probe_rays=PROBE_RAYS, stream=None, workspace=None, trees=None):
    """What the surrogate reads of a batch of one-receiver rooms: descriptors,
    the 0-50 ms histogram, the probe's tail energies, the prior, the base
    curve and the network input."""
    if trees is None:
        trees = [rt.rt_build_tree(r.vertices, r.tris, r.material_id, r.surface_id, stream=stream) for r in scene_list]
    desc = np.stack([descriptors(r) for r in scene_list])
    early, q1 = early_histograms(scene_list, early_rays, stream=stream, workspace=workspace, trees=trees)
    probe, q2 = probe_histograms(scene_list, probe_rays, stream=stream, workspace=workspace, trees=trees)
    early, probe = _np(early), _np(probe)[:, :, FIRST_TAIL:]
    prior = tail_prior_edc_db(desc, stream=stream)
    return dict(desc=desc, early=early, probe=probe, prior=prior, base=base_db(probe, prior),
                X=features(desc, early, probe, prior), queries=q1 + q2, trees=trees)


def respond(scene_list, sur: "Surrogate", early_rays=65_536, full_rays=1_000_000, stream=None, workspace=None):
    """Impulse-response energy envelopes [n][8][200] (10 ms bins, 0-2 s) of
    one-receiver rooms in surrogate-tail mode: traced 0-50 ms plus the
    predicted tail where the gate passes; full tracing for the others.
    Returns (envelopes, fallback mask)."""
    sh = short_traces(scene_list, early_rays, stream=stream, workspace=workspace)
    pred = sur.predict_db(sh["X"], sh["base"], stream=stream)
    ok = sur.gate(sh["desc"], sh["X"], pred, sh["prior"])
    env = combine(sh["early"], edc_to_energy(pred))
    if not ok.all():
        bad = np.nonzero(~ok)[0]
        full, _ = full_histograms([scene_list[k] for k in bad], full_rays, stream=stream, workspace=workspace,
                                  trees=[sh["trees"][k] for k in bad])
        env[bad] = _np(full)
    return env, ~ok


def extrapolated_tail_db(X: np.ndarray) -> np.ndarray:
    """The method without the network at the same cost: the traced 0-50 ms
    decay, fitted (least squares on 10 log10 energy of the 10-50 ms bins) and
    continued exponentially to 2 s.  [n][8 * 195] dB."""
    early = X[:, X_EARLY].reshape(len(X), 8, N_EARLY)
    t = (np.arange(N_EARLY) + 0.5) / EARLY_FS
    sel = slice(10, N_EARLY)
    A = np.stack([t[sel], np.ones(N_EARLY - 10)], 1)
    coef = np.einsum("ij,nbj->nbi", np.linalg.pinv(A), early[:, :, sel])
    tt = (np.arange(FIRST_TAIL, N_TAIL_BINS) + 0.5) / TAIL_FS
    slope = np.minimum(coef[..., 0], -1.0)          # never a rising tail
    db_1ms = coef[..., 1][..., None] + slope[..., None] * tt
    return (db_1ms + 10.0).reshape(len(X), -1)      # ten 1 ms bins per 10 ms bin


def eyring_tail_energy(desc: np.ndarray, X: np.ndarray) -> np.ndarray:
    """The method without the network, statistical form: an exponential tail
    at Eyring's rate c S (-ln(1 - alpha_f)) / (4 V) per band, joined to the
    traced 40-50 ms energy.  [n][8][195] energy per 10 ms bin."""
    V, Sa = 10 ** desc[:, 0], 10 ** desc[:, 1]
    a = np.clip(desc[:, 2:10], 1e-6, 0.999)
    rate = C_SOUND * Sa[:, None] * (-np.log(1 - a)) / (4 * V[:, None]) + desc[:, D_AIR]   # 1/s, energy
    early = 10 ** (X[:, X_EARLY].reshape(len(X), 8, N_EARLY) / 10.0)
    e45 = early[:, :, 40:50].sum(-1)                                             # energy in 40-50 ms
    t = (np.arange(FIRST_TAIL, N_TAIL_BINS) + 0.5) / TAIL_FS
    return e45[:, :, None] * np.exp(-rate[:, :, None] * (t[None, None, :] - 0.045))


def timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0
