"""Surrogate-tail mode: orchestration of libroomrays' surrogate calls.

The learned late reverberation of a room (no counterpart in the paper): a
short 0-50 ms trace, a 2 s tail probe with few rays, the room's descriptors
and the specular tail prior feed an ensemble of BF16 tensor-core networks
that predicts the room's 8-band tail decay; rooms whose descriptors leave
the training range or whose prediction disagrees with their traces fall back
to full tracing.  Every step runs in the library (include/roomrays.h,
rt_surrogate_* and rt_rir_surrogate); this module builds trees, marshals
room lists and loops over batches of rooms.
"""
from __future__ import annotations

import time

import numpy as np

from . import rt

C_SOUND = 343.2
TAIL_FS = 100.0                  # envelope bins: 10 ms
N_ENV = rt.SUR_N_ENV             # 0-2 s
PROBE_RAYS = 16_384
EARLY_RAYS = 65_536


def build_trees(scene_list, stream=None):
    return [rt.rt_build_tree(s.vertices, s.tris, s.material_id, s.surface_id, stream=stream) for s in scene_list]


def rooms_of(scene_list, trees):
    """rt_room dicts of one-receiver rooms (receiver 0 listens to source 0)."""
    return [dict(tree=t, sources=s.sources, rcv_center=s.rcv_center, rcv_radius=s.rcv_radius,
                 rcv_source=s.rcv_source, band_absorption=s.alpha) for t, s in zip(trees, scene_list)]


def volumes(scene_list):
    return np.array([float(s.meta["V"]) for s in scene_list])


def _air(scene_list):
    beta = np.asarray(scene_list[0].beta, np.float32)
    if any(not np.array_equal(np.asarray(s.beta, np.float32), beta) for s in scene_list):
        raise ValueError("rooms of one call share one air absorption")
    return beta if np.any(beta) else None


def inputs(scene_list, trees=None, early_rays=EARLY_RAYS, probe_rays=PROBE_RAYS, stream=None, workspace=None,
           rooms_per_launch=16):
    """What the surrogate reads of the rooms (CUDA tensors: desc, early,
    probe, prior_db, base_db, X) and the trees."""
    trees = trees or build_trees(scene_list, stream)
    out = rt.rt_surrogate_inputs(rooms_of(scene_list, trees), volumes(scene_list), early_rays=early_rays,
                                 probe_rays=probe_rays, rooms_per_launch=rooms_per_launch,
                                 air_beta=_air(scene_list), c=C_SOUND, stream=stream, workspace=workspace)
    out["trees"] = trees
    return out


def reference(scene_list, trees=None, full_rays=1_000_000, stream=None, workspace=None, rooms_per_launch=16):
    """Full traces (the method itself): envelopes [n][8][200] and tail decay
    curves [n][8][195], CUDA tensors."""
    trees = trees or build_trees(scene_list, stream)
    return rt.rt_surrogate_reference(rooms_of(scene_list, trees), full_rays=full_rays,
                                     rooms_per_launch=rooms_per_launch, air_beta=_air(scene_list), c=C_SOUND,
                                     stream=stream, workspace=workspace)


def respond(scene_list, model, full_rays=1_000_000, early_rays=EARLY_RAYS, probe_rays=PROBE_RAYS, stream=None,
            workspace=None, rooms_per_launch=16, trees=None):
    """Surrogate-tail envelopes [n][8][200] (CUDA tensor, 10 ms bins) and the
    rooms that fell back to full tracing (numpy bool [n])."""
    trees = trees or build_trees(scene_list, stream)
    resp, fb = rt.rt_rir_surrogate(rooms_of(scene_list, trees), volumes(scene_list), model,
                                   early_rays=early_rays, probe_rays=probe_rays, full_rays=full_rays,
                                   rooms_per_launch=rooms_per_launch, air_beta=_air(scene_list), c=C_SOUND,
                                   stream=stream, workspace=workspace)
    return resp.data, fb


def decay_times(env, stream=None):
    """EDT and T30 (s) [n][8] of envelopes [n][8][200] (rt_room_parameters)."""
    p = rt.rt_room_parameters(env, TAIL_FS, stream=stream)
    return p[:, :, rt.ROOM_PARAMS.index("EDT")], p[:, :, rt.ROOM_PARAMS.index("T30")]


def train(data, n_nets=4, steps=6000, batch=1024, lr=1e-3, seed=0, stream=None, **kw):
    """Train on a data set (dict of CUDA tensors X, tail_db, desc, base_db,
    prior_db over the same rooms); returns an rt.SurrogateModel."""
    return rt.rt_surrogate_train(data["X"], data["tail_db"], data["desc"], data["base_db"], data["prior_db"],
                                 n_nets=n_nets, steps=steps, batch=batch, lr=lr, seed=seed, stream=stream, **kw)


def timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0
