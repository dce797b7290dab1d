"""Thin Python binding of libroomrays (include/roomrays.h), same names.

Argument marshalling only: every step of the path runs in the CUDA library.
Host inputs may be numpy arrays or CPU torch tensors (pinned or not);
device inputs are CUDA torch tensors.  Device outputs are exposed as torch
tensors that keep their owning handle alive.  There is no CPU fallback: if
the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libroomrays.so")
N_BANDS = 8

RT_OK, RT_ERR_INVALID_ARG, RT_ERR_DEGENERATE_MESH, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_CAPACITY, \
    RT_ERR_STEP_LIMIT, RT_ERR_STACK, RT_ERR_INTERNAL = range(9)
STATUS_NAMES = {0: "RT_OK", 1: "RT_ERR_INVALID_ARG", 2: "RT_ERR_DEGENERATE_MESH", 3: "RT_ERR_OOM",
                4: "RT_ERR_CUDA", 5: "RT_ERR_CAPACITY", 6: "RT_ERR_STEP_LIMIT", 7: "RT_ERR_STACK",
                8: "RT_ERR_INTERNAL"}
RT_MEM_HOST, RT_MEM_DEVICE = 0, 1

RT_TAIL_AUTOTUNE = -2

EXPORTED = ["rt_build_tree", "rt_build_tree_median", "rt_build_tree_sah", "rt_tree_free", "rt_tree_info", "rt_trace", "rt_trace_batch", "rt_image_sources_view",
            "rt_workspace_create", "rt_workspace_free", "rt_workspace_graph_launches",
            "rt_image_sources_free", "rt_rir", "rt_rir_static", "rt_response_get", "rt_response_download",
            "rt_response_free",
            "rt_last_error", "rt_api_version", "rt_launch_count", "rt_measure_l2_bandwidth", "rt_set_allocator",
            "rt_mlp_create", "rt_mlp_free", "rt_mlp_info", "rt_mlp_forward", "rt_mlp_gradients", "rt_mlp_train_step",
            "rt_mlp_copy", "rt_mlp_set_weight_decay", "rt_mlp_get_step", "rt_mlp_set_step", "rt_tail_prior",
            "rt_room_parameters", "rt_pressure_rir",
            "rt_surrogate_inputs", "rt_surrogate_reference", "rt_surrogate_train", "rt_surrogate_free",
            "rt_surrogate_info", "rt_surrogate_save", "rt_surrogate_load", "rt_surrogate_predict",
            "rt_surrogate_gate", "rt_surrogate_envelope", "rt_rir_surrogate", "rt_nearest_hits", "rt_gemm_bf16"]


class RtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


P = C.c_void_p


class rt_mesh(C.Structure):
    _fields_ = [("vertices", P), ("n_vertices", C.c_int64), ("tris", P), ("n_tris", C.c_int64),
                ("material_id", P), ("surface_id", P), ("memory", C.c_int)]


class rt_sources(C.Structure):
    _fields_ = [("pos", P), ("n", C.c_int32), ("axis", P), ("pattern", P)]


def _sources(sources, src_axis=None, src_pattern=None):
    """rt_sources over host copies (returned with it, to keep them alive).
    src_axis [S][3] unit axes and src_pattern [S] (a in [0, 1/2]) make the
    sources directional; None keeps them omnidirectional."""
    src, ps = _host(np.asarray(sources, np.float64).reshape(-1, 3), np.float64)
    keep = [src]
    pax = ppa = None
    if src_axis is not None:
        ax, pax = _host(np.asarray(src_axis, np.float64).reshape(-1, 3), np.float64)
        pat = np.zeros(len(src)) if src_pattern is None else src_pattern
        pa, ppa = _host(np.asarray(pat, np.float64).reshape(-1), np.float64)
        if len(ax) != len(src) or len(pa) != len(src):
            raise ValueError("src_axis and src_pattern need one entry per source")
        keep += [ax, pa]
    return rt_sources(ps, len(src), pax, ppa), keep


class rt_receivers(C.Structure):
    _fields_ = [("center", P), ("radius", P), ("source_of", P), ("n", C.c_int32)]


class rt_trace_params(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("ray_begin", C.c_int64), ("ray_count", C.c_int64),
                ("n_bounces", C.c_int32), ("max_distance", C.c_double), ("air_beta", P), ("c", C.c_double),
                ("block_size", C.c_int32), ("max_node_visits", C.c_int32), ("tail_rays", C.c_int32),
                ("stream", P), ("debug_t", P),
                ("debug_state", P), ("debug_cost", P), ("workspace", P), ("replay_hist", P),
                ("compaction_period", C.c_int32), ("stack_entries", C.c_int32)]


def _check_debug(debug_t, debug_state, debug_cost, n_bounces, n_traced):
    """The optional per-query outputs cover n_bounces x n_traced queries."""
    q = int(n_bounces) * int(n_traced)
    if debug_t is not None:
        _cuda(debug_t, "debug_t", "float32", min_numel=q)
    if debug_state is not None:
        _cuda(debug_state, "debug_state", "float32", min_numel=6 * q)
    if debug_cost is not None:
        _cuda(debug_cost, "debug_cost", "int32", min_numel=2 * q)


def _replay_ptr(replay):
    """Hit history of an earlier trace: an ImageSources or a CUDA int32 tensor
    [n_bounces][n_traced]."""
    if replay is None:
        return None
    if isinstance(replay, ImageSources):
        return P(replay.view.hist)
    if not (_is_cuda_tensor(replay) and str(replay.dtype) == "torch.int32" and replay.is_contiguous()):
        raise ValueError("replay: an ImageSources or a contiguous CUDA int32 tensor [n_bounces][n_traced]")
    return P(replay.data_ptr())


class rt_room(C.Structure):
    _fields_ = [("tree", P), ("sources", rt_sources), ("receivers", rt_receivers), ("band_absorption", P),
                ("n_materials", C.c_int32)]


class rt_is_view(C.Structure):
    _fields_ = [("n", C.c_int64), ("rcv", P), ("order", P), ("count", P), ("rep_ray", P), ("pos", P),
                ("dist", P), ("time", P), ("energy", P), ("n_traced", C.c_int64), ("n_bounces", C.c_int32),
                ("hist", P), ("ray_energy", P), ("ray_length", P), ("ray_hits", P), ("n_records", C.c_int64),
                ("rec_rcv", P), ("rec_ray", P), ("rec_order", P), ("rec_length", P), ("queries", C.c_int64),
                ("hash_collisions", C.c_int64), ("block_size", C.c_int32), ("tail_rays", C.c_int64),
                ("ms_rays", C.c_float), ("ms_bounces", C.c_float), ("ms_image_sources", C.c_float),
                ("n_rcv", C.c_int32), ("compaction_period", C.c_int32), ("stack_entries", C.c_int32)]


class rt_response_view(C.Structure):
    _fields_ = [("n_rcv", C.c_int32), ("n_bins", C.c_int64), ("fs", C.c_double), ("data", P)]


class rt_surrogate_trace_params(C.Structure):
    _fields_ = [("early_rays", C.c_int32), ("probe_rays", C.c_int32), ("full_rays", C.c_int32),
                ("rooms_per_launch", C.c_int32), ("air_beta", P), ("c", C.c_double), ("stream", P),
                ("workspace", P)]


class rt_surrogate_train_params(C.Structure):
    _fields_ = [("n_nets", C.c_int32), ("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float),
                ("weight_decay", C.c_float), ("input_noise", C.c_float), ("val_frac", C.c_float),
                ("log_every", C.c_int32), ("seed", C.c_uint64), ("stream", P)]


ALLOC_FN = C.CFUNCTYPE(P, C.c_size_t, P, P)
FREE_FN = C.CFUNCTYPE(None, P, P, P)

_lib = None
_lock = threading.Lock()


def lib():
    """Load libroomrays.so (built by paper_1811_05784_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libroomrays.so is not built ({LIB_PATH}); run "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            st = C.c_int
            L.rt_build_tree.restype = st
            L.rt_build_tree.argtypes = [C.POINTER(rt_mesh), P, C.POINTER(P)]
            L.rt_build_tree_median.restype = st
            L.rt_build_tree_median.argtypes = [C.POINTER(rt_mesh), P, C.POINTER(P)]
            L.rt_build_tree_sah.restype = st
            L.rt_build_tree_sah.argtypes = [C.POINTER(rt_mesh), P, C.POINTER(P)]
            L.rt_tree_free.argtypes = [P]
            L.rt_tree_info.restype = st
            L.rt_tree_info.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]
            L.rt_trace.restype = st
            L.rt_trace.argtypes = [P, C.POINTER(rt_sources), C.POINTER(rt_receivers), P, C.c_int32,
                                   C.POINTER(rt_trace_params), C.POINTER(P)]
            L.rt_trace_batch.restype = st
            L.rt_trace_batch.argtypes = [C.POINTER(rt_room), C.c_int32, C.POINTER(rt_trace_params), C.POINTER(P)]
            L.rt_workspace_create.restype = st
            L.rt_workspace_create.argtypes = [C.POINTER(P)]
            L.rt_workspace_free.argtypes = [P]
            L.rt_workspace_graph_launches.restype = C.c_int64
            L.rt_workspace_graph_launches.argtypes = [P]
            L.rt_image_sources_view.restype = st
            L.rt_image_sources_view.argtypes = [P, C.POINTER(rt_is_view)]
            L.rt_image_sources_free.argtypes = [P]
            L.rt_rir.restype = st
            L.rt_rir.argtypes = [P, C.c_double, C.c_double, P, C.POINTER(P)]
            L.rt_rir_static.restype = st
            L.rt_rir_static.argtypes = [P, P, P, C.c_int64, C.c_int32, C.c_double, C.c_int64, P, P]
            L.rt_response_get.restype = st
            L.rt_response_get.argtypes = [P, C.POINTER(rt_response_view)]
            L.rt_response_download.restype = st
            L.rt_response_download.argtypes = [P, P, P]
            L.rt_response_free.argtypes = [P]
            L.rt_last_error.restype = C.c_char_p
            L.rt_api_version.restype = C.c_int32
            L.rt_launch_count.restype = C.c_int64
            L.rt_measure_l2_bandwidth.restype = st
            L.rt_measure_l2_bandwidth.argtypes = [C.POINTER(C.c_double), P]
            L.rt_mlp_create.restype = st
            L.rt_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, C.POINTER(P)]
            L.rt_mlp_free.argtypes = [P]
            L.rt_mlp_info.restype = st
            L.rt_mlp_info.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int64), P]
            L.rt_mlp_forward.restype = st
            L.rt_mlp_forward.argtypes = [P, P, C.c_int32, P, P]
            L.rt_mlp_gradients.restype = st
            L.rt_mlp_gradients.argtypes = [P, P, P, C.c_int32, C.POINTER(C.c_float), P]
            L.rt_mlp_train_step.restype = st
            L.rt_mlp_train_step.argtypes = [P, P, P, C.c_int32, C.c_float, C.POINTER(C.c_float), P]
            L.rt_mlp_copy.restype = st
            L.rt_mlp_copy.argtypes = [P, C.c_int32, P, C.c_int32, P]
            L.rt_mlp_set_weight_decay.restype = st
            L.rt_mlp_set_weight_decay.argtypes = [P, C.c_float]
            L.rt_mlp_get_step.restype = st
            L.rt_mlp_get_step.argtypes = [P, C.POINTER(C.c_int64)]
            L.rt_mlp_set_step.restype = st
            L.rt_mlp_set_step.argtypes = [P, C.c_int64]
            L.rt_room_parameters.restype = st
            L.rt_room_parameters.argtypes = [P, C.c_int32, C.c_int64, C.c_double, P, P]
            L.rt_pressure_rir.restype = st
            L.rt_pressure_rir.argtypes = [P, C.c_double, C.c_int64, C.c_int32, P, P]
            L.rt_tail_prior.restype = st
            L.rt_tail_prior.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_int32, P, P]
            for name, args in (
                    ("rt_surrogate_inputs", [P, P, C.c_int32, C.POINTER(rt_surrogate_trace_params), P, P, P, P, P, P]),
                    ("rt_surrogate_reference", [P, C.c_int32, C.POINTER(rt_surrogate_trace_params), P, P]),
                    ("rt_surrogate_train", [P, P, P, P, P, C.c_int32, C.POINTER(rt_surrogate_train_params),
                                            C.POINTER(P)]),
                    ("rt_surrogate_info", [P, C.POINTER(C.c_int32), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                           C.POINTER(C.c_int32), P]),
                    ("rt_surrogate_save", [P, P, C.c_size_t, C.POINTER(C.c_size_t)]),
                    ("rt_surrogate_load", [P, C.c_size_t, P, C.POINTER(P)]),
                    ("rt_surrogate_predict", [P, P, P, C.c_int32, P, P]),
                    ("rt_surrogate_gate", [P, P, P, P, P, C.c_int32, P, P, P]),
                    ("rt_surrogate_envelope", [P, P, C.c_int32, C.c_int32, P, P]),
                    ("rt_rir_surrogate", [P, P, C.c_int32, P, C.POINTER(rt_surrogate_trace_params), C.POINTER(P),
                                          P])):
                getattr(L, name).restype = st
                getattr(L, name).argtypes = args
            L.rt_surrogate_free.argtypes = [P]
            L.rt_gemm_bf16.restype = st
            L.rt_gemm_bf16.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, P, C.c_int32, P, C.c_int64,
                                       C.POINTER(C.c_float), P]
            L.rt_nearest_hits.restype = st
            L.rt_nearest_hits.argtypes = [P, P, P, P, C.c_int64, C.c_int32, P, P, P, P]
            L.rt_set_allocator.restype = st
            L.rt_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
            _lib = L
    return _lib


def rt_last_error() -> str:
    return lib().rt_last_error().decode()


def rt_api_version() -> int:
    return int(lib().rt_api_version())


def rt_launch_count() -> int:
    """Kernel launches made by libroomrays in this process."""
    return int(lib().rt_launch_count())


def rt_measure_l2_bandwidth(stream=None) -> float:
    """L2 read bandwidth (GB/s) measured by the library's probe kernel."""
    v = C.c_double()
    _check(lib().rt_measure_l2_bandwidth(C.byref(v), _stream_ptr(stream)))
    return v.value


ROOM_PARAMS = ("EDT", "T20", "T30", "C80", "D50", "Ts", "SPL")


def rt_room_parameters(H, fs, stream=None):
    """Room-acoustic parameters [n_rcv][8][7] (numpy, ROOM_PARAMS order) of
    CUDA histograms H [n_rcv][8][n_bins] (e.g. Response.data)."""
    if not _is_cuda_tensor(H):
        raise ValueError("rt_room_parameters: H must be a CUDA tensor")
    H = H.contiguous().float()
    R, nb = int(H.shape[0]), int(H.shape[-1])
    if H.dim() != 3 or H.shape[1] != N_BANDS:
        raise ValueError("rt_room_parameters: histograms [n_rcv][8][n_bins]")
    out = np.zeros((R, N_BANDS, len(ROOM_PARAMS)), np.float64)
    _check(lib().rt_room_parameters(P(H.data_ptr()), R, nb, float(fs), out.ctypes.data_as(P), _stream_ptr(stream)))
    return out


def rt_pressure_rir(image_sources, fs, n_out, n_taps=4095, out=None, stream=None):
    """Pressure responses [n_rcv][n_out] (CUDA float tensor) of image sources,
    synthesised with octave-band FIR filters of n_taps (odd) taps."""
    import torch
    R = image_sources.n_rcv
    if out is None:
        out = torch.empty((R, int(n_out)), dtype=torch.float32, device="cuda")
    if int(n_out) >= 1:  # the library reports invalid sizes itself
        _cuda(out, "rt_pressure_rir: out", "float32", (R, int(n_out)))
    _check(lib().rt_pressure_rir(image_sources._h, float(fs), int(n_out), int(n_taps), P(out.data_ptr()),
                                 _stream_ptr(stream)))
    return out


def rt_tail_prior(rates, air, level, n_nodes, t0, dt, n_bins, out=None, stream=None):
    """Direction-integrated specular tail [n][8][n_bins] (CUDA float tensor)
    from per-axis decay rates [n][3][8], air rates [n][8] and levels [n]
    (CUDA tensors), with an n_nodes x n_nodes Gauss-Legendre direction rule."""
    import torch
    if not all(_is_cuda_tensor(x) for x in (rates, air, level)):
        raise ValueError("rt_tail_prior: rates, air and level must be CUDA tensors")
    rates, air, level = (x.contiguous().float() for x in (rates, air, level))
    n = rates.shape[0]
    if rates.shape != (n, 3, N_BANDS) or air.shape != (n, N_BANDS) or level.shape != (n,):
        raise ValueError("rt_tail_prior: rates [n][3][8], air [n][8], level [n]")
    if out is None:
        out = torch.empty((n, N_BANDS, int(n_bins)), dtype=torch.float32, device=rates.device)
    if int(n_bins) >= 1 and n >= 1:  # the library reports invalid sizes itself
        _cuda(out, "rt_tail_prior: out", "float32", (n, N_BANDS, int(n_bins)))
    _check(lib().rt_tail_prior(P(rates.data_ptr()), P(air.data_ptr()), P(level.data_ptr()), int(n), int(n_nodes),
                               float(t0), float(dt), int(n_bins), P(out.data_ptr()), _stream_ptr(stream)))
    return out


def _check(status):
    if status != RT_OK:
        raise RtError(status, rt_last_error())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return P(stream)
    return P(stream.cuda_stream)


def _is_cuda_tensor(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _cuda(t, name, dtype=None, shape=None, min_numel=None):
    """t itself if it is a contiguous CUDA tensor of the given dtype (a torch
    dtype name such as "float32"), shape and at least min_numel elements;
    ValueError otherwise, before anything is launched: a device pointer the
    library reads or writes must cover what it touches."""
    ok = _is_cuda_tensor(t) and t.is_contiguous()
    if ok and dtype is not None:
        ok = str(t.dtype) == "torch." + dtype
    if ok and shape is not None:
        ok = tuple(t.shape) == tuple(int(x) for x in shape)
    if ok and min_numel is not None:
        ok = t.numel() >= int(min_numel)
    if not ok:
        want = "a contiguous CUDA " + (dtype or "") + " tensor"
        if shape is not None:
            want += f" of shape {tuple(int(x) for x in shape)}"
        if min_numel is not None:
            want += f" of at least {int(min_numel)} elements"
        raise ValueError(f"{name}: {want}")
    return t


def _host(x, dtype):
    """Host array view (numpy, or CPU torch tensor such as pinned memory)."""
    if hasattr(x, "is_cuda"):
        t = x.contiguous()
        assert str(t.dtype).replace("torch.", "") == np.dtype(dtype).name, (t.dtype, dtype)
        return t, P(t.data_ptr())
    a = np.ascontiguousarray(x, dtype=dtype)
    return a, P(a.ctypes.data)


def _device_tensor(ptr, shape, dtype, owner):
    import torch
    n = int(np.prod(shape)) if len(shape) else 1
    if n == 0 or not ptr:
        return torch.empty(shape, dtype=dtype, device="cuda")

    class _CAI:
        pass

    typestr = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4", torch.int64: "<i8"}[dtype]
    h = _CAI()
    h.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                  "data": (int(ptr), False), "version": 3, "strides": None, "stream": None}
    h._owner = owner
    return torch.as_tensor(h, device="cuda")


# ----------------------------------------------------------------------------
class Tree:
    """rt_tree handle (LBVH of a mesh)."""

    def __init__(self, handle):
        self._h = handle

    def info(self):
        nn, nt = C.c_int64(), C.c_int64()
        dp, ns = C.c_int32(), C.c_int32()
        _check(lib().rt_tree_info(self._h, C.byref(nn), C.byref(nt), C.byref(dp), C.byref(ns)))
        return {"n_nodes": nn.value, "n_tris": nt.value, "depth": dp.value, "n_surfaces": ns.value}

    def free(self):
        if self._h:
            lib().rt_tree_free(self._h)
            self._h = None

    __del__ = free


def rt_build_tree(vertices, tris, material_id, surface_id=None, stream=None, median=False, sah=False) -> Tree:
    """Build the LBVH of a triangle mesh (host numpy / CPU tensors or CUDA
    tensors); median=True builds the paper's median-split tree instead
    (rt_build_tree_median), sah=True the LBVH with SAH top levels
    (rt_build_tree_sah)."""
    if median and sah:
        raise ValueError("rt_build_tree: median and sah exclude each other")
    dev = _is_cuda_tensor(vertices)
    keep = []
    if dev:
        import torch
        v = vertices.contiguous().to(torch.float64)
        t = tris.contiguous().to(torch.int32)
        m = material_id.contiguous().to(torch.int32)
        s = None if surface_id is None else surface_id.contiguous().to(torch.int32)
        keep += [v, t, m, s]
        mesh = rt_mesh(P(v.data_ptr()), v.shape[0], P(t.data_ptr()), t.shape[0], P(m.data_ptr()),
                       P(s.data_ptr()) if s is not None else None, RT_MEM_DEVICE)
    else:
        v, pv = _host(vertices, np.float64)
        t, pt = _host(tris, np.int32)
        m, pm = _host(material_id, np.int32)
        if surface_id is not None:
            s, ps = _host(surface_id, np.int32)
        else:
            s, ps = None, None
        keep += [v, t, m, s]
        mesh = rt_mesh(pv, len(v), pt, len(t), pm, ps, RT_MEM_HOST)
    out = P()
    fn = lib().rt_build_tree_median if median else (lib().rt_build_tree_sah if sah else lib().rt_build_tree)
    _check(fn(C.byref(mesh), _stream_ptr(stream), C.byref(out)))
    return Tree(out)


RT_GEMM_TMA, RT_GEMM_STAGED = 0, 1


def rt_gemm_bf16(A, B, kernel=RT_GEMM_TMA, out=None, stream=None, workspace=None, timed=False):
    """C = A B^T (CUDA bfloat16 A [M][K], B [N][K]) -> CUDA float32 [M][N].
    workspace: CUDA float32 tensor for the partial sums of a product cut
    along K (None: not cut).  timed=True returns (C, device ms of the
    product's kernels)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or B.shape[1] != K:
        raise ValueError("rt_gemm_bf16: bfloat16 A [M][K] and B [N][K]")
    if not (_is_cuda_tensor(A) and _is_cuda_tensor(B)):
        raise ValueError("rt_gemm_bf16: A and B must be CUDA tensors")
    if workspace is not None and (workspace.dtype != torch.float32 or not workspace.is_contiguous()):
        raise ValueError("rt_gemm_bf16: the workspace is a contiguous float32 tensor")
    A, B = A.contiguous(), B.contiguous()
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _cuda(out, "rt_gemm_bf16: out", "float32", (M, N))
    if workspace is not None:
        _cuda(workspace, "rt_gemm_bf16: workspace", "float32")
    ms = C.c_float(0.0)
    _check(lib().rt_gemm_bf16(P(A.data_ptr()), P(B.data_ptr()), int(M), int(N), int(K), P(out.data_ptr()),
                              int(kernel), P(workspace.data_ptr()) if workspace is not None else None,
                              int(workspace.numel()) if workspace is not None else 0,
                              C.byref(ms) if timed else None, _stream_ptr(stream)))
    return (out, ms.value) if timed else out


RT_NEAREST_STACK, RT_NEAREST_LEVELS = 0, 1


def rt_nearest_hits(tree: Tree, origins, directions, exclude_surface=None, method=RT_NEAREST_STACK, stream=None):
    """Nearest triangles of n rays (CUDA float32 [n][3] origins and
    directions, optional CUDA int32 [n] surface to skip): (hit int32 [n],
    t float32 [n], (node visits, triangle tests)); method RT_NEAREST_STACK
    (per-ray stack traversal) or RT_NEAREST_LEVELS (the paper's level-by-level
    distribution of rays through the tree)."""
    import torch
    n = int(origins.shape[0])
    for x, name in ((origins, "origins"), (directions, "directions")):
        if not (_is_cuda_tensor(x) and x.dtype == torch.float32 and x.is_contiguous() and tuple(x.shape) == (n, 3)):
            raise ValueError(f"rt_nearest_hits: {name} must be a contiguous CUDA float32 tensor [n][3]")
    if exclude_surface is not None and not (_is_cuda_tensor(exclude_surface) and exclude_surface.dtype == torch.int32
                                            and exclude_surface.is_contiguous() and exclude_surface.numel() == n):
        raise ValueError("rt_nearest_hits: exclude_surface must be a contiguous CUDA int32 tensor [n]")
    hit = torch.empty(n, dtype=torch.int32, device=origins.device)
    t = torch.empty(n, dtype=torch.float32, device=origins.device)
    stats = np.zeros(2, np.int64)
    _check(lib().rt_nearest_hits(tree._h, P(origins.data_ptr()), P(directions.data_ptr()),
                                 P(exclude_surface.data_ptr()) if exclude_surface is not None else None, n,
                                 int(method), P(hit.data_ptr()), P(t.data_ptr()), P(stats.ctypes.data),
                                 _stream_ptr(stream)))
    return hit, t, (int(stats[0]), int(stats[1]))


class ImageSources:
    """rt_image_sources handle.  Its device arrays are exposed as torch tensors
    created on access; each tensor keeps the handle alive, and the handle keeps
    no tensor (no reference cycle, so memory returns as soon as both are gone)."""

    _FIELDS = {  # name: (view field, shape key, dtype name)
        "rcv": ("rcv", "n", "int32"), "order": ("order", "n", "int32"), "count": ("count", "n", "int32"),
        "rep_ray": ("rep_ray", "n", "int32"), "pos": ("pos", "n3", "float64"), "dist": ("dist", "n", "float64"),
        "time": ("time", "n", "float64"), "energy": ("energy", "n8", "float64"),
        "hist": ("hist", "hist", "int32"), "ray_energy": ("ray_energy", "t8", "float32"),
        "ray_length": ("ray_length", "t", "float32"), "ray_hits": ("ray_hits", "t", "int32"),
        "rec_rcv": ("rec_rcv", "r", "int32"), "rec_ray": ("rec_ray", "r", "int32"),
        "rec_order": ("rec_order", "r", "int32"), "rec_length": ("rec_length", "r", "float32"),
    }

    def __init__(self, handle):
        self._h = handle
        v = rt_is_view()
        _check(lib().rt_image_sources_view(handle, C.byref(v)))
        self.view = v
        self.n = v.n
        self.n_traced, self.n_bounces = v.n_traced, v.n_bounces
        self.n_records = v.n_records
        self.queries = v.queries
        self.hash_collisions = v.hash_collisions
        self.ms_rays, self.ms_bounces, self.ms_image_sources = v.ms_rays, v.ms_bounces, v.ms_image_sources
        self.block_size, self.tail_rays = v.block_size, v.tail_rays
        self.compaction_period, self.stack_entries = v.compaction_period, v.stack_entries
        self.n_rcv = v.n_rcv

    def __getattr__(self, name):
        f = ImageSources._FIELDS.get(name)
        if f is None:
            raise AttributeError(name)
        import torch
        v = self.__dict__["view"]
        n, t, r = v.n, v.n_traced, v.n_records
        shape = {"n": (n,), "n3": (n, 3), "n8": (n, N_BANDS), "hist": (v.n_bounces, t), "t8": (t, N_BANDS),
                 "t": (t,), "r": (r,)}[f[1]]
        return _device_tensor(getattr(v, f[0]), shape, getattr(torch, f[2]), self)

    def free(self):
        """Release the device memory now (tensors taken from it become invalid)."""
        if self.__dict__.get("_h"):
            lib().rt_image_sources_free(self._h)
            self._h = None

    def __del__(self):
        self.free()


def rt_trace(tree: Tree, sources, rcv_center, rcv_radius, rcv_source, band_absorption, n_rays, n_bounces,
             ray_begin=0, ray_count=0, max_distance=0.0, air_beta=None, c=343.2, block_size=0,
             max_node_visits=0, tail_rays=0, stream=None, debug_t=None, debug_state=None,
             debug_cost=None, workspace=None, replay=None, src_axis=None, src_pattern=None, compaction_period=0,
             stack_entries=0) -> ImageSources:
    """Propagate rays and build image sources (host inputs; see roomrays.h).
    replay: the result (or its hist) of an earlier trace of the same rays --
    the queries then re-test the recorded triangles, for new receivers.
    src_axis / src_pattern: directional sources (see _sources)."""
    S, keep_src = _sources(sources, src_axis, src_pattern)
    per_src = int(ray_count) if int(ray_count) > 0 else int(n_rays) - int(ray_begin)
    _check_debug(debug_t, debug_state, debug_cost, n_bounces,
                 max(per_src, 0) * np.asarray(sources, np.float64).reshape(-1, 3).shape[0])
    rc, prc = _host(np.asarray(rcv_center, np.float64).reshape(-1, 3), np.float64)
    rr, prr = _host(np.asarray(rcv_radius, np.float64).reshape(-1), np.float64)
    rs, prs = _host(np.asarray(rcv_source, np.int32).reshape(-1), np.int32)
    al, pal = _host(np.asarray(band_absorption, np.float32).reshape(-1, N_BANDS), np.float32)
    if air_beta is not None:
        be, pbe = _host(np.asarray(air_beta, np.float32).reshape(N_BANDS), np.float32)
    else:
        be, pbe = None, None
    R = rt_receivers(prc, prr, prs, len(rc))
    prm = rt_trace_params(int(n_rays), int(ray_begin), int(ray_count), int(n_bounces), float(max_distance), pbe,
                          float(c), int(block_size), int(max_node_visits), int(tail_rays), _stream_ptr(stream),
                          P(debug_t.data_ptr()) if debug_t is not None else None,
                          P(debug_state.data_ptr()) if debug_state is not None else None,
                          P(debug_cost.data_ptr()) if debug_cost is not None else None,
                          workspace._h if workspace is not None else None, _replay_ptr(replay),
                          int(compaction_period), int(stack_entries))
    out = P()
    _check(lib().rt_trace(tree._h, C.byref(S), C.byref(R), pal, len(al), C.byref(prm), C.byref(out)))
    res = ImageSources(out)
    res.n_rcv = len(rc)
    return res


class Response:
    """rt_response handle: [n_rcv, 8, n_bins] float32 device histograms
    (``data`` is created on access and keeps the handle alive)."""

    def __init__(self, handle):
        self._h = handle
        v = rt_response_view()
        _check(lib().rt_response_get(handle, C.byref(v)))
        self.view = v
        self.n_rcv, self.n_bins, self.fs = v.n_rcv, v.n_bins, v.fs

    @property
    def data(self):
        import torch
        v = self.view
        return _device_tensor(v.data, (max(v.n_rcv, 1), N_BANDS, v.n_bins), torch.float32, self)

    def download(self, out=None, stream=None):
        """Copy to host through rt_response_download (out: numpy or CPU tensor)."""
        need = max(self.n_rcv, 1) * N_BANDS * self.n_bins
        if out is None:
            out = np.empty((max(self.n_rcv, 1), N_BANDS, self.n_bins), np.float32)
        if hasattr(out, "data_ptr"):
            if out.is_cuda or str(out.dtype) != "torch.float32" or not out.is_contiguous() or out.numel() < need:
                raise ValueError(f"download: out must be a contiguous host float32 buffer of {need} elements")
            ptr = out.data_ptr()
        else:
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size < need:
                raise ValueError(f"download: out must be a contiguous host float32 buffer of {need} elements")
            ptr = out.ctypes.data
        _check(lib().rt_response_download(self._h, P(ptr), _stream_ptr(stream)))
        return out

    def free(self):
        if getattr(self, "_h", None):
            lib().rt_response_free(self._h)
            self._h = None

    def __del__(self):
        self.free()


def rt_rir(image_sources: ImageSources, fs, duration=0.0, stream=None) -> Response:
    out = P()
    _check(lib().rt_rir(image_sources._h, float(fs), float(duration), _stream_ptr(stream), C.byref(out)))
    return Response(out)


class Workspace:
    """rt_workspace: scratch and the bounce-loop CUDA graph reused across traces."""

    def __init__(self):
        h = P()
        _check(lib().rt_workspace_create(C.byref(h)))
        self._h = h

    @property
    def graph_launches(self) -> int:
        return int(lib().rt_workspace_graph_launches(self._h))

    def free(self):
        if getattr(self, "_h", None):
            lib().rt_workspace_free(self._h)
            self._h = None

    def __del__(self):
        self.free()


def _rooms(rooms):
    """rt_room array over host copies of a list of room dicts (keys tree,
    sources, rcv_center, rcv_radius, rcv_source, band_absorption, optionally
    src_axis, src_pattern); returns (array, kept copies, receiver count)."""
    keep, arr = [], (rt_room * len(rooms))()
    n_rcv = 0
    for k, r in enumerate(rooms):
        S, keep_src = _sources(r["sources"], r.get("src_axis"), r.get("src_pattern"))
        rc, prc = _host(np.asarray(r["rcv_center"], np.float64).reshape(-1, 3), np.float64)
        rr, prr = _host(np.asarray(r["rcv_radius"], np.float64).reshape(-1), np.float64)
        rs, prs = _host(np.asarray(r["rcv_source"], np.int32).reshape(-1), np.int32)
        al, pal = _host(np.asarray(r["band_absorption"], np.float32).reshape(-1, N_BANDS), np.float32)
        keep += keep_src + [rc, rr, rs, al]
        arr[k] = rt_room(r["tree"]._h, S, rt_receivers(prc, prr, prs, len(rc)), pal, len(al))
        n_rcv += len(rc)
    return arr, keep, n_rcv


def rt_trace_batch(rooms, n_rays, n_bounces, ray_begin=0, ray_count=0, max_distance=0.0, air_beta=None, c=343.2,
                   block_size=0, max_node_visits=0, tail_rays=0, stream=None, workspace=None,
                   replay=None, debug_t=None, debug_state=None, debug_cost=None, compaction_period=0,
                   stack_entries=0) -> ImageSources:
    """Trace many rooms in one persistent launch.  `rooms` is a list of dicts
    with keys tree, sources, rcv_center, rcv_radius, rcv_source,
    band_absorption (and optionally src_axis, src_pattern).  Receivers are
    numbered room after room.  replay and the debug outputs: see rt_trace."""
    per_src = int(ray_count) if int(ray_count) > 0 else int(n_rays) - int(ray_begin)
    n_src = sum(np.asarray(r["sources"], np.float64).reshape(-1, 3).shape[0] for r in rooms)
    _check_debug(debug_t, debug_state, debug_cost, n_bounces, max(per_src, 0) * n_src)
    arr, keep, n_rcv = _rooms(rooms)
    if air_beta is not None:
        be, pbe = _host(np.asarray(air_beta, np.float32).reshape(N_BANDS), np.float32)
    else:
        be, pbe = None, None
    prm = rt_trace_params(int(n_rays), int(ray_begin), int(ray_count), int(n_bounces), float(max_distance), pbe,
                          float(c), int(block_size), int(max_node_visits), int(tail_rays), _stream_ptr(stream),
                          P(debug_t.data_ptr()) if debug_t is not None else None,
                          P(debug_state.data_ptr()) if debug_state is not None else None,
                          P(debug_cost.data_ptr()) if debug_cost is not None else None,
                          workspace._h if workspace is not None else None, _replay_ptr(replay),
                          int(compaction_period), int(stack_entries))
    out = P()
    _check(lib().rt_trace_batch(arr, len(rooms), C.byref(prm), C.byref(out)))
    res = ImageSources(out)
    res.n_rcv = n_rcv
    return res


RT_RIR_STATIC_MAX_SOURCES = 524288


def rt_rir_static(image_sources: ImageSources, fs, duration, out=None, stream=None):
    """Histograms of image sources without any device allocation inside the
    library (static scratch; see roomrays.h).  `out` is a contiguous CUDA
    float32 tensor [n_rcv, 8, ceil(duration * fs)] that the call zero-fills
    and sums into; if not given, torch allocates it here (outside the
    library).  A wrong `out` raises ValueError before anything is launched."""
    n_bins = int(np.ceil(duration * fs))
    n_rcv = max(image_sources_n_rcv(image_sources), 1)
    if n_bins < 1:
        raise ValueError("rt_rir_static: duration * fs must give at least one bin")
    shape = (n_rcv, N_BANDS, n_bins)
    if out is None:
        import torch
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
    elif not (_is_cuda_tensor(out) and str(out.dtype) == "torch.float32" and out.is_contiguous()
              and tuple(out.shape) == shape):
        raise ValueError(f"rt_rir_static: out must be a contiguous CUDA float32 tensor of shape {shape}, got "
                         f"{tuple(getattr(out, 'shape', ()))} {getattr(out, 'dtype', type(out))} on "
                         f"{getattr(out, 'device', 'host')}")
    v = image_sources.view
    _check(lib().rt_rir_static(P(v.time), P(v.rcv), P(v.energy), int(v.n), int(n_rcv), float(fs), int(n_bins),
                               P(out.data_ptr()), _stream_ptr(stream)))
    return out


def image_sources_n_rcv(image_sources: ImageSources) -> int:
    return image_sources.n_rcv


_alloc_keep = []


def rt_set_allocator(alloc=None, free=None, ctx=None):
    """Install Python allocation callbacks (both None restores the default)."""
    if alloc is None and free is None:
        _check(lib().rt_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _alloc_keep.clear()
        return
    a, f = ALLOC_FN(alloc), FREE_FN(free)
    _alloc_keep[:] = [a, f]
    _check(lib().rt_set_allocator(a, f, ctx))


def scene_args(scene):
    """Keyword arguments of rt_trace for a scenes.Scene."""
    return dict(sources=scene.sources, rcv_center=scene.rcv_center, rcv_radius=scene.rcv_radius,
                rcv_source=scene.rcv_source, band_absorption=scene.alpha, n_rays=scene.n_rays,
                n_bounces=scene.n_bounces, max_distance=scene.max_distance,
                air_beta=scene.beta if np.any(scene.beta) else None, c=scene.c,
                src_axis=getattr(scene, "src_axis", None), src_pattern=getattr(scene, "src_pattern", None))


class MLP:
    """rt_mlp handle: the surrogate network, trained and run by libroomrays."""

    def __init__(self, n_in, n_hidden, n_out, seed=0, stream=None):
        h = P()
        _check(lib().rt_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), _stream_ptr(stream), C.byref(h)))
        self._h = h
        a, b, c, n = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        off = (C.c_int64 * 6)()
        _check(lib().rt_mlp_info(h, C.byref(a), C.byref(b), C.byref(c), C.byref(n), off))
        self.n_in, self.n_hidden, self.n_out, self.n_params = a.value, b.value, c.value, n.value
        self.offsets = [int(x) for x in off]

    def _inputs(self, x, target=None):
        if not _is_cuda_tensor(x) or x.dim() != 2 or x.shape[1] != self.n_in:
            raise ValueError(f"rt_mlp: x must be a CUDA tensor [batch][{self.n_in}]")
        x = x.contiguous().float()
        if target is not None:
            if not _is_cuda_tensor(target) or tuple(target.shape) != (x.shape[0], self.n_out):
                raise ValueError(f"rt_mlp: target must be a CUDA tensor [batch][{self.n_out}]")
            target = target.contiguous().float()
        return x, target

    def forward(self, x, y=None, stream=None):
        import torch
        x, _ = self._inputs(x)
        if y is None:
            y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        _cuda(y, "rt_mlp: y", "float32", (x.shape[0], self.n_out))
        _check(lib().rt_mlp_forward(self._h, P(x.data_ptr()), int(x.shape[0]), P(y.data_ptr()), _stream_ptr(stream)))
        return y

    def gradients(self, x, target, stream=None):
        loss = C.c_float()
        x, target = self._inputs(x, target)
        _check(lib().rt_mlp_gradients(self._h, P(x.data_ptr()), P(target.data_ptr()), int(x.shape[0]),
                                      C.byref(loss), _stream_ptr(stream)))
        return loss.value

    def train_step(self, x, target, lr, stream=None, want_loss=True):
        loss = C.c_float()
        x, target = self._inputs(x, target)
        _check(lib().rt_mlp_train_step(self._h, P(x.data_ptr()), P(target.data_ptr()), int(x.shape[0]), float(lr),
                                       C.byref(loss) if want_loss else None, _stream_ptr(stream)))
        return loss.value if want_loss else None

    def copy(self, what, host=None, to_device=False, stream=None):
        if host is None:
            host = np.empty(self.n_params, np.float32)
        host = np.ascontiguousarray(host, np.float32)
        _check(lib().rt_mlp_copy(self._h, int(what), P(host.ctypes.data), int(bool(to_device)), _stream_ptr(stream)))
        return host

    def blocks(self, flat):
        """Split a parameter-sized vector into W1, b1, W2, b2, W3, b3."""
        I, H, O = self.n_in, self.n_hidden, self.n_out
        shapes = [(H, I), (H,), (H, H), (H,), (O, H), (O,)]
        return [flat[o:o + int(np.prod(sh))].reshape(sh) for o, sh in zip(self.offsets, shapes)]

    def set_weight_decay(self, wd):
        _check(lib().rt_mlp_set_weight_decay(self._h, float(wd)))

    @property
    def step(self):
        v = C.c_int64()
        _check(lib().rt_mlp_get_step(self._h, C.byref(v)))
        return v.value

    @step.setter
    def step(self, value):
        _check(lib().rt_mlp_set_step(self._h, int(value)))

    def free(self):
        if getattr(self, "_h", None):
            lib().rt_mlp_free(self._h)
            self._h = None

    def __del__(self):
        self.free()


# ----------------------------------------------------------------------------
# surrogate-tail mode (see roomrays.h): every room one source, one receiver
# ----------------------------------------------------------------------------
SUR_N_DESC, SUR_N_EARLY, SUR_N_TAIL, SUR_N_ENV, SUR_N_FEAT = 47, 50, 195, 200, 951


def _sur_params(early_rays=0, probe_rays=0, full_rays=0, rooms_per_launch=0, air_beta=None, c=0.0, stream=None,
                workspace=None):
    be, pbe = (None, None) if air_beta is None else _host(np.asarray(air_beta, np.float32).reshape(N_BANDS),
                                                            np.float32)
    prm = rt_surrogate_trace_params(int(early_rays), int(probe_rays), int(full_rays), int(rooms_per_launch), pbe,
                                    float(c), _stream_ptr(stream), workspace._h if workspace is not None else None)
    return prm, be


def _dev(shape):
    import torch
    return torch.empty(shape, dtype=torch.float32, device="cuda")


def _ptr(t):
    return P(t.data_ptr()) if t is not None else None


def _f32(t, shape, name):
    if not (_is_cuda_tensor(t) and str(t.dtype) == "torch.float32" and t.is_contiguous() and tuple(t.shape) == shape):
        raise ValueError(f"{name}: a contiguous CUDA float32 tensor of shape {shape}")
    return t


def rt_surrogate_inputs(rooms, volume, **kw):
    """desc, early, probe, prior_db, base_db and X (CUDA tensors) of one-
    receiver rooms; kw: early_rays, probe_rays, rooms_per_launch, air_beta, c,
    stream, workspace."""
    n = len(rooms)
    arr, keep, _ = _rooms(rooms)
    vol, pvol = _host(np.asarray(volume, np.float64).reshape(-1), np.float64)
    if len(vol) != n:
        raise ValueError("rt_surrogate_inputs: one volume per room")
    prm, kb = _sur_params(**kw)
    out = {"desc": _dev((n, SUR_N_DESC)), "early": _dev((n, N_BANDS, SUR_N_EARLY)),
           "probe": _dev((n, N_BANDS, SUR_N_TAIL)), "prior_db": _dev((n, N_BANDS, SUR_N_TAIL)),
           "base_db": _dev((n, N_BANDS, SUR_N_TAIL)), "X": _dev((n, SUR_N_FEAT))}
    _check(lib().rt_surrogate_inputs(arr, pvol, n, C.byref(prm), *(_ptr(out[k]) for k in
                                     ("desc", "early", "probe", "prior_db", "base_db", "X"))))
    return out


def rt_surrogate_reference(rooms, **kw):
    """Full traces of one-receiver rooms: (env [n][8][200], tail_db [n][8][195])
    CUDA tensors; kw: full_rays, rooms_per_launch, air_beta, c, stream, workspace."""
    n = len(rooms)
    arr, keep, _ = _rooms(rooms)
    prm, kb = _sur_params(**kw)
    env, tdb = _dev((n, N_BANDS, SUR_N_ENV)), _dev((n, N_BANDS, SUR_N_TAIL))
    _check(lib().rt_surrogate_reference(arr, n, C.byref(prm), _ptr(env), _ptr(tdb)))
    return env, tdb


class SurrogateModel:
    """rt_surrogate handle: the trained tail networks, their normalisation,
    training range and gate tolerances."""

    def __init__(self, handle):
        self._h = handle

    def info(self):
        nn, nh = C.c_int32(), C.c_int32()
        j, pr = C.c_float(), C.c_float()
        _check(lib().rt_surrogate_info(self._h, C.byref(nn), C.byref(j), C.byref(pr), C.byref(nh), None))
        hist = np.zeros(3 * nh.value, np.float32)
        _check(lib().rt_surrogate_info(self._h, None, None, None, None, P(hist.ctypes.data)))
        return {"n_nets": nn.value, "join_db": j.value, "probe_db": pr.value, "history": hist.reshape(-1, 3)}

    def to_bytes(self) -> bytes:
        n = C.c_size_t()
        _check(lib().rt_surrogate_save(self._h, None, 0, C.byref(n)))
        buf = (C.c_ubyte * n.value)()
        _check(lib().rt_surrogate_save(self._h, buf, n.value, C.byref(n)))
        return bytes(buf)

    def save(self, path):
        with open(path, "wb") as f:
            f.write(self.to_bytes())

    @staticmethod
    def from_bytes(data: bytes, stream=None):
        buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
        h = P()
        _check(lib().rt_surrogate_load(buf, len(data), _stream_ptr(stream), C.byref(h)))
        return SurrogateModel(h)

    @staticmethod
    def load(path, stream=None):
        with open(path, "rb") as f:
            return SurrogateModel.from_bytes(f.read(), stream)

    def predict(self, X, base_db, stream=None):
        n = int(X.shape[0])
        _f32(X, (n, SUR_N_FEAT), "X")
        _f32(base_db, (n, N_BANDS, SUR_N_TAIL), "base_db")
        out = _dev((n, N_BANDS, SUR_N_TAIL))
        _check(lib().rt_surrogate_predict(self._h, _ptr(X), _ptr(base_db), n, _ptr(out), _stream_ptr(stream)))
        return out

    def gate(self, desc, X, pred_db, prior_db, stream=None):
        """(pass [n] bool, gaps [n][2] = join, probe in dB) as numpy arrays."""
        n = int(X.shape[0])
        _f32(desc, (n, SUR_N_DESC), "desc")
        _f32(X, (n, SUR_N_FEAT), "X")
        for t, name in ((pred_db, "pred_db"), (prior_db, "prior_db")):
            _f32(t, (n, N_BANDS, SUR_N_TAIL), name)
        ok = np.zeros(n, np.int32)
        gaps = np.zeros((n, 2), np.float32)
        _check(lib().rt_surrogate_gate(self._h, _ptr(desc), _ptr(X), _ptr(pred_db), _ptr(prior_db), n,
                                       P(ok.ctypes.data), P(gaps.ctypes.data), _stream_ptr(stream)))
        return ok.astype(bool), gaps

    def free(self):
        if getattr(self, "_h", None):
            lib().rt_surrogate_free(self._h)
            self._h = None

    def __del__(self):
        self.free()


def rt_surrogate_train(X, tail_db, desc, base_db, prior_db, n_nets=0, steps=0, batch=0, lr=0.0, weight_decay=0.0,
                       input_noise=0.0, val_frac=0.0, log_every=0, seed=0, stream=None) -> SurrogateModel:
    n = int(X.shape[0])
    _f32(X, (n, SUR_N_FEAT), "X")
    _f32(desc, (n, SUR_N_DESC), "desc")
    for t, name in ((tail_db, "tail_db"), (base_db, "base_db"), (prior_db, "prior_db")):
        _f32(t, (n, N_BANDS, SUR_N_TAIL), name)
    prm = rt_surrogate_train_params(int(n_nets), int(steps), int(batch), float(lr), float(weight_decay),
                                    float(input_noise), float(val_frac), int(log_every), int(seed),
                                    _stream_ptr(stream))
    h = P()
    _check(lib().rt_surrogate_train(_ptr(X), _ptr(tail_db), _ptr(desc), _ptr(base_db), _ptr(prior_db), n,
                                    C.byref(prm), C.byref(h)))
    return SurrogateModel(h)


def rt_surrogate_envelope(early, tail, tail_is_db, stream=None):
    """Envelopes [n][8][200] (CUDA): early [n][8][50] + a tail [n][8][195]
    given as per-bin energies or as a decay curve in dB."""
    n = int(early.shape[0])
    _f32(early, (n, N_BANDS, SUR_N_EARLY), "early")
    _f32(tail, (n, N_BANDS, SUR_N_TAIL), "tail")
    env = _dev((n, N_BANDS, SUR_N_ENV))
    _check(lib().rt_surrogate_envelope(_ptr(early), _ptr(tail), int(bool(tail_is_db)), n, _ptr(env),
                                       _stream_ptr(stream)))
    return env


def rt_rir_surrogate(rooms, volume, model: SurrogateModel, **kw):
    """Surrogate-tail responses of one-receiver rooms: (Response [n][8][200]
    at 100 Hz, used_fallback numpy bool [n]); kw: early_rays, probe_rays,
    full_rays, rooms_per_launch, air_beta, c, stream, workspace."""
    n = len(rooms)
    arr, keep, _ = _rooms(rooms)
    vol, pvol = _host(np.asarray(volume, np.float64).reshape(-1), np.float64)
    if len(vol) != n:
        raise ValueError("rt_rir_surrogate: one volume per room")
    prm, kb = _sur_params(**kw)
    fb = np.zeros(n, np.int32)
    h = P()
    _check(lib().rt_rir_surrogate(arr, pvol, n, model._h, C.byref(prm), C.byref(h), P(fb.ctypes.data)))
    return Response(h), fb.astype(bool)
