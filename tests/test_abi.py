"""Host-side checks of the C ABI library and of the oracle's independence."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "roomrays.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_exports_every_declared_symbol():
    from paper_1811_05784_gb300 import build, rt
    build.build()
    lib = rt.lib()
    declared = _declared()
    assert {"rt_build_tree", "rt_trace", "rt_rir"} <= set(declared)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(rt.EXPORTED) == declared
    assert rt.rt_api_version() == 1


def test_error_reporting_without_gpu():
    """Argument checks run before any CUDA call."""
    from paper_1811_05784_gb300 import rt
    mesh = rt.rt_mesh()
    out = ctypes.c_void_p()
    st = rt.lib().rt_build_tree(ctypes.byref(mesh), None, ctypes.byref(out))
    assert st == rt.RT_ERR_INVALID_ARG
    assert "n_tris" in rt.rt_last_error()
    assert rt.lib().rt_trace(None, None, None, None, 0, None, ctypes.byref(out)) == rt.RT_ERR_INVALID_ARG


def test_oracle_and_cuda_path_share_no_code():
    pkg = os.path.join(ROOT, "paper_1811_05784_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "rt_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1811_05784_gb300", txt, re.M), f
            assert not re.search(r"#include.*roomrays", txt), f


STRUCTS = ("rt_mesh", "rt_sources", "rt_receivers", "rt_trace_params", "rt_room", "rt_is_view",
           "rt_response_view", "rt_surrogate_trace_params", "rt_surrogate_train_params")


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors have the C compiler's size and field offsets for
    every public struct of roomrays.h (a field added on one side only would
    shift every later field)."""
    import shutil
    import subprocess
    from paper_1811_05784_gb300 import rt
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "roomrays.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(rt, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        name, field, value = line.split()
        cls = getattr(rt, name)
        want = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(value) == want, (name, field, int(value), want)
        seen += 1
    assert seen == sum(1 + len(getattr(rt, n)._fields_) for n in STRUCTS)


def test_static_histogram_binding_rejects_a_wrong_output_before_any_call():
    """rt.rt_rir_static checks a caller-supplied output (device, dtype,
    contiguity, shape) before it reaches the library: a wrong buffer would
    otherwise be written past its end on the device."""
    import numpy as np
    from paper_1811_05784_gb300 import rt

    class _Fake:          # only n_rcv is read before the output check
        n_rcv = 2

        @property
        def view(self):
            raise AssertionError("the library was reached")

    for bad in (np.zeros((2, 8, 100), np.float32), [[0.0]], np.zeros(3)):
        with pytest.raises(ValueError):
            rt.rt_rir_static(_Fake(), 100.0, 1.0, out=bad)
    torch = pytest.importorskip("torch")
    for bad in (torch.zeros((2, 8, 100)), torch.zeros((2, 8, 99)), torch.zeros((2, 8, 100), dtype=torch.float64)):
        with pytest.raises(ValueError):
            rt.rt_rir_static(_Fake(), 100.0, 1.0, out=bad)


def test_binding_rejects_host_tensors_and_short_buffers_before_any_call():
    """Every binding call that hands a caller's tensor to the library checks
    it first: host tensors (their pointers would reach kernels), wrong
    dtypes, and output or per-query buffers too small for what the library
    writes, all raise ValueError without the library being reached."""
    import numpy as np
    from paper_1811_05784_gb300 import rt
    torch = pytest.importorskip("torch")
    a = torch.zeros((16, 8), dtype=torch.bfloat16)  # host tensors
    with pytest.raises(ValueError):
        rt.rt_gemm_bf16(a, a)
    with pytest.raises(ValueError):
        rt.rt_room_parameters(torch.zeros((1, 8, 10)), 48000.0)
    with pytest.raises(ValueError):
        rt.rt_tail_prior(torch.zeros((1, 3, 8)), torch.zeros((1, 8)), torch.zeros(1), 8, 0.05, 0.01, 10)
    # per-query debug outputs sized for 2 bounces x 10 rays of one source
    kw = dict(sources=[[0.0, 0.0, 1.0]], rcv_center=[[1.0, 0.0, 1.0]], rcv_radius=[0.5], rcv_source=[0],
              band_absorption=np.zeros((1, 8)), n_rays=10, n_bounces=2)
    for bad in (dict(debug_t=torch.zeros(20)), dict(debug_state=torch.zeros(120)),
                dict(debug_cost=torch.zeros(40, dtype=torch.int32))):
        with pytest.raises(ValueError):
            rt.rt_trace(None, **kw, **bad)
    with pytest.raises(ValueError):
        rt.rt_trace_batch([dict(tree=None, **{k: v for k, v in kw.items() if k not in ("n_rays", "n_bounces")})],
                          10, 2, debug_t=torch.zeros(20))

    class _Response:
        n_rcv, n_bins = 1, 10
        download = rt.Response.download

    for bad in (np.zeros(79, np.float32), np.zeros(80, np.float64), torch.zeros(79)):
        with pytest.raises(ValueError):
            _Response().download(out=bad)


def test_tree_builder_flags_exclude_each_other_before_any_call():
    """rt_build_tree builds the LBVH, the paper's median-split tree or the
    LBVH with SAH top levels; asking for two at once raises ValueError before
    the library is reached (it need not even be built)."""
    import numpy as np
    from paper_1811_05784_gb300 import rt
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    with pytest.raises(ValueError):
        rt.rt_build_tree(V, np.array([[0, 1, 2]], np.int32), np.zeros(1, np.int32), median=True, sah=True)
