"""The kernels use 16- and 32-byte vector accesses (the traversal reads the
tree in 32-byte sectors), so a caller's device allocator must hand out
256-byte aligned blocks, as cudaMalloc does.  A block that is not goes back
to the caller's free function before any kernel sees it and the call fails
with RT_ERR_OOM; rt_gemm_bf16 refuses operands off a 16-byte boundary."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import scenes  # noqa: E402
from paper_1811_05784_gb300 import rt  # noqa: E402


def test_a_misaligned_allocator_is_refused():
    sc = scenes.shoebox(n_rays=100, n_bounces=2)
    held = {}

    def alloc(nbytes, stream, ctx):
        t = torch.empty(int(nbytes) + 64, dtype=torch.uint8, device="cuda")
        p = (t.data_ptr() + 255) // 256 * 256 + 16  # 16 bytes past a 256-byte boundary
        if p + int(nbytes) > t.data_ptr() + t.numel():
            t = torch.empty(int(nbytes) + 512, dtype=torch.uint8, device="cuda")
            p = (t.data_ptr() + 255) // 256 * 256 + 16
        held[p] = t
        return p

    def free(p, stream, ctx):
        held.pop(p, None)

    torch.cuda.synchronize()
    rt.rt_set_allocator(alloc, free)
    try:
        with pytest.raises(rt.RtError) as e:
            rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    finally:
        torch.cuda.synchronize()
        rt.rt_set_allocator(None, None)
    assert e.value.status == rt.RT_ERR_OOM and "256-byte aligned" in str(e.value)
    assert not held  # every block went back
    # the default allocator's tree traces as before
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    isrc = rt.rt_trace(tree, **rt.scene_args(sc))
    assert isrc.queries > 0


def test_gemm_operands_off_a_16_byte_boundary_are_refused():
    A = torch.zeros((16, 8), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(16 * 16 + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(rt.RtError):
        rt.rt_gemm_bf16(A, A, out=C[1:].view(16, 16))
