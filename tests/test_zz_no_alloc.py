"""dds_stress_noalloc, the evaluation entry point that allocates no device memory.

Some callers cannot call cudaMalloc while they run: their device memory belongs to
another allocator that must account for every byte, or they may not allocate once
their loop has started.  For them the library offers an evaluation whose work
buffers live in a fixed device area it declares itself.  These tests call that
entry point through the C ABI twice in a row (different densities, so stale
contents of the shared area would show) and compare each result with dds_stress,
check that a call changes no device allocation (free device memory is the same
before and after it), and check that a grid too large for the area is refused with
a clear error.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_STRESS = 1e-5     # the rel-L2 tolerance of the other stress tests


@pytest.fixture(scope="module")
def dds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_01830_gb300 as mod
    mod.load_library()
    return mod


def rel_l2_per_component(got, ref):
    got = np.asarray(got, np.float64).reshape(6, -1)
    ref = np.asarray(ref, np.float64).reshape(6, -1)
    scale = max(np.linalg.norm(ref[c]) for c in range(6))
    return np.array([np.linalg.norm(got[c] - ref[c]) / max(np.linalg.norm(ref[c]), 1e-6 * scale)
                     for c in range(6)])


def problems():
    t, b = W.gan_families()
    return [
        W.gaussian_disk_32(),
        W.random_problem(W.Geometry(40, 24, 10, 0.2e-6, 0.2e-6, 0.05e-6), t, b, seed=21),
        W.random_problem(W.Geometry(64, 64, 32, 0.3e-6, 0.3e-6, 0.1e-6), t[[0, 1, 9, 12]], b[[0, 1, 9, 12]], seed=22),
    ]


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_noalloc_matches_stress_on_two_calls(dds, idx):
    p = problems()[idx]
    ctx = dds.context_for(p)
    rho1 = torch.from_numpy(np.ascontiguousarray(p.rho, dtype=np.float32)).cuda()
    rho2 = (0.5 * torch.flip(rho1, dims=[3]) + 0.25 * rho1).contiguous()
    for rho in (rho1, rho2):
        ref = ctx.stress(rho)
        out = torch.full_like(ref, float("nan"))
        dds.dds_stress_noalloc(ctx.handle, rho.data_ptr(), dds.DDS_F32, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2_per_component(got, ref.cpu().numpy()).max() <= TOL_STRESS
    ctx.close()


def test_noalloc_call_allocates_no_device_memory(dds):
    p = problems()[2]
    ctx = dds.context_for(p)             # set-up: builds the kernels and places the area
    rho = torch.from_numpy(np.ascontiguousarray(p.rho, dtype=np.float32)).cuda()
    out = torch.empty((6,) + p.geom.shape, dtype=torch.float32, device="cuda")
    # warm-up call: the driver loads the evaluation kernels' code at their first launch
    dds.dds_stress_noalloc(ctx.handle, rho.data_ptr(), dds.DDS_F32, out.data_ptr())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        dds.dds_stress_noalloc(ctx.handle, rho.data_ptr(), dds.DDS_F32, out.data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.isfinite(out).all()
    ctx.close()


def test_noalloc_refuses_grids_beyond_the_fixed_area(dds):
    p = W.random_problem(W.Geometry(256, 256, 16, 0.5e-6, 0.5e-6, 0.2e-6), [[0, 0, 1]], [[W.A_LATT, 0, 0]], seed=23)
    ctx = dds.context_for(p)
    rho = torch.zeros((1, 16, 256, 256), device="cuda")
    out = torch.zeros((6, 16, 256, 256), device="cuda")
    with pytest.raises(dds.DDSError) as ei:
        dds.dds_stress_noalloc(ctx.handle, rho.data_ptr(), dds.DDS_F32, out.data_ptr())
    assert ei.value.code == dds.DDS_ERR_UNSUPPORTED
    assert "work space" in str(ei.value)
    ctx.close()
