"""Captured batches (dds_graph_*): several density sets on several grids replayed by
one graph launch give exactly the results of the same evaluations launched directly
(the same kernels on the same inputs), and follow densities refilled in place."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_01830_gb300 as mod
    mod.load_library()
    return mod


def build(dds, shape, cells, fams):
    t, b = W.gan_families()
    g = W.Geometry(*shape, *cells)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(t[fams], b[fams]).build_kernels()
    return ctx, g, len(fams)


def densities(g, F, nb, seed):
    return torch.stack([torch.from_numpy(W.random_problem(g, *[a[:F] for a in W.gan_families()], seed=seed + i)
                                         .rho.astype(np.float32)) for i in range(nb)]).cuda().contiguous()


def test_graph_replays_the_direct_evaluations(dds):
    c1, g1, F1 = build(dds, (40, 24, 10), (0.2e-6, 0.2e-6, 0.05e-6), [0, 1, 9, 12])
    c2, g2, F2 = build(dds, (64, 48, 16), (0.5e-6, 0.5e-6, 0.2e-6), [2, 7])
    r1 = densities(g1, F1, 3, seed=10)
    r2 = densities(g2, F2, 2, seed=20).to(torch.bfloat16)
    graph = dds.StressGraph([(c1, r1), (c2, r2)])
    assert graph.nodes >= 2 * 5
    for round_ in range(2):
        if round_ == 1:                      # new densities, same buffers
            r1.copy_(densities(g1, F1, 3, seed=30))
            r2.copy_(densities(g2, F2, 2, seed=40).to(torch.bfloat16))
        graph.launch()
        torch.cuda.synchronize()
        want1 = c1.stress_multi(r1)
        want2 = c2.stress_multi(r2)
        torch.cuda.synchronize()
        assert torch.equal(graph.sigma[0], want1)
        assert torch.equal(graph.sigma[1], want2)
    graph.close()
    c1.close()
    c2.close()


def test_graph_capture_errors(dds):
    c1, g1, F1 = build(dds, (16, 16, 4), (1e-6, 1e-6, 0.25e-6), [0])
    r = densities(g1, F1, 1, seed=1)
    dds.dds_profile_enable(c1.handle, True)
    with pytest.raises(dds.DDSError) as e:
        dds.StressGraph([(c1, r)])
    assert e.value.code == dds.DDS_ERR_INVALID_ARG
    dds.dds_profile_enable(c1.handle, False)
    c2 = dds.StressContext(0)
    c2.set_geometry(16, 16, 4, 1e-6, 1e-6, 0.25e-6, W.MU_GAN, W.NU_GAN)
    with pytest.raises(dds.DDSError) as e:
        dds.dds_graph_capture([c2.handle], [1], [r.data_ptr()], [dds.DDS_F32], [r.data_ptr()])
    assert e.value.code == dds.DDS_ERR_NOT_READY
    c1.close()
    c2.close()
