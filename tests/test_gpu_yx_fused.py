"""GPU parity of the fused inverse y + x pass (one thread-block cluster per output
plane, the plane exchanged through distributed shared memory): against the FP64
direct sum of Eq. 10 on sampled cells, and against the two separate inverse passes
on the same context settings, for every padded plane size the fused pass takes
(py x px/2 of 256 x 128, 512 x 128, 256 x 256, 512 x 256), ragged and odd extents,
rows that leave whole CTAs of a cluster empty, batches, the Eq. 20 statistics and the
fixed-work-area entry point."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_STRESS = 1e-5


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
    return np.array([np.linalg.norm(got[c] - ref[c]) / max(np.linalg.norm(ref[c]), 1e-6 * scale) for c in range(6)])


def context(dds, p, fused):
    g = p.geom
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    ctx.set_option(dds.DDS_OPT_YX_FUSED, 1 if fused else 0)
    return ctx.build_kernels()


CASES = [   # (nx, ny, nz), families, expected (py, px / 2, cluster), seed
    ((100, 70, 5), slice(0, 18), (256, 128, 8), 41),        # rows 70: CTAs 5..7 of 8 hold none
    ((255, 200, 3), [0, 9, 13], (512, 256, 16), 42),       # odd nx, ragged y
    ((129, 65, 4), [1, 4, 6, 13, 17], (256, 256, 16), 43),  # smallest nx of px 512, ny of py 256
    ((128, 256, 2), [2, 11], (512, 128, 8), 44),            # ny = py / 2: every row of every CTA
    ((65, 128, 6), slice(0, 18), (256, 128, 8), 45),        # smallest nx of px 256, ny = py / 2
]


def sample_targets(g, n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, g.n_cells, size=n)
    last_row = (g.nz - 1) * g.nx * g.ny + (g.ny - 1) * g.nx + np.arange(g.nx)        # y = ny - 1
    corners = [0, g.n_cells - 1, g.nx - 1, (g.ny - 1) * g.nx]
    return np.unique(np.concatenate([pts, corners, last_row[::7]]))


@pytest.mark.parametrize("shape,fams,expect,seed", CASES)
def test_fused_inverse_vs_direct_sum_and_separate_passes(dds, shape, fams, expect, seed):
    t18, b18 = W.gan_families()
    g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.1e-6)
    p = W.random_problem(g, t18[fams], b18[fams], seed=seed)
    fused = context(dds, p, True)
    q = fused.query()
    assert (q["py"], q["px"] // 2, q["yx_cluster"]) == expect
    assert fused.launches_per_stress + 1 == context(dds, p, False).launches_per_stress
    rho = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    got = fused.stress(rho).cpu().numpy().reshape(6, -1)
    sep = context(dds, p, False)
    assert sep.query()["yx_cluster"] == 0
    alt = sep.stress(rho).cpu().numpy().reshape(6, -1)
    assert rel_l2_per_component(got, alt).max() <= 1e-6
    tg = sample_targets(g, 40, seed)
    ref = oracle.stress_direct(g, p.t, p.b, p.rho, targets=tg, use_table=False).T
    assert rel_l2_per_component(got[:, tg], ref).max() <= TOL_STRESS


def test_fused_inverse_batches_statistics_and_fixed_area(dds):
    t18, b18 = W.gan_families()
    g = W.Geometry(100, 90, 6, 0.2e-6, 0.2e-6, 0.05e-6)
    probs = [W.random_problem(g, t18, b18, seed=50 + i) for i in range(3)]
    rho = torch.from_numpy(np.stack([p.rho for p in probs]).astype(np.float32)).cuda()
    fused, sep = context(dds, probs[0], True), context(dds, probs[0], False)
    assert fused.query()["yx_cluster"] == 8
    # batch of three density sets: each set as alone, and as the separate passes
    many = fused.stress_multi(rho).cpu().numpy()
    for i in range(3):
        one = fused.stress(rho[i].contiguous()).cpu().numpy()
        assert rel_l2_per_component(many[i], one).max() <= 1e-6
    assert rel_l2_per_component(many[2], sep.stress_multi(rho).cpu().numpy()[2]).max() <= 1e-6
    # Eq. 20 statistics accumulated in the fused pass
    s_f = fused.stress_stats(rho[1].contiguous())[1].cpu().numpy()
    s_s = sep.stress_stats(rho[1].contiguous())[1].cpu().numpy()
    assert np.allclose(s_f, s_s, rtol=1e-5, atol=0)
    # the fixed-work-area entry point runs the same passes
    sig = torch.empty((6,) + fused.shape, dtype=torch.float32, device="cuda")
    dds.dds_stress_noalloc(fused.handle, rho[0].contiguous().data_ptr(), dds.DDS_F32, sig.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(sig.cpu().numpy(), fused.stress(rho[0].contiguous()).cpu().numpy())


def test_fused_inverse_not_taken_where_it_does_not_apply(dds):
    t18, b18 = W.gan_families()
    g = W.Geometry(100, 70, 5, 0.2e-6, 0.2e-6, 0.1e-6)        # a plane it takes, option not set
    p = W.random_problem(g, t18[:2], b18[:2], seed=1)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b).build_kernels()
    assert ctx.query()["yx_cluster"] == 0                    # separate passes by default
    for shape in ((64, 64, 4), (300, 300, 2)):            # px / 2 = 64; py = 1024
        g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.1e-6)
        p = W.random_problem(g, t18[:2], b18[:2], seed=1)
        assert context(dds, p, True).query()["yx_cluster"] == 0
