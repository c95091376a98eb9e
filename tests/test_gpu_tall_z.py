"""GPU parity of the fused z pass on tall grids (padded z size 128 or 256), where the
three-stage register kernel is the default schedule: against the FP64 direct sum of
Eq. 10 for 1 to 6 combined fields, ragged and half-full z extents (nz = pz/2 is the
largest the padding allows), the Nyquist columns of odd and even nx, FP16 spectra,
BF16 densities, batches, and against the shared-memory schedule of the same pass."""
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


def families(kind):
    t, b = W.gan_families()
    if kind == "six":     # the 18 GaN families (5 fields) and an x-directed edge family
        t = np.concatenate([t, [[1.0, 0.0, 0.0]]])
        b = np.concatenate([b, [[0.0, W.A_LATT, 0.0]]])
        return t, b
    return t[kind], b[kind]


def context(dds, p, z_lanes=None, fp16=False):
    g = p.geom
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    if z_lanes is not None:
        ctx.set_option(dds.DDS_OPT_Z_LANES, z_lanes)
    if fp16:
        ctx.set_option(dds.DDS_OPT_SPECTRA_FP16, 1)
    return ctx.build_kernels()


CASES = [   # (nx, ny, nz), families, expected (pz, fields), seed
    ((12, 8, 40), [0], (128, 1), 31),
    ((10, 9, 64), [0, 9], (128, 2), 32),                    # nz = pz / 2
    ((9, 8, 33), [0, 7, 8], (128, 3), 33),                  # odd nx, smallest nz of pz 128
    ((8, 7, 65), [0, 1, 2, 9, 10], (256, 4), 34),           # smallest nz of pz 256
    ((6, 8, 100), list(range(18)), (256, 5), 35),
    ((7, 6, 128), "six", (256, 6), 36),                     # nz = pz / 2, six fields
    ((17, 5, 50), [1, 4, 6, 13, 17], (128, 5), 37),         # M = 32, odd nx
    ((5, 16, 71), "six", (256, 6), 38),
]


@pytest.mark.parametrize("shape,fams,expect,seed", CASES)
def test_tall_grids_vs_direct_sum(dds, shape, fams, expect, seed):
    g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6)
    p = W.random_problem(g, *families(fams), seed=seed)
    ctx = context(dds, p)
    q = ctx.query()
    assert (q["pz"], q["n_fields"]) == expect
    rho = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    got = ctx.stress(rho).cpu().numpy()
    ref = oracle.stress_direct(g, p.t, p.b, p.rho).T
    assert rel_l2_per_component(got, ref).max() <= TOL_STRESS
    # the shared-memory schedule of the same pass: the same result up to FP32 rounding
    other = context(dds, p, z_lanes=-1)
    alt = other.stress(rho).cpu().numpy()
    assert rel_l2_per_component(alt, got).max() <= 1e-6
    # a batch of two density sets: each equals its single evaluation
    rho2 = torch.stack([rho, torch.flip(rho, dims=[3])]).contiguous()
    s2 = ctx.stress_multi(rho2).cpu().numpy()
    assert rel_l2_per_component(s2[0], got).max() <= 1e-6
    assert rel_l2_per_component(s2[1], ctx.stress(rho2[1].clone()).cpu().numpy()).max() <= 1e-6
    ctx.close()
    other.close()


@pytest.mark.parametrize("shape,fams,expect,seed", [CASES[1], CASES[4], CASES[5]])
def test_tall_grids_fp16_spectra_and_bf16_densities(dds, shape, fams, expect, seed):
    g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6)
    p = W.random_problem(g, *families(fams), seed=seed)
    ref = oracle.stress_direct(g, p.t, p.b, p.rho).T
    ctx = context(dds, p, fp16=True)
    assert (ctx.query()["pz"], ctx.query()["n_fields"]) == expect
    got = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2_per_component(got, ref).max() <= 5e-4            # FP16 spectra bound
    ctx.close()
    ctx = context(dds, p)
    got = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda().to(torch.bfloat16)).cpu().numpy()
    rho16 = torch.from_numpy(p.rho.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    exact = oracle.stress_direct(g, p.t, p.b, rho16).T
    assert rel_l2_per_component(got, exact).max() <= TOL_STRESS
    ctx.close()


def test_three_stage_schedule_is_selectable_and_checked(dds):
    # DDS_OPT_Z_LANES = -2 forces the three-stage kernel; grids it cannot take are refused
    g = W.Geometry(8, 8, 40, 0.2e-6, 0.2e-6, 0.05e-6)
    p = W.random_problem(g, *families([0, 9]), seed=40)
    forced = context(dds, p, z_lanes=-2)
    auto = context(dds, p)
    rho = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    assert np.array_equal(forced.stress(rho).cpu().numpy(), auto.stress(rho).cpu().numpy())
    forced.close()
    auto.close()
    flat = W.random_problem(W.Geometry(8, 8, 8, 0.2e-6, 0.2e-6, 0.05e-6), *families([0, 9]), seed=41)
    ctx = dds.StressContext(0)
    g = flat.geom
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(flat.t, flat.b)
    ctx.set_option(dds.DDS_OPT_Z_LANES, -2)
    with pytest.raises(dds.DDSError) as e:
        ctx.build_kernels()
    assert e.value.code == dds.DDS_ERR_UNSUPPORTED
    ctx.close()
