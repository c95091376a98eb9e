"""dds_stress_subset: one context (one set of kernel spectra per geometry, Sec. 2.3) serves
any subset of its families, because Eq. 3b sums over the families present and the
coefficients are linear in b.  Checked against the FP64 direct sum of Eq. 10 over the
subset's families alone, and against dds_stress_multi with the absent families' densities
set to zero (same arithmetic)."""
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


@pytest.mark.parametrize("shape,fams,seed", [
    ((24, 20, 12), [3], 51),                 # one edge family of the 18
    ((17, 9, 40), [0, 13], 52),              # edge + mixed, padded z 128 (three-stage z pass)
    ((12, 14, 70), [2, 5, 8, 17], 53),       # padded z 256
    ((31, 7, 5), [16, 1, 9], 54),            # unordered indices
])
def test_subset_of_the_gan_families(dds, shape, fams, seed):
    t18, b18 = W.gan_families()
    g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(t18, b18).build_kernels()
    p = W.random_problem(g, t18[fams], b18[fams], seed=seed)
    rho = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    got = ctx.stress_subset(fams, rho).cpu().numpy()
    ref = oracle.stress_direct(g, p.t, p.b, p.rho).T
    assert rel_l2_per_component(got, ref).max() <= TOL_STRESS
    # the full-context evaluation with zeros for the absent families
    full = torch.zeros((1, 18) + g.shape, dtype=torch.float32, device="cuda")
    full[0, fams] = rho
    alt = ctx.stress_multi(full)[0].cpu().numpy()
    assert rel_l2_per_component(got, alt).max() <= 1e-6
    # a batch of two sets with the same subset
    rho2 = torch.stack([rho, 0.5 * torch.flip(rho, dims=[1])]).contiguous()
    s2 = ctx.stress_subset(fams, rho2).cpu().numpy()
    assert rel_l2_per_component(s2[0], got).max() <= 1e-6
    assert rel_l2_per_component(s2[1], ctx.stress_subset(fams, rho2[1].clone()).cpu().numpy()).max() <= 1e-6
    ctx.close()


def test_subset_rejects_bad_indices(dds):
    t18, b18 = W.gan_families()
    g = W.Geometry(8, 8, 4, 0.2e-6, 0.2e-6, 0.05e-6)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(t18, b18).build_kernels()
    rho = torch.zeros((2,) + g.shape, device="cuda")
    for fams in ([0, 0], [0, 18], [-1, 2]):
        with pytest.raises(dds.DDSError) as e:
            ctx.stress_subset(fams, rho)
        assert e.value.code == dds.DDS_ERR_INVALID_ARG
    ctx.close()
