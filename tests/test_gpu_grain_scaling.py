"""Grain-size scaling of the stress fluctuations (Sec. 6.4-6.5, Eqs. 21-27) on the GPU path.

One periodic columnar grain pattern (100 grains on a square of side 10 D, vertical
edge dislocations with a per-grain in-plane Burgers vector, height-independent
density) is scaled with the grain size D at a fixed layer thickness H, evaluated with
in-plane periodic boundary conditions, and the in-plane standard deviation of each
stress component is taken over the middle layers.  The paper's shell model predicts

  * tall grains (H >> D): the decay power m = 1 of Eq. 22 and s_tot ~ D (Eq. 27);
  * flat grains (H << D): m = 2 and s_tot independent of D (Eq. 26).

The fitted exponents of s(D) must match: 1 within 0.05 for tall, 0 within 0.05 for
flat layers.  (Tall layers use far-field cells only: at H/D ~ 10^3 every offset would
be near and the subdivision would dominate the run time without affecting the law.)
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UM = 1e-6


@pytest.fixture(scope="module")
def dds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_01830_gb300 as mod
    mod.load_library()
    return mod


def fluctuations(dds, p, shells, n_near=None):
    """In-plane standard deviation of each component, averaged over the middle layers."""
    g = p.geom
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, shells)
    if n_near is not None:
        ctx.set_option(dds.DDS_OPT_NEAR_RADIUS, n_near)
    ctx.build_kernels()
    sig = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda())
    s = sig.double().reshape(6, g.nz, -1).std(dim=2).cpu().numpy()
    ctx.close()
    k0 = g.nz // 4
    k1 = max(k0 + 1, 3 * g.nz // 4)
    return s[:, k0:k1].mean(axis=1)


def exponents(dds, n, nz, H, Ds, n_near=None):
    s = np.array([fluctuations(dds, W.scaled_polycrystal(n, nz, D, H), shells=2, n_near=n_near) for D in Ds])
    return {c: np.polyfit(np.log(Ds), np.log(s[:, i]), 1)[0] for i, c in ((0, "xx"), (1, "yy"), (3, "xy"), (2, "zz"))}


def test_tall_grains_fluctuate_in_proportion_to_grain_size(dds):
    ex = exponents(dds, 64, 8, 2000 * UM, [1 * UM, 2 * UM, 4 * UM], n_near=0.0)
    for c, e in ex.items():
        assert abs(e - 1.0) <= 0.05, (c, e)


def test_flat_grains_fluctuate_independently_of_grain_size(dds):
    ex = exponents(dds, 64, 2, 0.2 * UM, [10 * UM, 20 * UM, 40 * UM])
    for c, e in ex.items():
        assert abs(e) <= 0.05, (c, e)
