"""GPU parity of the in-plane periodic boundary conditions (Sec. 4, Eq. 12-13).

With n replica shells every coefficient is the sum over the replicas of the source
cell displaced by (k Lx, l Ly, 0), |k|, |l| <= n.  The FP64 table entries match the
oracle's replica sums to 1e-12 of each component's largest magnitude; FP32 stresses
match the oracle's direct sum with the same replica coefficients to a relative L2
error of 1e-5 per component.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_TABLE = 1e-12
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
    return np.array([np.linalg.norm(got[c] - ref[c]) / max(np.linalg.norm(ref[c]), 1e-6 * scale)
                     for c in range(6)])


def all_offsets(g):
    k, j, i = np.meshgrid(np.arange(-(g.nz - 1), g.nz), np.arange(-(g.ny - 1), g.ny),
                          np.arange(-(g.nx - 1), g.nx), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)


@pytest.mark.parametrize("shape,cells,n_shells", [
    ((6, 5, 4), (0.2e-6, 0.2e-6, 0.05e-6), 2),     # subdivided near field inside the system
    ((2, 2, 3), (0.2e-6, 0.2e-6, 0.05e-6), 3),     # replicas themselves fall in the near field
    ((5, 7, 2), (1e-6, 1e-6, 0.25e-6), 4),
])
def test_replica_table_matches_oracle(dds, shape, cells, n_shells):
    g = W.Geometry(*shape, *cells)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, n_shells)
    ijk = all_offsets(g)
    t_all, b_all = W.gan_families()
    for f in (0, 9):
        got = ctx.table_at(t_all[f], b_all[f], ijk)
        ref = np.array([oracle.interaction_pbc(g, *o, t_all[f], b_all[f], n_shells) for o in ijk])
        for c in range(6):
            assert np.abs(got[:, c] - ref[:, c]).max() <= TOL_TABLE * np.abs(ref[:, c]).max(), (f, c)
    ctx.close()


@pytest.mark.parametrize("shape,cells,fams,n_shells,seed", [
    ((12, 10, 6), (0.2e-6, 0.2e-6, 0.05e-6), [0, 8, 13], 4, 1),
    ((9, 16, 5), (1e-6, 1e-6, 0.25e-6), [2, 5], 6, 2),
    ((16, 16, 4), (0.5e-6, 0.5e-6, 0.2e-6), list(range(18)), 2, 3),
])
def test_periodic_stress_matches_oracle(dds, shape, cells, fams, n_shells, seed):
    g = W.Geometry(*shape, *cells)
    t, b = W.gan_families()
    p = W.random_problem(g, t[fams], b[fams], seed=seed)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, n_shells).build_kernels()
    sigma = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda())
    got = sigma.cpu().numpy()
    ctx.close()
    ref = oracle.stress_direct(g, p.t, p.b, p.rho, n_shells=n_shells).T
    assert rel_l2_per_component(got, ref).max() <= TOL_STRESS


def test_periodic_stress_equals_open_stress_of_the_tiled_system(dds):
    # Eq. 12-13 by construction: with n shells, the periodic stress in the system is
    # the open-boundary stress, on the central tile, of (2n+1) x (2n+1) copies of the
    # system laid side by side (a size the oracle would take minutes for).
    g = W.Geometry(32, 24, 8, 0.2e-6, 0.2e-6, 0.05e-6)
    n = 2
    t, b = W.gan_families()
    p = W.random_problem(g, t[[1, 10]], b[[1, 10]], seed=11)
    rho = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, n).build_kernels()
    got = ctx.stress(rho).cpu().numpy()
    ctx.close()
    r = 2 * n + 1
    tiled = rho.repeat(1, 1, r, r).contiguous()
    big = dds.StressContext(0)
    big.set_geometry(r * g.nx, r * g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    big.build_kernels()
    ref = big.stress(tiled).cpu().numpy()[:, :, n * g.ny:(n + 1) * g.ny, n * g.nx:(n + 1) * g.nx]
    big.close()
    assert rel_l2_per_component(got, ref).max() <= TOL_STRESS


def test_shell_option_validation(dds):
    ctx = dds.StressContext(0)
    ctx.set_geometry(4, 4, 2, 1e-6, 1e-6, 0.25e-6, W.MU_GAN, W.NU_GAN)
    for bad in (-1, 2.5, 1e6):
        with pytest.raises(RuntimeError):
            ctx.set_option(dds.DDS_OPT_PBC_SHELLS, bad)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, 0)
    ctx.close()


def test_replica_table_sampled_at_full_size(dds):
    # the GaN layer's geometry with two replica shells, sampled offsets (far, near, corners)
    g = W.Geometry(256, 256, 128, 0.2e-6, 0.2e-6, 0.05e-6)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, 2)
    rng = np.random.default_rng(5)
    ijk = np.concatenate([rng.integers(-255, 256, size=(40, 2)), rng.integers(-127, 128, size=(40, 1))], axis=1)
    ijk = np.concatenate([ijk, rng.integers(-3, 4, size=(20, 3)),
                          np.array([[255, 255, 127], [-255, 0, 0], [0, 0, 0], [0, -255, 1]])])
    t_all, b_all = W.gan_families()
    for f in (4, 13):
        got = ctx.table_at(t_all[f], b_all[f], ijk)
        ref = np.array([oracle.interaction_pbc(g, *o, t_all[f], b_all[f], 2) for o in ijk])
        for c in range(6):
            assert np.abs(got[:, c] - ref[:, c]).max() <= TOL_TABLE * np.abs(ref[:, c]).max(), (f, c)
    ctx.close()


# ------------------------------------------------ periodic reading (option) --
def periodic_context(dds, p, n_shells):
    g = p.geom
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, n_shells).set_option(dds.DDS_OPT_PBC_PERIODIC, 1)
    return ctx


def test_periodic_table_matches_oracle(dds):
    g = W.Geometry(8, 6, 3, 0.2e-6, 0.2e-6, 0.05e-6)       # ties at half a period in x and y
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
    ctx.set_option(dds.DDS_OPT_PBC_SHELLS, 3).set_option(dds.DDS_OPT_PBC_PERIODIC, 1)
    ijk = all_offsets(g)
    t_all, b_all = W.gan_families()
    for f in (0, 9):
        got = ctx.table_at(t_all[f], b_all[f], ijk)
        ref = np.array([oracle.interaction_periodic(g, *o, t_all[f], b_all[f], 3) for o in ijk])
        for c in range(6):
            scale = np.abs(ref[:, c]).max()
            if scale > 0:
                assert np.abs(got[:, c] - ref[:, c]).max() <= TOL_TABLE * scale, (f, c)
    ctx.close()


@pytest.mark.parametrize("shape,fams,n_shells", [
    ((24, 32, 6), [0, 9], 3),                 # ragged x (still padded), y periodic
    ((17, 64, 4), [1, 2, 9, 14], 2),
    ((32, 32, 40), list(range(18)), 2),       # padded z 128: the three-stage z pass
])
def test_periodic_stress_matches_oracle(dds, shape, fams, n_shells):
    t18, b18 = W.gan_families()
    g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6)
    p = W.random_problem(g, t18[fams], b18[fams], seed=70 + n_shells)
    ctx = periodic_context(dds, p, n_shells).build_kernels()
    q = ctx.query()
    assert q["py"] == g.ny                      # unpadded in y
    rho = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    got = ctx.stress(rho).cpu().numpy()
    tg = np.arange(g.n_cells) if g.n_cells <= 5000 else np.random.default_rng(1).integers(0, g.n_cells, 600)
    ref = oracle.stress_direct(g, p.t, p.b, p.rho, targets=tg, n_shells=n_shells, periodic=True).T
    assert rel_l2_per_component(got.reshape(6, -1)[:, tg], ref).max() <= TOL_STRESS
    # a cyclic convolution: shifting rho cyclically in x and y shifts sigma
    sh = torch.roll(rho, shifts=(5, 3), dims=(2, 3)).contiguous()
    got2 = ctx.stress(sh).cpu().numpy()
    assert rel_l2_per_component(got2, np.roll(got, (5, 3), axis=(2, 3))).max() <= TOL_STRESS
    ctx.close()


def test_periodic_reading_meets_the_other_at_the_papers_shell_count(dds):
    # Sec. 4 / Fig. 7: 15-20 shells bring every coefficient within 3% of the shell limit.
    # Both readings share that limit, so at 20 shells their device coefficients agree within
    # twice the 3% band (the stresses of a random density differ more: each reading cuts the
    # slowly converging image sum at a different last ring).
    g = W.Geometry(16, 16, 8, 1e-6, 1e-6, 1e-6)
    rng = np.random.default_rng(3)
    ijk = np.stack([rng.integers(0, 16, 40), rng.integers(0, 16, 40), rng.integers(-7, 8, 40)], axis=1)
    t_all, b_all = W.gan_families()
    tabs = []
    for periodic in (1, 0):
        ctx = dds.StressContext(0)
        ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
        ctx.set_option(dds.DDS_OPT_PBC_SHELLS, 20).set_option(dds.DDS_OPT_PBC_PERIODIC, periodic)
        tabs.append([ctx.table_at(t_all[f], b_all[f], ijk) for f in (0, 9)])
        ctx.close()
    for a, b in zip(*tabs):
        for c in range(6):
            scale = max(np.abs(a[:, c]).max(), np.abs(b[:, c]).max())
            if scale > 1e-12 * max(np.abs(a).max(), 1e-300):
                assert np.abs(a[:, c] - b[:, c]).max() <= 2 * 0.03 * scale, c


def test_periodic_reading_refuses_unsuitable_grids(dds):
    t18, b18 = W.gan_families()
    for shape, shells, code in (((16, 48, 4), 2, "UNSUPPORTED"), ((16, 32, 4), 0, "INVALID_ARG")):
        g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6)
        p = W.random_problem(g, t18[[0]], b18[[0]], seed=1)
        ctx = periodic_context(dds, p, shells)
        with pytest.raises(dds.DDSError) as e:
            ctx.build_kernels()
        assert e.value.code == getattr(dds, "DDS_ERR_" + code)
        ctx.close()
