"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: the FP64 coefficient table matches the oracle's to 1e-12 of each
component's largest magnitude; FP32 stresses match the FP64 direct sum of Eq. 10
to a relative L2 error of 1e-5 per component (denominator max(||sigma_c||,
1e-6 max_c' ||sigma_c'||)).
"""
import math

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
    out = []
    for c in range(6):
        den = max(np.linalg.norm(ref[c]), 1e-6 * scale)
        out.append(np.linalg.norm(got[c] - ref[c]) / den)
    return np.array(out)


def gpu_stress(dds, p, dtype=torch.float32, n_near=None, fp16_spectra=False):
    ctx = dds.StressContext(0)
    g = p.geom
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    if n_near is not None:
        ctx.set_option(dds.DDS_OPT_NEAR_RADIUS, n_near)
    if fp16_spectra:
        ctx.set_option(dds.DDS_OPT_SPECTRA_FP16, 1)
    ctx.build_kernels()
    rho = torch.from_numpy(p.rho.astype(np.float32)).to("cuda", dtype=dtype).contiguous()
    sigma = ctx.stress(rho)
    torch.cuda.synchronize()
    out = sigma.cpu().numpy()
    ctx.close()
    return out


def all_offsets(g):
    k, j, i = np.meshgrid(np.arange(-(g.nz - 1), g.nz), np.arange(-(g.ny - 1), g.ny),
                          np.arange(-(g.nx - 1), g.nx), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)


# ------------------------------------------------------------ table (P11) --
@pytest.mark.parametrize("cells", [(1e-6, 1e-6, 0.25e-6), (0.5e-6, 0.5e-6, 0.2e-6), (0.2e-6, 0.2e-6, 0.02e-6)])
def test_fp64_table_matches_oracle(dds, cells):
    g = W.Geometry(12, 10, 7, *cells)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
    ijk = all_offsets(g)
    t_all, b_all = W.gan_families()
    for t, b in [(t_all[0], b_all[0]), (t_all[9], b_all[9]),
                 ([0.0, 0.5, math.sqrt(3) / 2], [W.A_LATT / 2, math.sqrt(3) * W.A_LATT / 2, W.C_LATT])]:
        got = ctx.table_at(t, b, ijk).reshape(2 * g.nz - 1, 2 * g.ny - 1, 2 * g.nx - 1, 6)
        ref = oracle.gtable(g, t, b)
        for c in range(6):
            m = np.abs(ref[..., c]).max()
            assert np.abs(got[..., c] - ref[..., c]).max() <= TOL_TABLE * m, c
    ctx.close()


def test_fp64_table_sampled_at_full_size(dds):
    g = W.Geometry(256, 256, 128, 0.2e-6, 0.2e-6, 0.05e-6)
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
    rng = np.random.default_rng(0)
    ijk = np.concatenate([rng.integers(-255, 256, size=(200, 3)) * np.array([1, 1, 0]) +
                          rng.integers(-127, 128, size=(200, 1)) * np.array([0, 0, 1]),
                          rng.integers(-4, 5, size=(100, 3)),
                          np.array([[255, 255, 127], [-255, -255, -127], [0, 0, 0], [0, 0, 1]])])
    t_all, b_all = W.gan_families()
    for f in (2, 11):
        got = ctx.table_at(t_all[f], b_all[f], ijk)
        ref = np.array([oracle.interaction(g, *o, t_all[f], b_all[f]) for o in ijk])
        for c in range(6):
            assert np.abs(got[:, c] - ref[:, c]).max() <= TOL_TABLE * np.abs(ref[:, c]).max()
    ctx.close()


# ------------------------------------------------------ stress vs oracle ---
def test_gaussian_disk_32_full(dds):
    p = W.gaussian_disk_32()
    got = gpu_stress(dds, p)
    ref = oracle.stress_direct(p.geom, p.t, p.b, p.rho).T
    assert rel_l2_per_component(got, ref).max() <= TOL_STRESS


@pytest.mark.parametrize("shape,cells,fams,seed", [
    ((40, 24, 10), (0.2e-6, 0.2e-6, 0.05e-6), list(range(18)), 1),     # ragged sizes, all 18 families
    ((33, 17, 9), (1e-6, 1e-6, 0.25e-6), [0, 7, 8], 2),                  # odd nx, one field per family
    ((16, 64, 3), (0.5e-6, 0.5e-6, 0.2e-6), [1, 4, 6, 13, 17], 3),
    ((64, 16, 16), (0.3e-6, 0.3e-6, 0.3e-6), [5, 10], 4),                # cubic cells (no subdivision)
    ((7, 1, 1), (1e-6, 1e-6, 1e-6), [3, 12], 6),                         # a single line
    ((101, 12, 4), (0.2e-6, 0.2e-6, 0.05e-6), [0, 9], 7),                 # M = 128, odd nx
    ((128, 9, 3), (0.5e-6, 0.5e-6, 0.2e-6), [4, 11, 16], 8),              # M = 128, full half line
    ((129, 6, 3), (0.2e-6, 0.2e-6, 0.05e-6), [2], 9),                     # M = 256, odd nx, one family
    ((250, 5, 2), (1e-6, 1e-6, 0.25e-6), [1, 6, 12], 10),                 # M = 256
    ((300, 3, 2), (0.5e-6, 0.5e-6, 0.2e-6), [7, 14], 11),                 # M = 512
    ((17, 5, 4), (0.2e-6, 0.2e-6, 0.05e-6), [5], 12),                     # M = 32, odd nx, one family
    ((244, 7, 3), (0.2e-6, 0.2e-6, 0.05e-6), [0, 3, 9, 14], 13),          # M = 256, 4-value loads, summed
    ((12, 9, 5), (1e-6, 1e-6, 0.25e-6), [6], 14),                         # M = 16, 4-value loads
])
def test_random_densities_vs_direct_sum(dds, shape, cells, fams, seed):
    g = W.Geometry(*shape, *cells)
    t, b = W.gan_families()
    p = W.random_problem(g, t[fams], b[fams], seed=seed)
    got = gpu_stress(dds, p)
    ref = oracle.stress_direct(g, p.t, p.b, p.rho).T
    assert rel_l2_per_component(got, ref).max() <= TOL_STRESS


def test_single_cell_has_only_the_vanishing_self_term(dds):
    # Sec. 2.3: the self-interaction coefficient vanishes; one cell alone gives sigma = 0
    g = W.Geometry(1, 1, 1, 1e-6, 1e-6, 0.25e-6)
    t, b = W.gan_families()
    p = W.random_problem(g, t[[0, 9]], b[[0, 9]], seed=5)
    got = gpu_stress(dds, p)
    scale = g.mu * W.A_LATT * p.rho.max() * g.dz          # natural stress scale of one cell
    assert np.abs(got).max() <= 1e-9 * scale


def test_near_radius_option(dds):
    g = W.Geometry(20, 18, 12, 0.2e-6, 0.2e-6, 0.05e-6)
    t, b = W.gan_families()
    p = W.random_problem(g, t[[0, 8]], b[[0, 8]], seed=9)
    for n_near in (0.0, 5.0):
        got = gpu_stress(dds, p, n_near=n_near)
        ref = oracle.stress_direct(g, p.t, p.b, p.rho, n_near=n_near).T
        assert rel_l2_per_component(got, ref).max() <= TOL_STRESS


def sample_targets(g, n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, g.n_cells, size=n)
    corners = [0, g.n_cells - 1, g.nx - 1, (g.ny - 1) * g.nx, (g.nz - 1) * g.nx * g.ny]
    return np.unique(np.concatenate([pts, corners]))


def x_line(g, y, z):
    """Linear indices of the full x-line at (y, z)."""
    return z * g.nx * g.ny + y * g.nx + np.arange(g.nx)


def test_radial_disk_512_sampled(dds):
    # 96 random cells, the corners, and one full x-line through the disk centre
    p = W.radial_disk_512()
    got = gpu_stress(dds, p).reshape(6, -1)
    g = p.geom
    tg = np.unique(np.concatenate([sample_targets(g, 96, seed=1), x_line(g, g.ny // 2, g.nz // 2)]))
    ref = oracle.stress_direct(g, p.t, p.b, p.rho, targets=tg, use_table=False).T
    assert rel_l2_per_component(got[:, tg], ref).max() <= TOL_STRESS


def test_gan_layer_256_sampled(dds):
    # 48 random cells, the corners, and one full x-line in the dense bottom layers
    p = W.gan_layer_256(0)
    got = gpu_stress(dds, p).reshape(6, -1)
    g = p.geom
    tg = np.unique(np.concatenate([sample_targets(g, 48, seed=2), x_line(g, 101, 3)]))
    ref = oracle.stress_direct(g, p.t, p.b, p.rho, targets=tg, use_table=False).T
    assert rel_l2_per_component(got[:, tg], ref).max() <= TOL_STRESS


@pytest.mark.parametrize("r", [3, 5])
def test_sweep_realisation_sampled(dds, r):
    # the grain-size sweep (grid and grain diameter drawn per realisation), FP32 and BF16
    # densities; BF16 against the oracle on the bf16-rounded densities
    p = W.sweep_realisation(r)
    g = p.geom
    tg = np.unique(np.concatenate([sample_targets(g, 24, seed=r), x_line(g, g.ny // 3, 1)[::4]]))
    got = gpu_stress(dds, p).reshape(6, -1)
    ref = oracle.stress_direct(g, p.t, p.b, p.rho, targets=tg, use_table=False).T
    assert rel_l2_per_component(got[:, tg], ref).max() <= TOL_STRESS
    got16 = gpu_stress(dds, p, dtype=torch.bfloat16).reshape(6, -1)
    rho16 = torch.from_numpy(p.rho.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    t16 = tg[::3]
    ref16 = oracle.stress_direct(g, p.t, p.b, rho16, targets=t16, use_table=False).T
    assert rel_l2_per_component(got16[:, t16], ref16).max() <= TOL_STRESS


@pytest.mark.parametrize("grid,aspect,fam", [(0, 0, (3, 11)), (1, 1, (0,)), (3, 2, (1, 4, 8, 15)), (2, 0, (6, 7, 17))])
def test_serving_requests_sampled(dds, grid, aspect, fam):
    # requests of the serving mix: grid, cell aspect dz/dx, a subset of the 18 families,
    # evaluated as the server does -- one context of all 18 families per geometry
    a = W.ServingArrival(0.0, grid, aspect, fam, seed=11)
    c = W.serving_problem(a)
    g = c.geom
    ctx = dds.StressContext(0)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(c.t, c.b).build_kernels()
    got = ctx.stress_subset(list(fam), torch.from_numpy(np.ascontiguousarray(c.rho)).cuda()).cpu().numpy()
    ctx.close()
    got = got.reshape(6, -1)
    tg = np.unique(np.concatenate([sample_targets(g, 24, seed=7), x_line(g, g.ny // 2, 0)[::4]]))
    ref = oracle.stress_direct(g, c.t[list(fam)], c.b[list(fam)], c.rho.astype(np.float64), targets=tg,
                               use_table=False).T
    assert rel_l2_per_component(got[:, tg], ref).max() <= TOL_STRESS


# ------------------------------------------------------------- properties ---
def test_linearity_at_full_size(dds):
    p = W.gan_layer_256(0)
    ctx = dds.context_for(p)
    r1 = torch.from_numpy(p.rho.astype(np.float32)).cuda()
    r2 = torch.flip(r1, dims=[2]).contiguous()
    s1 = ctx.stress(r1).double()
    s2 = ctx.stress(r2).double()
    s12 = ctx.stress((2.0 * r1 - 0.5 * r2).contiguous()).double()
    torch.cuda.synchronize()
    lhs = (s12 - (2.0 * s1 - 0.5 * s2)).cpu().numpy().reshape(6, -1)
    ref = (2.0 * s1 - 0.5 * s2).cpu().numpy().reshape(6, -1)
    assert rel_l2_per_component(lhs + ref, ref).max() <= 1e-5
    ctx.close()


@pytest.mark.parametrize("shape,fams", [((24, 20, 8), [0, 9]),              # one family per group
                                        ((33, 10, 5), [0, 1, 2, 9, 10]),     # summed families, odd nx
                                        ((200, 6, 3), [0, 1, 9, 10]),        # M = 256, 4-value loads
                                        ((48, 10, 4), [2, 9])])              # M = 64, 4-value loads
def test_bf16_density_storage(dds, shape, fams):
    p = W.random_problem(W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6), *[a[fams] for a in W.gan_families()],
                         seed=11)
    got = gpu_stress(dds, p, dtype=torch.bfloat16)
    rho_bf16 = torch.from_numpy(p.rho.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    exact = oracle.stress_direct(p.geom, p.t, p.b, rho_bf16).T
    assert rel_l2_per_component(got, exact).max() <= TOL_STRESS     # exact on bf16-rounded densities
    full = oracle.stress_direct(p.geom, p.t, p.b, p.rho).T
    assert rel_l2_per_component(got, full).max() <= 4e-3            # bf16 rounding of rho: 2^-8 relative


# ---------------------------------------------------------- API surfaces ---
def test_host_entry_point_matches_device_entry_point(dds):
    p = W.gaussian_disk_32()
    ctx = dds.context_for(p)
    dev = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda()).cpu().numpy()
    host = ctx.stress_host(p.rho.astype(np.float32))
    assert np.array_equal(dev, host)
    ctx.close()


def test_pipelined_host_calls_match_device_calls(dds):
    # five calls in flight through the two staging sets, each with its own densities and
    # result buffer: every result equals the device-buffer evaluation of its densities
    p = W.random_problem(W.Geometry(96, 80, 40, 0.2e-6, 0.2e-6, 0.05e-6),
                         *[a[[0, 1, 9, 12]] for a in W.gan_families()], seed=8)
    ctx = dds.context_for(p)
    base = p.rho.astype(np.float32)
    rhos = [np.ascontiguousarray(base * (1.0 + 0.25 * k) if k % 2 == 0 else base[:, :, :, ::-1] * (1.0 + 0.1 * k))
            for k in range(5)]
    rhos = [torch.from_numpy(r).pin_memory().numpy() for r in rhos]
    outs = [torch.empty((6,) + p.geom.shape, dtype=torch.float32).pin_memory().numpy() for _ in rhos]
    for r, o in zip(rhos, outs):
        ctx.stress_host_async(r, o)
    ctx.stress_host_sync()
    for r, o in zip(rhos, outs):
        dev = ctx.stress(torch.from_numpy(r).cuda()).cpu().numpy()
        assert np.array_equal(dev, o)
    ctx.close()


def test_batched_matches_single_calls(dds):
    probs = [W.gaussian_disk_32(), W.random_problem(W.Geometry(20, 12, 6, 0.5e-6, 0.5e-6, 0.2e-6),
                                                    *[a[[2, 3, 14]] for a in W.gan_families()], seed=3)]
    ctxs = [dds.context_for(p) for p in probs]
    rhos = [torch.from_numpy(p.rho.astype(np.float32)).cuda() for p in probs]
    singles = [c.stress(r).cpu().numpy() for c, r in zip(ctxs, rhos)]
    outs = [torch.empty((6,) + c.shape, device="cuda") for c in ctxs]
    dds.dds_stress_batched([c.handle for c in ctxs], [r.data_ptr() for r in rhos], [dds.DDS_F32] * 2,
                           [o.data_ptr() for o in outs])
    torch.cuda.synchronize()
    for s, o in zip(singles, outs):
        assert np.array_equal(s, o.cpu().numpy())
    for c in ctxs:
        c.close()


def test_error_codes(dds):
    ctx = dds.StressContext(0)
    with pytest.raises(dds.DDSError) as ei:
        ctx.build_kernels()
    assert ei.value.code == dds.DDS_ERR_NOT_READY
    with pytest.raises(dds.DDSError) as ei:
        ctx.set_geometry(0, 4, 4, 1e-6, 1e-6, 1e-6, 1e9, 0.3)
    assert ei.value.code == dds.DDS_ERR_INVALID_ARG
    with pytest.raises(dds.DDSError) as ei:
        ctx.set_geometry(1024, 4, 4, 1e-6, 1e-6, 1e-6, 1e9, 0.3)
    assert ei.value.code == dds.DDS_ERR_UNSUPPORTED
    ctx.set_geometry(8, 8, 4, 1e-6, 1e-6, 1e-6, 1e9, 0.3)
    with pytest.raises(dds.DDSError) as ei:
        ctx.set_families([[0, 0, 0]], [[1e-10, 0, 0]])
    assert ei.value.code == dds.DDS_ERR_INVALID_ARG
    ctx.set_families([[0, 0, 1]], [[1e-10, 0, 0]])
    rho = torch.zeros((1, 4, 8, 8), device="cuda")
    with pytest.raises(dds.DDSError) as ei:
        ctx.stress(rho)
    assert ei.value.code == dds.DDS_ERR_NOT_READY
    ctx.build_kernels()
    assert float(ctx.stress(rho).abs().max()) == 0.0
    assert ctx.launches_per_stress == 5
    ctx.close()


# ------------------------------------------------------ reduced storage ----
TOL_FP16_SPECTRA = 5e-4     # stated bound of the FP16 kernel-spectrum storage mode


@pytest.mark.parametrize("case", ["gaussian_disk", "polycrystal_small"])
def test_fp16_spectra_within_stated_bound(dds, case):
    if case == "gaussian_disk":
        p = W.gaussian_disk_32()                                       # register z pass
    else:
        p = W.gan_polycrystal(W.Geometry(40, 32, 24, 0.2e-6, 0.2e-6, 0.05e-6), 1e-6, seed=7)  # 5 fields
    got = gpu_stress(dds, p, fp16_spectra=True)
    ref = oracle.stress_direct(p.geom, p.t, p.b, p.rho).T
    err = rel_l2_per_component(got, ref).max()
    print(f"FP16 spectra, {case}: rel-L2 {err:.2e}")
    assert err <= TOL_FP16_SPECTRA
    full = gpu_stress(dds, p)
    assert rel_l2_per_component(full, ref).max() <= TOL_STRESS


# ------------------------------------------------------------- batches -----
@pytest.mark.parametrize("case", ["thin", "tall"])
def test_multi_matches_single_evaluations(dds, case):
    if case == "thin":          # register z pass
        g = W.Geometry(64, 48, 16, 0.5e-6, 0.5e-6, 0.2e-6)
        t, b = W.gan_families()
        probs = [W.random_problem(g, t[[0, 9]], b[[0, 9]], seed=40 + i) for i in range(3)]
    else:                       # shared-memory z pass, 5 fields
        g = W.Geometry(32, 32, 40, 0.2e-6, 0.2e-6, 0.05e-6)
        probs = [W.gan_polycrystal(g, 1e-6, seed=50 + i) for i in range(3)]
    ctx = dds.context_for(probs[0])
    rhos = torch.stack([torch.from_numpy(np.ascontiguousarray(p.rho, dtype=np.float32)) for p in probs]).cuda()
    multi = ctx.stress_multi(rhos)
    singles = [ctx.stress(rhos[i].contiguous()) for i in range(len(probs))]
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert rel_l2_per_component(multi[i].cpu().numpy(), singles[i].cpu().numpy()).max() <= 1e-6
    ref = oracle.stress_direct(g, probs[1].t, probs[1].b, probs[1].rho).T
    assert rel_l2_per_component(multi[1].cpu().numpy(), ref).max() <= TOL_STRESS
    ctx.close()


# ---------------------------------------------------- Eq. 20 statistics ----
def plane_rms(sig):
    """Eq. 20: s_c(h_k) = sqrt(mean over the (x, y) plane of sigma_c^2), shape (6, nz)."""
    sig = np.asarray(sig, np.float64)
    return np.sqrt((sig ** 2).mean(axis=(-1, -2)))


def test_eq20_statistics_fused_into_the_evaluation(dds):
    p = W.gan_polycrystal(W.Geometry(40, 32, 24, 0.2e-6, 0.2e-6, 0.05e-6), 1e-6, seed=8)
    ctx = dds.context_for(p)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho, dtype=np.float32)).cuda()
    sig, s = ctx.stress_stats(rho)
    torch.cuda.synchronize()
    sig = sig.cpu().numpy()
    s = s.cpu().numpy()
    assert s.shape == (6, p.geom.nz)
    assert np.abs(s - plane_rms(sig)).max() <= 1e-6 * np.abs(s).max()
    ref = oracle.stress_direct(p.geom, p.t, p.b, p.rho).T.reshape(6, p.geom.nz, p.geom.ny, p.geom.nx)
    s_ref = plane_rms(ref)
    for c in range(6):
        assert np.linalg.norm(s[c] - s_ref[c]) <= TOL_STRESS * np.linalg.norm(s_ref[c])
    # same statistics for a batch of two sets
    rho2 = torch.stack([rho, 0.5 * rho]).contiguous()
    sig2, s2 = ctx.stress_stats(rho2)
    torch.cuda.synchronize()
    s2 = s2.cpu().numpy()
    assert np.abs(s2[0] - s).max() <= 1e-6 * np.abs(s).max()
    assert np.abs(s2[1] - 0.5 * s).max() <= 1e-5 * np.abs(s).max()
    ctx.close()


@pytest.mark.parametrize("shape", [(300, 8, 4), (200, 16, 6), (100, 12, 5), (20, 40, 3)])
def test_eq20_statistics_every_line_length(dds, shape):
    # x lines of 512, 256, 128 and 32 padded points (the persistent inverse x pass with 16,
    # 8, 8 and 4 threads per line): the fused sums equal the plane RMS of the returned sigma
    t18, b18 = W.gan_families()
    g = W.Geometry(*shape, 0.2e-6, 0.2e-6, 0.05e-6)
    p = W.random_problem(g, t18[[0, 9, 13]], b18[[0, 9, 13]], seed=sum(shape))
    ctx = dds.context_for(p)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho, dtype=np.float32)).cuda()
    sig, s = ctx.stress_stats(rho)
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    ref = plane_rms(sig.cpu().numpy())
    assert s.shape == (6, g.nz)
    assert np.abs(s - ref).max() <= 1e-6 * np.abs(ref).max()
    ctx.close()


# ------------------------------------------------------------- autotuner ---
@pytest.mark.parametrize("case", ["thin", "tall"])
def test_autotune_keeps_the_result(dds, case):
    if case == "thin":
        p = W.random_problem(W.Geometry(64, 48, 16, 0.5e-6, 0.5e-6, 0.2e-6), *[a[[0, 9]] for a in W.gan_families()],
                             seed=61)
    else:
        p = W.gan_polycrystal(W.Geometry(32, 32, 40, 0.2e-6, 0.2e-6, 0.05e-6), 1e-6, seed=62)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho, dtype=np.float32)).cuda()
    plain = dds.context_for(p)
    ref = plain.stress(rho).cpu().numpy()
    tuned = dds.StressContext(0)
    g = p.geom
    tuned.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu).set_families(p.t, p.b)
    ms = tuned.autotune()
    assert ms > 0
    tuned.build_kernels()
    got = tuned.stress(rho).cpu().numpy()
    assert rel_l2_per_component(got, ref).max() <= 1e-6
    plain.close()
    tuned.close()


def test_no_bounded_wait_gave_up(dds):
    # the bulk-copy waits of the x passes record a timeout in the device status word
    p = W.random_problem(W.Geometry(200, 40, 6, 0.2e-6, 0.2e-6, 0.05e-6), *[a[[0, 9]] for a in W.gan_families()],
                         seed=3)
    got = gpu_stress(dds, p)
    assert np.isfinite(got).all()
    torch.cuda.synchronize()
    assert dds.dds_device_status(0) == dds.DDS_OK
