"""GPU parity of the free-surface relaxation (Sec. 5, Eqs. 14-18) through the C ABI.

The FP32 steps match the FP64 oracle step for step: after K steps from the same
state, u and the total stress agree to a relative L2 error (per component,
denominator max(||x_c||, 1e-6 max_c' ||x_c'||)) below TOL_STEP(K) = 1e-6 + K * 2^-24.
Each step rounds u once to FP32 (relative 2^-24 = 6e-8) and the explicit scheme at
the stated time step does not amplify errors, so K steps add at most K such
roundings.  The total stress is compared relative to its largest component (the
surface z-components cancel to zero, leaving FP32 residues of 2^-24 |sigma^dis|).
Converged states are checked against the closed forms of the oracle pins (uniform
load, plate under a sinusoidal surface load).
"""
import numpy as np
import pytest

import oracle
import oracle.relax as R
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MU, NU = W.MU_GAN, W.NU_GAN


def tol_step(k):
    return 1e-6 + k * 2.0 ** -24


@pytest.fixture(scope="module")
def dds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_01830_gb300 as mod
    mod.load_library()
    return mod


def rel_l2(got, ref):
    got = np.asarray(got, np.float64).reshape(got.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    scale = max(np.linalg.norm(r) for r in ref)
    return max(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-6 * scale) for g, r in zip(got, ref))


def rel_l2_total(got, ref):
    """Stress error relative to the largest component's norm: on the free surfaces the
    z-components of sigma^dis + sigma(u) cancel to zero, and FP32 leaves a residue of
    about 2^-24 |sigma^dis| there, which a per-component norm would magnify."""
    got = np.asarray(got, np.float64).reshape(got.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    scale = max(np.linalg.norm(r) for r in ref)
    return max(np.linalg.norm(g - r) for g, r in zip(got, ref)) / scale


def context(dds, shape, h):
    nz, ny, nx = shape
    ctx = dds.StressContext(0)
    ctx.set_geometry(nx, ny, nz, *h, MU, NU)
    return ctx


def smooth_load(shape, h, seed):
    """A seeded load with the scales of a dislocation stress: a few random Fourier modes
    in x, y (periodic) and smooth in z, amplitude ~1e8 Pa."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z = (np.arange(nz) * h[2])[:, None, None]
    y = (np.arange(ny) / ny)[None, :, None]
    x = (np.arange(nx) / nx)[None, None, :]
    sig = np.zeros((6,) + shape)
    for c in range(6):
        for _ in range(3):
            m, n = rng.integers(-2, 3, size=2)
            q = rng.normal() / (nz * h[2])
            sig[c] += rng.normal() * 1e8 * np.cos(2 * np.pi * (m * x + n * y) + q * z + rng.uniform(0, 6.3))
    return sig


@pytest.mark.parametrize("shape,h,steps", [
    ((6, 10, 12), (0.5e-6, 0.5e-6, 0.2e-6), [1, 10, 200]),
    ((4, 16, 16), (1e-6, 1e-6, 1e-6), [3, 100]),
    ((2, 7, 9), (0.2e-6, 0.2e-6, 0.05e-6), [1, 50]),       # two layers, odd sides
    ((3, 1, 32), (1e-6, 1e-6, 1e-6), [40]),                # plane strain (ny = 1)
    ((35, 9, 66), (0.2e-6, 0.2e-6, 0.05e-6), [1, 20]),     # two x tiles of the pair kernel, two z chunks
    ((34, 5, 67), (0.2e-6, 0.2e-6, 0.05e-6), [1, 20]),     # odd nx: one-cell kernel, two z chunks
])
def test_steps_match_oracle(dds, shape, h, steps):
    sig = smooth_load(shape, h, seed=sum(shape))
    ctx = context(dds, shape, h)
    sig_d = torch.from_numpy(sig.astype(np.float32)).cuda()
    u_d = torch.zeros((3,) + shape, device="cuda")
    u_ref = np.zeros((3,) + shape)
    done = 0
    for k in steps:
        u_d, tot_d = ctx.relax(sig_d, k - done, u=u_d)
        u_ref = R.relax(sig.astype(np.float32).astype(np.float64), h, MU, NU, k - done, u0=u_ref)
        done = k
        torch.cuda.synchronize()
        tot_ref = R.total_stress(u_ref, sig.astype(np.float32).astype(np.float64), h, MU, NU)
        assert rel_l2(u_d.cpu().numpy(), u_ref) <= tol_step(k), k
        assert rel_l2_total(tot_d.cpu().numpy(), tot_ref) <= tol_step(k), k
    ctx.close()


def test_zero_steps_returns_the_load_plus_the_start_state(dds):
    shape, h = (3, 5, 6), (1e-6, 1e-6, 0.5e-6)
    sig = smooth_load(shape, h, seed=4)
    ctx = context(dds, shape, h)
    u, tot = ctx.relax(torch.from_numpy(sig.astype(np.float32)).cuda(), 0)
    ref = R.total_stress(np.zeros((3,) + shape), sig.astype(np.float32).astype(np.float64), h, MU, NU)
    assert np.abs(u.cpu().numpy()).max() == 0.0
    assert rel_l2_total(tot.cpu().numpy(), ref) <= 1e-6
    ctx.close()


def test_uniform_load_relaxes_to_the_closed_form(dds):
    S = np.array([2e7, -5e6, 1e8, 3e6, 3e7, -4e7])
    shape, h = (6, 4, 4), (1e-6, 1e-6, 0.5e-6)
    sig = np.broadcast_to(S[:, None, None, None], (6,) + shape).astype(np.float32).copy()
    ctx = context(dds, shape, h)
    _, tot = ctx.relax(torch.from_numpy(sig).cuda(), 4000)
    A, B = R.moduli(MU, NU)
    lam = A - 2 * B
    want = np.array([S[0] - lam * S[2] / A, S[1] - lam * S[2] / A, 0.0, S[3], 0.0, 0.0])
    got = tot.cpu().numpy().astype(np.float64)
    for c in range(6):
        assert np.abs(got[c] - want[c]).max() <= 1e-5 * np.abs(S).max(), c
    ctx.close()


def test_surfaces_are_traction_free_after_every_call(dds):
    shape, h = (5, 12, 10), (0.5e-6, 0.5e-6, 0.2e-6)
    sig = smooth_load(shape, h, seed=7).astype(np.float32)
    ctx = context(dds, shape, h)
    sig_d = torch.from_numpy(sig).cuda()
    u = None
    for k in (1, 5, 30):
        u, tot = ctx.relax(sig_d, k, u=u)
        t = tot.cpu().numpy()
        for c in (4, 5, 2):
            assert np.abs(t[c][[0, -1]]).max() <= 1e-5 * np.abs(sig).max(), (k, c)
    ctx.close()


def test_plate_under_sinusoidal_surface_load(dds):
    # the oracle pin's Airy-function solution, reached by the GPU relaxation
    nx, nz, s = 32, 9, 1e8
    L = 32e-6
    dx = L / nx
    k = 2 * np.pi / L
    H = (nz - 1) * dx
    x, z = np.arange(nx) * dx, np.arange(nz) * dx
    sig = np.zeros((6, nz, 1, nx), np.float32)
    sig[2] = (s * np.cos(k * x))[None, None, :]
    ctx = context(dds, (nz, 1, nx), (dx, dx, dx))
    _, tot = ctx.relax(torch.from_numpy(sig).cuda(), 3000)
    got = tot.cpu().numpy().astype(np.float64)
    # closed form, as in the oracle pin
    def basis(zz):
        ch, sh = np.cosh(k * zz), np.sinh(k * zz)
        return (np.array([ch, zz * ch, sh, zz * sh]), np.array([k * sh, ch + zz * k * sh, k * ch, sh + zz * k * ch]),
                np.array([k * k * ch, 2 * k * sh + zz * k * k * ch, k * k * sh, 2 * k * ch + zz * k * k * sh]))
    rows, rhs = [], []
    for zz in (0.0, H):
        g, gp, _ = basis(zz)
        rows += [g, gp]
        rhs += [s / k ** 2, 0.0]
    C = np.linalg.solve(np.array(rows), np.array(rhs))
    g, gp, gpp = (C @ b for b in basis(z))
    cx, sx = np.cos(k * x)[None, :], np.sin(k * x)[None, :]
    want = sig.astype(np.float64).copy()
    want[0, :, 0] += gpp[:, None] * cx
    want[2, :, 0] += -k * k * g[:, None] * cx
    want[4, :, 0] += k * gp[:, None] * sx
    want[1, :, 0] += NU * (gpp[:, None] - k * k * g[:, None]) * cx
    assert np.abs(got - want).max() / s < 5e-3
    ctx.close()


def test_dislocation_stress_then_relaxation_matches_oracle_pipeline(dds):
    # the hot path's sigma^dis feeds the relaxation; against the oracle's direct sum + relaxation
    g = W.Geometry(16, 12, 6, 0.5e-6, 0.5e-6, 0.2e-6)
    t, b = W.gan_families()
    p = W.random_problem(g, t[[0, 9]], b[[0, 9]], seed=21)
    ctx = dds.context_for(p)
    sig_d = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda())
    u, tot = ctx.relax(sig_d, 60)
    torch.cuda.synchronize()
    sig_ref = oracle.stress_direct(g, p.t, p.b, p.rho).T.reshape(6, g.nz, g.ny, g.nx)
    h = (g.dx, g.dy, g.dz)
    u_ref = R.relax(sig_ref, h, MU, NU, 60)
    tot_ref = R.total_stress(u_ref, sig_ref, h, MU, NU)
    assert rel_l2_total(tot.cpu().numpy(), tot_ref) <= 1e-5 + tol_step(60)
    assert rel_l2(u.cpu().numpy(), u_ref) <= 1e-5 + tol_step(60)
    ctx.close()


def test_relax_error_codes(dds):
    ctx = dds.StressContext(0)
    sig = torch.zeros((6, 1, 4, 4), device="cuda")
    with pytest.raises(dds.DDSError) as e:
        ctx.relax(sig, 1)                      # no geometry
    ctx.set_geometry(4, 4, 1, 1e-6, 1e-6, 1e-6, MU, NU)
    with pytest.raises(dds.DDSError) as e:
        ctx.relax(sig, 1)                      # one layer
    assert e.value.code == dds.DDS_ERR_UNSUPPORTED
    ctx.set_geometry(4, 4, 2, 1e-6, 1e-6, 1e-6, MU, NU)
    with pytest.raises(dds.DDSError) as e:
        ctx.relax(torch.zeros((6, 2, 4, 4), device="cuda"), -1)
    assert e.value.code == dds.DDS_ERR_INVALID_ARG
    ctx.close()


@pytest.mark.parametrize("workload", ["radial_disk_512x512x16", "gan_layer_256x256x128"])
def test_full_size_steps_match_oracle(dds, workload):
    # the bench grids, in the launch configuration bench.py times: the dislocation stress of
    # the workload (GPU) relaxed for a few steps, every cell against the FP64 oracle's steps
    # from the same FP32 load
    p = W.CONFIGS[workload]()
    g = p.geom
    ctx = dds.context_for(p)
    sig_d = ctx.stress(torch.from_numpy(p.rho.astype(np.float32)).cuda())
    K = 3
    u, tot = ctx.relax(sig_d, K)
    torch.cuda.synchronize()
    sig = sig_d.cpu().numpy().astype(np.float64)
    h = (g.dx, g.dy, g.dz)
    u_ref = R.relax(sig, h, g.mu, g.nu, K)
    tot_ref = R.total_stress(u_ref, sig, h, g.mu, g.nu)
    assert rel_l2(u.cpu().numpy(), u_ref) <= tol_step(K)
    assert rel_l2_total(tot.cpu().numpy(), tot_ref) <= tol_step(K)
    ctx.close()
