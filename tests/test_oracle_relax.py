"""Pins of the relaxation oracle (Sec. 5, Eqs. 14-18) against closed forms.

Each pin fixes the reference by something other than itself: a uniform load whose
relaxed stress is known exactly, a plate under a sinusoidal surface load with its
Airy-function solution, plane waves through the Navier operator and the divergence,
and the traction-free surfaces the ghost layers must produce at every step.
"""
import numpy as np
import pytest

import oracle.relax as R

MU, NU = 68.0e9, 0.23


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_moduli_are_lame_constants():
    # A = lambda + 2 mu, B = mu (Eq. 14 with E = 2 mu (1 + nu))
    A, B = R.moduli(MU, NU)
    lam = 2 * MU * NU / (1 - 2 * NU)
    assert abs(A - (lam + 2 * MU)) <= 1e-12 * A and abs(B - MU) <= 1e-12 * B


def test_zero_load_stays_zero():
    sig = np.zeros((6, 4, 5, 6))
    u = R.relax(sig, (1e-6, 1e-6, 0.5e-6), MU, NU, 50)
    assert np.abs(u).max() == 0.0


def test_uniform_load_relaxes_to_the_closed_form():
    # sigma^dis = S uniform: f = 0; free surfaces and periodic sides admit only u linear in z,
    # u_x = -S_xz z / mu, u_y = -S_yz z / mu, u_z = -S_zz z / A, so the total stress has
    # zero z-components and sigma_xx = S_xx - lambda S_zz / A (same for yy), sigma_xy = S_xy.
    S = np.array([2e7, -5e6, 1e8, 3e6, 3e7, -4e7])
    sig = np.broadcast_to(S[:, None, None, None], (6, 6, 4, 4)).copy()
    h = (1e-6, 1e-6, 0.5e-6)
    u = R.relax(sig, h, MU, NU, 4000)
    st = R.total_stress(u, sig, h, MU, NU)
    A, B = R.moduli(MU, NU)
    lam = A - 2 * B
    want = np.array([S[0] - lam * S[2] / A, S[1] - lam * S[2] / A, 0.0, S[3], 0.0, 0.0])
    for c in range(6):
        assert np.abs(st[c] - want[c]).max() <= 1e-9 * np.abs(S).max(), c


def test_surfaces_are_traction_free_at_every_step():
    # Eq. 16b: the ghost layers make sigma_xz, sigma_yz, sigma_zz of the total stress vanish
    # on the first and last layers after each step, whatever the interior state
    rng = np.random.default_rng(0)
    sig = rng.normal(size=(6, 5, 6, 7)) * 1e8
    h = (0.5e-6, 0.5e-6, 0.2e-6)
    u = None
    for n in (0, 1, 7):
        u = R.relax(sig, h, MU, NU, n, u0=u) if n else np.zeros((3, 5, 6, 7))
        st = R.total_stress(u, sig, h, MU, NU)
        for c in (R.XZ, R.YZ, R.ZZ):
            assert np.abs(st[c][[0, -1]]).max() <= 1e-7 * np.abs(sig).max(), (n, c)


def _plane_waves(shape, h, L):
    """Two plane waves u = d sin(q.r) periodic in x and y, sampled on the film cells and
    the ghost layers; returns u_ext (3, nz+2, ny, nx) and the analytic Navier operator."""
    nz, ny, nx = shape
    A, B = R.moduli(MU, NU)
    z = (np.arange(-1, nz + 1) * h[2])[:, None, None]
    y = (np.arange(ny) * h[1])[None, :, None]
    x = (np.arange(nx) * h[0])[None, None, :]
    waves = [((1, 2), 1.3 / (nz * h[2]), np.array([0.3, -1.0, 0.7])),
             ((2, -1), -0.8 / (nz * h[2]), np.array([1.0, 0.4, -0.5]))]
    ue = np.zeros((3, nz + 2, ny, nx))
    nav = np.zeros((3, nz, ny, nx))
    for (m, n), qz, d in waves:
        q = np.array([2 * np.pi * m / L[0], 2 * np.pi * n / L[1], qz])
        ph = q[0] * x + q[1] * y + q[2] * z
        for a in range(3):
            ue[a] += d[a] * np.sin(ph)
            # (lambda + mu) grad div u + mu lap u = -[(A - B) q (q.d) + B |q|^2 d] sin(q.r)
            nav[a] += -((A - B) * q[a] * (q @ d) + B * (q @ q) * d[a]) * np.sin(ph)[1:-1]
    return ue, nav


def test_navier_operator_is_second_order():
    errs = []
    for n in (16, 32):
        L = (8e-6, 8e-6)
        shape = (n // 2, n, n)
        h = (L[0] / n, L[1] / n, 4e-6 / (n // 2))
        ue, want = _plane_waves(shape, h, L)
        got = R.navier(ue, h, MU, NU)
        errs.append(rel(got, want))
    assert errs[0] < 0.1 and 3.5 < errs[0] / errs[1] < 4.5, errs


def test_divergence_force_is_second_order():
    # Eq. 15 on smooth fields, including the one-sided differences on the surface layers
    errs = []
    for n in (32, 64):
        L = 8e-6
        h = (L / n, L / n, 3e-6 / n)
        nz = n
        z = (np.arange(nz) * h[2])[:, None, None]
        y = (np.arange(n) * h[1])[None, :, None]
        x = (np.arange(n) * h[0])[None, None, :]
        k = 2 * np.pi / L
        qz = 1.7 / 3e-6
        sig = np.zeros((6, nz, n, n))
        want = np.zeros((3, nz, n, n))
        for c in range(6):
            m = 1 + c % 2
            ph = k * m * x + k * (c % 3) * y + qz * (1 + 0.2 * c) * z
            sig[c] = np.cos(ph) * (1 + c)
            grad = [-(1 + c) * np.sin(ph) * g for g in (k * m, k * (c % 3), qz * (1 + 0.2 * c))]
            for a in range(3):
                for b in range(3):
                    if R.PAIR[a][b] == c:
                        want[a] += grad[b]
        errs.append(rel(R.force(sig, h), want))
    assert errs[0] < 0.05 and 3.5 < errs[0] / errs[1] < 4.5, errs


def _plate(nx, nz, steps, s=1e8):
    """Layer 0 <= z <= H under sigma^dis_zz = s cos(kx) (no other component): f = 0 and the
    free surfaces carry sigma_zz(u) = -s cos(kx), sigma_xz(u) = 0.  Plane strain; the Airy
    function cos(kx) g(z), g = (C1 + C2 z) cosh kz + (C3 + C4 z) sinh kz, with
    g(0) = g(H) = s / k^2, g'(0) = g'(H) = 0, gives sigma(u) in closed form."""
    L = 32e-6
    dx = L / nx
    h = (dx, dx, dx)
    k = 2 * np.pi / L
    H = (nz - 1) * dx
    x = np.arange(nx) * dx
    z = np.arange(nz) * dx
    sig = np.zeros((6, nz, 1, nx))
    sig[R.ZZ] = s * np.cos(k * x)[None, None, :]

    def basis(zz):
        ch, sh = np.cosh(k * zz), np.sinh(k * zz)
        g = np.array([ch, zz * ch, sh, zz * sh])
        gp = np.array([k * sh, ch + zz * k * sh, k * ch, sh + zz * k * ch])
        gpp = np.array([k * k * ch, 2 * k * sh + zz * k * k * ch, k * k * sh, 2 * k * ch + zz * k * k * sh])
        return g, gp, gpp

    rows, rhs = [], []
    for zz in (0.0, H):
        g, gp, _ = basis(zz)
        rows += [g, gp]
        rhs += [s / k ** 2, 0.0]
    C = np.linalg.solve(np.array(rows), np.array(rhs))
    g, gp, gpp = (C @ b for b in basis(z))
    cx, sx = np.cos(k * x)[None, :], np.sin(k * x)[None, :]
    want = sig.copy()
    want[R.XX, :, 0] += gpp[:, None] * cx
    want[R.ZZ, :, 0] += -k * k * g[:, None] * cx
    want[R.XZ, :, 0] += k * gp[:, None] * sx
    want[R.YY, :, 0] += NU * ((gpp[:, None] - k * k * g[:, None]) * cx)      # plane strain
    u = R.relax(sig, h, MU, NU, steps)
    st = R.total_stress(u, sig, h, MU, NU)
    return np.abs(st - want).max() / s


def test_plate_under_sinusoidal_surface_load_matches_airy_solution():
    e1 = _plate(32, 9, 3000)
    e2 = _plate(64, 17, 9000)
    assert e1 < 5e-3 and 3.5 < e1 / e2 < 4.5, (e1, e2)


def test_time_step_of_the_paper_is_stable():
    # dt = min(h)^2 / (5A - 3B): with no load every mode decays; random start, anisotropic cells
    rng = np.random.default_rng(1)
    h = (0.4e-6, 0.4e-6, 0.1e-6)
    u0 = rng.normal(size=(3, 6, 8, 8))
    sig = np.zeros((6, 6, 8, 8))
    norms = [np.abs(u0).max()]
    u = u0
    for _ in range(10):
        u = R.relax(sig, h, MU, NU, 200, u0=u)
        norms.append(np.abs(u).max())
    assert all(b <= a * (1 + 1e-12) for a, b in zip(norms, norms[1:])), norms
    assert norms[-1] < 0.5 * norms[0]


def test_two_layers_is_the_minimum():
    with pytest.raises(ValueError):
        R.relax(np.zeros((6, 1, 4, 4)), (1e-6, 1e-6, 1e-6), MU, NU, 1)
