"""FP64 reference of the free-surface stress relaxation (Sec. 5, Eqs. 14-18).

TEST INFRASTRUCTURE ONLY: imported by the tests and the CPU-baseline legs of
``bench.py``; never by the product path, and it shares no code with the CUDA
library.  Plain numpy, vectorised over the grid, in the paper's order:

  * Eq. 14/17: the displacement u relaxes by explicit Euler steps of
        du/dt = A grad div u - B rot rot u + f,
    A = E(1-nu)/((1+nu)(1-2nu)), B = E/(2(1+nu)) (E = 2 mu (1+nu)), with the
    time step dt = min(dx, dy, dz)^2 / (5A - 3B) the paper states;
  * Eq. 15: f_a = sum_b d sigma^dis_ab / d b;
  * Eq. 16a: u periodic in x and y;
  * Eq. 16c / 18a-18b: free top and bottom surfaces through one layer of ghost
    cells below the first and above the last film layer, refreshed from the
    film values after every step.

Discretisation (the paper names the scheme, not every difference):
  * second differences (u[+1] - 2u + u[-1]) / h^2; mixed derivatives
    (u[+a+b] - u[+a-b] - u[-a+b] + u[-a-b]) / (4 h_a h_b); first derivatives
    central, (u[+1] - u[-1]) / (2h);
  * the surfaces lie on the cell centres of the first and last film layers, where
    the boundary conditions of Eq. 16c are centred (Eq. 18a);
  * d sigma^dis / dz inside the film is central; on the first and last layers it
    is the second-order one-sided difference (first order when nz = 2);
  * the total stress is sigma^dis + sigma(u), sigma(u) by Hooke's law with the
    same central differences (ghost cells on the surface layers).

Arrays are [component][z][y][x]; stresses in the order xx, yy, zz, xy, xz, yz.
"""
from __future__ import annotations

import numpy as np

XX, YY, ZZ, XY, XZ, YZ = range(6)
# stress component of the pair (a, b), a, b in {0: x, 1: y, 2: z}
PAIR = ((XX, XY, XZ), (XY, YY, YZ), (XZ, YZ, ZZ))


def moduli(mu: float, nu: float):
    """A and B of Eq. 14 from the shear modulus and Poisson's ratio."""
    E = 2.0 * mu * (1.0 + nu)
    A = E * (1.0 - nu) / ((1.0 + nu) * (1.0 - 2.0 * nu))
    B = E / (2.0 * (1.0 + nu))
    return A, B


def time_step(h, mu: float, nu: float) -> float:
    """dt = min(h)^2 / (5A - 3B) (Sec. 5, von Neumann estimate)."""
    A, B = moduli(mu, nu)
    return min(h) ** 2 / (5.0 * A - 3.0 * B)


# -- finite differences on the periodic (x, y) plane ---------------------------
def _dx(g, h):    # d/dx, axis -1
    return (np.roll(g, -1, axis=-1) - np.roll(g, 1, axis=-1)) / (2.0 * h)


def _dy(g, h):    # d/dy, axis -2
    return (np.roll(g, -1, axis=-2) - np.roll(g, 1, axis=-2)) / (2.0 * h)


def force(sig: np.ndarray, h) -> np.ndarray:
    """Eq. 15: f_a = d sig_ax/dx + d sig_ay/dy + d sig_az/dz, shape (3, nz, ny, nx)."""
    nz = sig.shape[1]
    f = np.zeros((3,) + sig.shape[1:])
    for a in range(3):
        f[a] = _dx(sig[PAIR[a][0]], h[0]) + _dy(sig[PAIR[a][1]], h[1])
        s = sig[PAIR[a][2]]
        dz = np.zeros_like(s)
        if nz >= 3:
            dz[1:-1] = (s[2:] - s[:-2]) / (2.0 * h[2])
            dz[0] = (-3.0 * s[0] + 4.0 * s[1] - s[2]) / (2.0 * h[2])
            dz[-1] = (3.0 * s[-1] - 4.0 * s[-2] + s[-3]) / (2.0 * h[2])
        elif nz == 2:
            dz[:] = (s[1] - s[0]) / h[2]
        f[a] += dz
    return f


def surface_terms(sig: np.ndarray, mu: float, nu: float):
    """Eq. 16c: phi_xz, phi_yz, phi_zz on the bottom and top layers, shape (2, 3, ny, nx)."""
    E = 2.0 * mu * (1.0 + nu)
    phi = np.zeros((2, 3) + sig.shape[2:])
    for s, k in ((0, 0), (1, -1)):
        phi[s, 0] = -(1.0 + nu) / E * sig[XZ, k]
        phi[s, 1] = -(1.0 + nu) / E * sig[YZ, k]
        phi[s, 2] = -(1.0 + nu) * (1.0 - 2.0 * nu) / E * sig[ZZ, k]
    return phi


def with_ghosts(u: np.ndarray, phi: np.ndarray, h, nu: float) -> np.ndarray:
    """u extended by the ghost layers below and above the film (Eq. 18b and its
    counterparts for u_y, u_z and the top surface), shape (3, nz + 2, ny, nx)."""
    nz = u.shape[1]
    if nz < 2:
        raise ValueError("the free-surface relaxation needs at least two layers")
    ue = np.zeros((3, nz + 2) + u.shape[2:])
    ue[:, 1:-1] = u
    two_dz = 2.0 * h[2]
    # bottom: centred at the first layer, ghost below (Eq. 18b)
    b, b2 = u[:, 0], u[:, 1]
    ue[0, 0] = b2[0] + two_dz * (_dx(b[2], h[0]) - 2.0 * phi[0, 0])
    ue[1, 0] = b2[1] + two_dz * (_dy(b[2], h[1]) - 2.0 * phi[0, 1])
    ue[2, 0] = b2[2] - two_dz / (1.0 - nu) * (phi[0, 2] - nu * (_dx(b[0], h[0]) + _dy(b[1], h[1])))
    # top: centred at the last layer, ghost above
    t, t2 = u[:, -1], u[:, -2]
    ue[0, -1] = t2[0] + two_dz * (2.0 * phi[1, 0] - _dx(t[2], h[0]))
    ue[1, -1] = t2[1] + two_dz * (2.0 * phi[1, 1] - _dy(t[2], h[1]))
    ue[2, -1] = t2[2] + two_dz / (1.0 - nu) * (phi[1, 2] - nu * (_dx(t[0], h[0]) + _dy(t[1], h[1])))
    return ue


def _at(ue: np.ndarray, comp: int, s) -> np.ndarray:
    """Component comp of the extended u at the film cells shifted by s = (sx, sy, sz)
    cells (x, y periodic; |sz| <= 1 reaches into the ghost layers)."""
    nz = ue.shape[1] - 2
    g = ue[comp, 1 + s[2]:1 + s[2] + nz]
    return np.roll(np.roll(g, -s[1], axis=1), -s[0], axis=2)


def _unit(a: int, sign: int = 1):
    e = [0, 0, 0]
    e[a] = sign
    return e


def navier(ue: np.ndarray, h, mu: float, nu: float) -> np.ndarray:
    """A grad div u - B rot rot u on the film cells (Eq. 14 without f), from u
    extended by its ghost layers; shape (3, nz, ny, nx).  Component a:
        A d2u_a/da2 + B sum_{b != a} d2u_a/db2 + (A - B) sum_{b != a} d2u_b/(da db)
    (grad div u - rot rot u = laplacian u)."""
    A, B = moduli(mu, nu)

    def d2(c, a):
        return (_at(ue, c, _unit(a, 1)) - 2.0 * _at(ue, c, (0, 0, 0)) + _at(ue, c, _unit(a, -1))) / h[a] ** 2

    def mixed(c, a, b):
        def sh(sa, sb):
            s = [0, 0, 0]
            s[a] += sa
            s[b] += sb
            return _at(ue, c, s)
        return (sh(1, 1) - sh(1, -1) - sh(-1, 1) + sh(-1, -1)) / (4.0 * h[a] * h[b])

    out = np.zeros((3, ue.shape[1] - 2) + ue.shape[2:])
    for a in range(3):
        acc = A * d2(a, a)
        for b in range(3):
            if b != a:
                acc = acc + B * d2(a, b) + (A - B) * mixed(b, a, b)
        out[a] = acc
    return out


def relax(sig: np.ndarray, h, mu: float, nu: float, n_steps: int, u0: np.ndarray | None = None,
          dt: float | None = None) -> np.ndarray:
    """n_steps explicit steps of Eq. 17 from u0 (default 0); returns u (3, nz, ny, nx)."""
    sig = np.asarray(sig, dtype=np.float64)
    f = force(sig, h)
    phi = surface_terms(sig, mu, nu)
    dt = time_step(h, mu, nu) if dt is None else dt
    u = np.zeros((3,) + sig.shape[1:]) if u0 is None else np.array(u0, dtype=np.float64)
    for _ in range(int(n_steps)):
        ue = with_ghosts(u, phi, h, nu)
        u = u + dt * (navier(ue, h, mu, nu) + f)
    return u


def residual(u: np.ndarray, sig: np.ndarray, h, mu: float, nu: float) -> np.ndarray:
    """A grad div u - B rot rot u + f at the film cells (zero at equilibrium)."""
    ue = with_ghosts(u, surface_terms(sig, mu, nu), h, nu)
    return navier(ue, h, mu, nu) + force(sig, h)


def displacement_stress(u: np.ndarray, sig: np.ndarray, h, mu: float, nu: float) -> np.ndarray:
    """sigma(u) by Hooke's law, lambda div u delta + mu (du_a/db + du_b/da), shape (6, nz, ny, nx)."""
    A, B = moduli(mu, nu)
    lam = A - 2.0 * B
    ue = with_ghosts(u, surface_terms(sig, mu, nu), h, nu)
    grad = np.zeros((3, 3) + u.shape[1:])          # grad[a][b] = d u_a / d b
    for a in range(3):
        grad[a, 0] = _dx(u[a], h[0])
        grad[a, 1] = _dy(u[a], h[1])
        grad[a, 2] = (ue[a, 2:] - ue[a, :-2]) / (2.0 * h[2])
    div = grad[0, 0] + grad[1, 1] + grad[2, 2]
    out = np.zeros((6,) + u.shape[1:])
    for a in range(3):
        for b in range(a, 3):
            v = B * (grad[a, b] + grad[b, a])
            if a == b:
                v = v + lam * div
            out[PAIR[a][b]] = v
    return out


def total_stress(u: np.ndarray, sig: np.ndarray, h, mu: float, nu: float) -> np.ndarray:
    """sigma^dis + sigma(u): the stress of the film with free surfaces."""
    return np.asarray(sig, dtype=np.float64) + displacement_stress(u, sig, h, mu, nu)
