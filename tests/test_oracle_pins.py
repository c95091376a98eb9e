"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the textbook
field of an infinite straight dislocation (the limit of Eq. 4a/Eq. 5), the
independent Eq. 4a routine, exact identities (telescoping of Eq. 5, oddness,
linearity in b and rho, rotation covariance), the multipole error law of
Sec. 2.3, brute force (FFT convolution == direct sum of Eq. 10) and the
magnitudes and symmetries the paper states for its disk example (Sec. 3).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

MU, NU = 68.0e9, 0.23
BB = 3.19e-10


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def textbook_infinite(x, y, b, mu=MU, nu=NU):
    """Infinite straight dislocation along +z (Hirth & Lothe), components xx,yy,zz,xy,xz,yz.
    This is the z'_A -> -inf, z'_B -> +inf limit of Eq. 4a with Eq. 5."""
    D = mu / (2 * math.pi * (1 - nu))
    r2 = x * x + y * y
    bx, by, bz = b
    xx = -D * bx * y * (3 * x * x + y * y) / r2 ** 2 + D * by * x * (x * x - y * y) / r2 ** 2
    yy = D * bx * y * (x * x - y * y) / r2 ** 2 + D * by * x * (x * x + 3 * y * y) / r2 ** 2
    zz = -2 * nu * D * bx * y / r2 + 2 * nu * D * by * x / r2
    xy = D * bx * x * (x * x - y * y) / r2 ** 2 + D * by * y * (x * x - y * y) / r2 ** 2
    xz = -mu * bz * y / (2 * math.pi * r2)
    yz = mu * bz * x / (2 * math.pi * r2)
    return np.array([xx, yy, zz, xy, xz, yz])


def rot_random(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def to33(s):
    return np.array([[s[0], s[3], s[4]], [s[3], s[1], s[5]], [s[4], s[5], s[2]]])


# ---------------------------------------------------------------- P1 ------
@pytest.mark.parametrize("b", [(BB, 0, 0), (0, BB, 0), (0, 0, BB), (BB, -0.4 * BB, 0.7 * BB)])
def test_eq6_long_segment_is_textbook_line(b):
    x, y = 0.7e-6, -1.3e-6
    half = 1.5e6 * math.hypot(x, y)        # L / r ~ 1e6: finite-length term ~1e-12
    got = oracle.segment_eq6([x, y, 0.0], [0, 0, -half], [0, 0, half], [0, 0, 1], b, MU, NU)
    assert rel(got, textbook_infinite(x, y, b)) < 1e-10


def test_eq4_long_segment_is_textbook_line():
    x, y = -0.4e-6, 0.9e-6
    half = 1.0e3 * math.hypot(x, y)
    b = (BB, 0.3 * BB, -0.8 * BB)
    got = oracle.segment_eq4([x, y, 0.0], -half, half, b, MU, NU)
    assert rel(got, textbook_infinite(x, y, b)) < 1e-5     # (r/L)^2 ~ 1e-6 plus roundoff


# ---------------------------------------------------------------- P2 ------
def test_eq6_matches_independent_eq4_for_vertical_segments():
    rng = np.random.default_rng(11)
    for _ in range(200):
        b = rng.normal(size=3) * BB
        zA = rng.uniform(-2e-6, 0)
        zB = zA + rng.uniform(0.05e-6, 2e-6)
        obs = rng.normal(size=3) * 1e-6
        obs[2] = zA - rng.uniform(0.01e-6, 5e-6)            # Eq. 4a's region: below z'_A
        ref = oracle.segment_eq4(obs, zA, zB, b, MU, NU)
        got = oracle.segment_eq6(obs, [0, 0, zA], [0, 0, zB], [0, 0, 1], b, MU, NU)
        assert rel(got, ref) < 1e-11


def test_eq6_rotation_covariance_general_direction():
    rng = np.random.default_rng(5)
    for _ in range(50):
        Q = rot_random(rng)
        b = rng.normal(size=3) * BB
        obs = rng.normal(size=3) * 1e-6
        A = np.array([0, 0, -0.3e-6])
        B = np.array([0, 0, 0.5e-6])
        s = to33(oracle.segment_eq6(obs, A, B, [0, 0, 1], b, MU, NU))
        sr = to33(oracle.segment_eq6(Q @ obs, Q @ A, Q @ B, Q @ np.array([0, 0, 1.0]), Q @ b, MU, NU))
        assert rel(Q @ s @ Q.T, sr) < 1e-11


def test_eq6_two_forms_differ_only_by_constants():
    rng = np.random.default_rng(7)
    for _ in range(100):
        t = rng.normal(size=3)
        t /= np.linalg.norm(t)
        b = rng.normal(size=3) * BB
        A = rng.normal(size=3) * 1e-7
        B = A + t * rng.uniform(0.1e-6, 1e-6)
        n = np.cross(t, rng.normal(size=3))
        obs = 0.5 * (A + B) + n / np.linalg.norm(n) * rng.uniform(0.2e-6, 2e-6)
        s1 = oracle.segment_eq6(obs, A, B, t, b, MU, NU, form=+1)
        s2 = oracle.segment_eq6(obs, A, B, t, b, MU, NU, form=-1)
        assert rel(s1, s2) < 1e-10


def test_eq6_on_axis_observers():
    # below the segment on its axis: Eq. 4a is regular there (lambda > 0)
    b = (BB, -0.5 * BB, 0.8 * BB)
    zA, zB = -0.2e-6, 0.3e-6
    below = np.array([0.0, 0.0, -1.1e-6])
    ref = oracle.segment_eq4(below, zA, zB, b, MU, NU)
    got = oracle.segment_eq6(below, [0, 0, zA], [0, 0, zB], [0, 0, 1], b, MU, NU)
    assert rel(got, ref) < 1e-12
    # above the segment on its axis: the field is odd about the segment midpoint
    mid = 0.5 * (zA + zB)
    above = np.array([0.0, 0.0, 2 * mid - below[2]])
    got_above = oracle.segment_eq6(above, [0, 0, zA], [0, 0, zB], [0, 0, 1], b, MU, NU)
    assert np.all(np.isfinite(got_above))
    assert rel(got_above, -ref) < 1e-12


def test_eq6_linear_in_b_and_flip():
    rng = np.random.default_rng(3)
    t = np.array([0.0, math.sin(0.27), math.cos(0.27)])
    A, B = -0.2e-6 * t, 0.2e-6 * t
    obs = np.array([0.3e-6, -0.1e-6, 0.45e-6])
    b1, b2 = rng.normal(size=3) * BB, rng.normal(size=3) * BB
    s1 = oracle.segment_eq6(obs, A, B, t, b1, MU, NU)
    s2 = oracle.segment_eq6(obs, A, B, t, b2, MU, NU)
    s12 = oracle.segment_eq6(obs, A, B, t, b1 + b2, MU, NU)
    assert rel(s12, s1 + s2) < 1e-12
    assert rel(oracle.segment_eq6(obs, A, B, t, -b1, MU, NU), -s1) < 1e-15
    # the same physical segment described as (-t, -b, B -> A)
    assert rel(oracle.segment_eq6(obs, B, A, -t, -b1, MU, NU), s1) < 1e-12


# ------------------------------------------------- subcells and chords ----
def test_subcell_rule():
    assert oracle.subcells([0.2, 0.2, 0.05]) == (4, 4, 1)
    assert oracle.subcells([0.5, 0.5, 0.2]) == (3, 3, 1)
    assert oracle.subcells([0.2, 0.2, 0.02]) == (10, 10, 1)
    assert oracle.subcells([1.0, 1.0, 1.0]) == (1, 1, 1)
    assert oracle.subcells([1.0, 0.5, 0.25]) == (4, 2, 1)


def test_chord():
    assert oracle.chord([0.2, 0.2, 0.05], [0, 0, 1]) == pytest.approx(0.05, rel=1e-15)
    t = [0.0, 0.5, math.sqrt(3) / 2]
    assert oracle.chord([0.5, 0.5, 0.2], t) == pytest.approx(min(0.5 / 0.5, 0.2 / (math.sqrt(3) / 2)), rel=1e-15)


# ---------------------------------------------------------------- P3 ------
@pytest.mark.parametrize("cells,ij", [((1e-6, 1e-6, 1e-6), (2, 1)), ((1e-6, 1e-6, 0.25e-6), (4, 1))])
def test_column_telescopes_to_one_segment(cells, ij):
    """Sum over a column of vertical-dislocation coefficients = one long segment (Eq. 5)."""
    g = W.Geometry(8, 8, 16, *cells, MU, NU)
    b = (BB, 0.4 * BB, -0.6 * BB)
    i, j = ij
    K = 7
    total = np.zeros(6)
    for k in range(-K, K + 1):
        total += oracle.interaction(g, i, j, k, [0, 0, 1], b)
    dx, dy, dz = cells
    ref = oracle.segment_eq4([i * dx, j * dy, 0.0], -(K + 0.5) * dz, (K + 0.5) * dz, b, MU, NU)
    assert rel(total / (dx * dy), ref) < 1e-11


# ---------------------------------------------------------------- P4 ------
def test_table_is_odd_and_self_term_vanishes():
    g = W.Geometry(10, 9, 6, 1e-6, 1e-6, 0.25e-6, MU, NU)
    t = np.array([0.0, 0.5, math.sqrt(3) / 2])
    tab = oracle.gtable(g, t, (BB / 2, math.sqrt(3) * BB / 2, 1.6 * BB))
    m = np.abs(tab).max()
    assert rel(tab[::-1, ::-1, ::-1], -tab) < 1e-13
    assert np.abs(tab[g.nz - 1, g.ny - 1, g.nx - 1]).max() < 1e-14 * m


# ---------------------------------------------------------------- P5 ------
def test_linearity_in_b_and_rho():
    g = W.Geometry(6, 5, 4, 1e-6, 1e-6, 0.25e-6, MU, NU)
    t = W.t_mixed()
    b1, b2 = np.array([BB, 0, 0.5 * BB]), np.array([-0.3 * BB, BB, 0])
    for ijk in [(0, 0, 1), (1, -1, 2), (5, 4, -3)]:
        G1 = oracle.interaction(g, *ijk, t, b1)
        G2 = oracle.interaction(g, *ijk, t, b2)
        assert rel(oracle.interaction(g, *ijk, t, b1 + b2), G1 + G2) < 1e-12
        assert rel(oracle.interaction(g, *ijk, t, -b1), -G1) < 1e-15
    p1 = W.random_problem(g, [t], [b1], seed=1)
    p2 = W.random_problem(g, [t], [b1], seed=2)
    s1 = oracle.stress_direct(g, p1.t, p1.b, p1.rho)
    s2 = oracle.stress_direct(g, p2.t, p2.b, p2.rho)
    s12 = oracle.stress_direct(g, p1.t, p1.b, 2.0 * p1.rho - 3.0 * p2.rho)
    assert rel(s12, 2.0 * s1 - 3.0 * s2) < 1e-12


# ---------------------------------------------------------------- P7 ------
def test_near_field_error_falls_as_inverse_square():
    """Sec. 2.3: the single-term (monopole) coefficient differs from the subdivided one by
    higher multipoles, which fall off at least as (h / |Delta|)^2 relative to G."""
    g = W.Geometry(40, 40, 40, 1e-6, 1e-6, 0.25e-6, MU, NU)
    t, b = [0, 0, 1], (BB, 0, 0)
    errs = []
    for i in (2, 4, 8):
        sub = oracle.interaction(g, i, 1, 0, t, b, n_near=1e3)     # always subdivided
        mono = oracle.interaction(g, i, 1, 0, t, b, n_near=0.0)    # never subdivided
        errs.append(rel(mono, sub))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 3.0 and errs[0] / errs[1] > 2.5
    assert errs[2] < 5e-3


# ---------------------------------------------------------------- P8 ------
@pytest.mark.parametrize("cells", [(1e-6, 1e-6, 1e-6), (1e-6, 1e-6, 0.25e-6)])
def test_single_column_reproduces_infinite_dislocation(cells):
    """A column of cells each holding one threading dislocation (rho * dx * dy = 1)
    gives the textbook field of one straight line, up to its finite length."""
    dx, dy, dz = cells
    nz = int(round(256e-6 / dz))
    g = W.Geometry(24, 24, nz, dx, dy, dz, MU, NU)
    b = (BB, 0.0, 0.5 * BB)
    rho = np.zeros((1, g.nz, g.ny, g.nx))
    rho[0, :, 4, 4] = 1.0 / (dx * dy)
    k = nz // 2
    pts = [(4 + 9, 4 + 3), (4 + 12, 4 - 2), (4 - 3, 4 + 14), (4 + 2, 4 + 2)]
    targets = [(k * g.ny + j) * g.nx + i for i, j in pts]
    s = oracle.stress_direct(g, [[0, 0, 1]], [b], rho, targets=targets, use_table=False)
    for q, (i, j) in enumerate(pts):
        x = (i - 4) * dx
        y = (j - 4) * dy
        ref = textbook_infinite(x, y, b)
        z_line_mid = (k + 0.5) * dz - 0.5 * nz * dz
        tol = 0.03 if abs(i - 4) + abs(j - 4) > 6 else 0.15   # (2,2) is a near-field cell
        assert rel(s[q], ref) < tol, (i, j, s[q], ref, z_line_mid)


# ---------------------------------------------------------------- P9 ------
def test_gaussian_disk_mirror_parities():
    p = W.gaussian_disk_32()
    s = oracle.stress_direct(p.geom, p.t, p.b, p.rho).T.reshape(6, 8, 32, 32)
    my = s[:, :, ::-1, :]
    mx = s[:, :, :, ::-1]
    m = np.abs(s).max(axis=(1, 2, 3))
    odd_y = {0, 1, 2, 4}
    odd_x = {3, 4}
    for c in range(6):
        sy = -1 if c in odd_y else 1
        sx = -1 if c in odd_x else 1
        assert np.abs(my[c] - sy * s[c]).max() < 1e-12 * m[c], c
        assert np.abs(mx[c] - sx * s[c]).max() < 1e-12 * m[c], c


# ---------------------------------------------------------------- P10 -----
def fft_convolution(geom, tables, rho):
    """Zero-padded FFT convolution of per-family tables with densities (numpy FP64)."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    P = (2 * nz, 2 * ny, 2 * nx)
    iz = np.arange(-(nz - 1), nz) % P[0]
    iy = np.arange(-(ny - 1), ny) % P[1]
    ix = np.arange(-(nx - 1), nx) % P[2]
    out = np.zeros((6, nz, ny, nx))
    for f, tab in enumerate(tables):
        R = np.fft.rfftn(rho[f], s=P, axes=(0, 1, 2))
        for c in range(6):
            Gp = np.zeros(P)
            Gp[np.ix_(iz, iy, ix)] = tab[..., c]
            out[c] += np.fft.irfftn(np.fft.rfftn(Gp) * R, s=P, axes=(0, 1, 2))[:nz, :ny, :nx]
    return out


@pytest.mark.parametrize("shape,cells", [((6, 5, 4), (1e-6, 1e-6, 0.25e-6)), ((7, 3, 5), (0.5e-6, 0.5e-6, 0.2e-6))])
def test_fft_convolution_equals_direct_sum(shape, cells):
    g = W.Geometry(*shape, *cells, MU, NU)
    t, b = W.gan_families()
    sel = [0, 3, 7, 12]
    p = W.random_problem(g, t[sel], b[sel], seed=4)
    direct = oracle.stress_direct(g, p.t, p.b, p.rho).T.reshape(6, g.nz, g.ny, g.nx)
    tables = [oracle.gtable(g, p.t[f], p.b[f]) for f in range(p.n_families)]
    via_fft = fft_convolution(g, tables, p.rho)
    for c in range(6):
        assert np.linalg.norm(via_fft[c] - direct[c]) <= 1e-12 * np.linalg.norm(direct[c])


# ----------------------------------------------- golden: Sec. 3 disk ------
def _read_golden(name):
    vals = {}
    from pathlib import Path
    for line in (Path(__file__).parent / "golden" / name).read_text().splitlines():
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split(None, 1)
            vals[k] = v.strip()
    return vals


def _disk_problem(n, gold):
    D = float(gold["diameter_m"])
    h = float(gold["thickness_m"])
    E = float(gold["young_pa"])
    nu = float(gold["poisson"])
    mu = E / (2 * (1 + nu))
    nz = n // 5
    g = W.Geometry(n, n, nz, D / n, D / n, h / nz, mu, nu)
    x = (np.arange(n) + 0.5) * g.dx - D / 2
    z = (np.arange(nz) + 0.5) * g.dz
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    rho = (float(gold["rho_max_m2"]) * np.exp(-r2 / (2 * float(gold["decay_radial_m"]) ** 2))[None]
           * np.exp(-z / float(gold["decay_vertical_m"]))[:, None, None])
    rho = rho * (r2 < (D / 2) ** 2)[None]
    return g, rho[None]


def test_disk_example_magnitude_and_symmetry():
    gold = _read_golden("disk_sec3.txt")
    a = float(gold["lattice_a_m"])
    c = float(gold["lattice_c_m"])
    smax = float(gold["max_stress_pa"])
    cases = {"edge": ([0, 0, 1], [a, 0, 0]),
             "mixed": ([0, 0.5, math.sqrt(3) / 2], [a / 2, math.sqrt(3) * a / 2, c])}
    peaks = {}
    for n in (40, 80):
        g, rho = _disk_problem(n, gold)
        for name, (t, b) in cases.items():
            s = fft_convolution(g, [oracle.gtable(g, t, b)], rho)
            peaks[(name, n)] = np.abs(s).max()
            # "~50 GPa": the same order of magnitude (a wrong prefactor moves it 4x)
            assert 0.5 * smax < peaks[(name, n)] < 2.0 * smax, (name, n, peaks[(name, n)])
            if name == "edge":
                inside = rho[0, 0] > 0
                for comp in range(6):
                    plane = s[comp, g.nz // 2][inside]
                    big = np.abs(plane) > 1e-3 * np.abs(plane).max()
                    single = (np.all(plane[big] > 0) or np.all(plane[big] < 0))
                    assert single == (comp == 5), comp        # only sigma_yz keeps its sign
    # Sec. 2.3: halving the cell size does not noticeably change the result
    for name in cases:
        assert abs(peaks[(name, 80)] - peaks[(name, 40)]) < 0.05 * peaks[(name, 80)]


# ------------------------------------------- periodic boundary conditions ----
def test_replica_sum_equals_the_tiled_open_system():
    """Eq. 12: summing the replicas of every source cell (|k|,|l| <= n) is the open-boundary
    sum over the system tiled (2n+1) x (2n+1) times, seen from the central tile."""
    g = W.Geometry(6, 5, 3, 1e-6, 1e-6, 0.25e-6, MU, NU)
    t18, b18 = W.gan_families()
    p = W.random_problem(g, t18[[0, 9]], b18[[0, 9]], seed=3)
    n = 2
    T = 2 * n + 1
    pbc = oracle.stress_direct(g, p.t, p.b, p.rho, n_shells=n)
    gt = W.Geometry(g.nx * T, g.ny * T, g.nz, g.dx, g.dy, g.dz, MU, NU)
    tiled = np.tile(p.rho, (1, 1, T, T))
    tg = [(k * gt.ny + j + n * g.ny) * gt.nx + i + n * g.nx
          for k in range(g.nz) for j in range(g.ny) for i in range(g.nx)]
    ref = oracle.stress_direct(gt, p.t, p.b, tiled, targets=tg)
    assert rel(pbc, ref) < 1e-12


def test_replica_shells_converge_as_the_paper_states():
    gold = _read_golden("pbc_sec4.txt")
    acc = float(gold["accuracy"])
    g = W.Geometry(16, 16, 8, 1e-6, 1e-6, 1e-6, MU, NU)
    rng = np.random.default_rng(0)
    offs = list(zip(rng.integers(-15, 16, 30), rng.integers(-15, 16, 30), rng.integers(-7, 8, 30)))
    for t, b in [([0, 0, 1], [BB, 0, 0]), ([0, 0, 1], [0, 0, BB]), (W.t_mixed(), [BB, 0, 1.6 * BB])]:
        ref = np.array([oracle.interaction_pbc(g, *o, t, b, 80) for o in offs])
        scale = np.abs(ref).max(axis=0)
        for n in (int(gold["shells_low"]), int(gold["shells_high"])):
            F = np.array([oracle.interaction_pbc(g, *o, t, b, n) for o in offs])
            for c in range(6):
                if scale[c] > 1e-12 * scale.max():
                    assert np.abs(F[:, c] - ref[:, c]).max() < acc * scale[c], (t, b, n, c)


def test_replica_table_is_odd():
    g = W.Geometry(7, 6, 4, 1e-6, 1e-6, 0.25e-6, MU, NU)
    tab = oracle.gtable(g, W.t_mixed(), (BB, 0.3 * BB, 1.6 * BB), n_shells=3)
    assert rel(tab[::-1, ::-1, ::-1], -tab) < 1e-13


# ---------------------------------------------- periodic reading (Sec. 4) --
def test_periodic_reading_is_a_cyclic_convolution():
    """The periodic reading (replica shells centred on each source's minimal image) makes
    sigma exactly covariant under cyclic shifts of rho in x and y; the in-system-offset
    reading is not (the test has teeth)."""
    g = W.Geometry(8, 6, 3, 1e-6, 1e-6, 0.25e-6, MU, NU)
    t18, b18 = W.gan_families()
    p = W.random_problem(g, t18[[0, 9]], b18[[0, 9]], seed=4)
    shifted = np.roll(p.rho, (2, 3), axis=(2, 3))
    for periodic, tol in ((True, 1e-12), (False, None)):
        s0 = oracle.stress_direct(g, p.t, p.b, p.rho, n_shells=3, periodic=periodic).T.reshape(6, 3, 6, 8)
        s1 = oracle.stress_direct(g, p.t, p.b, shifted, n_shells=3, periodic=periodic).T.reshape(6, 3, 6, 8)
        err = rel(s1, np.roll(s0, (2, 3), axis=(2, 3)))
        if tol is not None:
            assert err < tol
        else:
            assert err > 1e-4


def test_periodic_table_is_odd_and_periodic():
    g = W.Geometry(8, 6, 4, 1e-6, 1e-6, 0.25e-6, MU, NU)
    tab = oracle.gtable(g, W.t_mixed(), (BB, 0.3 * BB, 1.6 * BB), n_shells=3, periodic=True)
    assert rel(tab[::-1, ::-1, ::-1], -tab) < 1e-13
    # offset i and i - nx are the same column of sources (index i + nx - 1 vs i - 1)
    assert rel(tab[:, :, g.nx:], tab[:, :, : g.nx - 1]) < 1e-15
    assert rel(tab[:, g.ny:, :], tab[:, : g.ny - 1, :]) < 1e-15
    # a half-period offset is the mean of its two minimal images
    t, b = (0, 0, 1), (BB, 0, 0)
    half = oracle.interaction_periodic(g, 4, 1, 2, t, b, 3)
    two = 0.5 * (oracle.interaction_pbc(g, 4, 1, 2, t, b, 3) + oracle.interaction_pbc(g, -4, 1, 2, t, b, 3))
    assert rel(half, two) < 1e-15


def test_periodic_reading_converges_as_the_paper_states_and_meets_the_other():
    gold = _read_golden("pbc_sec4.txt")
    acc = float(gold["accuracy"])
    g = W.Geometry(16, 16, 8, 1e-6, 1e-6, 1e-6, MU, NU)
    rng = np.random.default_rng(1)
    offs = list(zip(rng.integers(0, 16, 30), rng.integers(0, 16, 30), rng.integers(-7, 8, 30)))
    for t, b in [([0, 0, 1], [BB, 0, 0]), ([0, 0, 1], [0, 0, BB]), (W.t_mixed(), [BB, 0, 1.6 * BB])]:
        ref = np.array([oracle.interaction_periodic(g, *o, t, b, 80) for o in offs])
        scale = np.abs(ref).max(axis=0)
        for n in (int(gold["shells_low"]), int(gold["shells_high"])):
            F = np.array([oracle.interaction_periodic(g, *o, t, b, n) for o in offs])
            E = np.array([oracle.interaction_pbc(g, *o, t, b, n) for o in offs])   # the other reading
            for c in range(6):
                if scale[c] > 1e-12 * scale.max():
                    assert np.abs(F[:, c] - ref[:, c]).max() < acc * scale[c], (t, b, n, c)
                    assert np.abs(E[:, c] - ref[:, c]).max() < 2 * acc * scale[c], (t, b, n, c)


# ------------------------------------------------------- mirror parities --
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))   # xx, yy, zz, xy, xz, yz


def mirror_parity(a, b):
    """Parity of each component of G under the mirror x_a -> -x_a, for a line direction with
    t_a = 0 and b parallel or perpendicular to axis a.  Reflection Q maps the segment onto
    itself and the field of (t, b) at r onto det(Q) Q sigma Q^T of (t, Q b) at Q r, the
    det(Q) = -1 coming from the handedness of the Burgers circuit; Q b = s_b b."""
    s_b = -1.0 if b[a] != 0.0 else 1.0
    q = [(-1.0 if i == a else 1.0) for i in range(3)]
    return np.array([-s_b * q[i] * q[j] for i, j in PAIRS])


@pytest.mark.parametrize("cells", [(0.2e-6, 0.2e-6, 0.05e-6), (0.5e-6, 0.5e-6, 0.2e-6), (1e-6, 1e-6, 1e-6)])
def test_table_mirror_parities(cells):
    """The coefficient table (near field subdivided) is even or odd in x under the mirror
    x -> -x for every line direction in the y-z plane and Cartesian b, and in y as well for
    t = z, with the parities of the reflected field; the textbook edge field of an
    infinite line (Sec. 3, Fig. 5 discussion) shows the same parities.  Oblique b, or a
    line direction out of the mirror plane, break them (the test has teeth)."""
    g = W.Geometry(9, 8, 6, *cells, MU, NU)
    s15 = math.sin(math.radians(15.6))
    lines = [((0.0, 0.0, 1.0), (0, 1)), ((0.0, s15, math.sqrt(1 - s15 * s15)), (0,)),
             ((0.0, 0.5, math.sqrt(3) / 2), (0,))]
    for t, axes in lines:
        for d in range(3):
            b = np.zeros(3)
            b[d] = BB
            tab = oracle.gtable(g, t, b)
            m = np.abs(tab).max(axis=(0, 1, 2))
            for a in axes:
                flip = tab[:, :, ::-1] if a == 0 else tab[:, ::-1, :]
                p = mirror_parity(a, b)
                assert np.all(np.abs(flip - p * tab).max(axis=(0, 1, 2)) <= 1e-13 * m.max())
        # teeth: an oblique b has no x parity; a tilted line has no y parity
        tab = oracle.gtable(g, t, (BB, BB, 0.0))
        assert np.abs(tab[:, :, ::-1] - mirror_parity(0, (BB, 0, 0)) * tab).max() > 1e-3 * np.abs(tab).max()
    tab = oracle.gtable(g, lines[1][0], (BB, 0.0, 0.0))
    assert np.abs(tab[:, ::-1, :] - mirror_parity(1, (BB, 0, 0)) * tab).max() > 1e-3 * np.abs(tab).max()
    # the infinite edge line of Burgers vector along x: the same parities at a few points
    for x, y in [(1.3, 0.4), (0.2, 2.1)]:
        s = textbook_infinite(x, y, (BB, 0, 0))
        assert rel(textbook_infinite(-x, y, (BB, 0, 0)), mirror_parity(0, (BB, 0, 0)) * s) < 1e-14
        assert rel(textbook_infinite(x, -y, (BB, 0, 0)), mirror_parity(1, (BB, 0, 0)) * s) < 1e-14
