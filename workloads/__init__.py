"""Seeded synthetic inputs for the dislocation-density stress path.

This module only *generates inputs*: grid geometry, dislocation families
(line direction t, Burgers vector b) and site-dependent densities rho_f.
It contains none of the method's arithmetic (no segment stress, no
interaction coefficients, no FFT), so the FP64 oracle and the GPU path can
both consume what it produces without sharing any computation.

Units are SI throughout: lengths in metres, moduli in pascal, densities as
dislocation lines per unit area in m^-2 (the paper quotes cm^-2; 1 cm^-2 =
1e4 m^-2).  Arrays are C-ordered ``[F][nz][ny][nx]`` (x fastest), cell (i,j,k)
centred at ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz).

Workload shapes follow the paper's experiments: the disk with a radially /
vertically varying density of one dislocation type (Sec. 3, Eq. 11, Figs. 4-6)
and the columnar Voronoi polycrystal with per-grain Burgers vectors drawn from
the six hexagonal a-type directions, edge and mixed (Sec. 6, Eq. 19).

Random numbers come from the counter-based SplitMix64 generator (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
draw i of stream ``seed`` is mix(seed + (i+1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CM2 = 1.0e4          # 1 cm^-2 in m^-2
UM = 1.0e-6          # 1 micrometre in m
NM = 1.0e-9

# Material constants used by every configuration (isotropic, GaN-like).
MU_GAN = 68.0e9
NU_GAN = 0.23
A_LATT = 0.319 * NM   # a-type Burgers length used by the configurations
C_LATT = 0.519 * NM   # c-type Burgers length

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index) -> np.ndarray:
    """SplitMix64 output for draws ``index`` (array-like of ints) of stream ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, index) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Geometry:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    mu: float = MU_GAN
    nu: float = NU_GAN

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclass
class Problem:
    """One stress evaluation: geometry, F families and F density fields."""
    name: str
    geom: Geometry
    t: np.ndarray            # (F, 3) unit line directions
    b: np.ndarray            # (F, 3) Burgers vectors (m)
    rho: np.ndarray          # (F, nz, ny, nx) float64, m^-2
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.t = np.ascontiguousarray(self.t, dtype=np.float64).reshape(-1, 3)
        self.b = np.ascontiguousarray(self.b, dtype=np.float64).reshape(-1, 3)
        self.rho = np.ascontiguousarray(self.rho, dtype=np.float64)

    @property
    def n_families(self) -> int:
        return int(self.t.shape[0])


def hex_a(i: int, a: float = A_LATT) -> np.ndarray:
    """In-plane a-type Burgers vector number i (0..5): a (cos 60 i, sin 60 i, 0)."""
    ang = math.radians(60.0 * i)
    return np.array([a * math.cos(ang), a * math.sin(ang), 0.0])


T_Z = np.array([0.0, 0.0, 1.0])


def t_mixed(incline_deg: float = 15.6) -> np.ndarray:
    """Mixed-dislocation line direction tilted by ``incline_deg`` from z in the y-z plane."""
    a = math.radians(incline_deg)
    return np.array([0.0, math.sin(a), math.cos(a)])


def cell_centres_xy(geom: Geometry):
    x = (np.arange(geom.nx) + 0.5) * geom.dx
    y = (np.arange(geom.ny) + 0.5) * geom.dy
    return np.meshgrid(x, y, indexing="xy")   # (ny, nx)


def cell_centres_z(geom: Geometry) -> np.ndarray:
    return (np.arange(geom.nz) + 0.5) * geom.dz


# ---------------------------------------------------------------------------
# Configurations
# ---------------------------------------------------------------------------

def gaussian_disk_32() -> Problem:
    """32x32x8 grid of 1x1x0.25 um cells, one family of vertical edge dislocations
    (t = z, b = 0.319 nm along x), density 1e10 cm^-2 * exp(-r^2 / (2 * 8^2)) with r
    in cells from the grid centre, uniform in z (the Gaussian disk profile of Eq. 11
    without the z decay)."""
    g = Geometry(32, 32, 8, 1.0 * UM, 1.0 * UM, 0.25 * UM)
    i = np.arange(g.nx) - 15.5
    j = np.arange(g.ny) - 15.5
    r2 = j[:, None] ** 2 + i[None, :] ** 2
    plane = 1.0e10 * CM2 * np.exp(-r2 / (2.0 * 8.0 ** 2))
    rho = np.broadcast_to(plane, (1, g.nz, g.ny, g.nx)).astype(np.float64).copy()
    return Problem("gaussian_disk_32x32x8", g, T_Z[None, :].copy(),
                   np.array([[A_LATT, 0.0, 0.0]]), rho)


def radial_disk_512() -> Problem:
    """512x512x16 grid of 0.5x0.5x0.2 um cells; two families carrying the same density
    rho(r) = 1e9 (1 + 4 (r/R)^2) cm^-2 inside a disk of radius R = 240 cells about the
    grid centre, zero outside, uniform in z.  Family 1: vertical edge (t = z, b = a x).
    Family 2: mixed, t = (0, 1/2, sqrt3/2), b = (a/2, sqrt3 a/2, c), the mixed type of
    the paper's disk example (Sec. 3, Fig. 6)."""
    g = Geometry(512, 512, 16, 0.5 * UM, 0.5 * UM, 0.2 * UM)
    i = np.arange(g.nx) - 255.5
    j = np.arange(g.ny) - 255.5
    r = np.sqrt(j[:, None] ** 2 + i[None, :] ** 2)
    R = 240.0
    plane = np.where(r < R, 1.0e9 * CM2 * (1.0 + 4.0 * (r / R) ** 2), 0.0)
    rho1 = np.broadcast_to(plane, (g.nz, g.ny, g.nx))
    rho = np.stack([rho1, rho1]).astype(np.float64)
    s3 = math.sqrt(3.0)
    t = np.array([[0.0, 0.0, 1.0], [0.0, 0.5, s3 / 2.0]])
    b = np.array([[A_LATT, 0.0, 0.0], [A_LATT / 2.0, s3 * A_LATT / 2.0, C_LATT]])
    return Problem("radial_disk_512x512x16", g, t, b, rho)


def gan_families(incline_deg: float = 15.6):
    """The 18 families of the polycrystalline GaN-like layer: 6 vertical edge
    dislocations with b = a_i, then 12 mixed ones (tilted t, b = a_i + s c z,
    s = +1 for even slots, -1 for odd).  Returns (t, b) arrays of shape (18, 3)."""
    t = []
    b = []
    for i in range(6):
        t.append(T_Z)
        b.append(hex_a(i))
    tm = t_mixed(incline_deg)
    for i in range(6):
        for s in (1.0, -1.0):
            t.append(tm)
            b.append(hex_a(i) + np.array([0.0, 0.0, s * C_LATT]))
    return np.array(t), np.array(b)


def voronoi_columns(geom: Geometry, n_seeds: int, seed: int) -> np.ndarray:
    """Grain id per column (ny, nx): nearest of ``n_seeds`` seeds drawn uniformly in
    the layer plane (open boundary), ties to the lower id.  Vertical grain boundaries
    as in the paper's polycrystal (Sec. 6)."""
    Lx, Ly = geom.nx * geom.dx, geom.ny * geom.dy
    u = uniform01(seed, np.arange(2 * n_seeds))
    sx = Lx * u[0::2]
    sy = Ly * u[1::2]
    X, Y = cell_centres_xy(geom)
    xs = X.ravel()
    ys = Y.ravel()
    try:                                     # k-d tree when scipy is present (same nearest seed)
        from scipy.spatial import cKDTree
        _, idx = cKDTree(np.stack([sx, sy], axis=1)).query(np.stack([xs, ys], axis=1))
        return np.asarray(idx, dtype=np.int64).reshape(geom.ny, geom.nx)
    except ImportError:
        pass
    best = np.zeros(xs.size, dtype=np.int64)
    bestd = np.full(xs.size, np.inf)
    chunk = 64
    for k0 in range(0, n_seeds, chunk):     # ascending ids; argmin keeps the lowest id on ties
        d = (xs[:, None] - sx[None, k0:k0 + chunk]) ** 2 + (ys[:, None] - sy[None, k0:k0 + chunk]) ** 2
        j = np.argmin(d, axis=1)
        dj = d[np.arange(xs.size), j]
        m = dj < bestd
        best[m] = k0 + j[m]
        bestd[m] = dj[m]
    return best.reshape(geom.ny, geom.nx)


def gan_height_profile(geom: Geometry) -> np.ndarray:
    """rho(z) = 1e10 exp(-z / 0.5 um) + 1e8 cm^-2 at the cell-centre heights."""
    z = cell_centres_z(geom)
    return (1.0e10 * np.exp(-z / (0.5 * UM)) + 1.0e8) * CM2


def gan_polycrystal_parts(geom: Geometry, grain_diameter: float, seed: int):
    """The factors of ``gan_polycrystal``'s density: per family a column mask (F, ny, nx)
    and the height profile rho(z) (nz,), so that rho[f, z, y, x] = prof[z] * mask[f, y, x].
    Returns (t, b, mask, prof, n_grains)."""
    Lx, Ly = geom.nx * geom.dx, geom.ny * geom.dy
    n_seeds = max(1, int(round(Lx * Ly / (math.pi * (grain_diameter / 2.0) ** 2))))
    grains = voronoi_columns(geom, n_seeds, seed)
    u = uniform01(seed, 2 * n_seeds + np.arange(3 * n_seeds))
    edge_idx = np.minimum((6.0 * u[0::3]).astype(np.int64), 5)
    mix_idx = np.minimum((6.0 * u[1::3]).astype(np.int64), 5)
    mix_sign = (u[2::3] >= 0.5).astype(np.int64)         # 0 -> +c, 1 -> -c
    t, b = gan_families()
    F = t.shape[0]
    fam_edge = edge_idx[grains]                          # (ny, nx)
    fam_mix = 6 + 2 * mix_idx[grains] + mix_sign[grains]
    mask = np.stack([(fam_edge == f) | (fam_mix == f) for f in range(F)])
    return t, b, mask, gan_height_profile(geom), n_seeds


def gan_polycrystal(geom: Geometry, grain_diameter: float, seed: int,
                    name: str = "gan_polycrystal") -> Problem:
    """Columnar Voronoi polycrystal with mean grain diameter ``grain_diameter``.
    Each grain draws one edge family (b = a_i) and one mixed family (b = a_i +- c);
    both carry the height profile rho(z) in every cell of the grain."""
    t, b, mask, prof, n_seeds = gan_polycrystal_parts(geom, grain_diameter, seed)
    rho = prof[None, :, None, None] * mask[:, None, :, :].astype(np.float64)
    return Problem(name, geom, t, b, rho,
                   meta={"n_grains": n_seeds, "grain_diameter": grain_diameter, "seed": seed})



def gan_layer_256(seed: int = 0) -> Problem:
    """256x256x128 grid of 0.2x0.2x0.05 um cells, Voronoi grains of mean diameter 2 um,
    18 families (6 edge + 12 mixed), height profile 1e10 exp(-z/0.5um) + 1e8 cm^-2."""
    g = Geometry(256, 256, 128, 0.2 * UM, 0.2 * UM, 0.05 * UM)
    return gan_polycrystal(g, 2.0 * UM, seed, name="gan_layer_256x256x128")


def gan_layer_128(seed: int = 0) -> Problem:
    """The GaN layer's cells, grains, families and height profile on a 128x128x128 grid
    (one of the sweep grids): the same padded z size with a quarter of the columns, for
    profiling captures that must stay small."""
    g = Geometry(128, 128, 128, 0.2 * UM, 0.2 * UM, 0.05 * UM)
    return gan_polycrystal(g, 2.0 * UM, seed, name="gan_layer_128x128x128")


def gan_layer_256_thin(seed: int = 0) -> Problem:
    """The GaN layer's cells, grains, families and height profile on a 256x256x32 grid:
    the same in-plane transforms as the 256x256x128 layer (padded 512 x 512) on a quarter
    of its planes, for profiling captures that must stay small."""
    g = Geometry(256, 256, 32, 0.2 * UM, 0.2 * UM, 0.05 * UM)
    return gan_polycrystal(g, 2.0 * UM, seed, name="gan_layer_256x256x32")


SWEEP_GRIDS = [(128, 128, 64), (128, 128, 128), (256, 256, 64), (256, 256, 128)]


def periodic_voronoi(n: int, n_seeds: int, seed: int) -> np.ndarray:
    """Grain id per column (n, n) of a square cell grid with periodic sides: nearest of
    ``n_seeds`` seeds drawn uniformly in the unit square, distances taken to the nearest
    periodic image (ties to the lower id).  Scale-free: the same ids for every size."""
    u = uniform01(seed, np.arange(2 * n_seeds))
    sx, sy = u[0::2], u[1::2]
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c, indexing="xy")
    best = np.zeros(X.size, dtype=np.int64)
    bestd = np.full(X.size, np.inf)
    for k in range(n_seeds):                 # ascending ids; strict < keeps the lowest id on ties
        dx = np.abs(X.ravel() - sx[k])
        dy = np.abs(Y.ravel() - sy[k])
        dx = np.minimum(dx, 1.0 - dx)
        dy = np.minimum(dy, 1.0 - dy)
        d = dx * dx + dy * dy
        m = d < bestd
        best[m] = k
        bestd[m] = d[m]
    return best.reshape(n, n)


def scaled_polycrystal(n: int, nz: int, grain_size: float, thickness: float, n_grains: int = 100,
                       seed: int = 0, rho_d: float = 1.0e9 * CM2) -> Problem:
    """The grain-size study of Sec. 6.4-6.5: one fixed columnar grain pattern of
    ``n_grains`` periodic Voronoi grains on a square of side L = 10 D (so the mean grain
    area is D^2), scaled with D; vertical edge dislocations (t = z) whose Burgers vector
    a_i is drawn per grain from the six in-plane orientations; density rho_d uniform in
    height (the vertically homogeneous layer of Sec. 6.5).  n x n x nz cells over a
    layer of the given thickness.  Six families, one per orientation."""
    L = 10.0 * grain_size
    geom = Geometry(n, n, nz, L / n, L / n, thickness / nz)
    grains = periodic_voronoi(n, n_grains, seed)
    u = uniform01(seed, 2 * n_grains + np.arange(n_grains))
    orient = np.minimum((6.0 * u).astype(np.int64), 5)[grains]
    t = np.array([T_Z] * 6)
    b = np.array([hex_a(i) for i in range(6)])
    rho = np.zeros((6, nz, n, n))
    for f in range(6):
        rho[f] = rho_d * (orient == f)[None, :, :]
    return Problem(f"scaled_polycrystal_D{grain_size:.3g}_H{thickness:.3g}", geom, t, b, rho,
                   meta={"n_grains": n_grains, "grain_size": grain_size, "thickness": thickness, "seed": seed})


def sweep_spec(r: int):
    """Grid and grain diameter of realisation r of the grain-size sweep: grid drawn
    uniformly from SWEEP_GRIDS, grain diameter log-uniform in [0.5, 8] um."""
    u = uniform01(1000 + r, np.arange(2))
    nx, ny, nz = SWEEP_GRIDS[min(int(4 * u[0]), 3)]
    D = math.exp(math.log(0.5) + (math.log(8.0) - math.log(0.5)) * u[1]) * UM
    return Geometry(nx, ny, nz, 0.2 * UM, 0.2 * UM, 0.05 * UM), D


def sweep_realisation(r: int) -> Problem:
    """Realisation r of the grain-size sweep: cells 0.2x0.2x0.05 um, grid and grain
    diameter from sweep_spec(r), grain seed r."""
    g, D = sweep_spec(r)
    return gan_polycrystal(g, D, r, name=f"sweep_{r}")


# Serving stream: per request a grid, a cell aspect dz/dx (dx = dy = 0.2 um), 1 to 4
# families drawn from the 18 of gan_families(), and a grain seed (the request id).
SERVING_GRIDS = [(64, 64, 64), (128, 128, 64), (256, 256, 128), (512, 512, 64)]
SERVING_ASPECTS = [0.1, 0.25, 1.0]
SERVING_MAX_FAMILIES = 4


@dataclass
class ServingArrival:
    time: float              # s after the start of the stream
    grid: int                # index into SERVING_GRIDS
    aspect: int              # index into SERVING_ASPECTS
    fam: tuple               # 1..4 distinct indices into gan_families(), ascending
    seed: int                # grain seed of the request's polycrystal


def serving_stream(seed: int, duration: float, rate: float):
    """Poisson arrivals at `rate` per second for `duration` seconds, as a list of
    ServingArrival; request i draws its grid, aspect and family count uniformly, its
    families as a uniform random subset of the 18, and grain seed i."""
    out = []
    t = 0.0
    i = 0
    while True:
        u = uniform01(seed, np.arange(24 * i, 24 * i + 24))
        t += -math.log(1.0 - u[0]) / rate
        if t >= duration:
            return out
        k = 1 + min(int(SERVING_MAX_FAMILIES * u[3]), SERVING_MAX_FAMILIES - 1)
        order = np.argsort(u[4:22], kind="stable")         # a uniform random permutation of 18
        fam = tuple(sorted(int(f) for f in order[:k]))
        out.append(ServingArrival(t, min(int(4 * u[1]), 3), min(int(3 * u[2]), 2), fam, i))
        i += 1


@dataclass
class ServingCase:
    geom: Geometry
    t: np.ndarray            # (18, 3): every request of the geometry shares one context
    b: np.ndarray
    rho: np.ndarray          # (n, nz, ny, nx) float32 for the families fam
    fam: tuple


def serving_geometry(grid_idx: int, aspect_idx: int) -> Geometry:
    nx, ny, nz = SERVING_GRIDS[grid_idx]
    dx = 0.2 * UM
    return Geometry(nx, ny, nz, dx, dx, dx * SERVING_ASPECTS[aspect_idx])


def serving_slots(grid_idx: int, aspect_idx: int, grain_seed: int) -> np.ndarray:
    """The densities of up to four families of one request's polycrystal: Voronoi
    columns (2 um grains, seeds from grain_seed) whose grains take the four family slots
    in turn, each slot carrying the GaN height profile.  Shape (4, nz, ny, nx), float32;
    a request with k families uses the first k slots."""
    g = serving_geometry(grid_idx, aspect_idx)
    n_seeds = max(1, int(round(g.nx * g.dx * g.ny * g.dy / (math.pi * UM ** 2))))
    grains = voronoi_columns(g, n_seeds, grain_seed)
    prof = gan_height_profile(g).astype(np.float32)
    rho = np.empty((SERVING_MAX_FAMILIES, g.nz, g.ny, g.nx), dtype=np.float32)
    for q in range(SERVING_MAX_FAMILIES):
        mask = ((grains % SERVING_MAX_FAMILIES) == q).astype(np.float32)
        np.multiply(prof[:, None, None], mask[None], out=rho[q])
    return rho


def serving_problem(a: ServingArrival, slots: np.ndarray | None = None) -> ServingCase:
    """The request of arrival `a` (slots: serving_slots of its geometry and grain seed,
    when already made)."""
    g = serving_geometry(a.grid, a.aspect)
    if slots is None:
        slots = serving_slots(a.grid, a.aspect, a.seed)
    t18, b18 = gan_families()
    return ServingCase(g, t18, b18, slots[: len(a.fam)], a.fam)


def random_problem(geom: Geometry, t: np.ndarray, b: np.ndarray, seed: int,
                   scale: float = 1.0e10 * CM2) -> Problem:
    """Uniform random densities in [0, scale) for each family (parity tests)."""
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    F = t.shape[0]
    n = F * geom.n_cells
    rho = (scale * uniform01(seed, np.arange(n))).reshape(F, geom.nz, geom.ny, geom.nx)
    return Problem(f"random_{seed}", geom, t, b, rho)


CONFIGS = {
    "gaussian_disk_32x32x8": gaussian_disk_32,
    "radial_disk_512x512x16": radial_disk_512,
    "gan_layer_256x256x128": gan_layer_256,
    "gan_layer_128x128x128": gan_layer_128,
    "gan_layer_256x256x32": gan_layer_256_thin,
}
