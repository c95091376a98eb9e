"""Host-side input generators: determinism, published PRNG values, config facts."""
import math

import numpy as np

import workloads as W


def test_splitmix64_published_values():
    # first outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014 reference code)
    got = [int(v) for v in W.splitmix64(0, np.arange(3))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    u = W.uniform01(7, np.arange(100000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(u, W.uniform01(7, np.arange(100000)))


def test_gaussian_disk_config():
    p = W.gaussian_disk_32()
    assert p.rho.shape == (1, 8, 32, 32)
    assert p.rho.max() == 1e14 * math.exp(-0.5 / 128.0)      # 4 centre cells, r^2 = 0.5
    assert np.array_equal(p.rho[0, 0], p.rho[0, 7])


def test_radial_disk_config():
    p = W.radial_disk_512()
    assert p.rho.shape == (2, 16, 512, 512)
    plane = p.rho[0, 0]
    assert plane[255, 255] > 1e13 and plane[0, 0] == 0.0
    assert np.array_equal(p.rho[0], p.rho[1])
    assert np.allclose(np.linalg.norm(p.t, axis=1), 1.0)


def test_gan_polycrystal_small():
    g = W.Geometry(32, 32, 6, 0.2e-6, 0.2e-6, 0.05e-6)
    p = W.gan_polycrystal(g, 1e-6, seed=3)
    assert p.rho.shape == (18, 6, 32, 32)
    nz_per_cell = (p.rho > 0).sum(axis=0)
    assert np.all(nz_per_cell == 2)                       # one edge + one mixed family per column
    edge = (p.rho[:6] > 0).sum(axis=0)
    assert np.all(edge == 1)
    prof = W.gan_height_profile(g)
    assert np.allclose(p.rho.max(axis=(0, 2, 3)), prof)
    assert p.meta["n_grains"] == round((6.4e-6) ** 2 / (math.pi * 0.25e-12))
    p2 = W.gan_polycrystal(g, 1e-6, seed=3)
    assert np.array_equal(p.rho, p2.rho)


def test_periodic_voronoi_is_nearest_periodic_image():
    n, k, seed = 24, 10, 3
    g = W.periodic_voronoi(n, k, seed)
    u = W.uniform01(seed, np.arange(2 * k))
    sx, sy = u[0::2], u[1::2]
    for (j, i) in [(0, 0), (5, 23), (23, 11), (12, 12), (7, 0)]:
        x, y = (i + 0.5) / n, (j + 0.5) / n
        best = min(range(k), key=lambda s: (min(abs(x - sx[s]), 1 - abs(x - sx[s])) ** 2 +
                                            min(abs(y - sy[s]), 1 - abs(y - sy[s])) ** 2, s))
        assert g[j, i] == best


def test_scaled_polycrystal_scales_one_pattern():
    a = W.scaled_polycrystal(32, 4, 2e-6, 10e-6)
    b = W.scaled_polycrystal(32, 4, 8e-6, 10e-6)
    assert np.array_equal(a.rho, b.rho)
    assert abs(b.geom.dx / a.geom.dx - 4.0) < 1e-12 and a.geom.dz == b.geom.dz
    assert abs(a.geom.nx * a.geom.dx - 10 * 2e-6) < 1e-18
    # every column carries exactly one orientation, uniform in height
    assert np.all((a.rho > 0).sum(axis=0) == 1)
    assert np.all(a.rho[:, 0] == a.rho[:, -1])


def test_serving_stream_draws_family_subsets_and_seeds():
    a = W.serving_stream(0, 20.0, 200.0)
    assert abs(len(a) / 20.0 - 200.0) < 15                      # Poisson rate
    assert all(x.time < y.time for x, y in zip(a, a[1:]))
    assert [x.seed for x in a] == list(range(len(a)))            # one grain seed per request
    for x in a:
        assert 1 <= len(x.fam) <= 4 and list(x.fam) == sorted(set(x.fam)) and all(0 <= f < 18 for f in x.fam)
    counts = np.bincount([len(x.fam) for x in a], minlength=5)[1:]
    assert counts.min() > 0.8 * len(a) / 4                       # family counts uniform over 1..4
    per_family = np.bincount([f for x in a for f in x.fam], minlength=18)
    assert per_family.min() > 0.7 * per_family.mean()            # every family drawn
    assert W.serving_stream(0, 20.0, 200.0)[5] == a[5]           # seeded
    s = W.serving_slots(0, 1, 3)
    assert s.shape == (4, 64, 64, 64) and s.dtype == np.float32
    assert np.allclose(s.sum(axis=0), W.gan_height_profile(W.serving_geometry(0, 1))[:, None, None])
