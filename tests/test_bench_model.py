"""The byte model behind bench.py's roofline figures, on the CPU.

The algorithmic bytes of each pass are written out here from what the pass moves
(complex FP32 = 8 bytes, kernel spectra = one FP32 imaginary part per value) for the
two bench-sized grids, and compared with bench.pass_bytes / bench.floor_bytes and with
the per-launch figures quoted in the profiles (1.345 GB and 5.524 GB for the fused z pass
with every spectrum column stored; 3.519 GB for the GaN layer, whose five fields all have
the x-mirror parity, so that only the columns ky <= py/2 and the Nyquist column are
stored).
"""
from types import SimpleNamespace

import bench
import workloads as W


def padded(nx, ny, nz):
    p2 = lambda n: 1 << (2 * n - 1).bit_length()
    return max(32, p2(nx)), max(32, p2(ny)), max(16, p2(nz))


CASES = [   # (nx, ny, nz), families, fields, z-pass bytes quoted in the profiles
    ((512, 512, 16), 2, 2, 1_344_798_720),
    ((256, 256, 128), 18, 5, 5_524_422_656),
]


def test_pass_bytes_from_first_principles():
    for (nx, ny, nz), fin, fe, z_quoted in CASES:
        px, py, pz = padded(nx, ny, nz)
        q = {"n_fields": fe, "px": px, "py": py, "pz": pz}
        p = SimpleNamespace(geom=W.Geometry(nx, ny, nz, 1e-6, 1e-6, 1e-6), n_families=fin)
        cols = px // 2 + 1                         # half spectrum along x, Nyquist included
        n = nx * ny * nz
        after_x = cols * ny * nz * 8               # one field or component after the x pass
        after_y = cols * py * nz * 8               # ... after the y pass (z rows < nz)
        spectra = 6 * fe * cols * py * pz * 4
        want = {
            "x_fwd": 4 * fin * n + fe * after_x,
            "y_fwd": fe * after_x + fe * after_y,
            "z_fused": fe * after_y + spectra + 6 * after_y,
            "y_inv": 6 * after_y + 6 * after_x,
            "x_inv": 6 * after_x + 6 * 4 * n,
        }
        assert bench.pass_bytes(p, q) == want
        assert want["z_fused"] == z_quoted
        assert bench.floor_bytes(p, q) == 4 * fin * n + spectra + 6 * 4 * n


def test_mirror_stored_spectra_bytes():
    # GaN layer: main columns (kx < px/2, ky <= py/2) and all Nyquist columns (kx = px/2)
    nx, ny, nz, fin, fe = 256, 256, 128, 18, 5
    px, py, pz = padded(nx, ny, nz)
    stored_cols = (px // 2) * (py // 2 + 1) + py
    spectra = 6 * fe * pz * 4 * stored_cols
    q = {"n_fields": fe, "px": px, "py": py, "pz": pz, "spectra_bytes": spectra}
    p = SimpleNamespace(geom=W.Geometry(nx, ny, nz, 1e-6, 1e-6, 1e-6), n_families=fin)
    after_y = (px // 2 + 1) * py * nz * 8
    assert bench.pass_bytes(p, q)["z_fused"] == fe * after_y + spectra + 6 * after_y == 3_519_021_056
    assert abs(spectra / (6 * fe * (px // 2 + 1) * py * pz * 4) - 0.5039) < 1e-4


def test_pass_model_per_cell_closed_form():
    # per unpadded cell, with px = 2 nx, py = 2 ny, pz = 2 nz and nx large:
    # 4 F_in + 144 F_e + 312 bytes (x 8F_e, y 24F_e, z 112F_e + 96, y 144, x 72)
    nx, ny, nz, fin, fe = 4096, 64, 32, 3, 2
    q = {"n_fields": fe, "px": 2 * nx, "py": 2 * ny, "pz": 2 * nz}
    p = SimpleNamespace(geom=W.Geometry(nx, ny, nz, 1e-6, 1e-6, 1e-6), n_families=fin)
    per_cell = sum(bench.pass_bytes(p, q).values()) / (nx * ny * nz)
    assert abs(per_cell - (4 * fin + 144 * fe + 312)) / per_cell < 1e-3    # the Nyquist column


def test_roofline_per_cell_figures_match_the_exact_model():
    # the per-cell figures bench.py divides by the dominant kernel's time (the planned
    # schedule's model, spectra read in full) are the large-grid limit of pass_bytes
    nx, ny, nz, fin, fe = 4096, 64, 32, 18, 5
    q = {"n_fields": fe, "px": 2 * nx, "py": 2 * ny, "pz": 2 * nz}
    p = SimpleNamespace(geom=W.Geometry(nx, ny, nz, 1e-6, 1e-6, 1e-6), n_families=fin)
    exact = bench.pass_bytes(p, q)
    model = bench.pass_model_per_cell(p, q)
    assert model == {"x_fwd": 4 * fin + 8 * fe, "y_fwd": 24 * fe, "z_fused": 112 * fe + 96, "y_inv": 144,
                     "x_inv": 72}
    for k in exact:
        assert abs(exact[k] / (nx * ny * nz) - model[k]) / model[k] < 1e-3, k
    # the GaN layer: 656 bytes per cell for the fused z pass, 5.50 GB per launch
    g = W.Geometry(256, 256, 128, 1e-6, 1e-6, 1e-6)
    assert bench.pass_model_per_cell(SimpleNamespace(geom=g, n_families=18), {"n_fields": 5})["z_fused"] \
        * g.n_cells == 5_502_926_848
