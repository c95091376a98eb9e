"""Python binding of the FP64 CPU oracle (``dds_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product path.  It shares no
code with the CUDA library.  ``build()`` compiles the C file with gcc (OpenMP,
no fast-math, no floating-point contraction); the shared object is git-ignored.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "dds_oracle.c"
_LIB = _HERE / "libdds_oracle.so"
_lib = None


class OrcGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double * 3), ("mu", ctypes.c_double), ("nu", ctypes.c_double),
                ("n_near", ctypes.c_double), ("n_shells", ctypes.c_int), ("periodic", ctypes.c_int)]


def build(force: bool = False) -> Path:
    """Compile the oracle into ``oracle/libdds_oracle.so`` (skipped if up to date)."""
    if (not force and _LIB.exists()
            and _LIB.stat().st_mtime >= max(_SRC.stat().st_mtime, (_HERE / "dds_oracle.h").stat().st_mtime)):
        return _LIB
    tmp = _LIB.with_suffix(f".so.{os.getpid()}")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
           "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        ip = ctypes.POINTER(ctypes.c_int)
        gp = ctypes.POINTER(OrcGeom)
        lib.orc_segment_eq4.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                        ctypes.c_double, dp]
        lib.orc_segment_eq6.argtypes = [dp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, dp]
        lib.orc_segment_eq6.restype = ctypes.c_int
        lib.orc_subcells.argtypes = [dp, ip]
        lib.orc_chord.argtypes = [dp, dp]
        lib.orc_chord.restype = ctypes.c_double
        lib.orc_interaction.argtypes = [gp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_gtable.argtypes = [gp, dp, dp, dp]
        lib.orc_interaction_pbc.argtypes = [gp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_interaction_periodic.argtypes = [gp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_stress_direct.argtypes = [gp, ctypes.c_int, dp, dp, dp, ctypes.c_long, lp,
                                          ctypes.c_int, dp]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


def geom_struct(geom, n_near: float = 3.0, n_shells: int = 0, periodic: bool = False) -> OrcGeom:
    g = OrcGeom()
    g.nx, g.ny, g.nz = int(geom.nx), int(geom.ny), int(geom.nz)
    g.h[0], g.h[1], g.h[2] = float(geom.dx), float(geom.dy), float(geom.dz)
    g.mu, g.nu = float(geom.mu), float(geom.nu)
    g.n_near = float(n_near)
    g.n_shells = int(n_shells)
    g.periodic = int(bool(periodic))
    return g


def segment_eq4(obs, zA: float, zB: float, b, mu: float, nu: float) -> np.ndarray:
    """Eq. 4a-4c + Eq. 5: vertical segment (0,0,zA)->(0,0,zB); returns xx,yy,zz,xy,xz,yz."""
    lib = _load()
    out = np.zeros(6)
    lib.orc_segment_eq4(_dp(_vec(obs)), zA, zB, _dp(_vec(b)), mu, nu, _dp(out))
    return out


def segment_eq6(obs, A, B, t, b, mu: float, nu: float, form: int = 0) -> np.ndarray:
    """Eq. 6/7: straight segment A->B, unit direction t, Burgers b."""
    lib = _load()
    out = np.zeros(6)
    lib.orc_segment_eq6(_dp(_vec(obs)), _dp(_vec(A)), _dp(_vec(B)), _dp(_vec(t)), _dp(_vec(b)),
                        mu, nu, int(form), _dp(out))
    return out


def subcells(h) -> tuple:
    lib = _load()
    m = (ctypes.c_int * 3)()
    lib.orc_subcells(_dp(_vec(h)), m)
    return (m[0], m[1], m[2])


def chord(h, t) -> float:
    return float(_load().orc_chord(_dp(_vec(h)), _dp(_vec(t))))


def interaction(geom, i: int, j: int, k: int, t, b, n_near: float = 3.0) -> np.ndarray:
    """G(Delta) for offset (i,j,k) cells (observer minus source), one family."""
    lib = _load()
    g = geom_struct(geom, n_near)
    out = np.zeros(6)
    lib.orc_interaction(ctypes.byref(g), int(i), int(j), int(k), _dp(_vec(t)), _dp(_vec(b)), _dp(out))
    return out


def interaction_pbc(geom, i: int, j: int, k: int, t, b, n_shells: int, n_near: float = 3.0) -> np.ndarray:
    """Eq. 13: replica sum of G over |k|,|l| <= n_shells for offset (i,j,k), one family."""
    lib = _load()
    g = geom_struct(geom, n_near, n_shells)
    out = np.zeros(6)
    lib.orc_interaction_pbc(ctypes.byref(g), int(i), int(j), int(k), _dp(_vec(t)), _dp(_vec(b)), _dp(out))
    return out


def interaction_periodic(geom, i: int, j: int, k: int, t, b, n_shells: int, n_near: float = 3.0) -> np.ndarray:
    """Periodic reading of the replica sum: images of the minimal in-plane offset (i, j)
    mod (nx, ny) within n_shells periods, ties at half a period averaged; one family."""
    lib = _load()
    g = geom_struct(geom, n_near, n_shells, periodic=True)
    out = np.zeros(6)
    lib.orc_interaction_periodic(ctypes.byref(g), int(i), int(j), int(k), _dp(_vec(t)), _dp(_vec(b)), _dp(out))
    return out


def gtable(geom, t, b, n_near: float = 3.0, n_shells: int = 0, periodic: bool = False) -> np.ndarray:
    """Full table, shape (2nz-1, 2ny-1, 2nx-1, 6); index [k+nz-1, j+ny-1, i+nx-1]."""
    lib = _load()
    g = geom_struct(geom, n_near, n_shells, periodic)
    out = np.zeros((2 * geom.nz - 1, 2 * geom.ny - 1, 2 * geom.nx - 1, 6))
    lib.orc_gtable(ctypes.byref(g), _dp(_vec(t)), _dp(_vec(b)), _dp(out))
    return out


def stress_direct(geom, t, b, rho, targets=None, n_near: float = 3.0,
                  use_table: bool | None = None, n_shells: int = 0, periodic: bool = False) -> np.ndarray:
    """Eq. 10 summed over families by direct summation.

    rho: (F, nz, ny, nx) in m^-2; targets: linear cell indices (default: all cells).
    Returns (ntargets, 6).  With ``use_table`` (default: when the tables are small)
    each family's full coefficient table is built first."""
    lib = _load()
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1, 3))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1, 3))
    F = t.shape[0]
    rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(F, geom.nz, geom.ny, geom.nx))
    if targets is None:
        targets = np.arange(geom.n_cells)
    targets = np.ascontiguousarray(np.asarray(targets, dtype=np.int64).ravel())
    if use_table is None:
        n_off = (2 * geom.nx - 1) * (2 * geom.ny - 1) * (2 * geom.nz - 1)
        use_table = n_off * 48 <= 256 * 2 ** 20 and n_off <= 4 * targets.size * geom.n_cells
    g = geom_struct(geom, n_near, n_shells, periodic)
    out = np.zeros((targets.size, 6))
    lib.orc_stress_direct(ctypes.byref(g), F, _dp(t), _dp(b), _dp(rho), targets.size,
                          targets.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), int(bool(use_table)),
                          _dp(out))
    return out


def num_threads() -> int:
    return int(_load().orc_num_threads())
