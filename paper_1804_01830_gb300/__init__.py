"""GB300 dislocation-density stress: Python binding of ``libdds.so``.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/dds.h``.  The module-level
functions carry the C names (``dds_create``, ``dds_set_geometry``, ...);
``StressContext`` wraps them for convenience.  PyTorch supplies device memory
and streams.  If the library has not been built this module raises on import of
any entry point -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libdds.so"

DDS_OK = 0
DDS_ERR_INVALID_ARG = -1
DDS_ERR_NOT_READY = -2
DDS_ERR_OOM = -3
DDS_ERR_CUDA = -4
DDS_ERR_TIMEOUT = -5
DDS_ERR_UNSUPPORTED = -6
DDS_F32 = 0
DDS_BF16 = 1
DDS_OPT_NEAR_RADIUS = 1
DDS_OPT_Z_LANES = 2
DDS_OPT_SPECTRA_FP16 = 3
DDS_OPT_PBC_SHELLS = 4
DDS_OPT_PBC_PERIODIC = 5
DDS_OPT_YX_FUSED = 6

# Every symbol include/dds.h declares.
EXPORTS = ("dds_create", "dds_set_geometry", "dds_set_families", "dds_set_option", "dds_autotune",
           "dds_build_kernels", "dds_stress", "dds_stress_multi", "dds_stress_stats", "dds_stress_batched",
           "dds_stress_noalloc", "dds_stress_subset",
           "dds_stress_host", "dds_stress_host_async", "dds_stress_host_sync",
           "dds_table_at", "dds_query", "dds_footprint", "dds_spectra_bytes", "dds_contract_spectra", "dds_launches_per_stress", "dds_yx_cluster",
           "dds_profile_enable",
           "dds_profile_read", "dds_relax", "dds_graph_capture", "dds_graph_launch", "dds_graph_nodes",
           "dds_graph_destroy", "dds_device_status", "dds_last_error", "dds_destroy")

PASS_NAMES = ("x_fwd", "y_fwd", "z_fused", "y_inv", "x_inv")

_lib = None


class DDSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dds error {code}: {msg}")
        self.code = code


def load_library():
    """Load libdds.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(str(LIB_PATH))
    vp, dp, ip, lp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_long
    sig = {
        "dds_create": ([ctypes.POINTER(vp), ctypes.c_int], ctypes.c_int),
        "dds_set_geometry": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "dds_set_families": ([vp, ctypes.c_int, dp, dp], ctypes.c_int),
        "dds_set_option": ([vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
        "dds_build_kernels": ([vp, vp], ctypes.c_int),
        "dds_autotune": ([vp, vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "dds_stress": ([vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "dds_stress_batched": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), ip,
                                ctypes.POINTER(vp), vp], ctypes.c_int),
        "dds_stress_noalloc": ([vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "dds_stress_subset": ([vp, ctypes.c_int, ctypes.c_int, ip, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "dds_stress_multi": ([vp, ctypes.c_int, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "dds_stress_stats": ([vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "dds_stress_host": ([vp, vp, vp, vp], ctypes.c_int),
        "dds_stress_host_async": ([vp, vp, vp, vp], ctypes.c_int),
        "dds_stress_host_sync": ([vp], ctypes.c_int),
        "dds_table_at": ([vp, dp, dp, lp, ip, dp], ctypes.c_int),
        "dds_query": ([vp, ip, ip, ip, ip], ctypes.c_int),
        "dds_spectra_bytes": ([vp, ctypes.POINTER(ctypes.c_ulonglong)], ctypes.c_int),
        "dds_footprint": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)], ctypes.c_int),
        "dds_contract_spectra": ([vp, ctypes.c_int, vp, vp, ctypes.c_longlong, vp], ctypes.c_int),
        "dds_launches_per_stress": ([vp], ctypes.c_int),
        "dds_yx_cluster": ([vp], ctypes.c_int),
        "dds_profile_enable": ([vp, ctypes.c_int], ctypes.c_int),
        "dds_profile_read": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ip, ip], ctypes.c_int),
        "dds_relax": ([vp, vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "dds_graph_capture": ([ctypes.POINTER(vp), ctypes.c_int, ip, ctypes.POINTER(vp), ip, ctypes.POINTER(vp), vp,
                               ctypes.POINTER(vp)], ctypes.c_int),
        "dds_graph_launch": ([vp, vp], ctypes.c_int),
        "dds_graph_nodes": ([vp], ctypes.c_int),
        "dds_graph_destroy": ([vp], None),
        "dds_device_status": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "dds_last_error": ([vp], ctypes.c_char_p),
        "dds_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(ctx, rc: int):
    if rc != DDS_OK:
        msg = load_library().dds_last_error(ctx).decode() if ctx else ""
        raise DDSError(rc, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---- C-named entry points ---------------------------------------------------
def dds_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(None, load_library().dds_create(ctypes.byref(h), int(device)))
    return h


def dds_set_geometry(ctx, nx, ny, nz, dx, dy, dz, mu, nu):
    _check(ctx, load_library().dds_set_geometry(ctx, int(nx), int(ny), int(nz), float(dx), float(dy),
                                                float(dz), float(mu), float(nu)))


def dds_set_families(ctx, t, b):
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1, 3))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1, 3))
    _check(ctx, load_library().dds_set_families(ctx, t.shape[0], _dptr(t), _dptr(b)))


def dds_set_option(ctx, key: int, value: float):
    _check(ctx, load_library().dds_set_option(ctx, int(key), float(value)))


def dds_autotune(ctx, stream=None) -> float:
    """Pick the fastest fused-z schedule for this geometry (before build); returns its ms."""
    ms = ctypes.c_float()
    _check(ctx, load_library().dds_autotune(ctx, _stream_handle(stream), ctypes.byref(ms)))
    return float(ms.value)


def dds_build_kernels(ctx, stream=None):
    _check(ctx, load_library().dds_build_kernels(ctx, _stream_handle(stream)))


def dds_stress(ctx, rho_ptr: int, rho_dtype: int, sigma_ptr: int, stream=None):
    _check(ctx, load_library().dds_stress(ctx, ctypes.c_void_p(rho_ptr), int(rho_dtype),
                                          ctypes.c_void_p(sigma_ptr), _stream_handle(stream)))


def dds_stress_multi(ctx, nb: int, rho_ptr: int, rho_dtype: int, sigma_ptr: int, stream=None):
    _check(ctx, load_library().dds_stress_multi(ctx, int(nb), ctypes.c_void_p(rho_ptr), int(rho_dtype),
                                                ctypes.c_void_p(sigma_ptr), _stream_handle(stream)))


def dds_stress_subset(ctx, nb: int, fam, rho_ptr: int, rho_dtype: int, sigma_ptr: int, stream=None):
    fam = [int(f) for f in fam]
    arr = (ctypes.c_int * len(fam))(*fam)
    _check(ctx, load_library().dds_stress_subset(ctx, int(nb), len(fam), arr, ctypes.c_void_p(rho_ptr),
                                                 int(rho_dtype), ctypes.c_void_p(sigma_ptr),
                                                 _stream_handle(stream)))


def dds_stress_stats(ctx, nb: int, rho_ptr: int, rho_dtype: int, sigma_ptr: int, s_ptr: int, stream=None):
    _check(ctx, load_library().dds_stress_stats(ctx, int(nb), ctypes.c_void_p(rho_ptr), int(rho_dtype),
                                                ctypes.c_void_p(sigma_ptr), ctypes.c_void_p(s_ptr),
                                                _stream_handle(stream)))


def dds_stress_batched(ctxs, rho_ptrs, rho_dtypes, sigma_ptrs, stream=None):
    n = len(ctxs)
    arr_c = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    arr_r = (ctypes.c_void_p * n)(*rho_ptrs)
    arr_d = (ctypes.c_int * n)(*rho_dtypes)
    arr_s = (ctypes.c_void_p * n)(*sigma_ptrs)
    rc = load_library().dds_stress_batched(arr_c, n, arr_r, arr_d, arr_s, _stream_handle(stream))
    _check(ctxs[0] if n else None, rc)


def dds_stress_noalloc(ctx, rho_ptr: int, rho_dtype: int, sigma_ptr: int, stream=None):
    """dds_stress with its work buffers in the library's fixed device area (no allocation)."""
    _check(ctx, load_library().dds_stress_noalloc(ctx, ctypes.c_void_p(rho_ptr), int(rho_dtype),
                                                  ctypes.c_void_p(sigma_ptr), _stream_handle(stream)))


def dds_relax(ctx, sigma_dis_ptr: int, u_ptr: int, n_steps: int, sigma_tot_ptr: int = 0, stream=None):
    _check(ctx, load_library().dds_relax(ctx, ctypes.c_void_p(sigma_dis_ptr), ctypes.c_void_p(u_ptr), int(n_steps),
                                         ctypes.c_void_p(sigma_tot_ptr or None), _stream_handle(stream)))


def dds_stress_host(ctx, rho_host: np.ndarray, sigma_host: np.ndarray, stream=None):
    assert rho_host.dtype == np.float32 and rho_host.flags.c_contiguous
    assert sigma_host.dtype == np.float32 and sigma_host.flags.c_contiguous
    _check(ctx, load_library().dds_stress_host(ctx, ctypes.c_void_p(rho_host.ctypes.data),
                                               ctypes.c_void_p(sigma_host.ctypes.data),
                                               _stream_handle(stream)))


def dds_stress_host_async(ctx, rho_host: np.ndarray, sigma_host: np.ndarray, stream=None):
    assert rho_host.dtype == np.float32 and rho_host.flags.c_contiguous
    assert sigma_host.dtype == np.float32 and sigma_host.flags.c_contiguous
    _check(ctx, load_library().dds_stress_host_async(ctx, ctypes.c_void_p(rho_host.ctypes.data),
                                                     ctypes.c_void_p(sigma_host.ctypes.data),
                                                     _stream_handle(stream)))


def dds_stress_host_sync(ctx):
    _check(ctx, load_library().dds_stress_host_sync(ctx))


def dds_table_at(ctx, t, b, ijk) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(3))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(3))
    ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((ijk.shape[0], 6))
    _check(ctx, load_library().dds_table_at(ctx, _dptr(t), _dptr(b), ijk.shape[0],
                                            ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(out)))
    return out


def dds_query(ctx):
    v = [ctypes.c_int() for _ in range(4)]
    _check(ctx, load_library().dds_query(ctx, *[ctypes.byref(x) for x in v]))
    return {"n_fields": v[0].value, "px": v[1].value, "py": v[2].value, "pz": v[3].value,
            "spectra_bytes": dds_spectra_bytes(ctx), "yx_cluster": dds_yx_cluster(ctx)}


def dds_footprint(ctx, nb: int = 1) -> int:
    b = ctypes.c_ulonglong()
    _check(ctx, load_library().dds_footprint(ctx, int(nb), ctypes.byref(b)))
    return int(b.value)


def dds_spectra_bytes(ctx) -> int:
    b = ctypes.c_ulonglong()
    _check(ctx, load_library().dds_spectra_bytes(ctx, ctypes.byref(b)))
    return int(b.value)


def dds_contract_spectra(rho_hat_ptr: int, fe: int, g_ptr: int, sigma_hat_ptr: int, nk: int, stream=None):
    _check(None, load_library().dds_contract_spectra(ctypes.c_void_p(rho_hat_ptr), int(fe), ctypes.c_void_p(g_ptr),
                                                     ctypes.c_void_p(sigma_hat_ptr), int(nk),
                                                     _stream_handle(stream)))


def dds_launches_per_stress(ctx) -> int:
    return int(load_library().dds_launches_per_stress(ctx))


def dds_yx_cluster(ctx) -> int:
    """CTAs per cluster of the fused inverse y + x pass (0: two separate passes)."""
    v = int(load_library().dds_yx_cluster(ctx))
    _check(ctx, min(v, 0))
    return v


def dds_profile_enable(ctx, enable: bool = True):
    _check(ctx, load_library().dds_profile_enable(ctx, int(bool(enable))))


def dds_profile_read(ctx, max_steps: int) -> np.ndarray:
    """Per-pass milliseconds of the evaluations recorded since enabling, (steps, 5)."""
    out = np.zeros((max(int(max_steps), 1), 5), dtype=np.float32)
    ns, npass = ctypes.c_int(), ctypes.c_int()
    _check(ctx, load_library().dds_profile_read(ctx, int(max_steps),
                                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                ctypes.byref(ns), ctypes.byref(npass)))
    return out[: ns.value, : npass.value]


def dds_graph_capture(ctxs, nbs, rho_ptrs, dtypes, sigma_ptrs, stream=None) -> ctypes.c_void_p:
    """Capture the batch; returns the graph handle (raises DDSError)."""
    n = len(ctxs)
    h = ctypes.c_void_p()
    rc = load_library().dds_graph_capture((ctypes.c_void_p * n)(*ctxs), n, (ctypes.c_int * n)(*nbs),
                                          (ctypes.c_void_p * n)(*rho_ptrs), (ctypes.c_int * n)(*dtypes),
                                          (ctypes.c_void_p * n)(*sigma_ptrs), _stream_handle(stream),
                                          ctypes.byref(h))
    if rc != DDS_OK:
        raise DDSError(rc, dds_last_error(ctxs[0]) if n else "")
    return h


def dds_graph_launch(graph, stream=None):
    rc = load_library().dds_graph_launch(graph, _stream_handle(stream))
    if rc != DDS_OK:
        raise DDSError(rc, "graph launch failed")


def dds_graph_nodes(graph) -> int:
    return int(load_library().dds_graph_nodes(graph))


def dds_graph_destroy(graph):
    if graph:
        load_library().dds_graph_destroy(graph)


class StressGraph:
    """A captured batch: entries (context, densities) -> sigma replayed by one launch.

    entries: list of (StressContext, rho) with rho a contiguous CUDA tensor of shape
    (nb, F, nz, ny, nx) (float32 or bfloat16); the outputs (nb, 6, nz, ny, nx) are
    allocated here and exposed as ``sigma``.  Refill the rho tensors in place between
    launches."""

    def __init__(self, entries, stream=None):
        import torch
        self.entries = entries
        self.sigma = []
        ctxs, nbs, rhos, dts, sigs = [], [], [], [], []
        for ctx, rho in entries:
            if rho.dim() != 5 or not rho.is_cuda or not rho.is_contiguous():
                raise ValueError("rho must be a contiguous 5-d CUDA tensor (nb, F, nz, ny, nx)")
            dt = {torch.float32: DDS_F32, torch.bfloat16: DDS_BF16}.get(rho.dtype)
            if dt is None:
                raise ValueError(f"unsupported density dtype {rho.dtype}")
            sig = torch.empty((rho.shape[0], 6) + tuple(rho.shape[2:]), dtype=torch.float32, device=rho.device)
            self.sigma.append(sig)
            ctxs.append(ctx.handle)
            nbs.append(int(rho.shape[0]))
            rhos.append(rho.data_ptr())
            dts.append(dt)
            sigs.append(sig.data_ptr())
        self._handle = dds_graph_capture(ctxs, nbs, rhos, dts, sigs, stream)

    @property
    def nodes(self) -> int:
        return dds_graph_nodes(self._handle)

    def launch(self, stream=None):
        dds_graph_launch(self._handle, stream)

    def close(self):
        if self._handle:
            dds_graph_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dds_device_status(device: int = 0, reset: bool = False) -> int:
    """DDS_OK, or DDS_ERR_TIMEOUT if a bounded device wait gave up since the last reset."""
    return int(load_library().dds_device_status(int(device), int(bool(reset))))


def dds_last_error(ctx) -> str:
    return load_library().dds_last_error(ctx).decode()


def dds_destroy(ctx):
    if ctx:
        load_library().dds_destroy(ctx)


# ---- convenience wrapper ------------------------------------------------------
class StressContext:
    """One geometry + family set with its cached kernel spectra on one GPU."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.handle = dds_create(self.device)
        self.shape = None
        self.n_families = 0

    def close(self):
        if self.handle:
            dds_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, nx, ny, nz, dx, dy, dz, mu, nu):
        dds_set_geometry(self.handle, nx, ny, nz, dx, dy, dz, mu, nu)
        self.shape = (int(nz), int(ny), int(nx))
        return self

    def set_families(self, t, b):
        dds_set_families(self.handle, t, b)
        self.n_families = int(np.asarray(t).reshape(-1, 3).shape[0])
        return self

    def set_option(self, key, value):
        dds_set_option(self.handle, key, value)
        return self

    def autotune(self, stream=None) -> float:
        return dds_autotune(self.handle, stream)

    def build_kernels(self, stream=None):
        dds_build_kernels(self.handle, stream)
        return self

    def stress(self, rho, sigma=None, stream=None):
        """rho: CUDA tensor (F, nz, ny, nx) float32 or bfloat16 -> sigma (6, nz, ny, nx) float32."""
        import torch
        if not rho.is_cuda or not rho.is_contiguous():
            raise ValueError("rho must be a contiguous CUDA tensor")
        if tuple(rho.shape) != (self.n_families,) + self.shape:
            raise ValueError(f"rho has shape {tuple(rho.shape)}, expected {(self.n_families,) + self.shape}")
        dt = {torch.float32: DDS_F32, torch.bfloat16: DDS_BF16}.get(rho.dtype)
        if dt is None:
            raise ValueError(f"unsupported density dtype {rho.dtype}")
        if sigma is None:
            sigma = torch.empty((6,) + self.shape, dtype=torch.float32, device=rho.device)
        dds_stress(self.handle, rho.data_ptr(), dt, sigma.data_ptr(), stream)
        return sigma

    def stress_multi(self, rho, sigma=None, stream=None):
        """rho: CUDA tensor (nb, F, nz, ny, nx) -> sigma (nb, 6, nz, ny, nx); spectra shared by the sets."""
        import torch
        if not rho.is_cuda or not rho.is_contiguous() or rho.dim() != 5:
            raise ValueError("rho must be a contiguous 5-d CUDA tensor (nb, F, nz, ny, nx)")
        if tuple(rho.shape[1:]) != (self.n_families,) + self.shape:
            raise ValueError(f"rho has shape {tuple(rho.shape)}")
        dt = {torch.float32: DDS_F32, torch.bfloat16: DDS_BF16}.get(rho.dtype)
        if dt is None:
            raise ValueError(f"unsupported density dtype {rho.dtype}")
        nb = int(rho.shape[0])
        if sigma is None:
            sigma = torch.empty((nb, 6) + self.shape, dtype=torch.float32, device=rho.device)
        dds_stress_multi(self.handle, nb, rho.data_ptr(), dt, sigma.data_ptr(), stream)
        return sigma

    def footprint(self, nb: int = 1) -> int:
        """Device bytes a build will hold (spectra + work buffers for nb sets), before building."""
        return dds_footprint(self.handle, nb)

    def stress_subset(self, fam, rho, sigma=None, stream=None):
        """Only the families `fam` (indices into this context's families) carry density:
        rho CUDA tensor (len(fam), nz, ny, nx) or (nb, len(fam), nz, ny, nx) -> sigma
        (6, nz, ny, nx) or (nb, 6, nz, ny, nx); the other families count as zero."""
        import torch
        batched = rho.dim() == 5
        r = rho if batched else rho.unsqueeze(0)
        if not r.is_cuda or not r.is_contiguous():
            raise ValueError("rho must be a contiguous CUDA tensor")
        if tuple(r.shape[1:]) != (len(fam),) + self.shape:
            raise ValueError(f"rho has shape {tuple(rho.shape)}")
        dt = {torch.float32: DDS_F32, torch.bfloat16: DDS_BF16}.get(r.dtype)
        if dt is None:
            raise ValueError(f"unsupported density dtype {r.dtype}")
        nb = int(r.shape[0])
        if sigma is None:
            sigma = torch.empty((nb, 6) + self.shape, dtype=torch.float32, device=r.device)
        dds_stress_subset(self.handle, nb, fam, r.data_ptr(), dt, sigma.data_ptr(), stream)
        return sigma if batched else sigma[0]

    def stress_stats(self, rho, sigma=None, stream=None):
        """sigma and the Eq. 20 in-plane RMS per component and height: returns (sigma, s)
        with s of shape (6, nz) (or (nb, 6, nz) for a 5-d batch of densities)."""
        import torch
        batched = rho.dim() == 5
        r = rho if batched else rho.unsqueeze(0)
        if not r.is_cuda or not r.is_contiguous():
            raise ValueError("rho must be a contiguous CUDA tensor")
        if tuple(r.shape[1:]) != (self.n_families,) + self.shape:
            raise ValueError(f"rho has shape {tuple(rho.shape)}")
        dt = {torch.float32: DDS_F32, torch.bfloat16: DDS_BF16}.get(r.dtype)
        if dt is None:
            raise ValueError(f"unsupported density dtype {r.dtype}")
        nb = int(r.shape[0])
        if sigma is None:
            sigma = torch.empty((nb, 6) + self.shape, dtype=torch.float32, device=r.device)
        s = torch.empty((nb, 6, self.shape[0]), dtype=torch.float32, device=r.device)
        dds_stress_stats(self.handle, nb, r.data_ptr(), dt, sigma.data_ptr(), s.data_ptr(), stream)
        return (sigma, s) if batched else (sigma[0], s[0])

    def stress_host(self, rho_host: np.ndarray, sigma_host: np.ndarray | None = None, stream=None):
        rho_host = np.ascontiguousarray(rho_host, dtype=np.float32)
        if sigma_host is None:
            sigma_host = np.empty((6,) + self.shape, dtype=np.float32)
        dds_stress_host(self.handle, rho_host, sigma_host, stream)
        return sigma_host

    def stress_host_async(self, rho_host: np.ndarray, sigma_host: np.ndarray, stream=None):
        """Enqueue one host-buffer evaluation (C-contiguous float32 arrays that stay alive
        until stress_host_sync); copies overlap the neighbouring calls' evaluations."""
        dds_stress_host_async(self.handle, rho_host, sigma_host, stream)

    def stress_host_sync(self):
        dds_stress_host_sync(self.handle)

    def relax(self, sigma_dis, n_steps: int, u=None, total: bool = True, stream=None):
        """Free-surface relaxation (Sec. 5) of sigma_dis (CUDA float32, (6, nz, ny, nx)).
        u: CUDA float32 (3, nz, ny, nx) starting displacement, updated in place (default:
        zeros).  Returns (u, sigma_tot) with sigma_tot None unless total."""
        import torch
        shape = self.shape
        if not (sigma_dis.is_cuda and sigma_dis.dtype == torch.float32 and sigma_dis.is_contiguous()):
            raise ValueError("sigma_dis must be a contiguous CUDA float32 tensor")
        if sigma_dis.dim() != 4 or sigma_dis.shape[0] != 6 or (shape and tuple(sigma_dis.shape[1:]) != shape):
            raise ValueError(f"sigma_dis has shape {tuple(sigma_dis.shape)}, expected (6,) + {shape}")
        if u is None:
            u = torch.zeros((3,) + tuple(sigma_dis.shape[1:]), dtype=torch.float32, device=sigma_dis.device)
        elif not (u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()
                  and tuple(u.shape) == (3,) + tuple(sigma_dis.shape[1:])):
            raise ValueError("u must be a contiguous CUDA float32 tensor of shape (3, nz, ny, nx)")
        tot = torch.empty_like(sigma_dis) if total else None
        dds_relax(self.handle, sigma_dis.data_ptr(), u.data_ptr(), n_steps, tot.data_ptr() if total else 0, stream)
        return u, tot

    def table_at(self, t, b, ijk):
        return dds_table_at(self.handle, t, b, ijk)

    def query(self):
        return dds_query(self.handle)

    @property
    def launches_per_stress(self) -> int:
        return dds_launches_per_stress(self.handle)


def context_for(problem, device: int = 0, n_near: float | None = None, stream=None,
                autotune: bool = False) -> StressContext:
    """Context set up and built for a ``workloads.Problem``-like object (geom, t, b)."""
    g = problem.geom
    ctx = StressContext(device)
    ctx.set_geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.mu, g.nu)
    ctx.set_families(problem.t, problem.b)
    if n_near is not None:
        ctx.set_option(DDS_OPT_NEAR_RADIUS, n_near)
    if autotune:
        ctx.autotune(stream)
    ctx.build_kernels(stream)
    return ctx
