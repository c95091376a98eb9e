"""The C-ABI library loads and exports every symbol include/dds.h declares (no GPU
needed); host-side error paths that need no device."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_1804_01830_gb300 import build as libbuild
    libbuild.build()
    import paper_1804_01830_gb300 as dds
    return dds.load_library()


def declared_symbols():
    text = (ROOT / "include" / "dds.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dds_[a-z_]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    syms = declared_symbols()
    for name in ("dds_create", "dds_set_geometry", "dds_set_families", "dds_build_kernels", "dds_stress",
                 "dds_destroy", "dds_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_every_declared_symbol():
    import paper_1804_01830_gb300 as dds
    assert sorted(dds.EXPORTS) == declared_symbols()
    for name in declared_symbols():
        assert callable(getattr(dds, name))


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1804_01830_gb300 as dds
    with pytest.raises(dds.DDSError) as ei:
        dds.dds_create(0)
    assert ei.value.code == dds.DDS_ERR_INVALID_ARG


def test_null_context_is_rejected(lib):
    assert lib.dds_set_geometry(None, 8, 8, 8, 1e-6, 1e-6, 1e-6, 1e9, 0.3) == -1
    assert lib.dds_build_kernels(None, None) == -1
    assert lib.dds_stress(None, None, 0, None, None) == -1
    assert lib.dds_launches_per_stress(None) == 0
    lib.dds_destroy(None)
