"""dds_contract_spectra, the stand-alone Fourier-space contraction of Eq. 10 used by the
library-FFT comparison pipeline: against the same contraction written with PyTorch ops
in FP64, for every supported field count and a ragged length."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_01830_gb300 as mod
    mod.load_library()
    return mod


@pytest.mark.parametrize("fe", [1, 2, 3, 5, 8])
def test_contraction_matches_reference(dds, fe):
    nk = 100_003
    gen = torch.Generator(device="cuda").manual_seed(fe)
    rho = torch.randn((fe, nk), dtype=torch.complex64, device="cuda", generator=gen)
    g = torch.randn((6, fe, nk), dtype=torch.float32, device="cuda", generator=gen)
    out = torch.full((6, nk), complex(float("nan"), 0.0), dtype=torch.complex64, device="cuda")
    dds.dds_contract_spectra(rho.data_ptr(), fe, g.data_ptr(), out.data_ptr(), nk)
    torch.cuda.synchronize()
    ref = (1j * g.double()[:, :, :] * rho.to(torch.complex128)[None]).sum(dim=1)
    err = (out.to(torch.complex128) - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-6


def test_contraction_rejects_bad_arguments(dds):
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    g = torch.zeros(6 * 16, dtype=torch.float32, device="cuda")
    for fe in (0, 9):
        with pytest.raises(dds.DDSError) as e:
            dds.dds_contract_spectra(x.data_ptr(), fe, g.data_ptr(), x.data_ptr(), 1)
        assert e.value.code == dds.DDS_ERR_INVALID_ARG
    dds.dds_contract_spectra(x.data_ptr(), 1, g.data_ptr(), x.data_ptr(), 0)   # empty: no-op
