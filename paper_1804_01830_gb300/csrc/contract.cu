// dds_contract_spectra: the Fourier-space contraction of Eq. 10 as a kernel of its own,
// on full spectra in the layout of a library real-to-complex FFT.  The fused path never
// calls it (there the contraction lives inside the z transform); it exists so that the
// "library FFT + separate contraction" pipeline can be timed against the fused passes.
#include "dds_internal.h"

namespace dds {
namespace {

// sigma^_c(k) = sum_e (i g_ce(k)) rho^_e(k), one k per thread and iteration.
template <int FE>
__global__ void __launch_bounds__(256) k_contract(const float2 *__restrict__ rho, const float *__restrict__ g,
                                                  float2 *__restrict__ sig, long long nk) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nk;
       k += (long long)gridDim.x * blockDim.x) {
    float2 r[FE];
#pragma unroll
    for (int e = 0; e < FE; ++e) r[e] = __ldg(rho + e * nk + k);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int e = 0; e < FE; ++e) {
        const float gv = __ldg(g + ((long long)c * FE + e) * nk + k);
        s.x = fmaf(-gv, r[e].y, s.x);
        s.y = fmaf(gv, r[e].x, s.y);
      }
      sig[c * nk + k] = s;
    }
  }
}

template <int FE>
cudaError_t launch(const float2 *rho, const float *g, float2 *sig, long long nk, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  const long long want = (nk + 255) / 256, cap = 8LL * sms;
  const unsigned grid = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  k_contract<FE><<<grid, 256, 0, s>>>(rho, g, sig, nk);
  return cudaGetLastError();
}

}  // namespace
}  // namespace dds

extern "C" int dds_contract_spectra(const void *rho_hat, int fe, const float *g, void *sigma_hat, long long nk,
                                    void *cuda_stream) {
  using namespace dds;
  if (!rho_hat || !g || !sigma_hat || nk < 0 || fe < 1 || fe > 8) return DDS_ERR_INVALID_ARG;
  if (nk == 0) return DDS_OK;
  const float2 *r = static_cast<const float2 *>(rho_hat);
  float2 *o = static_cast<float2 *>(sigma_hat);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t err;
  switch (fe) {
    case 1: err = launch<1>(r, g, o, nk, s); break;
    case 2: err = launch<2>(r, g, o, nk, s); break;
    case 3: err = launch<3>(r, g, o, nk, s); break;
    case 4: err = launch<4>(r, g, o, nk, s); break;
    case 5: err = launch<5>(r, g, o, nk, s); break;
    case 6: err = launch<6>(r, g, o, nk, s); break;
    case 7: err = launch<7>(r, g, o, nk, s); break;
    default: err = launch<8>(r, g, o, nk, s); break;
  }
  if (err != cudaSuccess) {
    cudaGetLastError();
    return DDS_ERR_CUDA;
  }
  return DDS_OK;
}
