// FP16-spectra instantiation of the fused z pass (see zpass_impl.cuh).
#include "zpass_impl.cuh"

namespace dds {

cudaError_t dispatch_z_f16(const Shape &sh, const float2 *im, const float2 *in, const __half *ks, const float *kscale,
                           float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  return zp::dispatch_z_typed<__half>(sh, im, in, ks, kscale, om, on, tw, s);
}

}  // namespace dds
