// FP32-spectra instantiation of the fused z pass (see zpass_impl.cuh).
#include "zpass_impl.cuh"

namespace dds {

cudaError_t dispatch_z_f32(const Shape &sh, const float2 *im, const float2 *in, const float *ks, float2 *om,
                           float2 *on, const float2 *tw, cudaStream_t s) {
  return zp::dispatch_z_typed<float>(sh, im, in, ks, nullptr, om, on, tw, s);
}

cudaError_t dispatch_z(const Shape &sh, const float2 *im, const float2 *in, const void *ks, const float *kscale,
                       float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  if (kscale != nullptr)
    return dispatch_z_f16(sh, im, in, static_cast<const __half *>(ks), kscale, om, on, tw, s);
  return dispatch_z_f32(sh, im, in, static_cast<const float *>(ks), om, on, tw, s);
}

}  // namespace dds
