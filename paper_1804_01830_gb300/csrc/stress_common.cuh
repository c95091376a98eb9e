// Helpers shared by the translation units of the stress passes.
#pragma once
#include <cuda_fp16.h>

#include "dds_fft.cuh"
#include "dds_internal.h"

namespace dds {

constexpr int NT = 256;   // threads of the shared-memory z pass

// Tile shape of the y passes: W columns per tile, NT threads.  Small tiles keep
// several CTAs resident per SM so that one tile's copies overlap another tile's
// transform.
// y-pass tiles: W columns, NT threads.  The 512-row inverse takes 16 columns and 256
// threads (whole 128-byte rows; GaN layer 0.215 -> 0.207 ms); the 512-row forward keeps
// 8 and 128 (0.176 against 0.183 ms with 16).
template <int P, bool INV = false> struct YTile {
  static constexpr int W = P >= 1024 ? 4 : (P >= 512 ? (INV ? 16 : 8) : 16);
  static constexpr int NT = (P == 512 && INV) ? 256 : 128;
};

__device__ __forceinline__ float2 cmadd_i(float2 acc, float g, float2 r) {
  // acc + (i g) * r
  return make_float2(fmaf(-g, r.y, acc.x), fmaf(g, r.x, acc.y));
}

__device__ __forceinline__ float bf16_to_f32(uint16_t v) { return __uint_as_float(((uint32_t)v) << 16); }

template <typename K>
inline cudaError_t prep(K kernel, size_t smem) {
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess || smem <= 48 * 1024) return err;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Fused z pass (zpass_f32.cu, zpass_f16.cu).  ks: kernel spectra, FP32 or FP16 (kscale != nullptr:
// FP16 storage, value = stored * kscale[c * fe + e]).
cudaError_t dispatch_z(const Shape &sh, const float2 *im, const float2 *in, const void *ks, const float *kscale,
                       float2 *om, float2 *on, const float2 *tw, cudaStream_t s);
cudaError_t dispatch_z_f16(const Shape &sh, const float2 *im, const float2 *in, const __half *ks, const float *kscale,
                           float2 *om, float2 *on, const float2 *tw, cudaStream_t s);

}  // namespace dds
