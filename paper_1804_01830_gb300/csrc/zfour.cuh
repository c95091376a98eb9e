// Fused z pass for padded z sizes 128 and 256 (PZ = 8 R1), in three register stages
// of the four-step factorisation: forward n = n2 + 8 n1, k = k1 + R1 k2; inverse
// k = k1 + R1 k2, n = a + 8 b.  A CTA takes W adjacent columns (16 for PZ 128: rows of
// 128 bytes; 8 for PZ 256, so that two CTAs fit an SM) with R1 W threads:
//   stage 1  thread (field e, n2, column w) loads rows n2 + 8 n1 < nz straight from
//            global memory (row segments of W complex values), runs the R1-point DFT of the
//            half-zero input (two R1/2-point DFTs), twiddles by W_PZ^(n2 k1) and
//            writes T[e][k1][n2][w];
//   stage 2  thread (k1, w) reads its 8 values of every field, runs the 8-point DFTs
//            and keeps rho^_e(k1 + R1 k2) of all fields in registers; for each
//            component it loads its kernel spectra straight from global memory (laid
//            out per thread in 16-byte chunks), contracts (Eq. 10 in Fourier space),
//            runs the inverse 8-point DFT over k2, twiddles by conj W_PZ^(a k1) and
//            writes Y[c][a][k1][w] into the space of T;
//   stage 3  thread (c, a, w) reads the R1 values of k1, runs the inverse R1-point DFT
//            for the outputs b < R1/2 only (rows a + 8 b < nz <= PZ/2) and stores them.
// Shared memory is written and read once per stage; row strides of 9 W values (T) and
// (R1 + 1) W values (Y) keep every stage's half-warp accesses free of bank conflicts.
//
// Kernel spectra of fields with the x-mirror parity (ZSym) are stored for ky <= py/2
// only.  A tile at ky > py/2 works at the negated frequencies: the conjugate-direction
// transform is conj(transform(conj(x))), so it runs the same code on its conjugated,
// rescaled densities and conjugates what it stores (signs uniform over the tile).  Its
// thread (k1, w) then needs the values the same thread reads in the stored tile py - ky
// (g(kx, -ky, -kz) = s_b chi(c) g(kx, ky, kz)).  Launch order puts the tiles ky and
// py - ky of the same kx range next to each other, so the second read comes from L2.
#pragma once
#include "stress_common.cuh"

namespace dds {
namespace zp {

template <int PZ> struct ZF {
  static constexpr int W = zfour_width(PZ);   // columns per tile
  static constexpr int R2 = 8, R1 = PZ / 8, NT = R1 * W;
  static constexpr int SK = (R2 + 1) * W;     // T row (e, k1): 8 n2 x W columns + W
  static constexpr int SY = (R1 + 1) * W;     // Y row (c, a): R1 k1 x W columns + W
  static_assert(R1 == 16 || R1 == 32, "padded z size 128 or 256");
};

// shared memory of the kernel, in float2 values: T, or Y in the same space ...
template <int PZ> __host__ __device__ constexpr int zf_smem0(int fe) {
  return fe * ZF<PZ>::R1 * ZF<PZ>::SK > 6 * ZF<PZ>::R2 * ZF<PZ>::SY ? fe * ZF<PZ>::R1 * ZF<PZ>::SK
                                                                    : 6 * ZF<PZ>::R2 * ZF<PZ>::SY;
}
// ... plus the PZ twiddles exp(-2 pi i m / PZ), staged in shared memory: stages 1 and 2
// read them at scattered indices, and shared loads beat L1 hits here (1.18 -> 1.11 ms
// on the GaN layer)
template <int PZ> __host__ __device__ constexpr int zf_smem(int fe) { return zf_smem0<PZ>(fe) + PZ; }

// Launch order of the main tiles: the rows ky = 0 and py/2 (their own mirrors) first,
// then, for ky = 1 .. py/2 - 1 and each kx tile, the tile at ky followed by the tile at
// py - ky.
__device__ __forceinline__ void zf_tile_of(int L, int py, int ktiles, int *ky, int *kxt) {
  if (L < 2 * ktiles) {
    *ky = L < ktiles ? 0 : py / 2;
    *kxt = L < ktiles ? L : L - ktiles;
    return;
  }
  const int pair = (L - 2 * ktiles) >> 1, ky1 = 1 + pair / ktiles;
  *kxt = pair - (ky1 - 1) * ktiles;
  *ky = ((L - 2 * ktiles) & 1) ? py - ky1 : ky1;
}

// The kernel-spectrum values (e, k2 = 0..7) of fields e = e0 .. e0 + FE - 1 of one
// component for the calling thread, held raw in registers (FP32, or FP16 converted and
// scaled at use).  Layout of one (tile, component): 16-byte chunks [j][thread], value
// (e, k2) in chunk j = (8 e + k2) / (values per chunk).
template <typename GT, int FE> struct ZRaw;
template <int FE> struct ZRaw<float, FE> {
  float4 v[FE][2];
  __device__ __forceinline__ void load(const float *kc, int e0, int t, int nthreads) {
    const float4 *p = reinterpret_cast<const float4 *>(kc);
#pragma unroll
    for (int e = 0; e < FE; ++e) {
      v[e][0] = __ldg(p + (long)(2 * (e0 + e)) * nthreads + t);
      v[e][1] = __ldg(p + (long)(2 * (e0 + e) + 1) * nthreads + t);
    }
  }
  __device__ __forceinline__ float get(int e, int k2, float) const {
    const float4 q = v[e][k2 / 4];
    return (k2 % 4 == 0) ? q.x : (k2 % 4 == 1) ? q.y : (k2 % 4 == 2) ? q.z : q.w;
  }
};
template <int FE> struct ZRaw<__half, FE> {
  uint4 v[FE];
  __device__ __forceinline__ void load(const __half *kc, int e0, int t, int nthreads) {
    const uint4 *p = reinterpret_cast<const uint4 *>(kc);
#pragma unroll
    for (int e = 0; e < FE; ++e) v[e] = __ldg(p + (long)(e0 + e) * nthreads + t);
  }
  __device__ __forceinline__ float get(int e, int k2, float s) const {
    const uint4 q = v[e];
    const unsigned w = (k2 / 2 == 0) ? q.x : (k2 / 2 == 1) ? q.y : (k2 / 2 == 2) ? q.z : q.w;
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    return ((k2 % 2) ? f.y : f.x) * s;
  }
};

// Prefetch of [p, p + bytes) into L2 by the bulk-copy unit; p and bytes multiples of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

template <int PZ, int FE, typename GT>
__global__ void __launch_bounds__(ZF<PZ>::NT, 512 / ZF<PZ>::NT)
    k_zfour(Shape sh, const float2 *in_main, const float2 *in_nyq, const GT *kspec, const float *kscale,
            float2 *out_main, float2 *out_nyq, const float2 *tw) {
  constexpr int R1 = ZF<PZ>::R1, R2 = ZF<PZ>::R2, W = ZF<PZ>::W, NT = ZF<PZ>::NT;
  constexpr int SK = ZF<PZ>::SK, SY = ZF<PZ>::SY, H = R1 / 2;
  extern __shared__ __align__(16) float2 zsm[];
  const int tid = threadIdx.x;
  const int M = sh.M, py = sh.py, nz = sh.nz;
  const int ktiles = M / W, tiles_main = py * ktiles;
  // Consecutive blocks take the same column tile for the density sets of a batch,
  // so the tile's kernel spectra come from HBM once and from L2 for the others.
  const int tau = blockIdx.x / sh.nb;
  const int bset = (int)(blockIdx.x - tau * sh.nb);
  in_main += bset * ((long)FE * nz * py * M);
  in_nyq += bset * ((long)FE * py * nz);
  out_main += bset * (6L * nz * py * M);
  out_nyq += bset * (6L * py * nz);
  const bool nyq = tau >= tiles_main;
  int ky = 0, kxt = 0, nyq_idx = 0;
  if (!nyq) zf_tile_of(tau, py, ktiles, &ky, &kxt);
  else nyq_idx = tau - tiles_main;
  const bool sw = sh.zs.xall && !nyq && ky > py / 2;   // works at the negated frequencies
  float2 *twP = zsm + zf_smem0<PZ>(FE);
  for (int i = tid; i < PZ; i += NT) twP[i] = __ldg(tw + tw_offset(PZ) + i);
  __syncthreads();
  // the stored tile this tile reads: its own, or py - ky for a negated-frequency tile
  const long st = nyq ? (long)(sh.zs.xall ? py / 2 + 1 : py) * ktiles + nyq_idx
                      : (long)(sw ? py - ky : ky) * ktiles + kxt;
  const GT *ks = kspec + st * 6L * FE * PZ * W;
  // the tile's kernel spectra (6 FE PZ W values, contiguous) head for L2 now, so the
  // per-component loads of stage 2 find them there; a negated-frequency tile leaves
  // them to its partner launched beside it
  if (!sw) {
    constexpr unsigned BYTES = 6u * FE * PZ * W * sizeof(GT), CH = 8192, NCH = (BYTES + CH - 1) / CH;
    static_assert(BYTES % 16 == 0 && NCH <= NT, "prefetch chunks");
    if (tid < (int)NCH) prefetch_l2_bulk(reinterpret_cast<const char *>(ks) + tid * CH, min(CH, BYTES - tid * CH));
  }

  // stage 1: forward R1-point DFTs over n1 of the rows n2 + 8 n1 (n1 < R1/2 non-zero);
  // a negated-frequency tile transforms -s_b conj(rho) (s_b folds the spectra's sign)
  constexpr int NI = FE * R2 * W;              // items (field, n2, column)
  auto s1_load = [&](int item, float2 (&ev)[H]) {
    const int e = item / (R2 * W), r = item - e * (R2 * W), n2 = r / W, w = r - n2 * W;
#pragma unroll
    for (int n1 = 0; n1 < H; ++n1) {
      const int z = n2 + R2 * n1;
      ev[n1] = make_float2(0.f, 0.f);
      if (z < nz)
        ev[n1] = !nyq ? __ldg(in_main + (((long)e * nz + z) * py + ky) * M + kxt * W + w)
                      : __ldg(in_nyq + ((long)e * py + nyq_idx * W + w) * nz + z);
    }
  };
  auto s1_finish = [&](int item, float2 (&ev)[H]) {
    const int e = item / (R2 * W), r = item - e * (R2 * W), n2 = r / W, w = r - n2 * W;
    if (sw) {
      const float sy = ((sh.zs.sbneg >> e) & 1u) ? -1.0f : 1.0f;
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) ev[n1] = make_float2(-sy * ev[n1].x, sy * ev[n1].y);
    }
    float2 od[H];
#pragma unroll
    for (int n1 = 0; n1 < H; ++n1) od[n1] = rot_const<false>(ev[n1], n1, R1);
    dft_reg<H, false>(ev);                    // outputs k1 = 2 j
    dft_reg<H, false>(od);                    // outputs k1 = 2 j + 1
    float2 *T = zsm + (long)e * R1 * SK + n2 * W + w;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      T[(2 * j) * SK] = j == 0 ? ev[0] : cmul_tw<false>(ev[j], twP[n2 * 2 * j]);
      T[(2 * j + 1) * SK] = cmul_tw<false>(od[j], twP[n2 * (2 * j + 1)]);
    }
  };
  // items in pairs of rounds: both items' rows are requested before either is transformed
  // (five fields give 1.25 items per thread; GaN layer 1.11 -> 1.07 ms)
  for (int item = tid; item < NI; item += 2 * NT) {
    float2 a[H], b[H];
    const bool two = item + NT < NI;
    s1_load(item, a);
    if (two) s1_load(item + NT, b);
    s1_finish(item, a);
    if (two) s1_finish(item + NT, b);
  }
  __syncthreads();

  // stage 2: forward 8-point DFTs over n2, contraction, inverse 8-point DFTs over k2;
  // the spectra of the next component (of its first PF fields, as registers allow) load
  // while the current one is inverted and stored
  constexpr int PF = FE <= 4 ? FE : (FE == 5 ? 2 : 1);
  const int k1 = tid / W, w = tid - k1 * W;
  ZRaw<GT, PF> gr;
  gr.load(ks, 0, tid, NT);
  float2 f[FE][R2];
#pragma unroll
  for (int e = 0; e < FE; ++e) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) f[e][n2] = zsm[((long)e * R1 + k1) * SK + n2 * W + w];
    dft_reg<R2, false>(f[e]);
  }
  __syncthreads();                            // T is read: Y takes its space
#pragma unroll 1
  for (int c = 0; c < 6; ++c) {
    const GT *kc = ks + (long)c * FE * PZ * W;
    float2 s[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) s[k2] = make_float2(0.f, 0.f);
    // this component's other fields load now, before the prefetched ones are used
    ZRaw<GT, (FE > PF ? FE - PF : 1)> lt;
    if constexpr (FE > PF) lt.load(kc, PF, tid, NT);
#pragma unroll
    for (int e = 0; e < PF; ++e) {
      const float sc = kscale != nullptr ? __ldg(kscale + c * FE + e) : 1.0f;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) s[k2] = cmadd_i(s[k2], gr.get(e, k2, sc), f[e][k2]);
    }
    if (c < 5) gr.load(kc + (long)FE * PZ * W, 0, tid, NT);
#pragma unroll
    for (int e = PF; e < FE; ++e) {
      const float sc = kscale != nullptr ? __ldg(kscale + c * FE + e) : 1.0f;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) s[k2] = cmadd_i(s[k2], lt.get(e - PF, k2, sc), f[e][k2]);
    }
    dft_reg<R2, true>(s);                     // index a of n = a + 8 b
    float2 *Y = zsm + (long)c * R2 * SY + k1 * W + w;
    Y[0] = s[0];
#pragma unroll
    for (int a = 1; a < R2; ++a) Y[a * SY] = cmul_tw<true>(s[a], twP[a * k1]);
  }
  __syncthreads();

  // stage 3: inverse R1-point DFTs over k1, outputs b < R1/2: x(b) = E(b) + W_R1^-b O(b);
  // a negated-frequency tile stores chi(c) conj(x)
  for (int item = tid; item < 6 * R2 * W; item += NT) {
    const int c = item / (R2 * W), r = item - c * (R2 * W), a = r / W, wc = r - a * W;
    const float bx = sw ? ((c == 3 || c == 4) ? -1.0f : 1.0f) : 1.0f, by = sw ? -bx : 1.0f;
    const float2 *Y = zsm + ((long)c * R2 + a) * SY + wc;
    float2 ev[H], od[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      ev[j] = Y[(2 * j) * W];
      od[j] = Y[(2 * j + 1) * W];
    }
    dft_reg<H, true>(ev);
    dft_reg<H, true>(od);
#pragma unroll
    for (int b = 0; b < H; ++b) {
      const int z = a + R2 * b;
      if (z < nz) {
        const float2 u = cadd(ev[b], rot_const<true>(od[b], b, R1));
        const float2 v = make_float2(bx * u.x, by * u.y);
        // streaming stores: the next pass reads them after far more than L2 has gone by,
        // and they leave L2 to the mirror tiles' spectra (1.049 -> 1.041 ms); streaming
        // loads of the density rows cost more (1.088 ms), since neighbouring tiles share
        // their 128-byte lines
        if (!nyq) __stcs(out_main + (((long)c * nz + z) * py + ky) * M + kxt * W + wc, v);
        else __stcs(out_nyq + ((long)c * py + nyq_idx * W + wc) * nz + z, v);
      }
    }
  }
}

template <int PZ, int FE, typename GT>
cudaError_t launch_zfour(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                         float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t)zf_smem<PZ>(FE);
  constexpr int W = ZF<PZ>::W;
  if (sh.wz != W) return cudaErrorInvalidValue;
  const long tiles = ((long)sh.py * (sh.M / W) + sh.py / W) * sh.nb;
  cudaError_t err = prep(k_zfour<PZ, FE, GT>, smem);
  if (err != cudaSuccess) return err;
  k_zfour<PZ, FE, GT><<<(unsigned)tiles, ZF<PZ>::NT, smem, s>>>(sh, im, in, ks, ksc, om, on, tw);
  return cudaGetLastError();
}

template <int PZ, typename GT>
cudaError_t dispatch_zfour_fe(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                              float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  switch (sh.fe) {
    case 1: return launch_zfour<PZ, 1, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 2: return launch_zfour<PZ, 2, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 3: return launch_zfour<PZ, 3, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 4: return launch_zfour<PZ, 4, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 5: return launch_zfour<PZ, 5, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 6: return launch_zfour<PZ, 6, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace zp
}  // namespace dds
