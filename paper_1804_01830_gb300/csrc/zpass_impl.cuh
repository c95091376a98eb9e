// Fused z pass of the stress evaluation: per (kx, ky) column, the forward FFT
// along z of every field, the contraction with the cached kernel spectra
//   sigma^_c(k) = sum_e (i g_ce(k)) rho^_e(k)            (Eq. 10 in Fourier space)
// and the inverse FFT along z of the six components, keeping rows z < nz.
// Kernel spectra are stored as FP32, or as FP16 with one FP32 scale per
// (component, field); arithmetic is FP32 either way.
#pragma once
#include "stress_common.cuh"
#include "zfour.cuh"

namespace dds {
namespace zp {

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

// ------------------------------------------------------------- fused z ------
// Shared-memory variant for tall grids (or many fields).  A tile is W adjacent
// columns.  The fields are interleaved in one tile F[z][e W + w] and transformed
// together (fe W lines).  The kernel spectra of one component for the tile
// (fe x PZ x W values) stream into one of two buffers G by cp.async while the
// previous component is contracted, and while the inverse FFTs run; the six
// components are formed in S[z][c' W + w] and inverted three at a time.
// The inverse z transform of three components (3W lines of S, rows kz < PZ) in two
// register stages of PZ = R1 R2 (four-step factorisation), the second storing rows
// z < nz straight to global memory: S is read twice and written once, against the
// four sweeps and the copy-out of a Stockham tile.  The stage-1 results go back into S
// (after a barrier), transposed, with a row stride that keeps both stages free of bank
// conflicts; S holds PZ 3W + R1 ZPAD values.
template <int W> __host__ __device__ constexpr int zpad() { return W == 8 ? 8 : 3 * W; }
template <int PZ, int W> __host__ __device__ constexpr bool z_reg_inverse() { return Plan<PZ>::n == 2 && W <= 8; }
template <int PZ, int W> __host__ __device__ constexpr int z_s_extra() {
  return z_reg_inverse<PZ, W>() ? Plan<PZ>::r0 * zpad<W>() : 0;
}

template <int PZ, int W, typename Store>
__device__ __forceinline__ void inverse3_store(float2 *S, const float2 *twP, int tid, int nz, Store store) {
  constexpr int R1 = Plan<PZ>::r0, R2 = Plan<PZ>::r1, L3 = 3 * W, ST = R2 * L3 + zpad<W>();
  constexpr int I1 = (R2 * L3 + NT - 1) / NT, I2 = (R1 * L3 + NT - 1) / NT;
  float2 v[I1][R1];
#pragma unroll
  for (int it = 0; it < I1; ++it) {
    const int item = tid + it * NT;
    if ((R2 * L3) % NT != 0 && item >= R2 * L3) continue;
    const int n2 = item / L3, line = item - n2 * L3;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[it][n1] = S[(n2 + R2 * n1) * L3 + line];
  }
  __syncthreads();                            // S read: it now takes the stage-1 results
#pragma unroll
  for (int it = 0; it < I1; ++it) {
    const int item = tid + it * NT;
    if ((R2 * L3) % NT != 0 && item >= R2 * L3) continue;
    const int n2 = item / L3, line = item - n2 * L3;
    dft_reg<R1, true>(v[it]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 y = v[it][k1];
      if (k1 > 0) y = cmul_tw<true>(y, __ldg(twP + n2 * k1));
      S[k1 * ST + n2 * L3 + line] = y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < I2; ++it) {
    const int item = tid + it * NT;
    if ((R1 * L3) % NT != 0 && item >= R1 * L3) continue;
    const int k1 = item / L3, line = item - k1 * L3;
    float2 y[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) y[n2] = S[k1 * ST + n2 * L3 + line];
    dft_reg<R2, true>(y);
#pragma unroll
    for (int k2 = 0; k2 < R2 / 2; ++k2) {
      const int z = k1 + R1 * k2;
      if (z < nz) store(line, z, y[k2]);
    }
  }
}

template <int PZ, int W, int FEMAX, typename GT>
__global__ void __launch_bounds__(NT) k_zpass(Shape sh, const float2 *in_main, const float2 *in_nyq,
                                              const GT *kspec, const float *kscale, float2 *out_main,
                                              float2 *out_nyq, const float2 *tw) {
  constexpr int TS = PZ * W;                 // positions of one field in the tile
  constexpr int LF = FEMAX * W;              // most field lines
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int M = sh.M, py = sh.py, nz = sh.nz, fe = sh.fe;
  const int L = fe * W;
  float2 *F = smem;                                       // [PZ][fe W]
  float2 *S = smem + (long)PZ * L;                        // [PZ][3 W]
  GT *G0 = reinterpret_cast<GT *>(S + 3 * TS + z_s_extra<PZ, W>());   // [fe][PZ][W], two buffers
  GT *G1 = G0 + (long)fe * TS;
  const long ktiles = M / W;
  const long tiles_main = (long)py * ktiles;
  // Consecutive blocks take the same column tile for the density sets of a batch,
  // so the tile's kernel spectra come from HBM once and from L2 for the others.
  const long tau = blockIdx.x / sh.nb;
  const int bset = (int)(blockIdx.x - tau * sh.nb);
  in_main += bset * ((long)fe * nz * py * M);
  in_nyq += bset * ((long)fe * py * nz);
  out_main += bset * (6L * nz * py * M);
  out_nyq += bset * (6L * py * nz);
  const bool nyq = tau >= tiles_main;
  long ky = 0, kx0 = 0, ky0 = 0;
  if (!nyq) {
    ky = tau / ktiles;
    kx0 = (tau - ky * ktiles) * W;
  } else {
    ky0 = (tau - tiles_main) * W;
  }
  const GT *ks = kspec + tau * 6L * fe * TS;
  constexpr int PER16 = 16 / sizeof(GT);                   // values per 16-byte chunk
  const int gchunks = fe * TS / PER16;                    // 16-byte chunks of one component
  auto load_spectra = [&](int c, GT *dst) {
    const GT *src = ks + (long)c * fe * TS;
    for (int q = tid; q < gchunks; q += NT) cp_async16(dst + PER16 * q, src + PER16 * q);
    cp_async_commit();
  };
  // rows z < nz of every field; rows [nz, PZ/2) zero
  if (!nyq) {
    constexpr int H = W / 2;
    for (int p = tid; p < nz * fe * H; p += NT) {
      const int z = p / (fe * H), r = p - z * (fe * H), e = r / H, c2 = r - e * H;
      cp_async16(&F[z * L + e * W + 2 * c2], in_main + (((long)e * nz + z) * py + ky) * M + kx0 + 2 * c2);
    }
  } else {
    for (int p = tid; p < nz * fe * W; p += NT) {
      const int e = p / (nz * W), r = p - e * (nz * W), w = r / nz, z = r - w * nz;
      cp_async8(&F[z * L + e * W + w], in_nyq + ((long)e * py + ky0 + w) * nz + z);
    }
  }
  cp_async_commit();
  load_spectra(0, G0);
  for (int p = nz * L + tid; p < (PZ / 2) * L; p += NT) F[p] = make_float2(0.f, 0.f);
  cp_async_wait_group<1>();                               // fields have landed
  __syncthreads();
  const float2 *twP = tw + tw_offset(PZ);
  fft_tile_rt<PZ, LF, NT, false, true, false>(F, L, twP, tid);

  for (int c = 0; c < 6; ++c) {
    GT *Gc = (c & 1) ? G1 : G0;
    float sc[FEMAX];
#pragma unroll
    for (int e = 0; e < FEMAX; ++e) sc[e] = (kscale != nullptr && e < fe) ? __ldg(kscale + c * fe + e) : 1.0f;
    cp_async_wait_group<0>();                             // spectra of component c
    __syncthreads();
    if (c < 5) load_spectra(c + 1, (c & 1) ? G0 : G1);    // next component flies meanwhile
    const int c3 = c % 3;
    for (int p = tid; p < TS; p += NT) {                  // position p = kz W + w
      const int kz = p / W, w = p - kz * W;
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int e = 0; e < FEMAX; ++e)
        if (e < fe) a = cmadd_i(a, to_f32(Gc[(long)e * TS + p]) * sc[e], F[kz * L + e * W + w]);
      S[kz * (3 * W) + c3 * W + w] = a;
    }
    if (c3 == 2) {
      __syncthreads();
      if constexpr (z_reg_inverse<PZ, W>()) {
        inverse3_store<PZ, W>(S, twP, tid, nz, [&](int line, int z, float2 val) {
          const int cc = c - 2 + line / W, w = line % W;
          if (!nyq) out_main[(((long)cc * nz + z) * py + ky) * M + kx0 + w] = val;
          else out_nyq[((long)cc * py + ky0 + w) * nz + z] = val;
        });
      } else {
        fft_tile_rt<PZ, 3 * W, NT, true, false, true>(S, 3 * W, twP, tid);
        for (int p = tid; p < nz * 3 * W; p += NT) {
          const int z = p / (3 * W), r = p - z * (3 * W), cc = c - 2 + r / W, w = r % W;
          if (!nyq) out_main[(((long)cc * nz + z) * py + ky) * M + kx0 + w] = S[p];
          else out_nyq[((long)cc * py + ky0 + w) * nz + z] = S[p];
        }
      }
    }
  }
}

// ------------------------------------------------- fused z, registers only ---
// For pz = E G (E = 8 or 16 registers, G = 1..8 lanes per column): a warp owns
// CW = 32 / G adjacent columns; lane g of a column holds elements n = g + G m
// (m < E) of each field.  Four-step FFT: E-point DFT over m in registers, twiddle
// W_pz^(g k1), G-point DFT across the G lanes by shuffles.  Lane g then holds
// k = k1 + E bitrev_G(g); the contraction with the kernel spectra (laid out per warp
// tile, lane, k1) runs in registers, and the inverse retraces the steps.  No shared
// memory and no barriers; the next component's spectra load while the current one
// is inverted and stored.
template <int G>
__device__ __forceinline__ int bitrev_lane(int g) {
  if (G == 4) return ((g & 1) << 1) | (g >> 1);
  if (G == 8) return ((g & 1) << 2) | (g & 2) | (g >> 2);
  return g;
}

// a * W_8^q (forward) or a * conj(W_8^q) (inverse), q in 0..3 chosen per lane
template <bool INV>
__device__ __forceinline__ float2 rot8(float2 a, int q) {
  const float r = 0.70710678118654752440f;
  if (q == 0) return a;
  if (q == 2) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  if (q == 1) return INV ? make_float2(r * (a.x - a.y), r * (a.x + a.y)) : make_float2(r * (a.x + a.y), r * (a.y - a.x));
  return INV ? make_float2(-r * (a.x + a.y), r * (a.x - a.y)) : make_float2(r * (a.y - a.x), -r * (a.x + a.y));
}

template <int E, int G, bool INV>
__device__ __forceinline__ void cross_lane_dft(float2 (&v)[E], int g, int cw) {
  if constexpr (G == 1) return;
  if (!INV) {   // decimation in frequency: natural in, bit-reversed out
#pragma unroll
    for (int h = G / 2; h >= 1; h >>= 1) {
      const bool upper = (g & h) != 0;
      const int q = (g & (h - 1)) * (4 / h);
#pragma unroll
      for (int k = 0; k < E; ++k) {
        float2 p;
        p.x = __shfl_xor_sync(0xffffffffu, v[k].x, h * cw);
        p.y = __shfl_xor_sync(0xffffffffu, v[k].y, h * cw);
        v[k] = upper ? rot8<false>(csub(p, v[k]), q) : cadd(v[k], p);
      }
    }
  } else {      // decimation in time: bit-reversed in, natural out
#pragma unroll
    for (int h = 1; h < G; h <<= 1) {
      const bool upper = (g & h) != 0;
      const int q = (g & (h - 1)) * (4 / h);
#pragma unroll
      for (int k = 0; k < E; ++k) {
        float2 p;
        p.x = __shfl_xor_sync(0xffffffffu, v[k].x, h * cw);
        p.y = __shfl_xor_sync(0xffffffffu, v[k].y, h * cw);
        v[k] = upper ? csub(p, rot8<true>(v[k], q)) : cadd(v[k], rot8<true>(p, q));
      }
    }
  }
}

// E spectrum values of one lane in registers, FP32 or FP16 (converted at use).
template <typename GT, int E> struct GRaw;
template <int E> struct GRaw<float, E> {
  float4 v[E / 4];
  __device__ __forceinline__ void load(const float *p) {
#pragma unroll
    for (int i = 0; i < E / 4; ++i) v[i] = __ldg(reinterpret_cast<const float4 *>(p) + i);
  }
  // values 2 k2 and 2 k2 + 1
  __device__ __forceinline__ float2 get2(int k2, float) const {
    const float4 q = v[k2 / 2];
    return (k2 % 2 == 0) ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
  }
};
template <int E> struct GRaw<__half, E> {
  uint4 v[E / 8];
  __device__ __forceinline__ void load(const __half *p) {
#pragma unroll
    for (int i = 0; i < E / 8; ++i) v[i] = __ldg(reinterpret_cast<const uint4 *>(p) + i);
  }
  __device__ __forceinline__ float2 get2(int k2, float s) const {
    const uint4 q = v[k2 / 4];
    const unsigned w = (k2 % 4 == 0) ? q.x : (k2 % 4 == 1) ? q.y : (k2 % 4 == 2) ? q.z : q.w;
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    return make_float2(f.x * s, f.y * s);
  }
};

template <int E, int G, int FE, typename GT>
__global__ void __launch_bounds__(128) k_zreg(Shape sh, const float2 *in_main, const float2 *in_nyq,
                                              const GT *kspec, const float *kscale, float2 *out_main,
                                              float2 *out_nyq, const float2 *tw) {
  constexpr int P = G * E, CW = 32 / G;
  const int lane = threadIdx.x & 31;
  const long TB = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int M = sh.M, py = sh.py, nz = sh.nz, fe = sh.fe;
  const long wt_main = (long)py * (M / CW);
  const long wt_all = wt_main + py / CW;
  // Consecutive warps take the same columns for the density sets of a batch, so the
  // kernel spectra come from HBM once and from L1/L2 for the others.
  const long T = TB / sh.nb;
  const int bset = (int)(TB - T * sh.nb);
  if (T >= wt_all) return;                              // whole warp exits together
  in_main += bset * ((long)fe * nz * py * M);
  in_nyq += bset * ((long)fe * py * nz);
  out_main += bset * (6L * nz * py * M);
  out_nyq += bset * (6L * py * nz);
  const int g = lane / CW, wl = lane - g * CW;
  const bool nyq = T >= wt_main;
  long ky = 0, kx = 0;
  if (!nyq) {
    ky = T / (M / CW);
    kx = (T - ky * (M / CW)) * CW + wl;
  } else {
    ky = (T - wt_main) * CW + wl;
  }
  const float2 *twP = tw + tw_offset(P);

  float2 f[FE][E];
#pragma unroll
  for (int e = 0; e < FE; ++e) {
#pragma unroll
    for (int m = 0; m < E; ++m) f[e][m] = make_float2(0.f, 0.f);
    if (e < fe) {
#pragma unroll
      for (int m = 0; m < E / 2; ++m) {
        const int z = g + G * m;
        if (z < nz) {
          f[e][m] = !nyq ? __ldg(in_main + (((long)e * nz + z) * py + ky) * M + kx)
                         : __ldg(in_nyq + ((long)e * py + ky) * nz + z);
        }
      }
    }
  }
  // kernel spectra of component 0, in flight while the fields are transformed
  const GT *ks = kspec + (T * 6L * fe) * 32 * E;
  GRaw<GT, E> gv[FE];
  float sc[FE];
#pragma unroll
  for (int e = 0; e < FE; ++e) {
    sc[e] = 1.0f;
    if (e < fe) {
      gv[e].load(ks + ((long)e * 32 + lane) * E);
      if (kscale != nullptr) sc[e] = __ldg(kscale + e);
    }
  }
#pragma unroll
  for (int e = 0; e < FE; ++e) {
    if (e < fe) {
      dft_reg<E, false>(f[e]);
      if (G > 1) {
#pragma unroll
        for (int k = 1; k < E; ++k) f[e][k] = cmul_tw<false>(f[e][k], __ldg(twP + g * k));
      }
      cross_lane_dft<E, G, false>(f[e], g, CW);
    }
  }
  for (int c = 0; c < 6; ++c) {
    float2 s[E];
#pragma unroll
    for (int k = 0; k < E; ++k) s[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < FE; ++e) {
      if (e < fe) {
#pragma unroll
        for (int k2 = 0; k2 < E / 2; ++k2) {
          const float2 g2 = gv[e].get2(k2, sc[e]);
          s[2 * k2] = cmadd_i(s[2 * k2], g2.x, f[e][2 * k2]);
          s[2 * k2 + 1] = cmadd_i(s[2 * k2 + 1], g2.y, f[e][2 * k2 + 1]);
        }
      }
    }
    if (c < 5) {   // next component's spectra fly while this one is inverted and stored
#pragma unroll
      for (int e = 0; e < FE; ++e) {
        if (e < fe) {
          gv[e].load(ks + (((long)(c + 1) * fe + e) * 32 + lane) * E);
          if (kscale != nullptr) sc[e] = __ldg(kscale + (c + 1) * fe + e);
        }
      }
    }
    cross_lane_dft<E, G, true>(s, g, CW);
    if (G > 1) {
#pragma unroll
      for (int k = 1; k < E; ++k) s[k] = cmul_tw<true>(s[k], __ldg(twP + g * k));
    }
    dft_reg<E, true>(s);
#pragma unroll
    for (int m = 0; m < E / 2; ++m) {
      const int z = g + G * m;
      if (z < nz) {
        if (!nyq) out_main[(((long)c * nz + z) * py + ky) * M + kx] = s[m];
        else out_nyq[((long)c * py + ky) * nz + z] = s[m];
      }
    }
  }
}

template <int PZ, int W, int FEMAX, typename GT>
cudaError_t launch_z_fe(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                        float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  const size_t smem = (sizeof(float2) * (size_t)(sh.fe + 3) + 2 * sizeof(GT) * (size_t)sh.fe) * PZ * W +
                      sizeof(float2) * z_s_extra<PZ, W>();
  const long tiles = ((long)sh.py * (sh.M / W) + sh.py / W) * sh.nb;
  cudaError_t err = prep(k_zpass<PZ, W, FEMAX, GT>, smem);
  if (err != cudaSuccess) return err;
  k_zpass<PZ, W, FEMAX, GT><<<(unsigned)tiles, NT, smem, s>>>(sh, im, in, ks, ksc, om, on, tw);
  return cudaGetLastError();
}

template <int PZ, int W, typename GT>
cudaError_t launch_z(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                     float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  if (sh.fe <= 6) return launch_z_fe<PZ, W, 6, GT>(sh, im, in, ks, ksc, om, on, tw, s);
  return launch_z_fe<PZ, W, DDS_MAX_FIELDS, GT>(sh, im, in, ks, ksc, om, on, tw, s);
}

// Tile widths the planner can choose: W * PZ <= 2048, or W <= 8.
template <int PZ, int W, typename GT>
cudaError_t launch_z_if(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                        float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  if constexpr (W * PZ <= 2048 || W <= 8) return launch_z<PZ, W, GT>(sh, im, in, ks, ksc, om, on, tw, s);
  return cudaErrorInvalidValue;
}

template <int PZ, typename GT>
cudaError_t dispatch_z_w(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                         float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  switch (sh.wz) {
    case 4: return launch_z_if<PZ, 4, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 8: return launch_z_if<PZ, 8, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 16: return launch_z_if<PZ, 16, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 32: return launch_z_if<PZ, 32, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 64: return launch_z_if<PZ, 64, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int E, int G, int FE, typename GT>
cudaError_t launch_zreg(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                        float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  constexpr int CW = 32 / G;
  const long warps = ((long)sh.py * (sh.M / CW) + sh.py / CW) * sh.nb;
  k_zreg<E, G, FE, GT><<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(sh, im, in, ks, ksc, om, on, tw);
  return cudaGetLastError();
}

template <int E, int G, typename GT>
cudaError_t dispatch_zreg_fe(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                             float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  if (sh.fe <= 1) return launch_zreg<E, G, 1, GT>(sh, im, in, ks, ksc, om, on, tw, s);
  if (sh.fe <= 2) return launch_zreg<E, G, 2, GT>(sh, im, in, ks, ksc, om, on, tw, s);
  return launch_zreg<E, G, 4, GT>(sh, im, in, ks, ksc, om, on, tw, s);
}

template <typename GT>
cudaError_t dispatch_z_typed(const Shape &sh, const float2 *im, const float2 *in, const GT *ks, const float *ksc,
                             float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  if (sh.zfour) {
    if (sh.pz == 128) return dispatch_zfour_fe<128, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    if (sh.pz == 256) return dispatch_zfour_fe<256, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    return cudaErrorInvalidValue;
  }
  if (sh.zreg_g > 0) {
    switch (sh.pz * 16 + sh.zreg_g) {   // (pz, lanes per column) -> E = pz / G registers
      case 16 * 16 + 1: return dispatch_zreg_fe<16, 1, GT>(sh, im, in, ks, ksc, om, on, tw, s);
      case 16 * 16 + 2: return dispatch_zreg_fe<8, 2, GT>(sh, im, in, ks, ksc, om, on, tw, s);
      case 32 * 16 + 2: return dispatch_zreg_fe<16, 2, GT>(sh, im, in, ks, ksc, om, on, tw, s);
      case 32 * 16 + 4: return dispatch_zreg_fe<8, 4, GT>(sh, im, in, ks, ksc, om, on, tw, s);
      case 64 * 16 + 4: return dispatch_zreg_fe<16, 4, GT>(sh, im, in, ks, ksc, om, on, tw, s);
      case 64 * 16 + 8: return dispatch_zreg_fe<8, 8, GT>(sh, im, in, ks, ksc, om, on, tw, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (sh.pz) {
    case 16: return dispatch_z_w<16, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 32: return dispatch_z_w<32, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 64: return dispatch_z_w<64, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 128: return dispatch_z_w<128, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 256: return dispatch_z_w<256, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    case 512: return dispatch_z_w<512, GT>(sh, im, in, ks, ksc, om, on, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace zp
}  // namespace dds
