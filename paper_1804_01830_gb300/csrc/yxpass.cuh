// Fused inverse y and x passes (the last two of the five passes of Eq. 10's FFT
// evaluation), one thread-block cluster per output plane (component c, height z):
//
//   CTA r of the CL CTAs takes the W spectrum columns kx in [r W, r W + W) of the
//   plane, runs the inverse y FFT of those columns in the two register stages of
//   k_ypass_st, and stores each output row y < ny straight into the shared memory of
//   the CTA that owns the row (rows [q RMAX, q RMAX + RMAX) on CTA q), through the
//   cluster's distributed shared memory.  After a cluster barrier every CTA holds its
//   rows with all M bins and runs the complex-to-real x transform of k_x_inv_tma on
//   them.  The half-spectrum lines between the two transforms never reach HBM: the
//   pass reads the z pass's output once and writes sigma once.
//
// The Nyquist column kx = M rides in column 0.  For a real plane both columns kx = 0
// and kx = M are Hermitian in ky (their x transform is real on every row), so the
// inverse y transform of X[0] + i X[M] returns the two real columns as its real and
// imaginary parts, and the x transform takes them from there.
#pragma once
#include <cooperative_groups.h>

#include "xpass.cuh"
#include "ypass.cuh"

namespace dds {
namespace yx {

namespace cg = cooperative_groups;

// W columns per CTA, CL = M / W CTAs per cluster (at most 16), RMAX output rows per
// CTA (ny <= PY / 2: the padded y transform).  The y transform of 512 points runs as
// 32 x 16 (one stage-1 column per thread).  Shared memory: the y stage's tile, then
// the gathered rows (RMAX x (M + 8)) and the x stage's transposes after it where the
// tile leaves room, else behind it.
template <int PY, int M> struct Cfg {
  static constexpr int W = 16, CL = M / W, NT = 256;
  static constexpr int RMAX = PY / 2 / CL;
  static constexpr int YR1 = PY == 512 ? 32 : yr::YCfg<PY>::R1, YR2 = PY / YR1, YST = YR2 * W;
  static constexpr int XLD = M + 8;                       // gathered rows: stride M + 8
  static constexpr int XR1 = xr::InvCfg<M>::R1, XR2 = xr::InvCfg<M>::R2;   // x: XR2 threads per line
  static constexpr int XS = XR2 * (XR1 + 1);              // x-stage transpose stride per line
  static constexpr int A = PY * W > YR1 * YST ? PY * W : YR1 * YST;
  static constexpr int B = RMAX * XLD, C = RMAX * XS;
  static constexpr int XT_OFF = B;                        // transposes behind the gathered rows
  static constexpr int SMEM_F2 = A > B + C ? A : B + C;
  static_assert(CL >= 2 && CL <= 16 && CL * W == M, "cluster of 2..16 CTAs");
  static_assert(YR1 * YR2 == PY && (W * YR2) % NT == 0 && (W * YR1) % NT == 0, "y stage items");
  static constexpr int XLP = NT / XR2;                    // x-stage lines per round
  static_assert(RMAX * CL * 2 == PY, "rows y < PY / 2 spread over the cluster");
  static_assert(RMAX % XLP == 0 || (RMAX < XLP && (RMAX * XR2) % 32 == 0),
                "x stage: whole rounds of lines, or one round of whole warps");
};

template <int PY, int M>
__global__ void __launch_bounds__(Cfg<PY, M>::NT, 3)
k_yx_inv(Shape sh, const float2 *__restrict__ in_main, const float2 *__restrict__ in_nyq, float *__restrict__ sigma,
         const float2 *__restrict__ tw, double *stats) {
  using C = Cfg<PY, M>;
  constexpr int W = C::W, CL = C::CL, NT = C::NT, RMAX = C::RMAX, XLD = C::XLD;
  constexpr int R1 = C::YR1, R2 = C::YR2, ST = C::YST;
  extern __shared__ __align__(16) float2 sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int nz = sh.nz, ny = sh.ny;
  const long plane = (long)blockIdx.x / CL;         // (set * 6 + c) * nz + z
  const int e = (int)(plane / nz), z = (int)(plane - (long)e * nz);

  // ---- y stage: the PY rows of this CTA's W columns, by cp.async (16-byte pairs)
  {
    const float2 *in = in_main + (plane * PY) * M + r * W;
    constexpr int H = W / 2;
    for (int p = tid; p < PY * H; p += NT) {
      const int n = p / H, c2 = p - n * H;
      cp_async16(&sm[n * W + 2 * c2], &in[(long)n * M + 2 * c2]);
    }
  }
  constexpr int NQ = (PY + NT - 1) / NT;
  float2 nq[NQ];
  if (r == 0) {                                     // X[M] of every row ky, for column 0
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const int n = tid + j * NT;
      nq[j] = n < PY ? in_nyq[((long)e * PY + n) * nz + z] : make_float2(0.f, 0.f);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (r == 0) {                                     // column 0 <- X[0] + i X[M]
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const int n = tid + j * NT;
      if (n < PY) {
        const float2 a = sm[n * W];
        sm[n * W] = make_float2(a.x - nq[j].y, a.y + nq[j].x);
      }
    }
    __syncthreads();
  }

  // stage 1: items (n2, w), column fastest; all reads before the barrier, then writes
  constexpr int I1 = (W * R2 + NT - 1) / NT;
  float2 v[I1][R1];
#pragma unroll
  for (int it = 0; it < I1; ++it) {
    const int item = tid + it * NT;
    const int n2 = item / W, w = item - n2 * W;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1)
      v[it][n1] = ((W * R2) % NT == 0 || item < W * R2) ? sm[(n2 + R2 * n1) * W + w] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2 *twP = tw + tw_offset(PY);
#pragma unroll
  for (int it = 0; it < I1; ++it) {
    const int item = tid + it * NT;
    if ((W * R2) % NT != 0 && item >= W * R2) continue;
    const int n2 = item / W, w = item - n2 * W;
    dft_reg<R1, true>(v[it]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 y = v[it][k1];
      if (k1 > 0) y = cmul_tw<true>(y, __ldg(twP + n2 * k1));
      sm[k1 * ST + n2 * W + w] = y;
    }
  }
  __syncthreads();

  // stage 2: items (k1, w); rows k = k1 + R1 k2 < PY / 2 are kept
  constexpr int I2 = (W * R1 + NT - 1) / NT, K2 = R2 / 2;
  float2 o[I2][K2];
#pragma unroll
  for (int it = 0; it < I2; ++it) {
    const int item = tid + it * NT;
    const int k1 = item / W, w = item - k1 * W;
    float2 y[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2)
      y[n2] = ((W * R1) % NT == 0 || item < W * R1) ? sm[k1 * ST + n2 * W + w] : make_float2(0.f, 0.f);
    dft_reg<R2, true>(y);
#pragma unroll
    for (int k2 = 0; k2 < K2; ++k2) o[it][k2] = y[k2];
  }
  cluster.sync();           // every CTA has read its stage-2 inputs: the buffers take the rows
#pragma unroll
  for (int it = 0; it < I2; ++it) {
    const int item = tid + it * NT;
    if ((W * R1) % NT != 0 && item >= W * R1) continue;
    const int k1 = item / W, w = item - k1 * W;
#pragma unroll
    for (int k2 = 0; k2 < K2; ++k2) {
      const int k = k1 + R1 * k2;
      if (k < ny) {
        const int q = k / RMAX;
        float2 *dst = cluster.map_shared_rank(sm, q);
        dst[(k - q * RMAX) * XLD + r * W + w] = o[it][k2];
      }
    }
  }
  cluster.sync();           // rows complete (release / acquire across the cluster)

  // ---- x stage: line lw = row r RMAX + lw, XR2 threads per line, thread t owning
  // column t of the four-step factorisation (bins k = t + XR2 n1) and reading each
  // bin's mirror X[M - k] from the gathered row (c2r identities of k_x_inv_tma)
  constexpr int XR1 = C::XR1, XR2 = C::XR2, LD = XR1 + 1, XS = C::XS, XLP = C::XLP;
  const int t = tid % XR2;
  const float2 *twM = tw + tw_offset(M);
  const float2 *tw2 = tw + tw_offset(2 * M);
  const int nxh = (sh.nx + 1) >> 1;
  const bool even = (sh.nx & 1) == 0;
#pragma unroll 1
  for (int l0 = 0; l0 < RMAX; l0 += XLP) {
    const int lw = l0 + tid / XR2;
    const bool mine = lw < RMAX;
    const int yrow = r * RMAX + lw;
    const bool live = mine && yrow < ny;
    float2 *ls = sm + C::XT_OFF + lw * XS;
    if (mine) {
      const float2 *row = sm + lw * XLD;
      const float2 p0 = row[0];                     // X[0] + i X[M], both real
      float2 za[XR1];
#pragma unroll
      for (int n1 = 0; n1 < XR1; ++n1) {
        const int k = t + XR2 * n1;
        float2 a = row[k], am;
        if (k == 0) {
          a = make_float2(p0.x, 0.f);
          am = make_float2(p0.y, 0.f);
        } else {
          am = row[M - k];
        }
        za[n1] = xr::c2r_pre(a, am, __ldg(tw2 + k));
      }
      dft_reg<XR1, true>(za);
#pragma unroll
      for (int m1 = 0; m1 < XR1; ++m1) {
        const float2 y = m1 > 0 ? cmul_tw<true>(za[m1], __ldg(twM + t * m1)) : za[m1];
        ls[t * LD + m1] = y;
      }
    }
    __syncthreads();
    if (mine) {
      float ssq = 0.f;
      float *dst = sigma + (plane * ny + yrow) * sh.nx;
      const int m1 = t;                               // row m1 < XR1 of the second stage
      if (m1 < XR1) {
        float2 y[XR2];
#pragma unroll
        for (int c = 0; c < XR2; ++c) y[c] = ls[c * LD + m1];
        dft_reg<XR2, true>(y);
        if (live) {
#pragma unroll
          for (int m2 = 0; m2 < XR2 / 2; ++m2) {
            const int n = m1 + XR1 * m2;
            if (n < nxh) {
              if (even) {
                __stcs(reinterpret_cast<float2 *>(dst + 2 * n), y[m2]);
                ssq += y[m2].x * y[m2].x + y[m2].y * y[m2].y;
              } else {
                dst[2 * n] = y[m2].x;
                ssq += y[m2].x * y[m2].x;
                if (2 * n + 1 < sh.nx) {
                  dst[2 * n + 1] = y[m2].y;
                  ssq += y[m2].y * y[m2].y;
                }
              }
            }
          }
        }
      }
      if (stats != nullptr) {
#pragma unroll
        for (int off = XR2 / 2; off > 0; off >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, off, XR2);
        if (live && t == 0) atomicAdd(&stats[plane], (double)ssq);
      }
    }
  }
}

}  // namespace yx
}  // namespace dds
