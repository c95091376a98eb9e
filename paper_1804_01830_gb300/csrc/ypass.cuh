// y passes: the forward FFT along y (rows y < ny in, all P_y rows out) and the
// inverse (all rows in, rows y < ny out), on tiles of W adjacent columns (kx, or z for
// the Nyquist arrays) of P = R1 * R2 rows, in two register stages (four-step
// factorisation, n = n2 + R2 n1, k = k1 + R1 k2):
//   the tile's rows arrive in shared memory by cp.async (16-byte copies of column
//   pairs); stage 1: a thread takes the R1 rows n2 + R2 n1 of one column into
//   registers, runs the R1-point DFT and the twiddle W_P^{n2 k1} and writes the
//   results back transposed (the same buffer, after a barrier); stage 2: a thread
//   reads the R2 values of one k1 and one column, runs the R2-point DFT and stores
//   rows k1 + R1 k2 straight to global memory.
// Threads are numbered with the column fastest, so the shared-memory accesses of a
// warp are contiguous and its global stores are runs of W complex values per row.
// With zero padding (FULL false) the forward input is zero from row ny on and
// ny <= P/2, so stage 1 reads only n1 < R1/2 and splits the R1-point DFT into two
// R1/2-point DFTs; the inverse keeps rows k < ny <= P/2, so stage 2 computes only
// k2 < R2/2.  FULL (periodic in y, P = ny): every row is read and kept.
#pragma once
#include "stress_common.cuh"

namespace dds {
namespace yr {

template <int P> struct YCfg {
  static constexpr int R1 = Plan<P>::r0, R2 = Plan<P>::r1;
  static_assert(Plan<P>::n == 2 && R1 * R2 == P, "two-stage plan");
};

// Row stride of the transposed stage-1 results (R2 W values plus a shift that keeps
// both stages free of bank conflicts for every tile width used).
template <int P, int W> __host__ __device__ constexpr int y_stride() { return YCfg<P>::R2 * W + (W < 16 ? W : 0); }

template <int P, int W> __host__ __device__ constexpr int y_smem() {
  return P * W > YCfg<P>::R1 * y_stride<P, W>() ? P * W : YCfg<P>::R1 * y_stride<P, W>();
}

// Whether the tile stages the PY twiddles in shared memory (after its y_smem values):
// stage 1 reads them at scattered indices.  Forward passes up to 512 rows gain (GaN layer
// 0.190 -> 0.176 ms), and so does the 512-row inverse on its 16-column tiles (0.207 ->
// 0.201 ms; on 8-column tiles it lost a CTA per SM and 0.009 ms).  The full-row
// periodic passes take it up to 256 rows; 1024 rows lose in both directions.
template <int PY, bool INV, bool FULL> __host__ __device__ constexpr bool y_stw() {
  return PY <= 512 && (!FULL || PY <= 256);
}
template <int PY, int W, bool INV, bool FULL> __host__ __device__ constexpr int y_smem_all() {
  return y_smem<PY, W>() + (y_stw<PY, INV, FULL>() ? PY : 0);
}

template <int PY, int W, int NT, bool INV, bool FULL = false>
__global__ void __launch_bounds__(NT) k_ypass_st(Shape sh, int nf, const float2 *__restrict__ in_main,
                                                 const float2 *__restrict__ in_nyq, float2 *__restrict__ out_main,
                                                 float2 *__restrict__ out_nyq, const float2 *__restrict__ tw) {
  constexpr int R1 = YCfg<PY>::R1, R2 = YCfg<PY>::R2, ST = y_stride<PY, W>();
  extern __shared__ __align__(16) float2 sm[];              // y_smem_all<PY, W, INV, FULL>() values
  const int tid = threadIdx.x;
  const int M = sh.M, nz = sh.nz;
  const int rows_in = INV ? PY : sh.ny;
  const int rows_out = INV ? sh.ny : PY;
  const long ktiles = M / W;
  const long tiles_main = (long)nf * nz * ktiles;
  const long tau = blockIdx.x;
  const float2 *in;
  float2 *out;
  long rs;
  int ncols;
  const bool main_tile = tau < tiles_main;
  if (main_tile) {
    const int e = (int)(tau / (nz * ktiles));
    const long r = tau - (long)e * nz * ktiles;
    const int z = (int)(r / ktiles), kt = (int)(r - (long)z * ktiles);
    in = in_main + ((long)(e * nz + z) * rows_in) * M + kt * W;
    out = out_main + ((long)(e * nz + z) * rows_out) * M + kt * W;
    rs = M;
    ncols = W;
  } else {
    const long t2 = tau - tiles_main;
    const int ztiles = (nz + W - 1) / W;
    const int e = (int)(t2 / ztiles), zt = (int)(t2 - (long)e * ztiles);
    in = in_nyq + (long)e * rows_in * nz + zt * W;
    out = out_nyq + (long)e * rows_out * nz + zt * W;
    rs = nz;
    ncols = min(W, nz - zt * W);
  }
  // stage the rows: element (n, w) at sm[n W + w]
  if (main_tile) {                            // rows of W complex values, 16-byte aligned
    constexpr int H = W / 2;
    for (int p = tid; p < rows_in * H; p += NT) {
      const int n = p / H, c2 = p - n * H;
      cp_async16(&sm[n * W + 2 * c2], &in[n * rs + 2 * c2]);
    }
  } else {
    for (int p = tid; p < rows_in * W; p += NT) {
      const int n = p / W, w = p - n * W;
      if (w < ncols) cp_async8(&sm[n * W + w], &in[n * rs + w]);
      else sm[n * W + w] = make_float2(0.f, 0.f);
    }
  }
  constexpr bool STW = y_stw<PY, INV, FULL>();
  float2 *stw = sm + y_smem<PY, W>();
  if constexpr (STW)
    for (int i = tid; i < PY; i += NT) stw[i] = __ldg(tw + tw_offset(PY) + i);
  cp_async_wait_all();
  __syncthreads();

  // stage 1: items (n2, w), column fastest; all reads before the barrier, then writes
  constexpr int I1 = (W * R2 + NT - 1) / NT;
  constexpr int N1 = (INV || FULL) ? R1 : R1 / 2;   // non-zero inputs per column
  float2 v[I1][N1];
#pragma unroll
  for (int it = 0; it < I1; ++it) {
    const int item = tid + it * NT;
    const int n2 = item / W, w = item - n2 * W;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int n = n2 + R2 * n1;
      v[it][n1] = ((W * R2) % NT == 0 || item < W * R2) && n < rows_in ? sm[n * W + w] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const float2 *twP = STW ? stw : tw + tw_offset(PY);
#pragma unroll
  for (int it = 0; it < I1; ++it) {
    const int item = tid + it * NT;
    if ((W * R2) % NT != 0 && item >= W * R2) continue;
    const int n2 = item / W, w = item - n2 * W;
    float2 x[R1];
    if constexpr (!INV && !FULL) {
      constexpr int H = R1 / 2;
      float2 ev[H], od[H];
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) {
        ev[n1] = v[it][n1];
        od[n1] = rot_const<false>(v[it][n1], n1, R1);
      }
      dft_reg<H, false>(ev);
      dft_reg<H, false>(od);
#pragma unroll
      for (int j = 0; j < H; ++j) {
        x[2 * j] = ev[j];
        x[2 * j + 1] = od[j];
      }
    } else {
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = v[it][n1];
      dft_reg<R1, INV>(x);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 y = x[k1];
      if (k1 > 0) y = cmul_tw<INV>(y, STW ? twP[n2 * k1] : __ldg(twP + n2 * k1));
      sm[k1 * ST + n2 * W + w] = y;
    }
  }
  __syncthreads();

  // stage 2: items (k1, w)
  constexpr int I2 = (W * R1 + NT - 1) / NT;
  constexpr int K2 = (INV && !FULL) ? R2 / 2 : R2;
#pragma unroll
  for (int it = 0; it < I2; ++it) {
    const int item = tid + it * NT;
    if ((W * R1) % NT != 0 && item >= W * R1) continue;
    const int k1 = item / W, w = item - k1 * W;
    float2 y[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) y[n2] = sm[k1 * ST + n2 * W + w];
    dft_reg<R2, INV>(y);
    if (w < ncols) {
#pragma unroll
      for (int k2 = 0; k2 < K2; ++k2) {
        const int k = k1 + R1 * k2;
        if (k < rows_out) __stcs(out + (long)k * rs + w, y[k2]);
      }
    }
  }
}

}  // namespace yr
}  // namespace dds
