// Register-resident x passes: the real-to-complex FFT of the density lines and the
// complex-to-real FFT of the stress lines (the first and last of the five passes).
//
// A line of the half spectrum has M = R1 * R2 complex points and is handled by T
// threads.  Each thread keeps its share of the line in registers, so a line moves
// through shared memory exactly once, between the two DFT stages of the four-step
// factorisation
//
//   sum_n v[n] W^{kn},  n = n2 + R2 n1, k = k1 + R1 k2:
//     stage 1: R1-point DFTs over n1 (one per column n2), times W_M^{n2 k1}
//     stage 2: R2-point DFTs over n2 (one per row k1).
//
// Both passes also need, for every bin k, the bin M - k (the half-length real-FFT
// identities).  The column (or row) that holds the mirror of column c is R - c, so
// every thread owns a mirror pair of columns (inverse) or rows (forward) and the
// identities are evaluated in registers.
#pragma once
#include "bulk.cuh"
#include "stress_common.cuh"

namespace dds {
namespace xr {

// Inverse: R1 points per column, R2 columns, T = R2 / 2 threads per line, each
// owning columns t and R2 - t (thread 0: columns 0 and R2 / 2, both self-mirrored).
template <int M> struct InvCfg;
template <> struct InvCfg<16>  { static constexpr int R1 = 4,  R2 = 4; };
template <> struct InvCfg<32>  { static constexpr int R1 = 4,  R2 = 8; };
template <> struct InvCfg<64>  { static constexpr int R1 = 8,  R2 = 8; };
template <> struct InvCfg<128> { static constexpr int R1 = 8,  R2 = 16; };
template <> struct InvCfg<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct InvCfg<512> { static constexpr int R1 = 16, R2 = 32; };

// Forward: R1 points per column of which the first R1 / 2 are non-zero (the padded
// half of the line), R2 columns, T = R1 / 2 threads per line, each owning rows t and
// R1 - t of the second stage (thread 0: rows 0 and R1 / 2).
template <int M> struct FwdCfg;
template <> struct FwdCfg<16>  { static constexpr int R1 = 4,  R2 = 4; };
template <> struct FwdCfg<32>  { static constexpr int R1 = 8,  R2 = 4; };
template <> struct FwdCfg<64>  { static constexpr int R1 = 8,  R2 = 8; };
template <> struct FwdCfg<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct FwdCfg<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct FwdCfg<512> { static constexpr int R1 = 32, R2 = 16; };

constexpr int THREADS = 128;

// Shared-memory stride of one line: R rows of LD values, plus a shift that puts the
// lines sharing a half-warp on different banks (conflict-free for every config).
template <int T> __host__ __device__ constexpr int line_pad() { return T >= 16 ? 0 : T; }

// ------------------------------------------------------------- x inverse ---
// Z[k] = (X[k] + conj X[M-k]) + i conj(W_2M^k) (X[k] - conj X[M-k]); then
// z = IDFT_M(Z) gives sigma[2n] = Re z[n], sigma[2n+1] = Im z[n].
__device__ __forceinline__ float2 c2r_pre(float2 A, float2 Bm, float2 wk) {
  const float2 E = make_float2(A.x + Bm.x, A.y - Bm.y);
  const float2 D = make_float2(A.x - Bm.x, A.y + Bm.y);
  const float2 O = make_float2(D.x * wk.x + D.y * wk.y, D.y * wk.x - D.x * wk.y);
  return make_float2(E.x - O.y, E.y + O.x);
}

// The inverse pass is persistent: each CTA walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; the LPB input lines of a tile are contiguous and
// arrive in one bulk copy (TMA) into one of two shared-memory slots, issued two
// tiles ahead, so the copy of the next tile overlaps the transforms of this one.
// A slot, once its lines are in registers, serves as the tile's transpose buffer.
// stats != nullptr: the pass also accumulates sum_x sigma^2 of every line into
// stats[(set * 6 + c) * nz + z] (the per-height sums of Eq. 20).
template <int M> struct InvTma {
  static constexpr int R1 = InvCfg<M>::R1, R2 = InvCfg<M>::R2, T = R2 / 2;
  static constexpr int LPB = THREADS / T, S = R2 * (R1 + 1) + line_pad<T>();
  static constexpr int SLOT = (LPB * M > LPB * S ? LPB * M : LPB * S);       // float2 per slot
  // two slots, two barriers, then the M twiddles exp(-2 pi i m / M) and the first M of
  // exp(-2 pi i m / 2M) (the c2r identities use bins k < M only), staged once per
  // persistent CTA; at 256 points three CTAs still fit an SM (3 x 75.8 KB).  A thread's
  // twiddles then stay in its registers across the tiles (GaN layer 0.151 -> 0.127 ms)
  static constexpr size_t SMEM = sizeof(float2) * 2 * SLOT + 2 * sizeof(uint64_t) + sizeof(float2) * 2 * M;
};

__device__ __forceinline__ long nyq_index(const Shape &sh, long line) {
  const long cz = line / sh.ny;
  const int y = (int)(line - cz * sh.ny);
  const int c = (int)(cz / sh.nz), z = (int)(cz - (long)c * sh.nz);
  return ((long)c * sh.ny + y) * sh.nz + z;
}

template <int M>
__global__ void __launch_bounds__(THREADS)
k_x_inv_tma(Shape sh, const float2 *__restrict__ in_main, const float2 *__restrict__ in_nyq,
            float *__restrict__ sigma, const float2 *__restrict__ tw, double *stats, int *status) {
  using C = InvTma<M>;
  constexpr int R1 = C::R1, R2 = C::R2, T = C::T, RPT = R1 / T, LPB = C::LPB, LD = R1 + 1, S = C::S;
  static_assert(R1 * R2 == M && RPT >= 1 && RPT * T == R1, "x inverse config");
  extern __shared__ __align__(16) float2 dsm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(dsm + 2 * C::SLOT);
  float2 *stwM = reinterpret_cast<float2 *>(bar + 2);
  const int t = threadIdx.x % T, lw = threadIdx.x / T;
  const bool t0 = t == 0;
  const int ca = t, cb = t0 ? R2 / 2 : R2 - t;
  const long L = 6L * sh.nb * sh.nz * sh.ny;
  const long ntiles = (L + LPB - 1) / LPB;
  const long stride = gridDim.x;
  for (int i = threadIdx.x; i < M; i += THREADS) {
    stwM[i] = __ldg(tw + tw_offset(M) + i);
    stwM[M + i] = __ldg(tw + tw_offset(2 * M) + i);
  }
  const float2 *twM = stwM;
  const float2 *tw2 = stwM + M;
  const int nxh = (sh.nx + 1) >> 1;
  const bool even = (sh.nx & 1) == 0;

  auto issue = [&](long tile, int s) {        // one thread: bulk copy of a tile into slot s
    const long l0 = tile * LPB;
    const unsigned bytes = (unsigned)(min((long)LPB, L - l0) * M * sizeof(float2));
    mbar_arrive_expect_tx(&bar[s], bytes);
    bulk_g2s(dsm + s * C::SLOT, in_main + l0 * M, bytes, &bar[s]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0 only: copies issued and not yet waited for, and the barrier phase
  // (parity) each will complete; use j of slot j & 1 completes phase (j >> 1) & 1
  bool pending[2] = {false, false};
  unsigned pend_par[2] = {0u, 0u};
  if (threadIdx.x == 0) {
    if (blockIdx.x < ntiles) { issue(blockIdx.x, 0); pending[0] = true; }
    if (blockIdx.x + stride < ntiles) { issue(blockIdx.x + stride, 1); pending[1] = true; }
  }
  float2 xm_next = make_float2(0.f, 0.f);
  {
    const long line = (long)blockIdx.x * LPB + lw;
    if (t0 && blockIdx.x < ntiles && line < L) xm_next = in_nyq[nyq_index(sh, line)];
  }
  bool ok = true;
  for (long i = 0;; ++i) {
    const long tile = blockIdx.x + i * stride;
    if (tile >= ntiles) break;
    const int s = (int)(i & 1);
    const unsigned parity = (unsigned)((i >> 1) & 1);
    float2 *buf = dsm + s * C::SLOT;
    const long line = tile * LPB + lw;
    const bool live = line < L;
    const float2 xm = xm_next;
    {
      const long nline = (tile + stride) * LPB + lw;
      xm_next = (t0 && tile + stride < ntiles && nline < L) ? in_nyq[nyq_index(sh, nline)] : make_float2(0.f, 0.f);
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar[s], parity, status));
    if (!ok) break;
    if (threadIdx.x == 0) pending[s] = false;
    float2 a[R1], b[R1];
    const float2 *src = buf + lw * M;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      a[n1] = src[ca + R2 * n1];
      b[n1] = src[cb + R2 * n1];
    }
    __syncthreads();                          // raw lines read: the slot becomes the transpose buffer
    float2 za[R1], zb[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const float2 am = t0 ? (n1 == 0 ? xm : a[(R1 - n1) % R1]) : b[R1 - 1 - n1];
      const float2 bm = t0 ? b[R1 - 1 - n1] : a[R1 - 1 - n1];
      za[n1] = c2r_pre(a[n1], am, tw2[ca + R2 * n1]);
      zb[n1] = c2r_pre(b[n1], bm, tw2[cb + R2 * n1]);
    }
    dft_reg<R1, true>(za);
    dft_reg<R1, true>(zb);
    float2 *ls = buf + lw * S;
#pragma unroll
    for (int m1 = 0; m1 < R1; ++m1) {
      if (m1 > 0) {
        za[m1] = cmul_tw<true>(za[m1], twM[ca * m1]);
        zb[m1] = cmul_tw<true>(zb[m1], twM[cb * m1]);
      }
      ls[ca * LD + m1] = za[m1];
      ls[cb * LD + m1] = zb[m1];
    }
    __syncthreads();
    float ssq = 0.f;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int m1 = t + T * r;
      float2 y[R2];
#pragma unroll
      for (int c = 0; c < R2; ++c) y[c] = ls[c * LD + m1];
      dft_reg<R2, true>(y);
      if (live) {
        float *dst = sigma + line * sh.nx;
#pragma unroll
        for (int m2 = 0; m2 < R2 / 2; ++m2) {
          const int n = m1 + R1 * m2;
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
      for (int o = T / 2; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
      if (live && t0) atomicAdd(&stats[line / sh.ny], (double)ssq);
    }
    __syncthreads();                          // slot free: refill it two tiles ahead
    if (threadIdx.x == 0 && tile + 2 * stride < ntiles) {
      fence_proxy_async_smem();
      issue(tile + 2 * stride, s);
      pending[s] = true;
      pend_par[s] = (unsigned)(((i + 2) >> 1) & 1);
    }
  }
  if (!ok && threadIdx.x == 0) {              // gave up: let copies still in flight land first
    for (int s = 0; s < 2; ++s)
      if (pending[s]) {
        const unsigned long long t0ns = global_ns();
        while (!mbar_try_wait(&bar[s], pend_par[s]) && global_ns() - t0ns < WAIT_LIMIT_NS) {
        }
      }
  }
}

// ------------------------------------------------------------- x forward ---
// Z = DFT_M(z), z[n] = x[2n] + i x[2n+1]; X[k] = E + W_2M^k O with
// E = (Z[k] + conj Z[M-k]) / 2, O = -i (Z[k] - conj Z[M-k]) / 2, and
// X[M] = E - O at k = 0.  Each field is scaled by `scale` on output.
__device__ __forceinline__ float2 r2c_post(float2 a, float2 c, float2 wk, float scale) {
  const float2 E = make_float2(0.5f * (a.x + c.x), 0.5f * (a.y - c.y));
  const float2 O = make_float2(0.5f * (a.y + c.y), -0.5f * (a.x - c.x));
  return make_float2(scale * (E.x + (wk.x * O.x - wk.y * O.y)), scale * (E.y + (wk.x * O.y + wk.y * O.x)));
}

// Complex pair (x[2n], x[2n+1]) of one density line (zero beyond nx).
template <bool BF16>
__device__ __forceinline__ float2 load_pair(const void *rho, long o, int n2x, int nx, bool even) {
  if (BF16) {
    const uint16_t *r = (const uint16_t *)rho;
    if (even) {                                 // both values in one aligned 32-bit word
      const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(r + o));
      return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    return make_float2(bf16_to_f32(r[o]), n2x + 1 < nx ? bf16_to_f32(r[o + 1]) : 0.f);
  }
  const float *r = (const float *)rho;
  if (even) return __ldcs(reinterpret_cast<const float2 *>(r + o));
  return make_float2(r[o], n2x + 1 < nx ? r[o + 1] : 0.f);
}

// Four consecutive density values x[o .. o+3] (o a multiple of 4, row length a multiple
// of 4): one 16-byte load (FP32) or one 8-byte load (BF16).
template <bool BF16>
__device__ __forceinline__ float4 load_quad(const void *rho, long o) {
  if (BF16) {
    const uint2 w = __ldg(reinterpret_cast<const uint2 *>((const uint16_t *)rho + o));
    return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u),
                       __uint_as_float(w.y << 16), __uint_as_float(w.y & 0xffff0000u));
  }
  return __ldcs(reinterpret_cast<const float4 *>((const float *)rho + o));
}

// Groups with one family and one field (DIRECT) transform that family scaled by its
// coefficient; the others sum coef * rho over the group's families for each field.
// CTAs per SM the register budget is set for.  256 points: three, at most 170
// registers -- the summed-family kernel would otherwise take 176 and fit two; GaN layer
// 0.239 -> 0.233 ms.  128 points: four, 128 registers -- left free it takes 182 (two per
// SM), and bound to three it takes 163 and runs 18% slower.  512 points: direct groups
// four (radial disk 0.042 ms left free at 207 registers, 0.036 at three or four); summed
// families the compiler's choice (254 registers; bound to three they spill 312 bytes).
template <int M, bool DIRECT> constexpr int x_fwd_ctas() {
  return M == 256 ? 3 : (M == 128 ? 4 : (M == 512 && DIRECT ? 4 : 1));
}

template <int M, bool BF16, bool DIRECT>
__global__ void __launch_bounds__(THREADS, (x_fwd_ctas<M, DIRECT>()))
k_x_fwd_reg(Shape sh, Collapse col, GroupList gl, const void *__restrict__ rho_v, float2 *__restrict__ out_main,
            float2 *__restrict__ out_nyq, const float2 *__restrict__ tw) {
  constexpr int R1 = FwdCfg<M>::R1, R2 = FwdCfg<M>::R2, T = R1 / 2, CPT = R2 / T, H = R1 / 2;
  // thread t owns the adjacent columns n2 = CPT t + q; row stride and line shift keep
  // the shared-memory stages free of bank conflicts (2-way left for M = 16, 64)
  constexpr int LD = (M == 256) ? R2 + 2 : R2 + 1;
  constexpr int PADL = (M == 256) ? 1 : (CPT == 1 ? line_pad<T>() : 0);
  constexpr int LPB = THREADS / T, S = R1 * LD + PADL;
  static_assert(R1 * R2 == M && CPT >= 1 && CPT * T == R2 && CPT <= 2, "x forward config");
  __shared__ float2 sm[LPB * S];
  // lines of up to 256 points: the M and 2M twiddles staged in shared memory (GaN layer
  // 0.233 -> 0.220 ms; for 512 points, eight lines per CTA, the staging costs more than
  // it saves: radial disk 0.036 -> 0.044 ms)
  constexpr bool STW = M <= 256;
  __shared__ float2 stw[STW ? 3 * M : 1];
  const int t = threadIdx.x % T, lw = threadIdx.x / T;
  const long L = (long)sh.ny * sh.nz;
  const long N = L * sh.nx;
  const long line = (long)blockIdx.x * LPB + lw;
  const bool live = line < L;
  const bool t0 = t == 0;
  const int g = gl.g[blockIdx.y];
  const int bset = blockIdx.z;                       // density set of the batch
  const long set_off = (long)bset * sh.fin * N;
  const int nxh = (sh.nx + 1) >> 1;
  const bool even = (sh.nx & 1) == 0;
  const bool quad = (sh.nx & 3) == 0;               // rows and column pairs 16-byte aligned
  if constexpr (STW) {
    for (int i = threadIdx.x; i < M; i += THREADS) stw[i] = __ldg(tw + tw_offset(M) + i);
    for (int i = threadIdx.x; i < 2 * M; i += THREADS) stw[M + i] = __ldg(tw + tw_offset(2 * M) + i);
  }
  const float2 *twM = STW ? stw : tw + tw_offset(M);
  const float2 *tw2 = STW ? stw + M : tw + tw_offset(2 * M);
  const int ra = t, rb = t0 ? R1 / 2 : R1 - t;
  float2 *ls = sm + lw * S;

  // stage-1 inputs z[n2 + R2 n1], n2 = CPT t + q, n1 < R1 / 2, of every field of the
  // group: each family is read once and added into all fields (coef * rho).
  constexpr int NDM = DIRECT ? 1 : 3;
  const int nd = col.nd[g];
  float2 acc[NDM][CPT][H];
#pragma unroll
  for (int d = 0; d < NDM; ++d)
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) acc[d][q][n1] = make_float2(0.f, 0.f);
  const int nfam = DIRECT ? 1 : col.nf[g];
  if (live) {
#pragma unroll 2
    for (int f = 0; f < nfam; ++f) {
      const int fi = col.f0[g] + f;
      const long base = set_off + (long)col.fam[fi] * N + line * sh.nx;
      float2 v[CPT][H];
      if (CPT == 2 && quad) {                 // both columns' pairs in one 16-byte (8 for bf16) load
#pragma unroll
        for (int n1 = 0; n1 < H; ++n1) {
          const int n = CPT * t + R2 * n1;    // even; nxh even, so n + 1 < nxh with n
          if (n < nxh) {
            const float4 x = load_quad<BF16>(rho_v, base + 2 * n);
            v[0][n1] = make_float2(x.x, x.y);
            v[CPT - 1][n1] = make_float2(x.z, x.w);
          } else {
            v[0][n1] = v[CPT - 1][n1] = make_float2(0.f, 0.f);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < CPT; ++q)
#pragma unroll
          for (int n1 = 0; n1 < H; ++n1) {
            const int n = CPT * t + q + R2 * n1;
            v[q][n1] = n < nxh ? load_pair<BF16>(rho_v, base + 2 * n, 2 * n, sh.nx, even) : make_float2(0.f, 0.f);
          }
      }
      if (DIRECT) {
#pragma unroll
        for (int q = 0; q < CPT; ++q)
#pragma unroll
          for (int n1 = 0; n1 < H; ++n1) acc[0][q][n1] = v[q][n1];
      } else {
#pragma unroll
        for (int d = 0; d < NDM; ++d) {
          const float cf = col.coef[fi][d];
#pragma unroll
          for (int q = 0; q < CPT; ++q)
#pragma unroll
            for (int n1 = 0; n1 < H; ++n1) {
              acc[d][q][n1].x = fmaf(cf, v[q][n1].x, acc[d][q][n1].x);
              acc[d][q][n1].y = fmaf(cf, v[q][n1].y, acc[d][q][n1].y);
            }
        }
      }
    }
  }
  const float dscale = DIRECT ? col.coef[col.f0[g]][0] : 1.f;
  if constexpr (STW) __syncthreads();                // twiddles staged

#pragma unroll
  for (int d = 0; d < NDM; ++d) {
    if (d >= nd) break;
    const float scale = dscale;
    // stage 1: R1-point DFT of half-zero columns = two R1/2-point DFTs (even and odd
    // outputs), then twiddle W_M^{n2 k1}
    if (d > 0) __syncthreads();                      // previous field's stage 2 has read ls
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int n2 = CPT * t + q;
      float2 ev[H], od[H];
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) {
        ev[n1] = acc[d][q][n1];
        od[n1] = rot_const<false>(acc[d][q][n1], n1, R1);
      }
      dft_reg<H, false>(ev);
      dft_reg<H, false>(od);
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const int k0 = 2 * j, k1 = 2 * j + 1;
        float2 y0 = ev[j], y1 = od[j];
        if (k0 > 0) y0 = cmul_tw<false>(y0, twM[n2 * k0]);
        y1 = cmul_tw<false>(y1, twM[n2 * k1]);
        ls[k0 * LD + n2] = y0;
        ls[k1 * LD + n2] = y1;
      }
    }
    __syncthreads();
    // stage 2: rows ra and rb, R2-point DFTs -> Z[r + R1 k2]
    float2 ya[R2], yb[R2];
#pragma unroll
    for (int c = 0; c < R2; ++c) {
      ya[c] = ls[ra * LD + c];
      yb[c] = ls[rb * LD + c];
    }
    dft_reg<R2, false>(ya);
    dft_reg<R2, false>(yb);
    if (live) {
      const int e = bset * sh.fe + col.e0[g] + d;
      float2 *dst = out_main + ((long)e * L + line) * M;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const float2 am = t0 ? ya[(R2 - k2) % R2] : yb[R2 - 1 - k2];
        const float2 bm = t0 ? yb[R2 - 1 - k2] : ya[R2 - 1 - k2];
        const int ka = ra + R1 * k2, kb = rb + R1 * k2;
        __stcs(dst + ka, r2c_post(ya[k2], am, tw2[ka], scale));
        __stcs(dst + kb, r2c_post(yb[k2], bm, tw2[kb], scale));
      }
      if (t0) {
        const int z = (int)(line / sh.ny), y = (int)(line - (long)z * sh.ny);
        const float2 a0 = ya[0];
        const float2 E = make_float2(0.5f * (a0.x + a0.x), 0.5f * (a0.y - a0.y));
        const float2 O = make_float2(0.5f * (a0.y + a0.y), -0.5f * (a0.x - a0.x));
        out_nyq[((long)e * sh.ny + y) * sh.nz + z] = make_float2(scale * (E.x - O.x), scale * (E.y - O.y));
      }
    }
  }
}

}  // namespace xr
}  // namespace dds
