// FP32 evaluation of sigma_c = sum_e G_c^e * rho_e (Eq. 10) as a zero-padded FFT
// convolution (Sec. 2.3, first remark), in five passes over HBM:
//
//   x_fwd : densities of the F input families -> effective fields (linear in b),
//           real-to-complex FFT along x of the non-zero half of each padded line
//           (2M points, of which the last M are zero and never read);
//   y_fwd : FFT along y, input rows y < ny, output all py rows;
//   z     : per tile of (kx, ky) columns: FFT along z of every field (input rows
//           z < nz), contraction with the cached kernel spectra
//             sigma^_c(k) = sum_e (i g_ce(k)) rho^_e(k)      (g = Im G^ / P, G odd),
//           inverse FFT along z, keep rows z < nz;
//   y_inv : inverse FFT along y, keep rows y < ny;
//   x_inv : complex-to-real inverse FFT along x, keep x < nx.
//
// The Nyquist column kx = M of the half spectrum travels in separate small
// arrays.  Layouts (complex):
//   after x_fwd : main [e][z][y][kx < M],  nyq [e][y][z]
//   after y_fwd : main [e][z][ky][kx],     nyq [e][ky][z]
//   after z     : main [c][z][ky][kx],     nyq [c][ky][z]
//   after y_inv : main [c][z][y][kx],      nyq [c][y][z]
// Every tile keeps its lines interleaved in shared memory (lanes across lines),
// so global accesses are contiguous rows of W complex values.
#include "stress_common.cuh"

namespace dds {

namespace {


// ---------------------------------------------------------------- x forward --
template <int M, int W, int NT, bool BF16, bool DIRECT>
__global__ void __launch_bounds__(NT) k_x_fwd(Shape sh, Collapse col, GroupList gl, const void *rho_v,
                                              float2 *out_main, float2 *out_nyq, const float2 *tw) {
  constexpr int LD = W + 1, PB = Plan<M>::r0;
  constexpr int OWN = (W * (M / 2) + NT - 1) / NT;
  extern __shared__ float2 smem[];
  float2 *buf = smem;
  const int tid = threadIdx.x;
  const long L = (long)sh.ny * sh.nz;
  const long N = L * sh.nx;
  const long l0 = (long)blockIdx.x * W;
  const int g = gl.g[blockIdx.y];
  const int b = blockIdx.z;                       // density set of the batch
  rho_v = BF16 ? (const void *)((const uint16_t *)rho_v + (long)b * sh.fin * L * sh.nx)
               : (const void *)((const float *)rho_v + (long)b * sh.fin * L * sh.nx);
  const int nxh = (sh.nx + 1) >> 1;
  const bool even = (sh.nx & 1) == 0;
  const float2 *twM = tw + tw_offset(M);
  const float2 *tw2 = tw + tw_offset(2 * M);

  // A group with one family (coefficient c) needs no combination: its line pairs are
  // copied straight into the transposed tile and the spectrum is scaled by c.
  // Otherwise every family of the group is read once and accumulated into all of
  // the group's fields (at most three) in registers.
  const int nd = col.nd[g];
  float2 acc[DIRECT ? 1 : 3][OWN];
  if constexpr (!DIRECT) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int i = 0; i < OWN; ++i) acc[d][i] = make_float2(0.f, 0.f);
    for (int q = 0; q < col.nf[g]; ++q) {
      const float c0 = col.coef[col.f0[g] + q][0], c1 = col.coef[col.f0[g] + q][1],
                  c2 = col.coef[col.f0[g] + q][2];
      const long fbase = (long)col.fam[col.f0[g] + q] * N + l0 * sh.nx;
      float2 v[OWN];
#pragma unroll
      for (int i = 0; i < OWN; ++i) {
        v[i] = make_float2(0.f, 0.f);
        const int p = tid + i * NT;
        if (p < W * nxh) {
          const int w = p / nxh, n = p - w * nxh;
          if (l0 + w < L) {
            const long o = fbase + (long)w * sh.nx + 2 * n;
            if (BF16) {
              const uint16_t *r = (const uint16_t *)rho_v;
              v[i].x = bf16_to_f32(r[o]);
              v[i].y = (2 * n + 1 < sh.nx) ? bf16_to_f32(r[o + 1]) : 0.f;
            } else {
              const float *r = (const float *)rho_v;
              if (even) {
                v[i] = *reinterpret_cast<const float2 *>(r + o);
              } else {
                v[i].x = r[o];
                v[i].y = (2 * n + 1 < sh.nx) ? r[o + 1] : 0.f;
              }
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < OWN; ++i) {
        acc[0][i].x = fmaf(c0, v[i].x, acc[0][i].x);
        acc[0][i].y = fmaf(c0, v[i].y, acc[0][i].y);
        acc[1][i].x = fmaf(c1, v[i].x, acc[1][i].x);
        acc[1][i].y = fmaf(c1, v[i].y, acc[1][i].y);
        acc[2][i].x = fmaf(c2, v[i].x, acc[2][i].x);
        acc[2][i].y = fmaf(c2, v[i].y, acc[2][i].y);
      }
    }
  }
  for (int d = 0; d < nd; ++d) {
    float scale_out = 1.0f;
    if constexpr (DIRECT) {
      scale_out = col.coef[col.f0[g]][0];
      const float *r = (const float *)rho_v + (long)col.fam[col.f0[g]] * N + l0 * sh.nx;
      for (int p = tid; p < W * nxh; p += NT) {
        const int w = p / nxh, n = p - w * nxh;
        if (l0 + w < L) cp_async8(&buf[tidx<LD, PB, W>(n, w)], r + (long)w * sh.nx + 2 * n);
        else buf[tidx<LD, PB, W>(n, w)] = make_float2(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int i = 0; i < OWN; ++i) {
        const int p = tid + i * NT;
        if (p < W * nxh) {
          const int w = p / nxh, n = p - w * nxh;
          if constexpr (!DIRECT) buf[tidx<LD, PB, W>(n, w)] = d == 0 ? acc[0][i] : (d == 1 ? acc[1][i] : acc[2][i]);
        }
      }
    }
    for (int p = W * nxh + tid; p < W * (M / 2); p += NT) {   // zero the tail of the non-zero half
      const int w = p % W, n = p / W;
      buf[tidx<LD, PB, W>(n, w)] = make_float2(0.f, 0.f);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_tile<M, W, LD, NT, false, true, false, PB>(buf, twM, tid);
    const int e = b * sh.fe + col.e0[g] + d;
    for (int p = tid; p < W * M; p += NT) {
      const int w = p / M, k = p - w * M;
      const long line = l0 + w;
      if (line >= L) continue;
      const float2 a = buf[tidx<LD, PB, W>(k, w)];
      const float2 c = buf[tidx<LD, PB, W>((M - k) & (M - 1), w)];
      const float2 E = make_float2(0.5f * (a.x + c.x), 0.5f * (a.y - c.y));
      const float2 O = make_float2(0.5f * (a.y + c.y), -0.5f * (a.x - c.x));
      const float2 wk = __ldg(tw2 + k);
      float2 X;
      X.x = scale_out * (E.x + (wk.x * O.x - wk.y * O.y));
      X.y = scale_out * (E.y + (wk.x * O.y + wk.y * O.x));
      out_main[((long)e * L + line) * M + k] = X;
      if (k == 0) {
        const int z = (int)(line / sh.ny), y = (int)(line - (long)z * sh.ny);
        out_nyq[((long)e * sh.ny + y) * sh.nz + z] =
            make_float2(scale_out * (E.x - O.x), scale_out * (E.y - O.y));   // W^M = -1
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- y passes -----
// Forward: rows y < ny in, all py rows out.  Inverse: all py rows in, y < ny out.
template <int PY, int W, int NT, bool INV>
__global__ void __launch_bounds__(NT) k_ypass(Shape sh, int nf, const float2 *in_main, const float2 *in_nyq,
                                              float2 *out_main, float2 *out_nyq, const float2 *tw) {
  constexpr int LD = W, PB = Plan<PY>::r0;
  extern __shared__ float2 smem[];
  float2 *buf = smem;
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
  if (tau < tiles_main) {
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
  if (tau < tiles_main) {            // rows of W complex, 16-byte aligned: 16-byte copies
    constexpr int H = W / 2;
    for (int p = tid; p < rows_in * H; p += NT) {
      const int n = p / H, c2 = p - n * H;
      cp_async16(&buf[tidx<LD, PB, W>(n, 2 * c2)], &in[n * rs + 2 * c2]);
    }
  } else {
    for (int p = tid; p < rows_in * W; p += NT) {
      const int n = p / W, w = p - n * W;
      if (w < ncols) cp_async8(&buf[tidx<LD, PB, W>(n, w)], &in[n * rs + w]);
      else buf[tidx<LD, PB, W>(n, w)] = make_float2(0.f, 0.f);
    }
  }
  if (!INV) {
    for (int p = rows_in * W + tid; p < (PY / 2) * W; p += NT) buf[tidx<LD, PB, W>(p / W, p % W)] = make_float2(0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_tile<PY, W, LD, NT, INV, !INV, INV, PB>(buf, tw + tw_offset(PY), tid);
  if (tau < tiles_main) {            // 16-byte stores of column pairs
    constexpr int H = W / 2;
    for (int p = tid; p < rows_out * H; p += NT) {
      const int n = p / H, c2 = p - n * H;
      *reinterpret_cast<float4 *>(&out[n * rs + 2 * c2]) =
          *reinterpret_cast<const float4 *>(&buf[tidx<LD, PB, W>(n, 2 * c2)]);
    }
  } else {
    for (int p = tid; p < rows_out * W; p += NT) {
      const int n = p / W, w = p - n * W;
      if (w < ncols) out[n * rs + w] = buf[tidx<LD, PB, W>(n, w)];
    }
  }
}


// ---------------------------------------------------------------- x inverse --
// stats != nullptr: also accumulate sum_x sigma^2 of every line into
// stats[(set * 6 + c) * nz + z] (the per-height sums of Eq. 20).
template <int M, int W, int NT>
__global__ void __launch_bounds__(NT) k_x_inv(Shape sh, const float2 *in_main, const float2 *in_nyq,
                                              float *sigma, const float2 *tw, double *stats) {
  constexpr int LD = W + 1, PB = Plan<M>::r0;
  extern __shared__ float2 smem[];
  float2 *buf = smem;
  float2 *xm = smem + tile_elems<M, LD, PB, W>();
  const int tid = threadIdx.x;
  const long L = 6L * sh.nb * sh.nz * sh.ny;
  const long l0 = (long)blockIdx.x * W;
  for (int p = tid; p < W * M; p += NT) {
    const int w = p / M, k = p - w * M;
    if (l0 + w < L) cp_async8(&buf[tidx<LD, PB, W>(k, w)], &in_main[(l0 + w) * M + k]);
    else buf[tidx<LD, PB, W>(k, w)] = make_float2(0.f, 0.f);
  }
  if (tid < W) {
    const long line = l0 + tid;
    float2 v = make_float2(0.f, 0.f);
    if (line < L) {
      const long cz = line / sh.ny;
      const int y = (int)(line - cz * sh.ny);
      const int c = (int)(cz / sh.nz), z = (int)(cz - (long)c * sh.nz);
      v = in_nyq[((long)c * sh.ny + y) * sh.nz + z];
    }
    xm[tid] = v;
  }
  cp_async_wait_all();
  __syncthreads();
  // Z[k] = (X[k] + conj X[M-k]) + i W^-k (X[k] - conj X[M-k]); pairs (k, M-k) per thread
  const float2 *tw2 = tw + tw_offset(2 * M);
  for (int p = tid; p < W * (M / 2 + 1); p += NT) {
    const int w = p % W, k = p / W;
    const float2 A = buf[tidx<LD, PB, W>(k, w)];
    const float2 Bm = (k == 0) ? xm[w] : buf[tidx<LD, PB, W>(M - k, w)];   // X[M-k]
    {
      const float2 E = make_float2(A.x + Bm.x, A.y - Bm.y);
      const float2 D = make_float2(A.x - Bm.x, A.y + Bm.y);
      const float2 wk = __ldg(tw2 + k);                                  // W^k; use conj
      const float2 O = make_float2(D.x * wk.x + D.y * wk.y, D.y * wk.x - D.x * wk.y);
      buf[tidx<LD, PB, W>(k, w)] = make_float2(E.x - O.y, E.y + O.x);
    }
    if (k > 0 && k < M / 2) {
      const float2 E = make_float2(Bm.x + A.x, Bm.y - A.y);
      const float2 D = make_float2(Bm.x - A.x, Bm.y + A.y);
      const float2 wk = __ldg(tw2 + (M - k));
      const float2 O = make_float2(D.x * wk.x + D.y * wk.y, D.y * wk.x - D.x * wk.y);
      buf[tidx<LD, PB, W>(M - k, w)] = make_float2(E.x - O.y, E.y + O.x);
    }
  }
  __syncthreads();
  fft_tile<M, W, LD, NT, true, false, true, PB>(buf, tw + tw_offset(M), tid);
  const int nxh = (sh.nx + 1) >> 1;
  const bool even = (sh.nx & 1) == 0;
  float *lsum = reinterpret_cast<float *>(xm + W);     // per-line sums of squares (stats only)
  if (stats != nullptr && tid < W) lsum[tid] = 0.f;
  if (stats != nullptr) __syncthreads();
  for (int p = tid; p < W * nxh; p += NT) {
    const int w = p / nxh, n = p - w * nxh;
    const long line = l0 + w;
    if (line >= L) continue;
    const float2 v = buf[tidx<LD, PB, W>(n, w)];
    float *dst = sigma + line * sh.nx + 2 * n;
    if (even) {
      *reinterpret_cast<float2 *>(dst) = v;
    } else {
      dst[0] = v.x;
      if (2 * n + 1 < sh.nx) dst[1] = v.y;
    }
    if (stats != nullptr) atomicAdd(&lsum[w], v.x * v.x + ((2 * n + 1 < sh.nx) ? v.y * v.y : 0.f));
  }
  if (stats != nullptr) {
    __syncthreads();
    if (tid < W && l0 + tid < L) {
      const long line = l0 + tid;
      atomicAdd(&stats[line / sh.ny], (double)lsum[tid]);   // line / ny = (set * 6 + c) * nz + z
    }
  }
}

// s = sqrt(sum / (nx ny)) for every (set, component, height).
__global__ void k_stats_finish(const double *sums, long n, double inv_plane, float *s_out) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) s_out[i] = (float)sqrt(sums[i] * inv_plane);
}

// ------------------------------------------------------------ dispatch ------

template <int M, bool BF16, bool DIRECT>
cudaError_t launch_x_fwd_kind(const Shape &sh, const Collapse &col, const GroupList &gl, const void *rho,
                              float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  constexpr int W = XTile<M>::W, T = XTile<M>::NT;
  const size_t smem = sizeof(float2) * tile_elems<M, W + 1, Plan<M>::r0, W>();
  const long L = (long)sh.ny * sh.nz;
  dim3 grid((unsigned)((L + W - 1) / W), gl.n, sh.nb);
  cudaError_t err = prep(k_x_fwd<M, W, T, BF16, DIRECT>, smem);
  if (err != cudaSuccess) return err;
  k_x_fwd<M, W, T, BF16, DIRECT><<<grid, T, smem, s>>>(sh, col, gl, rho, om, on, tw);
  return cudaGetLastError();
}

// Groups with one family read that family straight into the tile (single-family
// kernel); the others accumulate their families in registers.
template <int M>
cudaError_t launch_x_fwd(const Shape &sh, const Collapse &col, const void *rho, bool bf16, float2 *om,
                         float2 *on, const float2 *tw, cudaStream_t s) {
  GroupList direct{}, accum{};
  for (int g = 0; g < col.ngroups; ++g) {
    const bool d = !bf16 && (sh.nx % 2 == 0) && col.nf[g] == 1 && col.nd[g] == 1;
    if (col.nd[g] == 0) continue;
    GroupList &gl = d ? direct : accum;
    gl.g[gl.n++] = g;
  }
  cudaError_t err = cudaSuccess;
  if (direct.n > 0) err = launch_x_fwd_kind<M, false, true>(sh, col, direct, rho, om, on, tw, s);
  if (err == cudaSuccess && accum.n > 0) {
    err = bf16 ? launch_x_fwd_kind<M, true, false>(sh, col, accum, rho, om, on, tw, s)
               : launch_x_fwd_kind<M, false, false>(sh, col, accum, rho, om, on, tw, s);
  }
  return err;
}

template <int PY, bool INV>
cudaError_t launch_y(const Shape &sh, int nf, const float2 *im, const float2 *in, float2 *om, float2 *on,
                     const float2 *tw, cudaStream_t s) {
  constexpr int W = YTile<PY>::W, T = YTile<PY>::NT;
  const size_t smem = sizeof(float2) * tile_elems<PY, W, Plan<PY>::r0, W>();
  const long tiles = (long)nf * sh.nz * (sh.M / W) + (long)nf * ((sh.nz + W - 1) / W);
  cudaError_t err = prep(k_ypass<PY, W, T, INV>, smem);
  if (err != cudaSuccess) return err;
  k_ypass<PY, W, T, INV><<<(unsigned)tiles, T, smem, s>>>(sh, nf, im, in, om, on, tw);
  return cudaGetLastError();
}


template <int M>
cudaError_t launch_x_inv(const Shape &sh, const float2 *im, const float2 *in, float *sigma, const float2 *tw,
                         cudaStream_t s, double *stats) {
  constexpr int W = XTile<M>::W, T = XTile<M>::NT;
  const size_t smem = sizeof(float2) * (tile_elems<M, W + 1, Plan<M>::r0, W>() + W) + sizeof(float) * W;
  const long L = 6L * sh.nb * sh.nz * sh.ny;
  cudaError_t err = prep(k_x_inv<M, W, T>, smem);
  if (err != cudaSuccess) return err;
  k_x_inv<M, W, T><<<(unsigned)((L + W - 1) / W), T, smem, s>>>(sh, im, in, sigma, tw, stats);
  return cudaGetLastError();
}

cudaError_t dispatch_x_fwd(const Shape &sh, const Collapse &col, const void *rho, bool bf16, float2 *om,
                           float2 *on, const float2 *tw, cudaStream_t s) {
  switch (sh.M) {
    case 16: return launch_x_fwd<16>(sh, col, rho, bf16, om, on, tw, s);
    case 32: return launch_x_fwd<32>(sh, col, rho, bf16, om, on, tw, s);
    case 64: return launch_x_fwd<64>(sh, col, rho, bf16, om, on, tw, s);
    case 128: return launch_x_fwd<128>(sh, col, rho, bf16, om, on, tw, s);
    case 256: return launch_x_fwd<256>(sh, col, rho, bf16, om, on, tw, s);
    case 512: return launch_x_fwd<512>(sh, col, rho, bf16, om, on, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool INV>
cudaError_t dispatch_y(const Shape &sh, int nf, const float2 *im, const float2 *in, float2 *om, float2 *on,
                       const float2 *tw, cudaStream_t s) {
  switch (sh.py) {
    case 32: return launch_y<32, INV>(sh, nf, im, in, om, on, tw, s);
    case 64: return launch_y<64, INV>(sh, nf, im, in, om, on, tw, s);
    case 128: return launch_y<128, INV>(sh, nf, im, in, om, on, tw, s);
    case 256: return launch_y<256, INV>(sh, nf, im, in, om, on, tw, s);
    case 512: return launch_y<512, INV>(sh, nf, im, in, om, on, tw, s);
    case 1024: return launch_y<1024, INV>(sh, nf, im, in, om, on, tw, s);
    default: return cudaErrorInvalidValue;
  }
}


cudaError_t dispatch_x_inv(const Shape &sh, const float2 *im, const float2 *in, float *sigma, const float2 *tw,
                           cudaStream_t s, double *stats = nullptr) {
  switch (sh.M) {
    case 16: return launch_x_inv<16>(sh, im, in, sigma, tw, s, stats);
    case 32: return launch_x_inv<32>(sh, im, in, sigma, tw, s, stats);
    case 64: return launch_x_inv<64>(sh, im, in, sigma, tw, s, stats);
    case 128: return launch_x_inv<128>(sh, im, in, sigma, tw, s, stats);
    case 256: return launch_x_inv<256>(sh, im, in, sigma, tw, s, stats);
    case 512: return launch_x_inv<512>(sh, im, in, sigma, tw, s, stats);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int stress_launch_count(const Shape &sh, const Collapse &col) {
  int direct = 0, accum = 0;
  for (int g = 0; g < col.ngroups; ++g) {
    if (col.nd[g] == 0) continue;
    if ((sh.nx % 2 == 0) && col.nf[g] == 1 && col.nd[g] == 1) direct = 1;
    else accum = 1;
  }
  return 4 + direct + accum;   // float32 densities; bfloat16 ones use the accumulating kernel
}

int enqueue_stress(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, cudaStream_t s, int nb,
                   double *stats, float *s_out) {
  Shape sh = ctx->shape;
  sh.nb = nb;
  const float2 *tw = ctx->tw.f32;
  cudaEvent_t *ev = nullptr;
  cudaError_t err = cudaSuccess;
  if (ctx->profiling) {
    const size_t need = 6 * (size_t)(ctx->prof_steps + 1);
    while (err == cudaSuccess && ctx->prof_events.size() < need) {
      cudaEvent_t e;
      err = cudaEventCreate(&e);
      if (err == cudaSuccess) ctx->prof_events.push_back(e);
    }
    if (err == cudaSuccess) {
      ev = &ctx->prof_events[6 * (size_t)ctx->prof_steps];
      ctx->prof_steps++;
      err = cudaEventRecord(ev[0], s);
    }
  }
  auto mark = [&](int i) {
    if (ev && err == cudaSuccess) err = cudaEventRecord(ev[i], s);
  };
  if (err == cudaSuccess) err = dispatch_x_fwd(sh, ctx->col, rho, rho_dtype == DDS_BF16, ctx->bufA, ctx->nyqA, tw, s);
  mark(1);
  if (err == cudaSuccess) err = dispatch_y<false>(sh, nb * sh.fe, ctx->bufA, ctx->nyqA, ctx->bufB, ctx->nyqB, tw, s);
  mark(2);
  if (err == cudaSuccess)
    err = dispatch_z(sh, ctx->bufB, ctx->nyqB, ctx->kspec, ctx->kscale, ctx->bufA, ctx->nyqA, tw, s);
  mark(3);
  if (err == cudaSuccess) err = dispatch_y<true>(sh, 6 * nb, ctx->bufA, ctx->nyqA, ctx->bufB, ctx->nyqB, tw, s);
  mark(4);
  if (err == cudaSuccess && stats != nullptr) err = cudaMemsetAsync(stats, 0, sizeof(double) * 6 * nb * sh.nz, s);
  if (err == cudaSuccess) err = dispatch_x_inv(sh, ctx->bufB, ctx->nyqB, sigma, tw, s, stats);
  if (err == cudaSuccess && stats != nullptr) {
    const long n = 6L * nb * sh.nz;
    k_stats_finish<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(stats, n, 1.0 / ((double)sh.nx * sh.ny), s_out);
    err = cudaGetLastError();
  }
  mark(5);
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress: kernel launch failed: %s", cudaGetErrorString(err));
  return DDS_OK;
}

// The five passes on caller-provided work buffers (used by dds_stress_noalloc).
int enqueue_stress_buffers(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, float2 *bufA, float2 *bufB,
                           float2 *nyqA, float2 *nyqB, cudaStream_t s) {
  const Shape &sh = ctx->shape;
  const float2 *tw = ctx->tw.f32;
  cudaError_t err = dispatch_x_fwd(sh, ctx->col, rho, rho_dtype == DDS_BF16, bufA, nyqA, tw, s);
  if (err == cudaSuccess) err = dispatch_y<false>(sh, sh.fe, bufA, nyqA, bufB, nyqB, tw, s);
  if (err == cudaSuccess) err = dispatch_z(sh, bufB, nyqB, ctx->kspec, ctx->kscale, bufA, nyqA, tw, s);
  if (err == cudaSuccess) err = dispatch_y<true>(sh, 6, bufA, nyqA, bufB, nyqB, tw, s);
  if (err == cudaSuccess) err = dispatch_x_inv(sh, bufB, nyqB, sigma, tw, s);
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress: kernel launch failed: %s", cudaGetErrorString(err));
  return DDS_OK;
}

}  // namespace dds
