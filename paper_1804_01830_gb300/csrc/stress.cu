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
// (With DDS_OPT_YX_FUSED the last two run as one cluster pass, yxpass.cuh.)
//
// The Nyquist column kx = M of the half spectrum travels in separate small
// arrays.  Layouts (complex):
//   after x_fwd : main [e][z][y][kx < M],  nyq [e][y][z]
//   after y_fwd : main [e][z][ky][kx],     nyq [e][ky][z]
//   after z     : main [c][z][ky][kx],     nyq [c][ky][z]
//   after y_inv : main [c][z][y][kx],      nyq [c][y][z]
// The y passes keep W columns interleaved in shared memory (lanes across
// columns), so global accesses are contiguous rows of W complex values; the x
// passes (xpass.cuh) keep each line in the registers of a few threads.
#include <algorithm>
#include <mutex>

#include "stress_common.cuh"
#include "xpass.cuh"
#include "ypass.cuh"
#include "yxpass.cuh"

namespace dds {

// Set by a bounded device wait that gave up (bulk.cuh); read by dds_device_status.
__device__ int g_wait_status;

namespace {

constexpr int MAX_DEV = 64;

// Per device: SM count and the address of g_wait_status (looked up once).
struct DevInfo {
  int sms = 0;
  int *status = nullptr;
};

cudaError_t dev_info(DevInfo *out) {
  static std::mutex mu;
  static DevInfo info[MAX_DEV];
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!info[dev].status) {
    err = cudaDeviceGetAttribute(&info[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    void *p = nullptr;
    if (err == cudaSuccess) err = cudaGetSymbolAddress(&p, g_wait_status);
    if (err != cudaSuccess) return err;
    info[dev].status = static_cast<int *>(p);
  }
  *out = info[dev];
  return cudaSuccess;
}

// Persistent grid: as many CTAs as fit on the device at once, at most one per tile.
template <typename K>
cudaError_t persistent_grid(K kernel, int threads, size_t smem, long tiles, const DevInfo &di, unsigned *grid) {
  int per_sm = 0;
  const cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (err != cudaSuccess) return err;
  const long g = std::max(1L, std::min(tiles, (long)std::max(per_sm, 1) * di.sms));
  *grid = (unsigned)g;
  return cudaSuccess;
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


// s = sqrt(sum / (nx ny)) for every (set, component, height).
__global__ void k_stats_finish(const double *sums, long n, double inv_plane, float *s_out) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) s_out[i] = (float)sqrt(sums[i] * inv_plane);
}

// ------------------------------------------------------------ dispatch ------

template <int M, bool BF16, bool DIRECT>
cudaError_t launch_x_fwd_kind(const Shape &sh, const Collapse &col, const GroupList &gl, const void *rho,
                              float2 *om, float2 *on, const float2 *tw, cudaStream_t s) {
  constexpr int LPB = xr::THREADS / (xr::FwdCfg<M>::R1 / 2);
  const long L = (long)sh.ny * sh.nz;
  dim3 grid((unsigned)((L + LPB - 1) / LPB), gl.n, sh.nb);
  cudaError_t err = prep(xr::k_x_fwd_reg<M, BF16, DIRECT>, 0);
  if (err != cudaSuccess) return err;
  xr::k_x_fwd_reg<M, BF16, DIRECT><<<grid, xr::THREADS, 0, s>>>(sh, col, gl, rho, om, on, tw);
  return cudaGetLastError();
}

// Groups with one family and one field transform that family directly; the others
// sum their families into each field first.
template <int M>
cudaError_t launch_x_fwd(const Shape &sh, const Collapse &col, const void *rho, bool bf16, float2 *om,
                         float2 *on, const float2 *tw, cudaStream_t s) {
  GroupList direct{}, accum{};
  for (int g = 0; g < col.ngroups; ++g) {
    const bool d = col.nf[g] == 1 && col.nd[g] == 1;
    if (col.nd[g] == 0) continue;
    GroupList &gl = d ? direct : accum;
    gl.g[gl.n++] = g;
  }
  cudaError_t err = cudaSuccess;
  if (direct.n > 0) {
    err = bf16 ? launch_x_fwd_kind<M, true, true>(sh, col, direct, rho, om, on, tw, s)
               : launch_x_fwd_kind<M, false, true>(sh, col, direct, rho, om, on, tw, s);
  }
  if (err == cudaSuccess && accum.n > 0) {
    err = bf16 ? launch_x_fwd_kind<M, true, false>(sh, col, accum, rho, om, on, tw, s)
               : launch_x_fwd_kind<M, false, false>(sh, col, accum, rho, om, on, tw, s);
  }
  return err;
}

template <int PY, bool INV>
cudaError_t launch_y(const Shape &sh, int nf, const float2 *im, const float2 *in, float2 *om, float2 *on,
                     const float2 *tw, cudaStream_t s) {
  constexpr int W = YTile<PY, INV>::W, T = YTile<PY, INV>::NT;
  const long tiles = (long)nf * sh.nz * (sh.M / W) + (long)nf * ((sh.nz + W - 1) / W);
  if (sh.py == sh.ny) {                   // periodic in y: no zero padding (py <= 512)
    if constexpr (PY <= 512) {
      const size_t smem = sizeof(float2) * yr::y_smem_all<PY, W, INV, true>();
      cudaError_t err = prep(yr::k_ypass_st<PY, W, T, INV, true>, smem);
      if (err != cudaSuccess) return err;
      yr::k_ypass_st<PY, W, T, INV, true><<<(unsigned)tiles, T, smem, s>>>(sh, nf, im, in, om, on, tw);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (INV && PY >= 1024) {
    // 1024-row inverse: the shared-memory Stockham tile with 16-byte row stores (radial
    // disk 512x512x16: 0.137 ms, against 0.152 for the register stages on 4-column
    // tiles and 0.146 on 8-column tiles of 256 threads)
    const size_t smem = sizeof(float2) * tile_elems<PY, W, Plan<PY>::r0, W>();
    cudaError_t err = prep(k_ypass<PY, W, T, INV>, smem);
    if (err != cudaSuccess) return err;
    k_ypass<PY, W, T, INV><<<(unsigned)tiles, T, smem, s>>>(sh, nf, im, in, om, on, tw);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(float2) * yr::y_smem_all<PY, W, INV, false>();
  cudaError_t err = prep(yr::k_ypass_st<PY, W, T, INV>, smem);
  if (err != cudaSuccess) return err;
  yr::k_ypass_st<PY, W, T, INV><<<(unsigned)tiles, T, smem, s>>>(sh, nf, im, in, om, on, tw);
  return cudaGetLastError();
}


// Persistent kernel with bulk-copied tiles for every line length (GaN layer 256x256x128:
// 185 -> 155 us against one CTA per tile; with its twiddles held in registers across
// tiles, 512 points too: radial disk 512x512x16 0.082 -> 0.078 ms against the one-tile
// register kernel it replaced).
template <int M>
cudaError_t launch_x_inv(const Shape &sh, const float2 *im, const float2 *in, float *sigma, const float2 *tw,
                         cudaStream_t s, double *stats) {
  using C = xr::InvTma<M>;
  const long L = 6L * sh.nb * sh.nz * sh.ny;
  DevInfo di;
  cudaError_t err = dev_info(&di);
  if (err == cudaSuccess) err = prep(xr::k_x_inv_tma<M>, C::SMEM);
  unsigned grid = 0;
  if (err == cudaSuccess)
    err = persistent_grid(xr::k_x_inv_tma<M>, xr::THREADS, C::SMEM, (L + C::LPB - 1) / C::LPB, di, &grid);
  if (err != cudaSuccess) return err;
  xr::k_x_inv_tma<M><<<grid, xr::THREADS, C::SMEM, s>>>(sh, im, in, sigma, tw, stats, di.status);
  return cudaGetLastError();
}

// Fused inverse y + x pass (yxpass.cuh): one cluster of Cfg::CL CTAs per output plane.
template <int PY, int M>
cudaError_t launch_yx_inv(const Shape &sh, const float2 *im, const float2 *in, float *sigma, const float2 *tw,
                          cudaStream_t s, double *stats) {
  using C = yx::Cfg<PY, M>;
  auto kernel = yx::k_yx_inv<PY, M>;
  const size_t smem = sizeof(float2) * C::SMEM_F2;
  cudaError_t err = prep(kernel, smem);
  if (err == cudaSuccess && C::CL > 8)
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(6L * sh.nb * sh.nz * C::CL), 1, 1);
  cfg.blockDim = dim3(C::NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C::CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  err = cudaLaunchKernelEx(&cfg, kernel, sh, im, in, sigma, tw, stats);
  return err != cudaSuccess ? err : cudaGetLastError();
}

// How many clusters of the fused pass the device holds at once (0: none fits).
template <int PY, int M>
int yx_clusters_resident() {
  using C = yx::Cfg<PY, M>;
  auto kernel = yx::k_yx_inv<PY, M>;
  const size_t smem = sizeof(float2) * C::SMEM_F2;
  if (prep(kernel, smem) != cudaSuccess) return 0;
  if (C::CL > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C::CL, 1, 1);
  cfg.blockDim = dim3(C::NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C::CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t dispatch_yx_inv(const Shape &sh, const float2 *im, const float2 *in, float *sigma, const float2 *tw,
                            cudaStream_t s, double *stats) {
  if (sh.py == 256 && sh.M == 128) return launch_yx_inv<256, 128>(sh, im, in, sigma, tw, s, stats);
  if (sh.py == 512 && sh.M == 128) return launch_yx_inv<512, 128>(sh, im, in, sigma, tw, s, stats);
  if (sh.py == 256 && sh.M == 256) return launch_yx_inv<256, 256>(sh, im, in, sigma, tw, s, stats);
  if (sh.py == 512 && sh.M == 256) return launch_yx_inv<512, 256>(sh, im, in, sigma, tw, s, stats);
  return cudaErrorInvalidValue;
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

int yx_inv_cluster(const Shape &sh) {
  if (sh.py == sh.ny || 2 * sh.ny > sh.py) return 0;       // the fused pass keeps rows y < py / 2
  int n = 0, cl = 0;
  if (sh.py == 256 && sh.M == 128) { n = yx_clusters_resident<256, 128>(); cl = yx::Cfg<256, 128>::CL; }
  else if (sh.py == 512 && sh.M == 128) { n = yx_clusters_resident<512, 128>(); cl = yx::Cfg<512, 128>::CL; }
  else if (sh.py == 256 && sh.M == 256) { n = yx_clusters_resident<256, 256>(); cl = yx::Cfg<256, 256>::CL; }
  else if (sh.py == 512 && sh.M == 256) { n = yx_clusters_resident<512, 256>(); cl = yx::Cfg<512, 256>::CL; }
  return n > 0 ? cl : 0;
}

int stress_launch_count(const Shape &sh, const Collapse &col) {
  int direct = 0, accum = 0;
  for (int g = 0; g < col.ngroups; ++g) {
    if (col.nd[g] == 0) continue;
    if (col.nf[g] == 1 && col.nd[g] == 1) direct = 1;
    else accum = 1;
  }
  return (sh.yxf > 0 ? 3 : 4) + direct + accum;
}

int enqueue_stress(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, cudaStream_t s, int nb,
                   double *stats, float *s_out, const Collapse *sub, int sub_fin) {
  Shape sh = ctx->shape;
  sh.nb = nb;
  if (sub) sh.fin = sub_fin;
  const Collapse &col = sub ? *sub : ctx->col;
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
  if (err == cudaSuccess) err = dispatch_x_fwd(sh, col, rho, rho_dtype == DDS_BF16, ctx->bufA, ctx->nyqA, tw, s);
  mark(1);
  if (err == cudaSuccess) err = dispatch_y<false>(sh, nb * sh.fe, ctx->bufA, ctx->nyqA, ctx->bufB, ctx->nyqB, tw, s);
  mark(2);
  if (err == cudaSuccess)
    err = dispatch_z(sh, ctx->bufB, ctx->nyqB, ctx->kspec, ctx->kscale, ctx->bufA, ctx->nyqA, tw, s);
  mark(3);
  if (err == cudaSuccess && sh.yxf == 0)
    err = dispatch_y<true>(sh, 6 * nb, ctx->bufA, ctx->nyqA, ctx->bufB, ctx->nyqB, tw, s);
  mark(4);
  if (err == cudaSuccess && stats != nullptr) err = cudaMemsetAsync(stats, 0, sizeof(double) * 6 * nb * sh.nz, s);
  if (err == cudaSuccess)
    err = sh.yxf > 0 ? dispatch_yx_inv(sh, ctx->bufA, ctx->nyqA, sigma, tw, s, stats)
                     : dispatch_x_inv(sh, ctx->bufB, ctx->nyqB, sigma, tw, s, stats);
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
  if (sh.yxf > 0) {
    if (err == cudaSuccess) err = dispatch_yx_inv(sh, bufA, nyqA, sigma, tw, s, nullptr);
  } else {
    if (err == cudaSuccess) err = dispatch_y<true>(sh, 6, bufA, nyqA, bufB, nyqB, tw, s);
    if (err == cudaSuccess) err = dispatch_x_inv(sh, bufB, nyqB, sigma, tw, s);
  }
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress: kernel launch failed: %s", cudaGetErrorString(err));
  return DDS_OK;
}

}  // namespace dds

extern "C" int dds_device_status(int cuda_device, int reset) {
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return DDS_ERR_CUDA;
  if (prev != cuda_device && cudaSetDevice(cuda_device) != cudaSuccess) return DDS_ERR_INVALID_ARG;
  int v = 0;
  cudaError_t err = cudaMemcpyFromSymbol(&v, dds::g_wait_status, sizeof(int));
  if (err == cudaSuccess && reset && v != 0) {
    const int zero = 0;
    err = cudaMemcpyToSymbol(dds::g_wait_status, &zero, sizeof(int));
  }
  if (prev != cuda_device) cudaSetDevice(prev);
  if (err != cudaSuccess) return DDS_ERR_CUDA;
  return v == 0 ? DDS_OK : DDS_ERR_TIMEOUT;
}
