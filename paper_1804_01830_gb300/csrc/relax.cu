// Relaxation of the dislocation stress to free top and bottom surfaces
// (Sec. 5, Eqs. 14-18), FP32.
//
// The displacement u (three components, [c][z][y][x], metres) relaxes by
// explicit Euler steps of Eq. 17,
//     u <- u + dt (A grad div u - B rot rot u + f),   f_a = sum_b d sigma^dis_ab / db (Eq. 15),
// with u periodic in x and y (Eq. 16a) and the traction-free surface conditions
// of Eq. 16c imposed through one ghost layer below the first and above the last
// film layer (Eq. 18b and its counterparts).  Ghost values are functions of the
// film values of the same step, so the step kernel evaluates them where it needs
// them instead of storing them.  Differences: second differences, 4-point mixed
// derivatives, central first derivatives; d sigma^dis / dz one-sided (second
// order) on the surface layers.  dt = min(h)^2 / (5A - 3B).
//
// The coefficients are folded with dt on the host (double, then rounded once),
// so every quantity the kernels touch is in units of u.  One step reads u and
// dt f and writes u: 36 bytes per cell from HBM.
#include <algorithm>

#include "dds_internal.h"

namespace dds {
namespace {

struct RelaxCoef {
  int nx, ny, nz;
  // dt-scaled operator: u_a += sum_b lap[a][b] (u_a[+b] - 2 u_a + u_a[-b])
  //                          + sum_{b != a} mix[a][b] (4-point cross of u_b in a, b)
  float lap[3][3];
  float mix[3][3];
  // ghost layers: first derivatives 1/(2 h) and the factors of Eq. 18b
  float inv2h[3];
  float two_dz;      // 2 dz
  float zfac;        // 2 dz / (1 - nu)
  float nu;
  // Hooke's law for sigma(u): lambda, mu
  float lam, mu;
  // phi of Eq. 16c from sigma^dis: -(1 + nu) / E and -(1 + nu)(1 - 2 nu) / E
  float phi_shear, phi_normal;
  // dt for f
  float dt;
};

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ long cidx(const RelaxCoef &r, int c, int k, int j, int i) {
  return (((long)c * r.nz + k) * r.ny + j) * r.nx + i;
}

// u_c at film cell (i, j, k) with i, j periodic and k in [-1, nz]: the ghost layers of
// Eq. 18b below (k = -1) and above (k = nz).  phi: [surface][3][ny][nx].
__device__ __forceinline__ float uext(const RelaxCoef &r, const float *__restrict__ u, const float *__restrict__ phi, int c,
                      int i, int j, int k) {
  i = wrap(i, r.nx);
  j = wrap(j, r.ny);
  if (k >= 0 && k < r.nz) return __ldg(u + cidx(r, c, k, j, i));
  const bool top = k >= r.nz;
  const int ks = top ? r.nz - 1 : 0;          // surface layer (centre of the condition)
  const int kn = top ? r.nz - 2 : 1;          // its inner neighbour
  const float sgn = top ? 1.f : -1.f;         // ghost = inner + sgn * 2dz * (condition terms)
  const float *ph = phi + (long)(top ? 3 : 0) * r.ny * r.nx + (long)j * r.nx + i;
  const long plane = (long)r.ny * r.nx;
  const float inner = __ldg(u + cidx(r, c, kn, j, i));
  if (c == 0) {   // (du_x/dz + du_z/dx) / 2 = phi_xz
    const float dxuz = (__ldg(u + cidx(r, 2, ks, j, wrap(i + 1, r.nx))) - __ldg(u + cidx(r, 2, ks, j, wrap(i - 1, r.nx)))) * r.inv2h[0];
    return inner + sgn * r.two_dz * (2.f * __ldg(ph) - dxuz);
  }
  if (c == 1) {   // (du_y/dz + du_z/dy) / 2 = phi_yz
    const float dyuz = (__ldg(u + cidx(r, 2, ks, wrap(j + 1, r.ny), i)) - __ldg(u + cidx(r, 2, ks, wrap(j - 1, r.ny), i))) * r.inv2h[1];
    return inner + sgn * r.two_dz * (2.f * __ldg(ph + plane) - dyuz);
  }
  // (1 - nu) du_z/dz + nu (du_x/dx + du_y/dy) = phi_zz
  const float dxux = (__ldg(u + cidx(r, 0, ks, j, wrap(i + 1, r.nx))) - __ldg(u + cidx(r, 0, ks, j, wrap(i - 1, r.nx)))) * r.inv2h[0];
  const float dyuy = (__ldg(u + cidx(r, 1, ks, wrap(j + 1, r.ny), i)) - __ldg(u + cidx(r, 1, ks, wrap(j - 1, r.ny), i))) * r.inv2h[1];
  return inner + sgn * r.zfac * (__ldg(ph + 2 * plane) - r.nu * (dxux + dyuy));
}

// dt f (Eq. 15) at every film cell and phi (Eq. 16c) on the two surface layers.
__global__ void k_relax_prep(RelaxCoef r, const float *__restrict__ sig, float *__restrict__ gf,
                             float *__restrict__ phi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= r.nx || j >= r.ny) return;
  // component index of the pair (a, b): xx yy zz xy xz yz
  constexpr int PAIR[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  const int ip = wrap(i + 1, r.nx), im = wrap(i - 1, r.nx), jp = wrap(j + 1, r.ny), jm = wrap(j - 1, r.ny);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int cx = PAIR[a][0], cy = PAIR[a][1], cz = PAIR[a][2];
    float d = (__ldg(sig + cidx(r, cx, k, j, ip)) - __ldg(sig + cidx(r, cx, k, j, im))) * r.inv2h[0] +
              (__ldg(sig + cidx(r, cy, k, jp, i)) - __ldg(sig + cidx(r, cy, k, jm, i))) * r.inv2h[1];
    float dz;
    if (r.nz >= 3) {
      if (k == 0)
        dz = (-3.f * __ldg(sig + cidx(r, cz, 0, j, i)) + 4.f * __ldg(sig + cidx(r, cz, 1, j, i)) - __ldg(sig + cidx(r, cz, 2, j, i))) * r.inv2h[2];
      else if (k == r.nz - 1)
        dz = (3.f * __ldg(sig + cidx(r, cz, k, j, i)) - 4.f * __ldg(sig + cidx(r, cz, k - 1, j, i)) + __ldg(sig + cidx(r, cz, k - 2, j, i))) * r.inv2h[2];
      else
        dz = (__ldg(sig + cidx(r, cz, k + 1, j, i)) - __ldg(sig + cidx(r, cz, k - 1, j, i))) * r.inv2h[2];
    } else {
      dz = (__ldg(sig + cidx(r, cz, 1, j, i)) - __ldg(sig + cidx(r, cz, 0, j, i))) * (2.f * r.inv2h[2]);
    }
    gf[cidx(r, a, k, j, i)] = r.dt * (d + dz);
  }
  if (k == 0 || k == r.nz - 1) {
    const long plane = (long)r.ny * r.nx;
    float *ph = phi + (long)(k == 0 ? 0 : 3) * plane + (long)j * r.nx + i;
    ph[0] = r.phi_shear * __ldg(sig + cidx(r, 4, k, j, i));
    ph[plane] = r.phi_shear * __ldg(sig + cidx(r, 5, k, j, i));
    ph[2 * plane] = r.phi_normal * __ldg(sig + cidx(r, 2, k, j, i));
  }
}

// One explicit step, u_out = u_in + dt (navier(u_in) + f), on a tile of TX x TY columns
// marching up a chunk of KZ layers: three planes (below, at, above the layer) of all
// three components, with a one-cell halo, rotate through shared memory, so every value
// of u is read from global memory about once per step (halo cells from L2).  The plane
// two layers ahead is loaded into registers while the current layer is updated; ghost
// planes are evaluated (uext) as they are loaded.
// (32-layer chunks: each chunk restarts its march with three plane loads; GaN grid
// 0.0986 -> 0.0948 ms per step against 16-layer chunks; 32x16 and 64x8 tiles were slower)
constexpr int TX = 32, TY = 8, KZ = 32, HX = TX + 2, HY = TY + 2;
constexpr int NT_TILE = TX * TY, PLANE = 3 * HY * HX, NQ = (PLANE + NT_TILE - 1) / NT_TILE;

__device__ __forceinline__ int mod(int i, int n) { return ((i % n) + n) % n; }

// The values of one plane (layer k, or a ghost layer) this thread stages: entry q of
// the [component][y][x] halo tile for q = threadIdx.x + NT_TILE * e, whose film
// element is u[base[e] + k * plane] (32-bit offsets: 3 nx ny nz < 2^31 for every grid
// the library accepts).
__device__ __forceinline__ void fetch_plane(const RelaxCoef &r, const float *__restrict__ u,
                                            const float *__restrict__ phi, const int (&base)[NQ], const int (&comp)[NQ],
                                            int k, int plane, float (&v)[NQ]) {
  if (k >= 0 && k < r.nz) {
    const int kp = k * plane;
#pragma unroll
    for (int e = 0; e < NQ; ++e)
      if (comp[e] >= 0) v[e] = __ldg(u + base[e] + kp);
  } else {
#pragma unroll
    for (int e = 0; e < NQ; ++e) {
      if (comp[e] < 0) continue;
      const int col = base[e] - comp[e] * r.nz * plane;
      const int j = col / r.nx, i = col - j * r.nx;
      v[e] = uext(r, u, phi, comp[e], i, j, k);
    }
  }
}

__device__ __forceinline__ void store_plane(const float (&v)[NQ], const int (&comp)[NQ], float *pl) {
#pragma unroll
  for (int e = 0; e < NQ; ++e)
    if (comp[e] >= 0) pl[threadIdx.x + NT_TILE * e] = v[e];
}

__global__ void __launch_bounds__(NT_TILE) k_relax_tile(RelaxCoef r, const float *__restrict__ u,
                                                        const float *__restrict__ gf, const float *__restrict__ phi,
                                                        float *__restrict__ u_out) {
  __shared__ float pl[3][3][HY][HX];          // [slot][component][y][x]
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kb = blockIdx.z * KZ, ke = min(kb + KZ, r.nz);
  const int i = i0 + tx, j = j0 + ty;
  const bool live = i < r.nx && j < r.ny;
  const int plane = r.ny * r.nx, cstride = r.nz * plane;
  const int own = j * r.nx + i;
  // the halo entries this thread stages, fixed for the whole march
  int base[NQ], comp[NQ];
#pragma unroll
  for (int e = 0; e < NQ; ++e) {
    const int q = threadIdx.x + NT_TILE * e;
    comp[e] = -1;
    base[e] = 0;
    if (q < PLANE) {
      const int c = q / (HY * HX), rem = q - c * HY * HX;
      const int hy = rem / HX, hx = rem - hy * HX;
      comp[e] = c;
      base[e] = c * cstride + mod(j0 + hy - 1, r.ny) * r.nx + mod(i0 + hx - 1, r.nx);
    }
  }
  int sb = 0, sm = 1, sa = 2;                 // slots of the layers below, at, above
  float v[NQ];
  fetch_plane(r, u, phi, base, comp, kb - 1, plane, v);
  store_plane(v, comp, &pl[sb][0][0][0]);
  fetch_plane(r, u, phi, base, comp, kb, plane, v);
  store_plane(v, comp, &pl[sm][0][0][0]);
  fetch_plane(r, u, phi, base, comp, kb + 1, plane, v);
  store_plane(v, comp, &pl[sa][0][0][0]);
  __syncthreads();
  const int x = tx + 1, y = ty + 1;
  for (int k = kb; k < ke; ++k) {
    const bool more = k + 1 < ke;
    if (more) fetch_plane(r, u, phi, base, comp, k + 2, plane, v);     // in flight during this layer
    if (live) {
      float (*B)[HY][HX] = pl[sb];
      float (*C)[HY][HX] = pl[sm];
      float (*A)[HY][HX] = pl[sa];
      const int o = k * plane + own;
      float out[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float c0 = C[a][y][x];
        float w = __ldg(gf + a * cstride + o);
        w = fmaf(r.lap[a][0], (C[a][y][x + 1] - c0) + (C[a][y][x - 1] - c0), w);
        w = fmaf(r.lap[a][1], (C[a][y + 1][x] - c0) + (C[a][y - 1][x] - c0), w);
        w = fmaf(r.lap[a][2], (A[a][y][x] - c0) + (B[a][y][x] - c0), w);
        out[a] = c0 + w;
      }
      // 4-point crosses: d2u_y/dxdy, d2u_z/dxdz into x; d2u_x/dxdy, d2u_z/dydz into y;
      // d2u_x/dxdz, d2u_y/dydz into z
      const float uy_xy = (C[1][y + 1][x + 1] + C[1][y - 1][x - 1]) - (C[1][y - 1][x + 1] + C[1][y + 1][x - 1]);
      const float ux_xy = (C[0][y + 1][x + 1] + C[0][y - 1][x - 1]) - (C[0][y - 1][x + 1] + C[0][y + 1][x - 1]);
      const float uz_xz = (A[2][y][x + 1] + B[2][y][x - 1]) - (B[2][y][x + 1] + A[2][y][x - 1]);
      const float ux_xz = (A[0][y][x + 1] + B[0][y][x - 1]) - (B[0][y][x + 1] + A[0][y][x - 1]);
      const float uz_yz = (A[2][y + 1][x] + B[2][y - 1][x]) - (B[2][y + 1][x] + A[2][y - 1][x]);
      const float uy_yz = (A[1][y + 1][x] + B[1][y - 1][x]) - (B[1][y + 1][x] + A[1][y - 1][x]);
      out[0] += r.mix[0][1] * uy_xy + r.mix[0][2] * uz_xz;
      out[1] += r.mix[1][0] * ux_xy + r.mix[1][2] * uz_yz;
      out[2] += r.mix[2][0] * ux_xz + r.mix[2][1] * uy_yz;
#pragma unroll
      for (int a = 0; a < 3; ++a) u_out[a * cstride + o] = out[a];
    }
    if (more) {
      __syncthreads();                        // every thread is done with the plane below
      const int t = sb;
      sb = sm;
      sm = sa;
      sa = t;
      store_plane(v, comp, &pl[sa][0][0][0]);
      __syncthreads();
    }
  }
}

// sigma_tot = sigma^dis + lambda div u delta + mu (du_a/db + du_b/da).
__global__ void k_relax_stress(RelaxCoef r, const float *__restrict__ u, const float *__restrict__ phi,
                               const float *__restrict__ sig, float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= r.nx || j >= r.ny) return;
  float g[3][3];   // g[a][b] = du_a / db
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g[a][0] = (uext(r, u, phi, a, i + 1, j, k) - uext(r, u, phi, a, i - 1, j, k)) * r.inv2h[0];
    g[a][1] = (uext(r, u, phi, a, i, j + 1, k) - uext(r, u, phi, a, i, j - 1, k)) * r.inv2h[1];
    g[a][2] = (uext(r, u, phi, a, i, j, k + 1) - uext(r, u, phi, a, i, j, k - 1)) * r.inv2h[2];
  }
  const float ld = r.lam * (g[0][0] + g[1][1] + g[2][2]);
  const float s[6] = {ld + 2.f * r.mu * g[0][0], ld + 2.f * r.mu * g[1][1], ld + 2.f * r.mu * g[2][2],
                      r.mu * (g[0][1] + g[1][0]), r.mu * (g[0][2] + g[2][0]), r.mu * (g[1][2] + g[2][1])};
#pragma unroll
  for (int c = 0; c < 6; ++c) out[cidx(r, c, k, j, i)] = __ldg(sig + cidx(r, c, k, j, i)) + s[c];
}

RelaxCoef relax_coef(const dds_ctx *ctx, double *dt_out) {
  RelaxCoef r{};
  r.nx = ctx->nx;
  r.ny = ctx->ny;
  r.nz = ctx->nz;
  const double mu = ctx->mu, nu = ctx->nu;
  const double E = 2.0 * mu * (1.0 + nu);
  const double A = E * (1.0 - nu) / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double B = E / (2.0 * (1.0 + nu));
  const double *h = ctx->h;
  const double hmin = std::min(h[0], std::min(h[1], h[2]));
  const double dt = hmin * hmin / (5.0 * A - 3.0 * B);
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) {
      r.lap[a][b] = (float)(dt * (a == b ? A : B) / (h[b] * h[b]));
      r.mix[a][b] = a == b ? 0.f : (float)(dt * (A - B) / (4.0 * h[a] * h[b]));
    }
    r.inv2h[a] = (float)(1.0 / (2.0 * h[a]));
  }
  r.two_dz = (float)(2.0 * h[2]);
  r.zfac = (float)(2.0 * h[2] / (1.0 - nu));
  r.nu = (float)nu;
  r.lam = (float)(A - 2.0 * B);
  r.mu = (float)B;
  r.phi_shear = (float)(-(1.0 + nu) / E);
  r.phi_normal = (float)(-(1.0 + nu) * (1.0 - 2.0 * nu) / E);
  r.dt = (float)dt;
  if (dt_out) *dt_out = dt;
  return r;
}

}  // namespace

int enqueue_relax(dds_ctx *ctx, const float *sig, float *u, int n_steps, float *sig_tot, cudaStream_t s) {
  const RelaxCoef r = relax_coef(ctx, nullptr);
  const size_t N = (size_t)r.nx * r.ny * r.nz;
  const size_t need = 3 * N + 3 * N + 6 * (size_t)r.nx * r.ny;     // dt f, u ping-pong, phi
  if (ctx->relax_n < need) {
    cudaFree(ctx->relax_buf);
    ctx->relax_buf = nullptr;
    ctx->relax_n = 0;
    if (cudaMalloc(&ctx->relax_buf, sizeof(float) * need) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, DDS_ERR_OOM, "relax: cannot allocate %.2f GB of work space", sizeof(float) * need / 1e9);
    }
    ctx->relax_n = need;
  }
  float *gf = ctx->relax_buf, *tmp = gf + 3 * N, *phi = tmp + 3 * N;
  const dim3 blk(32, 4, 1);
  const dim3 grid((unsigned)((r.nx + 31) / 32), (unsigned)((r.ny + 3) / 4), (unsigned)r.nz);
  k_relax_prep<<<grid, blk, 0, s>>>(r, sig, gf, phi);
  cudaError_t err = cudaGetLastError();
  // ping-pong so that the last step writes into u
  float *a = u, *b = tmp;
  if (n_steps % 2 == 1 && err == cudaSuccess) {
    err = cudaMemcpyAsync(tmp, u, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s);
    a = tmp;
    b = u;
  }
  const dim3 tgrid((unsigned)((r.nx + TX - 1) / TX), (unsigned)((r.ny + TY - 1) / TY), (unsigned)((r.nz + KZ - 1) / KZ));
  for (int t = 0; t < n_steps && err == cudaSuccess; ++t) {
    k_relax_tile<<<tgrid, NT_TILE, 0, s>>>(r, a, gf, phi, b);
    err = cudaGetLastError();
    std::swap(a, b);
  }
  if (err == cudaSuccess && sig_tot) {
    k_relax_stress<<<grid, blk, 0, s>>>(r, u, phi, sig, sig_tot);
    err = cudaGetLastError();
  }
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "relax: kernel launch failed: %s", cudaGetErrorString(err));
  return DDS_OK;
}

double relax_time_step(const dds_ctx *ctx) {
  double dt = 0.0;
  relax_coef(ctx, &dt);
  return dt;
}

}  // namespace dds
