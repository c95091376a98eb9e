// C ABI of libdds: validation, family collapse, FFT plan, buffers, entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "dds_fft.cuh"
#include "dds_internal.h"

namespace dds {

int fail(dds_ctx *ctx, int code, const char *fmt, ...) {
  if (ctx) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    ctx->err = msg;
  }
  return code;
}

// Subcells as close to cubic as possible (Sec. 2.3): per axis the integer m >= 1
// minimising |ln((h/m) / h_min)|; of the two integers around r = h / h_min the
// larger wins when m_lo * m_hi <= r^2 (ties included).
void subcell_counts(const double h[3], int m[3]) {
  const double hmin = std::min(h[0], std::min(h[1], h[2]));
  for (int a = 0; a < 3; ++a) {
    const double r = h[a] / hmin;
    int lo = (int)floor(r);
    if (lo < 1) lo = 1;
    const int hi = lo + 1;
    m[a] = ((double)lo * (double)hi <= r * r) ? hi : lo;
  }
}

double chord_length(const double h[3], const double t[3]) {
  double dl = INFINITY;
  for (int a = 0; a < 3; ++a)
    if (t[a] != 0.0) dl = std::min(dl, h[a] / fabs(t[a]));
  return dl;
}

// Near field: |(i dx, j dy, k dz)| < n_near * max(h), evaluated as
// ((x*x + y*y) + z*z) < r*r in IEEE double without contraction.
bool is_near(const double h[3], double n_near, int i, int j, int k) {
  const double hmax = std::max(h[0], std::max(h[1], h[2]));
  const double rn = n_near * hmax;
  const volatile double x = (double)i * h[0], y = (double)j * h[1], z = (double)k * h[2];
  const volatile double xx = x * x, yy = y * y, zz = z * z;
  const volatile double s = xx + yy;
  const volatile double s2 = s + zz;
  const volatile double r2 = rn * rn;
  return s2 < r2;
}

cudaError_t make_twiddles(Twiddles *tw) {
  std::vector<float2> f(TW_TOTAL);
  std::vector<double2> d(TW_TOTAL);
  for (int P = 16; P <= 2048; P *= 2) {
    for (int k = 0; k < P; ++k) {
      const double a = -2.0 * 3.14159265358979323846 * (double)k / (double)P;
      const double c = cos(a), s = sin(a);
      d[tw_offset(P) + k] = make_double2(c, s);
      f[tw_offset(P) + k] = make_float2((float)c, (float)s);
    }
  }
  cudaError_t err = cudaMalloc(&tw->f32, sizeof(float2) * TW_TOTAL);
  if (err == cudaSuccess) err = cudaMalloc(&tw->f64, sizeof(double2) * TW_TOTAL);
  if (err == cudaSuccess) err = cudaMemcpy(tw->f32, f.data(), sizeof(float2) * TW_TOTAL, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(tw->f64, d.data(), sizeof(double2) * TW_TOTAL, cudaMemcpyHostToDevice);
  return err;
}

void free_twiddles(Twiddles *tw) {
  cudaFree(tw->f32);
  cudaFree(tw->f64);
  tw->f32 = nullptr;
  tw->f64 = nullptr;
}

namespace {

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

void free_buffers(dds_ctx *ctx) {
  cudaFree(ctx->kspec);
  cudaFree(ctx->kscale);
  ctx->kscale = nullptr;
  cudaFree(ctx->bufA);
  cudaFree(ctx->bufB);
  cudaFree(ctx->nyqA);
  cudaFree(ctx->nyqB);
  ctx->kspec = nullptr;
  ctx->bufA = ctx->bufB = ctx->nyqA = ctx->nyqB = nullptr;
  ctx->kspec_floats = ctx->bufA_n = ctx->bufB_n = ctx->nyqA_n = ctx->nyqB_n = 0;
}

void invalidate(dds_ctx *ctx) { ctx->built = false; }

// Group families by line direction and choose effective fields per group.
int collapse(dds_ctx *ctx) {
  const int F = ctx->F;
  std::vector<int> group_of(F, -1);
  std::vector<int> leaders;
  for (int f = 0; f < F; ++f) {
    for (size_t g = 0; g < leaders.size(); ++g) {
      const int l = leaders[g];
      double dmax = 0.0;
      for (int a = 0; a < 3; ++a) dmax = std::max(dmax, fabs(ctx->t[3 * f + a] - ctx->t[3 * l + a]));
      if (dmax <= 1e-12) { group_of[f] = (int)g; break; }
    }
    if (group_of[f] < 0) {
      group_of[f] = (int)leaders.size();
      leaders.push_back(f);
    }
  }
  if ((int)leaders.size() > MAX_GROUPS)
    return fail(ctx, DDS_ERR_UNSUPPORTED, "set_families: %d distinct line directions (limit %d)",
                (int)leaders.size(), MAX_GROUPS);
  Collapse col;
  memset(&col, 0, sizeof(col));
  std::vector<double> ft, fb;
  int fe = 0, pos = 0;
  for (size_t g = 0; g < leaders.size(); ++g) {
    std::vector<int> fams;
    for (int f = 0; f < F; ++f)
      if (group_of[f] == (int)g) fams.push_back(f);
    int axes[3], nax = 0;
    double bmax = 0.0;
    for (int a = 0; a < 3; ++a) {
      bool any = false;
      for (int f : fams) {
        if (ctx->b[3 * f + a] != 0.0) any = true;
        bmax = std::max(bmax, fabs(ctx->b[3 * f + a]));
      }
      if (any) axes[nax++] = a;
    }
    const int k = (int)fams.size();
    const bool own = k <= nax;                 // each family is its own field
    const int nd = own ? k : nax;
    col.e0[g] = fe;
    col.nd[g] = nd;
    col.f0[g] = pos;
    col.nf[g] = k;
    const double *tl = &ctx->t[3 * leaders[g]];
    for (int d = 0; d < nd; ++d) {
      ft.insert(ft.end(), tl, tl + 3);
      if (own) {
        fb.insert(fb.end(), &ctx->b[3 * fams[d]], &ctx->b[3 * fams[d]] + 3);
      } else {
        double bv[3] = {0, 0, 0};
        bv[axes[d]] = bmax;
        fb.insert(fb.end(), bv, bv + 3);
      }
    }
    for (int q = 0; q < k; ++q) {
      const int f = fams[q];
      col.fam[pos + q] = f;
      for (int d = 0; d < 3; ++d) {
        double c = 0.0;
        if (d < nd) c = own ? (q == d ? 1.0 : 0.0) : ctx->b[3 * f + axes[d]] / bmax;
        col.coef[pos + q][d] = (float)c;
      }
    }
    pos += k;
    fe += nd;
  }
  if (fe > DDS_MAX_FIELDS)
    return fail(ctx, DDS_ERR_UNSUPPORTED, "set_families: %d effective fields (limit %d)", fe, DDS_MAX_FIELDS);
  col.ngroups = (int)leaders.size();
  ctx->col = col;
  ctx->fe = fe;
  ctx->field_t = ft;
  ctx->field_b = fb;
  return DDS_OK;
}

// Mirror x_a -> -x_a maps the segment of (t, b) onto itself and b onto +-b.
bool mirror_ok(const double *t, const double *b, int a) {
  const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
  return t[a] == 0.0 && (b[a] == 0.0 || (b[a1] == 0.0 && b[a2] == 0.0));
}

// Parity of component c (xx, yy, zz, xy, xz, yz) under that mirror: reflection Q takes
// the field of (t, b) at r to det(Q) Q sigma Q^T of (t, Q b) at Q r, det(Q) = -1 from
// the handedness of the Burgers circuit, Q b = s_b b.
int mirror_parity(const double *b, int a, int c) {
  static const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
  const int sb = b[a] != 0.0 ? -1 : 1;
  const int qi = I[c] == a ? -1 : 1, qj = J[c] == a ? -1 : 1;
  return -sb * qi * qj;
}

}  // namespace

size_t zfour_symmetry(const double *field_t, const double *field_b, int fe, Shape *sh) {
  ZSym &zs = sh->zs;
  memset(&zs, 0, sizeof(zs));
  static const int chi[6] = {1, 1, 1, -1, -1, 1};
  bool all = fe > 0;
  for (int e = 0; e < fe; ++e) {
    const double *t = field_t + 3 * e, *b = field_b + 3 * e;
    bool ok = mirror_ok(t, b, 0);
    // g(kx, -ky, -kz) = -p_x(c) g(kx, ky, kz), and -p_x(c) = s_b chi(c)
    const int sb = b[0] != 0.0 ? -1 : 1;
    for (int c = 0; c < 6 && ok; ++c) ok = -mirror_parity(b, 0, c) == sb * chi[c];
    all = all && ok;
    if (sb < 0) zs.sbneg |= 1u << e;
  }
  zs.xall = all ? 1u : 0u;
  if (!all) zs.sbneg = 0;
  return (size_t)zf_stored_tiles(*sh) * 6 * fe * sh->pz * sh->wz;
}

namespace {

// Padded sizes and the tile width of the fused z pass.
int make_plan(dds_ctx *ctx) {
  Shape sh;
  sh.nx = ctx->nx;
  sh.ny = ctx->ny;
  sh.nz = ctx->nz;
  sh.M = std::max(32, next_pow2(2 * ctx->nx)) / 2;
  sh.py = std::max(32, next_pow2(2 * ctx->ny));
  if (ctx->pbc_periodic) {
    // periodic reading: the convolution is cyclic in y (no padding); x keeps its padded
    // transform, whose table holds the periodic coefficients at offsets (-nx, nx)
    if (ctx->n_shells <= 0)
      return fail(ctx, DDS_ERR_INVALID_ARG, "plan: the periodic reading needs replica shells (DDS_OPT_PBC_SHELLS > 0)");
    if (ctx->ny < 32 || next_pow2(ctx->ny) != ctx->ny)
      return fail(ctx, DDS_ERR_UNSUPPORTED, "plan: the periodic reading needs ny a power of two >= 32 (ny = %d)",
                  ctx->ny);
    sh.py = ctx->ny;
  }
  sh.pz = std::max(16, next_pow2(2 * ctx->nz));
  sh.fin = ctx->F;
  sh.fe = ctx->fe;
  sh.wz = 0;
  sh.zreg_g = 0;
  sh.zfour = 0;
  sh.nb = 1;
  sh.yxf = ctx->yx_fused ? yx_inv_cluster(sh) : 0;
  if (sh.pz <= 64 && sh.fe <= 4 && ctx->z_lanes >= 0) {
    // register-only z pass: E = pz / G registers per lane, E in {8, 16}
    int G = ctx->z_lanes;
    if (G == 0) G = sh.pz / 16 < 1 ? 1 : (sh.fe >= 2 ? sh.pz / 8 : sh.pz / 16);   // default
    const int E = sh.pz / G;
    if ((E == 8 || E == 16) && sh.pz % G == 0 && sh.M >= 32 / G) {
      sh.zreg_g = G;
      ctx->shape = sh;
      return DDS_OK;
    }
    if (ctx->z_lanes > 0)
      return fail(ctx, DDS_ERR_UNSUPPORTED, "z pass: %d lanes per column not available for pz %d", G, sh.pz);
  }
  // three-stage register z pass: padded z 128 or 256, at most 6 fields (default there)
  const int fw = zfour_width(sh.pz);
  const bool four_ok = (sh.pz == 128 || sh.pz == 256) && sh.fe <= 6 && sh.M % fw == 0 && sh.py % fw == 0;
  if (ctx->z_lanes == -2 || (ctx->z_lanes == 0 && ctx->z_wz == 0 && four_ok)) {
    if (!four_ok)
      return fail(ctx, DDS_ERR_UNSUPPORTED, "z pass: the three-stage kernel needs pz 128 or 256 and <= 6 fields "
                  "(pz %d, %d fields)", sh.pz, sh.fe);
    sh.zfour = 1;
    sh.wz = fw;
    zfour_symmetry(ctx->field_t.data(), ctx->field_b.data(), sh.fe, &sh);
    ctx->shape = sh;
    return DDS_OK;
  }
  // shared-memory z pass: fe field lines and three component lines per column
  if (ctx->z_wz > 0) {                   // width fixed by the autotuner
    sh.wz = ctx->z_wz;
    ctx->shape = sh;
    return DDS_OK;
  }
  const size_t pref = 110 * 1024, cap = 220 * 1024;
  for (int pass = 0; pass < 2 && sh.wz == 0; ++pass) {
    for (int W : {64, 32, 16, 8, 4}) {
      if (W > sh.M || sh.py % W != 0) continue;
      if (W * sh.pz > 2048 && W > 8) continue;
      const size_t fe = (size_t)std::max(sh.fe, 1);
      const size_t smem = (sizeof(float2) * (fe + 3) + 2 * sizeof(float) * fe) * sh.pz * W;
      if (smem <= (pass == 0 ? pref : cap)) { sh.wz = W; break; }
    }
  }
  if (sh.wz == 0)
    return fail(ctx, DDS_ERR_UNSUPPORTED, "no z-pass tile fits shared memory (fields %d, pz %d)", sh.fe, sh.pz);
  ctx->shape = sh;
  return DDS_OK;
}

// Work buffers of the five passes for `nbatch` density sets (complex elements).
void work_sizes(const Shape &sh, int nbatch, size_t *a, size_t *b, size_t *na, size_t *nb) {
  const size_t fe = (size_t)std::max(sh.fe, 1) * nbatch, c6 = 6 * (size_t)nbatch;
  const size_t M = sh.M, ny = sh.ny, nz = sh.nz, py = sh.py;
  *a = std::max(fe * nz * ny * M, c6 * nz * py * M);
  *b = std::max(fe * nz * py * M, c6 * nz * ny * M);
  *na = std::max(fe * ny * nz, c6 * py * nz);
  *nb = std::max(fe * py * nz, c6 * ny * nz);
}

int alloc_work(dds_ctx *ctx, int nbatch) {
  size_t a, b, na, nb;
  work_sizes(ctx->shape, nbatch, &a, &b, &na, &nb);
  cudaFree(ctx->bufA);
  cudaFree(ctx->bufB);
  cudaFree(ctx->nyqA);
  cudaFree(ctx->nyqB);
  ctx->bufA = ctx->bufB = ctx->nyqA = ctx->nyqB = nullptr;
  ctx->bufA_n = ctx->bufB_n = ctx->nyqA_n = ctx->nyqB_n = 0;
  ctx->nb_cap = 0;
  cudaError_t err = cudaMalloc(&ctx->bufA, a * sizeof(float2));
  if (err == cudaSuccess) err = cudaMalloc(&ctx->bufB, b * sizeof(float2));
  if (err == cudaSuccess) err = cudaMalloc(&ctx->nyqA, na * sizeof(float2));
  if (err == cudaSuccess) err = cudaMalloc(&ctx->nyqB, nb * sizeof(float2));
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DDS_ERR_OOM, "cannot allocate %.2f GB of work buffers for %d density sets: %s",
                (a + b + na + nb) * 8.0 / 1e9, nbatch, cudaGetErrorString(err));
  }
  ctx->bufA_n = a;
  ctx->bufB_n = b;
  ctx->nyqA_n = na;
  ctx->nyqB_n = nb;
  ctx->nb_cap = nbatch;
  return DDS_OK;
}

int alloc_buffers(dds_ctx *ctx) {
  const Shape &sh = ctx->shape;
  const size_t fe = (size_t)std::max(sh.fe, 1);
  const size_t M = sh.M, py = sh.py, pz = sh.pz;
  size_t a, b, na, nb;
  work_sizes(sh, 1, &a, &b, &na, &nb);
  // one value per (k, component, field), or the three-stage pass's symmetric subset
  size_t ks = py * (M + 1) * pz * 6 * fe;
  if (sh.zfour) {
    Shape tmp = sh;
    ks = zfour_symmetry(ctx->field_t.data(), ctx->field_b.data(), sh.fe, &tmp);
  }
  free_buffers(ctx);
  cudaError_t err = cudaMalloc(&ctx->bufA, a * sizeof(float2));
  if (err == cudaSuccess) err = cudaMalloc(&ctx->bufB, b * sizeof(float2));
  if (err == cudaSuccess) err = cudaMalloc(&ctx->nyqA, na * sizeof(float2));
  if (err == cudaSuccess) err = cudaMalloc(&ctx->nyqB, nb * sizeof(float2));
  const size_t vbytes = ctx->spectra_fp16 ? 2 : sizeof(float);
  if (err == cudaSuccess) err = cudaMalloc(&ctx->kspec, ks * vbytes);
  if (err == cudaSuccess && ctx->spectra_fp16) err = cudaMalloc(&ctx->kscale, 6 * fe * sizeof(float));
  if (err != cudaSuccess) {
    cudaGetLastError();
    free_buffers(ctx);
    return fail(ctx, DDS_ERR_OOM, "build_kernels: cannot allocate %.2f GB of device buffers: %s",
                ((a + b + na + nb) * 8.0 + ks * (double)vbytes) / 1e9, cudaGetErrorString(err));
  }
  ctx->bufA_n = a;
  ctx->bufB_n = b;
  ctx->nyqA_n = na;
  ctx->nyqB_n = nb;
  ctx->nb_cap = 1;
  ctx->kspec_floats = ks;
  return DDS_OK;
}

bool finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

}  // namespace
}  // namespace dds

using namespace dds;

extern "C" {

int dds_create(dds_ctx **out, int cuda_device) {
  if (!out) return DDS_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
    cudaGetLastError();
    return DDS_ERR_INVALID_ARG;
  }
  dds_ctx *ctx = new (std::nothrow) dds_ctx();
  if (!ctx) return DDS_ERR_OOM;
  ctx->device = cuda_device;
  DeviceGuard guard(cuda_device);
  if (!guard.ok) {
    delete ctx;
    return DDS_ERR_CUDA;
  }
  if (make_twiddles(&ctx->tw) != cudaSuccess) {
    cudaGetLastError();
    free_twiddles(&ctx->tw);
    delete ctx;
    return DDS_ERR_OOM;
  }
  *out = ctx;
  return DDS_OK;
}

int dds_set_geometry(dds_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz, double mu,
                     double nu) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(ctx, DDS_ERR_INVALID_ARG, "set_geometry: grid %dx%dx%d must be positive", nx, ny, nz);
  if (nx > DDS_MAX_NXY || ny > DDS_MAX_NXY || nz > DDS_MAX_NZ)
    return fail(ctx, DDS_ERR_UNSUPPORTED, "set_geometry: grid %dx%dx%d exceeds %dx%dx%d", nx, ny, nz,
                DDS_MAX_NXY, DDS_MAX_NXY, DDS_MAX_NZ);
  if (!(dx > 0 && dy > 0 && dz > 0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
    return fail(ctx, DDS_ERR_INVALID_ARG, "set_geometry: cell edges must be positive and finite");
  if (!(mu > 0) || !isfinite(mu) || !(nu > -1.0 && nu < 0.5))
    return fail(ctx, DDS_ERR_INVALID_ARG, "set_geometry: need mu > 0 and -1 < nu < 0.5");
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->nz = nz;
  ctx->h[0] = dx;
  ctx->h[1] = dy;
  ctx->h[2] = dz;
  ctx->mu = mu;
  ctx->nu = nu;
  ctx->has_geom = true;
  if (ctx->tuned) {                      // a tuned schedule belongs to the old geometry
    ctx->z_lanes = 0;
    ctx->z_wz = 0;
    ctx->tuned = false;
  }
  invalidate(ctx);
  return DDS_OK;
}

int dds_set_families(dds_ctx *ctx, int F, const double *t, const double *b) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!t || !b) return fail(ctx, DDS_ERR_INVALID_ARG, "set_families: NULL pointer");
  if (F < 1 || F > DDS_MAX_FAMILIES)
    return fail(ctx, DDS_ERR_INVALID_ARG, "set_families: F = %d outside [1, %d]", F, DDS_MAX_FAMILIES);
  std::vector<double> tv(3 * F), bv(b, b + 3 * F);
  for (int f = 0; f < F; ++f) {
    if (!finite3(t + 3 * f) || !finite3(b + 3 * f))
      return fail(ctx, DDS_ERR_INVALID_ARG, "set_families: family %d has a non-finite vector", f);
    const double n = sqrt(t[3 * f] * t[3 * f] + t[3 * f + 1] * t[3 * f + 1] + t[3 * f + 2] * t[3 * f + 2]);
    if (!(n > 0)) return fail(ctx, DDS_ERR_INVALID_ARG, "set_families: family %d has t = 0", f);
    for (int a = 0; a < 3; ++a) tv[3 * f + a] = (fabs(n - 1.0) <= 1e-15) ? t[3 * f + a] : t[3 * f + a] / n;
  }
  const int F_old = ctx->F;
  std::vector<double> t_old = ctx->t, b_old = ctx->b;
  ctx->F = F;
  ctx->t = tv;
  ctx->b = bv;
  const int rc = collapse(ctx);
  if (rc != DDS_OK) {
    ctx->F = F_old;
    ctx->t = t_old;
    ctx->b = b_old;
    return rc;
  }
  ctx->has_fam = true;
  if (ctx->tuned) {
    ctx->z_lanes = 0;
    ctx->z_wz = 0;
    ctx->tuned = false;
  }
  invalidate(ctx);
  return DDS_OK;
}

int dds_set_option(dds_ctx *ctx, int key, double value) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  switch (key) {
    case DDS_OPT_Z_LANES:
      if (!(value == -2 || value == -1 || value == 0 || value == 1 || value == 2 || value == 4 || value == 8))
        return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: z lanes must be -2, -1, 0, 1, 2, 4 or 8");
      ctx->z_lanes = (int)value;
      ctx->z_wz = 0;
      ctx->tuned = false;
      invalidate(ctx);
      return DDS_OK;
    case DDS_OPT_SPECTRA_FP16:
      if (!(value == 0 || value == 1))
        return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: spectra storage must be 0 (FP32) or 1 (FP16)");
      ctx->spectra_fp16 = value == 1;
      invalidate(ctx);
      return DDS_OK;
    case DDS_OPT_PBC_SHELLS:
      if (!(value >= 0 && value <= 1000) || value != (double)(int)value)
        return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: replica shells must be an integer in [0, 1000]");
      ctx->n_shells = (int)value;
      invalidate(ctx);
      return DDS_OK;
    case DDS_OPT_PBC_PERIODIC:
      if (value != 0.0 && value != 1.0)
        return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: periodic reading must be 0 or 1");
      ctx->pbc_periodic = value != 0.0;
      invalidate(ctx);
      return DDS_OK;
    case DDS_OPT_YX_FUSED:
      if (value != 0.0 && value != 1.0)
        return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: fused inverse pass must be 0 or 1");
      ctx->yx_fused = value != 0.0;
      invalidate(ctx);
      return DDS_OK;
    case DDS_OPT_NEAR_RADIUS:
      if (!(value >= 0.0) || !isfinite(value))
        return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: near radius must be >= 0");
      ctx->n_near = value;
      invalidate(ctx);
      return DDS_OK;
    default:
      return fail(ctx, DDS_ERR_INVALID_ARG, "set_option: unknown key %d", key);
  }
}

int dds_build_kernels(dds_ctx *ctx, void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->has_geom || !ctx->has_fam)
    return fail(ctx, DDS_ERR_NOT_READY, "build_kernels: set geometry and families first");
  if (ctx->built) return DDS_OK;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  int rc = make_plan(ctx);
  if (rc != DDS_OK) return rc;
  rc = alloc_buffers(ctx);
  if (rc != DDS_OK) return rc;
  if (ctx->fe > 0) {
    rc = build_spectra(ctx, (cudaStream_t)cuda_stream);
    if (rc != DDS_OK) return rc;
  }
  // place the fixed work area of dds_stress_noalloc on this device now, during set-up
  const cudaError_t nerr = noalloc_prepare(ctx->device);
  if (nerr != cudaSuccess)
    return fail(ctx, DDS_ERR_CUDA, "build_kernels: cannot locate the fixed work area: %s", cudaGetErrorString(nerr));
  ctx->built = true;
  ctx->err.clear();
  return DDS_OK;
}

int dds_autotune(dds_ctx *ctx, void *cuda_stream, float *best_ms) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->has_geom || !ctx->has_fam)
    return fail(ctx, DDS_ERR_NOT_READY, "autotune: set geometry and families first");
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // candidate schedules of the fused z pass: (lanes, tile width)
  ctx->z_lanes = 0;
  ctx->z_wz = 0;
  int rc = make_plan(ctx);
  if (rc != DDS_OK) return rc;
  const Shape base = ctx->shape;
  std::vector<std::pair<int, int>> cand;
  if (base.pz <= 64 && base.fe <= 4) {
    for (int G : {1, 2, 4, 8}) {
      const int E = base.pz / G;
      if (base.pz % G == 0 && (E == 8 || E == 16) && base.M >= 32 / G) cand.push_back({G, 0});
    }
  }
  if ((base.pz == 128 || base.pz == 256) && base.fe <= 6 && base.M % zfour_width(base.pz) == 0 &&
      base.py % zfour_width(base.pz) == 0)
    cand.push_back({-2, 0});
  for (int W : {4, 8, 16, 32, 64}) {
    if (W > base.M || base.py % W != 0 || (W * base.pz > 2048 && W > 8)) continue;
    const size_t fe = (size_t)std::max(base.fe, 1);
    if ((sizeof(float2) * (fe + 3) + 2 * sizeof(float) * fe) * base.pz * W > 220 * 1024) continue;
    cand.push_back({-1, W});
  }
  if (cand.empty()) return fail(ctx, DDS_ERR_UNSUPPORTED, "autotune: no z-pass schedule applies");
  ctx->built = false;
  const size_t N = (size_t)ctx->nx * ctx->ny * ctx->nz;
  float *rho = nullptr, *sigma = nullptr;
  void *flush = nullptr;                  // written before each trial: trials start from a cold L2
  const size_t flush_bytes = 256u << 20;
  cudaError_t err = cudaMalloc(&rho, sizeof(float) * N * ctx->F);
  if (err == cudaSuccess) err = cudaMalloc(&sigma, sizeof(float) * N * 6);
  if (err == cudaSuccess) err = cudaMalloc(&flush, flush_bytes);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaMemsetAsync(rho, 0, sizeof(float) * N * ctx->F, s);
  float best = 1e30f;
  std::pair<int, int> pick = cand[0];
  for (size_t i = 0; i < cand.size() && err == cudaSuccess && rc == DDS_OK; ++i) {
    ctx->z_lanes = cand[i].first;
    ctx->z_wz = cand[i].second;
    rc = make_plan(ctx);
    if (rc != DDS_OK) break;
    if (ctx->shape.zreg_g != (cand[i].first > 0 ? cand[i].first : 0)) continue;   // planner declined
    if (ctx->shape.zfour != (cand[i].first == -2 ? 1 : 0)) continue;
    rc = alloc_buffers(ctx);
    if (rc != DDS_OK) break;
    const size_t vbytes = ctx->spectra_fp16 ? 2 : sizeof(float);
    err = cudaMemsetAsync(ctx->kspec, 0, ctx->kspec_floats * vbytes, s);   // timing only: values are irrelevant
    if (err == cudaSuccess && ctx->kscale) err = cudaMemsetAsync(ctx->kscale, 0, 6 * sizeof(float) * ctx->fe, s);
    for (int w = 0; w < 2 && rc == DDS_OK && err == cudaSuccess; ++w) rc = enqueue_stress(ctx, rho, DDS_F32, sigma, s);
    if (rc != DDS_OK || err != cudaSuccess) break;
    // median of five trials, each from a cold L2: one disturbed trial cannot decide
    float trial[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int r = 0; r < 5 && rc == DDS_OK && err == cudaSuccess; ++r) {
      err = cudaMemsetAsync(flush, r, flush_bytes, s);
      if (err == cudaSuccess) err = cudaEventRecord(e0, s);
      if (err == cudaSuccess) rc = enqueue_stress(ctx, rho, DDS_F32, sigma, s);
      if (err == cudaSuccess) err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&trial[r], e0, e1);
    }
    std::sort(trial, trial + 5);
    const float ms = trial[2];
    if (err == cudaSuccess && rc == DDS_OK && ms < best) {
      best = ms;
      pick = cand[i];
    }
  }
  cudaFree(rho);
  cudaFree(sigma);
  cudaFree(flush);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  free_buffers(ctx);
  ctx->z_lanes = pick.first;
  ctx->z_wz = pick.second;
  ctx->tuned = true;
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "autotune: %s", cudaGetErrorString(err));
  if (rc != DDS_OK) return rc;
  if (best_ms) *best_ms = best;
  return DDS_OK;
}

int dds_stress(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, DDS_ERR_NOT_READY, "stress: call dds_build_kernels first");
  if (!rho || !sigma) return fail(ctx, DDS_ERR_INVALID_ARG, "stress: NULL pointer");
  if (rho_dtype != DDS_F32 && rho_dtype != DDS_BF16)
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress: unknown density type %d", rho_dtype);
  if (((uintptr_t)rho & 15) || ((uintptr_t)sigma & 15))
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress: rho and sigma must be 16-byte aligned");
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (ctx->fe == 0) {
    const cudaError_t err = cudaMemsetAsync(sigma, 0, sizeof(float) * 6 * (size_t)ctx->nx * ctx->ny * ctx->nz, s);
    return err == cudaSuccess ? DDS_OK : fail(ctx, DDS_ERR_CUDA, "stress: %s", cudaGetErrorString(err));
  }
  return enqueue_stress(ctx, rho, rho_dtype, sigma, s);
}

int dds_relax(dds_ctx *ctx, const float *sigma_dis, float *u, int n_steps, float *sigma_tot, void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->has_geom) return fail(ctx, DDS_ERR_NOT_READY, "relax: call dds_set_geometry first");
  if (ctx->nz < 2) return fail(ctx, DDS_ERR_UNSUPPORTED, "relax: the free surfaces need at least two layers");
  if (!sigma_dis || !u) return fail(ctx, DDS_ERR_INVALID_ARG, "relax: NULL pointer");
  if (n_steps < 0) return fail(ctx, DDS_ERR_INVALID_ARG, "relax: negative step count %d", n_steps);
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  return enqueue_relax(ctx, sigma_dis, u, n_steps, sigma_tot, (cudaStream_t)cuda_stream);
}

int dds_stress_multi(dds_ctx *ctx, int nb, const void *rho, int rho_dtype, float *sigma, void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, DDS_ERR_NOT_READY, "stress_multi: call dds_build_kernels first");
  if (nb < 1 || nb > 4096) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_multi: nb = %d outside [1, 4096]", nb);
  if (!rho || !sigma) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_multi: NULL pointer");
  if (rho_dtype != DDS_F32 && rho_dtype != DDS_BF16)
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_multi: unknown density type %d", rho_dtype);
  if (((uintptr_t)rho & 15) || ((uintptr_t)sigma & 15))
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_multi: rho and sigma must be 16-byte aligned");
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (ctx->fe == 0) {
    const cudaError_t err =
        cudaMemsetAsync(sigma, 0, sizeof(float) * 6 * (size_t)nb * ctx->nx * ctx->ny * ctx->nz, s);
    return err == cudaSuccess ? DDS_OK : fail(ctx, DDS_ERR_CUDA, "stress_multi: %s", cudaGetErrorString(err));
  }
  if (nb > ctx->nb_cap) {
    // the current buffers may still be in use by work queued on any stream
    const cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_multi: %s", cudaGetErrorString(err));
    const int rc = alloc_work(ctx, nb);
    if (rc != DDS_OK) return rc;
  }
  return enqueue_stress(ctx, rho, rho_dtype, sigma, s, nb);
}

int dds_stress_subset(dds_ctx *ctx, int nb, int n, const int *fam, const void *rho, int rho_dtype, float *sigma,
                      void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, DDS_ERR_NOT_READY, "stress_subset: call dds_build_kernels first");
  if (nb < 1 || nb > 4096) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_subset: nb = %d outside [1, 4096]", nb);
  if (!fam || !rho || !sigma) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_subset: NULL pointer");
  if (n < 1 || n > ctx->F)
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_subset: n = %d outside [1, %d]", n, ctx->F);
  if (rho_dtype != DDS_F32 && rho_dtype != DDS_BF16)
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_subset: unknown density type %d", rho_dtype);
  if (((uintptr_t)rho & 15) || ((uintptr_t)sigma & 15))
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_subset: rho and sigma must be 16-byte aligned");
  std::vector<int> slot(ctx->F, -1);      // family -> its position in rho
  for (int i = 0; i < n; ++i) {
    if (fam[i] < 0 || fam[i] >= ctx->F || slot[fam[i]] >= 0)
      return fail(ctx, DDS_ERR_INVALID_ARG, "stress_subset: family index %d out of range or repeated", fam[i]);
    slot[fam[i]] = i;
  }
  // the context's collapse restricted to the given families (fields and coefficients
  // unchanged; a group without any of them contributes zero fields)
  Collapse sub = ctx->col;
  int pos = 0;
  for (int g = 0; g < ctx->col.ngroups; ++g) {
    const int f0 = pos;
    for (int q = 0; q < ctx->col.nf[g]; ++q) {
      const int src = ctx->col.f0[g] + q, i = slot[ctx->col.fam[src]];
      if (i < 0) continue;
      sub.fam[pos] = i;
      for (int d = 0; d < 3; ++d) sub.coef[pos][d] = ctx->col.coef[src][d];
      ++pos;
    }
    sub.f0[g] = f0;
    sub.nf[g] = pos - f0;
  }
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (ctx->fe == 0) {
    const cudaError_t err =
        cudaMemsetAsync(sigma, 0, sizeof(float) * 6 * (size_t)nb * ctx->nx * ctx->ny * ctx->nz, s);
    return err == cudaSuccess ? DDS_OK : fail(ctx, DDS_ERR_CUDA, "stress_subset: %s", cudaGetErrorString(err));
  }
  if (nb > ctx->nb_cap) {
    const cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_subset: %s", cudaGetErrorString(err));
    const int rc = alloc_work(ctx, nb);
    if (rc != DDS_OK) return rc;
  }
  return enqueue_stress(ctx, rho, rho_dtype, sigma, s, nb, nullptr, nullptr, &sub, n);
}

int dds_stress_stats(dds_ctx *ctx, int nb, const void *rho, int rho_dtype, float *sigma, float *s_out,
                     void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, DDS_ERR_NOT_READY, "stress_stats: call dds_build_kernels first");
  if (nb < 1 || nb > 4096) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_stats: nb = %d outside [1, 4096]", nb);
  if (!rho || !sigma || !s_out) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_stats: NULL pointer");
  if (rho_dtype != DDS_F32 && rho_dtype != DDS_BF16)
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_stats: unknown density type %d", rho_dtype);
  if (((uintptr_t)rho & 15) || ((uintptr_t)sigma & 15))
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_stats: rho and sigma must be 16-byte aligned");
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t ns = 6 * (size_t)nb * ctx->nz;
  if (ctx->fe == 0) {
    cudaError_t err = cudaMemsetAsync(sigma, 0, sizeof(float) * 6 * (size_t)nb * ctx->nx * ctx->ny * ctx->nz, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(s_out, 0, sizeof(float) * ns, s);
    return err == cudaSuccess ? DDS_OK : fail(ctx, DDS_ERR_CUDA, "stress_stats: %s", cudaGetErrorString(err));
  }
  if (nb > ctx->nb_cap || (int)ns > ctx->stats_cap) {
    const cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_stats: %s", cudaGetErrorString(err));
    if (nb > ctx->nb_cap) {
      const int rc = alloc_work(ctx, nb);
      if (rc != DDS_OK) return rc;
    }
    if ((int)ns > ctx->stats_cap) {
      cudaFree(ctx->stats);
      ctx->stats = nullptr;
      ctx->stats_cap = 0;
      if (cudaMalloc(&ctx->stats, sizeof(double) * ns) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DDS_ERR_OOM, "stress_stats: cannot allocate %zu bytes", sizeof(double) * ns);
      }
      ctx->stats_cap = (int)ns;
    }
  }
  return enqueue_stress(ctx, rho, rho_dtype, sigma, s, nb, ctx->stats, s_out);
}

int dds_stress_batched(dds_ctx **ctxs, int n, const void **rho, const int *rho_dtype, float **sigma,
                       void *cuda_stream) {
  if (!ctxs || n < 0 || (n > 0 && (!rho || !sigma))) return DDS_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int rc = dds_stress(ctxs[i], rho[i], rho_dtype ? rho_dtype[i] : DDS_F32, sigma[i], cuda_stream);
    if (rc != DDS_OK) return rc;
  }
  return DDS_OK;
}

struct dds_graph {
  int device = 0;
  int n = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int dds_graph_capture(dds_ctx **ctxs, int n, const int *nb, const void **rho, const int *rho_dtype, float **sigma,
                      void *cuda_stream, dds_graph **out) {
  if (!out) return DDS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || n < 1 || !nb || !rho || !sigma) return DDS_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    dds_ctx *c = ctxs[i];
    if (!c) return DDS_ERR_INVALID_ARG;
    if (c->device != ctxs[0]->device) return fail(c, DDS_ERR_INVALID_ARG, "graph_capture: contexts on different devices");
    if (!c->built) return fail(c, DDS_ERR_NOT_READY, "graph_capture: call dds_build_kernels first");
    if (c->profiling) return fail(c, DDS_ERR_INVALID_ARG, "graph_capture: disable per-pass profiling first");
    if (nb[i] < 1 || nb[i] > 4096) return fail(c, DDS_ERR_INVALID_ARG, "graph_capture: nb = %d outside [1, 4096]", nb[i]);
    const int dt = rho_dtype ? rho_dtype[i] : DDS_F32;
    if (dt != DDS_F32 && dt != DDS_BF16) return fail(c, DDS_ERR_INVALID_ARG, "graph_capture: unknown density type %d", dt);
    if (!rho[i] || !sigma[i] || ((uintptr_t)rho[i] & 15) || ((uintptr_t)sigma[i] & 15))
      return fail(c, DDS_ERR_INVALID_ARG, "graph_capture: rho and sigma must be non-NULL and 16-byte aligned");
  }
  DeviceGuard guard(ctxs[0]->device);
  if (!guard.ok) return fail(ctxs[0], DDS_ERR_CUDA, "cannot make device %d current", ctxs[0]->device);
  cudaStream_t user = (cudaStream_t)cuda_stream;
  // work buffers for every batch, then one evaluation of each entry outside the capture
  // (finishes the library's lazy per-device set-up; writes sigma)
  for (int i = 0; i < n; ++i) {
    if (nb[i] > ctxs[i]->nb_cap) {
      const cudaError_t err = cudaDeviceSynchronize();
      if (err != cudaSuccess) return fail(ctxs[i], DDS_ERR_CUDA, "graph_capture: %s", cudaGetErrorString(err));
      const int rc = alloc_work(ctxs[i], nb[i]);
      if (rc != DDS_OK) return rc;
    }
    if (ctxs[i]->fe == 0) continue;
    const int rc = enqueue_stress(ctxs[i], rho[i], rho_dtype ? rho_dtype[i] : DDS_F32, sigma[i], user, nb[i]);
    if (rc != DDS_OK) return rc;
  }
  cudaError_t err = cudaStreamSynchronize(user);
  if (err != cudaSuccess) return fail(ctxs[0], DDS_ERR_CUDA, "graph_capture: %s", cudaGetErrorString(err));
  cudaStream_t cs = nullptr;
  err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (err != cudaSuccess) return fail(ctxs[0], DDS_ERR_CUDA, "graph_capture: %s", cudaGetErrorString(err));
  err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = DDS_OK;
  for (int i = 0; i < n && err == cudaSuccess && rc == DDS_OK; ++i) {
    if (ctxs[i]->fe == 0) {
      err = cudaMemsetAsync(sigma[i], 0, sizeof(float) * 6 * (size_t)nb[i] * ctxs[i]->nx * ctxs[i]->ny * ctxs[i]->nz, cs);
      continue;
    }
    rc = enqueue_stress(ctxs[i], rho[i], rho_dtype ? rho_dtype[i] : DDS_F32, sigma[i], cs, nb[i]);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t end = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (err == cudaSuccess) err = end;
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess && rc == DDS_OK) err = cudaGraphInstantiate(&exec, graph, 0);
  if (err != cudaSuccess || rc != DDS_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != DDS_OK ? rc : fail(ctxs[0], DDS_ERR_CUDA, "graph_capture: %s", cudaGetErrorString(err));
  }
  dds_graph *g = new (std::nothrow) dds_graph;
  if (!g) {
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return DDS_ERR_OOM;
  }
  g->device = ctxs[0]->device;
  g->n = n;
  g->graph = graph;
  g->exec = exec;
  *out = g;
  return DDS_OK;
}

int dds_graph_launch(dds_graph *g, void *cuda_stream) {
  if (!g) return DDS_ERR_INVALID_ARG;
  DeviceGuard guard(g->device);
  if (!guard.ok) return DDS_ERR_CUDA;
  const cudaError_t err = cudaGraphLaunch(g->exec, (cudaStream_t)cuda_stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return DDS_ERR_CUDA;
  }
  return DDS_OK;
}

int dds_graph_nodes(const dds_graph *g) {
  if (!g) return DDS_ERR_INVALID_ARG;
  size_t nodes = 0;
  if (cudaGraphGetNodes(g->graph, nullptr, &nodes) != cudaSuccess) return DDS_ERR_CUDA;
  return (int)nodes;
}

void dds_graph_destroy(dds_graph *g) {
  if (!g) return;
  {
    DeviceGuard guard(g->device);   // frees proceed even if it failed: they need no current device
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
  }
  delete g;
}

int dds_stress_host_async(dds_ctx *ctx, const float *rho_host, float *sigma_host, void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, DDS_ERR_NOT_READY, "stress_host: call dds_build_kernels first");
  if (!rho_host || !sigma_host) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_host: NULL pointer");
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  const size_t N = (size_t)ctx->nx * ctx->ny * ctx->nz;
  const size_t rb = sizeof(float) * N * ctx->F, sb = sizeof(float) * N * 6;
  cudaError_t err = cudaSuccess;
  if (!ctx->s_in) {
    err = cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking);
    for (int j = 0; j < 2 && err == cudaSuccess; ++j) {
      err = cudaEventCreateWithFlags(&ctx->ev_in[j], cudaEventDisableTiming);
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ctx->ev_comp[j], cudaEventDisableTiming);
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ctx->ev_out[j], cudaEventDisableTiming);
    }
    if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_host: %s", cudaGetErrorString(err));
  }
  if (ctx->h2d_rho_bytes < rb || ctx->h2d_sigma_bytes < sb) {
    // earlier calls may still use the old buffers
    err = cudaDeviceSynchronize();
    if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_host: %s", cudaGetErrorString(err));
    for (int j = 0; j < 2; ++j) {
      cudaFree(ctx->h2d_rho[j]);
      cudaFree(ctx->h2d_sigma[j]);
      ctx->h2d_rho[j] = nullptr;
      ctx->h2d_sigma[j] = nullptr;
    }
    ctx->h2d_rho_bytes = ctx->h2d_sigma_bytes = 0;
    for (int j = 0; j < 2 && err == cudaSuccess; ++j) {
      err = cudaMalloc(&ctx->h2d_rho[j], rb);
      if (err == cudaSuccess) err = cudaMalloc(&ctx->h2d_sigma[j], sb);
    }
    if (err != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, DDS_ERR_OOM, "stress_host: cannot allocate 2 x %zu bytes of staging", rb + sb);
    }
    ctx->h2d_rho_bytes = rb;
    ctx->h2d_sigma_bytes = sb;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int j = (int)(ctx->host_calls & 1);
  // staging set j: its densities are free once the call two back has evaluated, its
  // stresses once that call's results reached the host (waits on unrecorded events pass)
  err = cudaStreamWaitEvent(ctx->s_in, ctx->ev_comp[j], 0);
  if (err == cudaSuccess) err = cudaMemcpyAsync(ctx->h2d_rho[j], rho_host, rb, cudaMemcpyHostToDevice, ctx->s_in);
  if (err == cudaSuccess) err = cudaEventRecord(ctx->ev_in[j], ctx->s_in);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(s, ctx->ev_in[j], 0);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(s, ctx->ev_out[j], 0);
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_host: H2D copy: %s", cudaGetErrorString(err));
  const int rc = dds_stress(ctx, ctx->h2d_rho[j], DDS_F32, ctx->h2d_sigma[j], cuda_stream);
  if (rc != DDS_OK) return rc;
  err = cudaEventRecord(ctx->ev_comp[j], s);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(ctx->s_out, ctx->ev_comp[j], 0);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(sigma_host, ctx->h2d_sigma[j], sb, cudaMemcpyDeviceToHost, ctx->s_out);
  if (err == cudaSuccess) err = cudaEventRecord(ctx->ev_out[j], ctx->s_out);
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_host: D2H copy: %s", cudaGetErrorString(err));
  ctx->host_calls++;
  return DDS_OK;
}

int dds_stress_host_sync(dds_ctx *ctx) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->s_out) return DDS_OK;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaError_t err = cudaStreamSynchronize(ctx->s_in);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->s_out);
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "stress_host_sync: %s", cudaGetErrorString(err));
  return DDS_OK;
}

int dds_stress_host(dds_ctx *ctx, const float *rho_host, float *sigma_host, void *cuda_stream) {
  const int rc = dds_stress_host_async(ctx, rho_host, sigma_host, cuda_stream);
  return rc != DDS_OK ? rc : dds_stress_host_sync(ctx);
}

int dds_table_at(dds_ctx *ctx, const double t[3], const double b[3], long n, const int *ijk_host,
                 double *out_host) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->has_geom) return fail(ctx, DDS_ERR_NOT_READY, "table_at: set geometry first");
  if (!t || !b || (n > 0 && (!ijk_host || !out_host)) || n < 0)
    return fail(ctx, DDS_ERR_INVALID_ARG, "table_at: bad arguments");
  if (!finite3(t) || !finite3(b)) return fail(ctx, DDS_ERR_INVALID_ARG, "table_at: non-finite t or b");
  const double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  if (!(tn > 0)) return fail(ctx, DDS_ERR_INVALID_ARG, "table_at: t = 0");
  double tu[3];
  for (int a = 0; a < 3; ++a) tu[a] = (fabs(tn - 1.0) <= 1e-15) ? t[a] : t[a] / tn;
  if (n == 0) return DDS_OK;
  for (long q = 0; q < n; ++q) {
    const int i = ijk_host[3 * q], j = ijk_host[3 * q + 1], k = ijk_host[3 * q + 2];
    if (abs(i) >= ctx->nx || abs(j) >= ctx->ny || abs(k) >= ctx->nz)
      return fail(ctx, DDS_ERR_INVALID_ARG, "table_at: offset (%d,%d,%d) outside the grid", i, j, k);
  }
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  int *d_ijk = nullptr;
  double *d_out = nullptr;
  cudaError_t err = cudaMalloc(&d_ijk, sizeof(int) * 3 * n);
  if (err == cudaSuccess) err = cudaMalloc(&d_out, sizeof(double) * 6 * n);
  if (err == cudaSuccess) err = cudaMemcpy(d_ijk, ijk_host, sizeof(int) * 3 * n, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = launch_table_at(make_coef_geom(ctx), tu, b, n, d_ijk, d_out, 0);
  if (err == cudaSuccess) err = cudaMemcpy(out_host, d_out, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost);
  cudaFree(d_ijk);
  cudaFree(d_out);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DDS_ERR_CUDA, "table_at: %s", cudaGetErrorString(err));
  }
  return DDS_OK;
}

int dds_query(const dds_ctx *ctx, int *n_fields, int *px, int *py, int *pz) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return DDS_ERR_NOT_READY;
  if (n_fields) *n_fields = ctx->fe;
  if (px) *px = 2 * ctx->shape.M;
  if (py) *py = ctx->shape.py;
  if (pz) *pz = ctx->shape.pz;
  return DDS_OK;
}

int dds_footprint(dds_ctx *ctx, int nb, unsigned long long *bytes) {
  if (!ctx || !bytes) return DDS_ERR_INVALID_ARG;
  if (nb < 1 || nb > 4096) return fail(ctx, DDS_ERR_INVALID_ARG, "footprint: nb = %d outside [1, 4096]", nb);
  if (!ctx->has_geom || !ctx->has_fam) return fail(ctx, DDS_ERR_NOT_READY, "footprint: set geometry and families first");
  const Shape saved = ctx->shape;
  const int rc = make_plan(ctx);            // host-only; restored below
  const Shape sh = ctx->shape;
  ctx->shape = saved;
  if (rc != DDS_OK) return rc;
  const size_t fe = (size_t)std::max(sh.fe, 1);
  size_t ks = (size_t)sh.py * (sh.M + 1) * sh.pz * 6 * fe;
  if (sh.zfour) {
    Shape tmp = sh;
    ks = zfour_symmetry(ctx->field_t.data(), ctx->field_b.data(), sh.fe, &tmp);
  }
  size_t a, b, na, nbuf;
  work_sizes(sh, nb, &a, &b, &na, &nbuf);
  *bytes = (unsigned long long)(ks * (ctx->spectra_fp16 ? 2 : 4) + (a + b + na + nbuf) * sizeof(float2));
  return DDS_OK;
}

int dds_spectra_bytes(const dds_ctx *ctx, unsigned long long *bytes) {
  if (!ctx || !bytes) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return DDS_ERR_NOT_READY;
  *bytes = (unsigned long long)ctx->kspec_floats * (ctx->spectra_fp16 ? 2 : 4);
  return DDS_OK;
}

int dds_launches_per_stress(const dds_ctx *ctx) {
  if (!ctx || !ctx->built) return 0;
  return ctx->fe == 0 ? 0 : stress_launch_count(ctx->shape, ctx->col);
}

int dds_yx_cluster(const dds_ctx *ctx) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return DDS_ERR_NOT_READY;
  return ctx->shape.yxf;
}

int dds_profile_enable(dds_ctx *ctx, int enable) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  ctx->profiling = enable != 0;
  ctx->prof_steps = 0;
  return DDS_OK;
}

int dds_profile_read(dds_ctx *ctx, int max_steps, float *ms_out, int *n_steps, int *n_passes) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (max_steps < 0 || (max_steps > 0 && !ms_out))
    return fail(ctx, DDS_ERR_INVALID_ARG, "profile_read: bad arguments");
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "cannot make device %d current", ctx->device);
  const int steps = std::min(max_steps, ctx->prof_steps);
  for (int st = 0; st < steps; ++st) {
    cudaEvent_t *ev = &ctx->prof_events[6 * (size_t)st];
    cudaError_t err = cudaEventSynchronize(ev[5]);
    for (int p = 0; p < 5 && err == cudaSuccess; ++p) err = cudaEventElapsedTime(&ms_out[5 * st + p], ev[p], ev[p + 1]);
    if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "profile_read: %s", cudaGetErrorString(err));
  }
  if (n_steps) *n_steps = steps;
  if (n_passes) *n_passes = 5;
  ctx->prof_steps = 0;
  return DDS_OK;
}

const char *dds_last_error(const dds_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void dds_destroy(dds_ctx *ctx) {
  if (!ctx) return;
  {
    DeviceGuard guard(ctx->device);   // frees proceed even if it failed: they need no current device
    free_buffers(ctx);
    free_twiddles(&ctx->tw);
    for (int j = 0; j < 2; ++j) {
      cudaFree(ctx->h2d_rho[j]);
      cudaFree(ctx->h2d_sigma[j]);
      if (ctx->ev_in[j]) cudaEventDestroy(ctx->ev_in[j]);
      if (ctx->ev_comp[j]) cudaEventDestroy(ctx->ev_comp[j]);
      if (ctx->ev_out[j]) cudaEventDestroy(ctx->ev_out[j]);
    }
    if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
    if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
    cudaFree(ctx->stats);
    cudaFree(ctx->relax_buf);
    for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
  }
  delete ctx;
}

}  // extern "C"
