// Internal declarations shared by the translation units of libdds.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dds.h"

namespace dds {

constexpr int MAX_GROUPS = 8;

// Families collapsed by line direction (the coefficients are linear in b):
// group g owns effective fields [e0, e0 + nd) and families fam[f0 .. f0 + nf);
// field e0 + d receives coef[f0 + q][d] * rho_{fam[f0 + q]}.
struct Collapse {
  int ngroups;
  int e0[MAX_GROUPS], nd[MAX_GROUPS], f0[MAX_GROUPS], nf[MAX_GROUPS];
  int fam[DDS_MAX_FAMILIES];
  float coef[DDS_MAX_FAMILIES][3];
};

// Subset of groups handled by one launch of the x forward pass.
struct GroupList {
  int n;
  int g[MAX_GROUPS];
};

// Symmetry of the kernel spectra used by the three-stage z pass (Shape::zfour).  The
// mirror x -> -x maps the coefficient table of a field with t_x = 0 and b parallel or
// perpendicular to x onto +-itself (reflection covariance of the segment field); with
// the table's oddness this gives g(kx, -ky, -kz) = -p_x(c) g(kx, ky, kz), where
// -p_x(c) = s_b chi(c): s_b = -1 for b along x (else +1), chi(c) = -1 for xy, xz.
// When every field has it (xall), only the main tiles with ky <= py/2 are stored: a
// tile at ky > py/2 works at the negated frequencies -(k1 + R1 k2) and reads the same
// thread's values of the stored tile py - ky.  sbneg bit e: s_b = -1 for field e.
struct ZSym {
  unsigned xall, sbneg;
};

// Geometry of one evaluation as the device kernels see it.
struct Shape {
  int nx, ny, nz;     // grid
  int M;              // px / 2 (complex length of the x transform)
  int py, pz;         // padded y and z sizes
  int fin, fe;        // input families, effective fields
  int wz;             // columns per tile of the fused z pass (shared-memory variant)
  int zreg_g;         // > 0: register-only z pass, pz = 16 * zreg_g, zreg_g lanes per column
  int zfour;          // 1: three-stage register z pass (pz 128 or 256, wz = zfour_width(pz))
  int nb;             // density sets evaluated together (batch); fields are [b][e], outputs [b][c]
  ZSym zs;            // zfour: stored-spectrum symmetries and layout
  int yxf;            // > 0: fused inverse y + x pass, one cluster of yxf CTAs per plane
};

// Columns per tile of the three-stage z pass (Shape::zfour) for padded z size pz.
__host__ __device__ constexpr int zfour_width(int pz) { return pz >= 256 ? 8 : 16; }

// Tiles of the three-stage z pass whose kernel spectra are stored: the main tiles
// (all ky, or ky <= py/2 under xall), then the py / W Nyquist-column tiles.
__host__ __device__ inline long zf_stored_tiles(const Shape &sh) {
  return (long)(sh.zs.xall ? sh.py / 2 + 1 : sh.py) * (sh.M / sh.wz) + sh.py / sh.wz;
}

// Fills sh->zs for the effective fields (t, b given per field, fe <= 6) and returns
// the number of kernel-spectrum values the three-stage z pass stores.
size_t zfour_symmetry(const double *field_t, const double *field_b, int fe, Shape *sh);

// FP64 description of a box coefficient (Eq. 9b times the cell volume).
struct CoefGeom {
  double h[3];        // cell edges
  double hs[3];       // subcell edges
  int m[3];           // subcells per axis
  double mu, nu;
  double rn2;         // squared near-field radius (n_near * max h)^2
  int nx, ny;         // grid (replica periods)
  int n_shells;       // > 0: replica shells of the in-plane periodic boundary conditions
  int periodic;       // with n_shells > 0: shells centred on each source's minimal image
};

// Twiddle tables exp(-2 pi i k / P) for P = 16 .. 2048 (see dds_fft.cuh).
struct Twiddles {
  float2 *f32 = nullptr;
  double2 *f64 = nullptr;
};

}  // namespace dds

struct dds_ctx {
  int device = 0;
  // geometry
  bool has_geom = false;
  int nx = 0, ny = 0, nz = 0;
  double h[3] = {0, 0, 0};
  double mu = 0, nu = 0;
  double n_near = 3.0;
  int n_shells = 0;                     // in-plane periodic boundary conditions (Sec. 4); 0: open
  bool pbc_periodic = false;            // periodic reading of the replica sum, FFT periodic in y
  int z_lanes = 0;                      // fused z pass: 0 auto, -1 shared-memory kernel, G lanes/column
  int z_wz = 0;                         // shared-memory z tile width chosen by dds_autotune (0: planner)
  bool tuned = false;                   // z_lanes / z_wz were set by dds_autotune
  // families
  bool has_fam = false;
  int F = 0;
  std::vector<double> t, b;             // F x 3 each (t normalised)
  // collapse
  int fe = 0;
  std::vector<double> field_t, field_b;  // fe x 3 each
  dds::Collapse col{};
  // plan
  dds::Shape shape{};
  bool built = false;
  // device memory
  dds::Twiddles tw;
  void *kspec = nullptr;                // kernel spectra (layout of the z pass), FP32 or FP16
  float *kscale = nullptr;              // FP16 storage: scale per (component, field); else null
  size_t kspec_floats = 0;              // number of stored values
  bool spectra_fp16 = false;            // option: store the kernel spectra as FP16
  bool yx_fused = false;                // option: fused inverse y + x pass where it applies
  float2 *bufA = nullptr, *bufB = nullptr;        // main work buffers
  float2 *nyqA = nullptr, *nyqB = nullptr;        // Nyquist-column buffers
  size_t bufA_n = 0, bufB_n = 0, nyqA_n = 0, nyqB_n = 0;
  int nb_cap = 1;                       // density sets the work buffers hold
  double *stats = nullptr;              // Eq. 20 sums, [set][6][nz]
  float *relax_buf = nullptr;           // relaxation: dt f, u ping-pong, surface terms
  size_t relax_n = 0;
  int stats_cap = 0;
  // staging for the host-buffer entry points: two sets, used by consecutive calls in
  // turn so that one call's copies overlap another call's evaluation
  void *h2d_rho[2] = {nullptr, nullptr};
  float *h2d_sigma[2] = {nullptr, nullptr};
  size_t h2d_rho_bytes = 0, h2d_sigma_bytes = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;     // copy streams (non-blocking)
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  long host_calls = 0;
  // per-pass profiling
  bool profiling = false;
  std::vector<cudaEvent_t> prof_events;   // 6 per recorded evaluation
  int prof_steps = 0;
  std::string err;
};

namespace dds {

// Twiddle tables, created once per context.
cudaError_t make_twiddles(Twiddles *tw);
void free_twiddles(Twiddles *tw);

// Subcell rule and chord (host side).
void subcell_counts(const double h[3], int m[3]);
double chord_length(const double h[3], const double t[3]);
bool is_near(const double h[3], double n_near, int i, int j, int k);

// FP64 coefficients at a list of offsets (device arrays), near flags per offset.
cudaError_t launch_table_at(const CoefGeom &g, const double t[3], const double b[3], long n,
                            const int *d_ijk, double *d_out, cudaStream_t s);

CoefGeom make_coef_geom(const dds_ctx *ctx);

// Build the FP32 kernel spectra of all effective fields into ctx->kspec.
int build_spectra(dds_ctx *ctx, cudaStream_t s);

// Enqueue one stress evaluation.
// sub: a restricted family collapse whose family indices point into rho's sub_fin
// families (dds_stress_subset); default: the context's own.
int enqueue_stress(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, cudaStream_t s, int nb = 1,
                   double *stats = nullptr, float *s_out = nullptr, const Collapse *sub = nullptr,
                   int sub_fin = 0);
int stress_launch_count(const Shape &sh, const Collapse &col);

// CTAs per cluster of the fused inverse y + x pass for this shape on the current
// device (the plane fits one cluster's shared memory and the device can hold such a
// cluster), else 0: the plan keeps the separate y and x inverse passes.
int yx_inv_cluster(const Shape &sh);

// Free-surface relaxation (Sec. 5): n_steps explicit steps on u, then sigma_tot.
int enqueue_relax(dds_ctx *ctx, const float *sig, float *u, int n_steps, float *sig_tot, cudaStream_t s);
int enqueue_stress_buffers(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, float2 *bufA, float2 *bufB,
                           float2 *nyqA, float2 *nyqB, cudaStream_t s);

// Locates the fixed work area of dds_stress_noalloc on device `dev` (current), which
// loads it onto the device if it is not there yet.
cudaError_t noalloc_prepare(int dev);

// Set ctx->err (printf-style) and return code.
int fail(dds_ctx *ctx, int code, const char *fmt, ...);

// Makes `dev` the current device for the guard's lifetime and restores the previous
// one afterwards.  ok is false when cudaSetDevice failed (then nothing may be enqueued:
// the work would land on whatever device is current).
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  }
  ~DeviceGuard() {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cudaGetLastError();
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard &) = delete;
  DeviceGuard &operator=(const DeviceGuard &) = delete;
};

}  // namespace dds
