// FP64 interaction coefficients and their FP32 Fourier spectra.
//
// Coefficient of a box (cell or subcell) of edges hb for observer offset r from
// its centre (Eq. 9b times the box volume, Eq. 2 / Eq. 10):
//   g(r) = (V / dl) * sigma^AB(r),  dl = chord of the box through its centre along t,
// with sigma^AB the stress of the straight segment A = -dl/2 t, B = +dl/2 t
// (Eq. 6, Eq. 7a, Eq. 7b, prefactor mu / pi, evaluated at B minus at A).
// Near offsets (|r0 - r_i| < n_near * max h, Sec. 2.3) use
//   G = (1/M) sum_{u in target subcells} sum_{v in source subcells} g_sub(Delta + u - v)
// which is evaluated grouped by the subcell difference d = u - v (multiplicity
// prod_a (m_a - |d_a|)).  The self pair (observer on the segment midpoint) is 0.
//
// The table of G over all offsets is wrapped into the zero-padded periodic grid
// (offset D -> index D mod P), transformed by an FP64 R2C FFT, and because the
// table is odd (G(-D) = -G(D)) its spectrum is purely imaginary: only Im / (Px Py Pz)
// is kept, in FP32, laid out per tile of the fused z pass.
#include <math.h>

#include <cuda_fp16.h>

#include "dds_fft.cuh"
#include "dds_internal.h"

namespace dds {

namespace {

struct V3 {
  double x, y, z;
};
__host__ __device__ __forceinline__ V3 v3(double x, double y, double z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// Bracket of Eq. 6 at one segment end, divided by R_t^2.  R joins the observer and
// the end point (either orientation, see segment_stress).  S in xx,yy,zz,xy,xz,yz.
__device__ void eq6_end(V3 R, V3 t, V3 b, double k1, double S[6]) {
  const double Rn = sqrt(dot(R, R));
  const double L = dot(R, t);
  const V3 Rt = R + Rn * t;
  const double iRt2 = 1.0 / dot(Rt, Rt);
  const V3 rho = R - L * t;
  const V3 u = cross(b, Rt);          // enters [b R_t t]^sym
  const V3 w = cross(b, t);           // enters [b t R_t]^sym
  const double k2 = 0.5 * k1 * dot(u, t);   // (b, R_t, t) / (2 (1 - nu))
  const double LR = L / Rn;
  const int ia[6] = {0, 1, 2, 0, 0, 1};
  const int ic[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int a = ia[q], c = ic[q];
    const double ta = comp(t, a), tc = comp(t, c);
    const double Ra = comp(Rt, a), Rc = comp(Rt, c);
    const double s1 = 0.5 * (comp(u, a) * tc + comp(u, c) * ta);
    const double s2 = 0.5 * (comp(w, a) * Rc + comp(w, c) * Ra);
    const double phi = 2.0 * iRt2 * (comp(rho, a) * Rc + comp(rho, c) * Ra + LR * Ra * Rc);
    const double dl = (a == c) ? 1.0 : 0.0;
    S[q] = iRt2 * (s1 - k1 * s2 - k2 * (dl + ta * tc + phi));
  }
}

// Stress (Pa) of the segment from -hl t to +hl t at observer r (relative to the
// segment centre), Burgers vector b.  Zero for the observer at the centre.
__device__ void segment_stress(V3 r, double hl, V3 t, V3 b, double mu, double nu, double out[6]) {
  if (r.x == 0.0 && r.y == 0.0 && r.z == 0.0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    return;
  }
  V3 RA = (-hl) * t - r;   // observer -> A
  V3 RB = hl * t - r;      // observer -> B
  const double cA = dot(RA, t) / sqrt(dot(RA, RA));
  const double cB = dot(RB, t) / sqrt(dot(RB, RB));
  if (cA + cB < 0.0) {     // observer ahead of the segment: use the other form of Eq. 6
    RA = (-1.0) * RA;
    RB = (-1.0) * RB;
  }
  const double k1 = 1.0 / (1.0 - nu);
  double SA[6], SB[6];
  eq6_end(RA, t, b, k1, SA);
  eq6_end(RB, t, b, k1, SB);
  const double pref = mu * 0.31830988618379067154;   // mu / pi
#pragma unroll
  for (int q = 0; q < 6; ++q) out[q] = pref * (SB[q] - SA[q]);
}

__device__ __forceinline__ double box_chord(const double hb[3], V3 t) {
  double dl = 1e300;
  const double tt[3] = {t.x, t.y, t.z};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (tt[a] != 0.0) dl = fmin(dl, hb[a] / fabs(tt[a]));
  return dl;
}

// g(r) for a box of edges hb: (V / dl) sigma^AB(r).
__device__ void box_coef(V3 r, const double hb[3], V3 t, V3 b, double mu, double nu, double out[6]) {
  const double dl = box_chord(hb, t);
  const double vol = hb[0] * hb[1] * hb[2];
  segment_stress(r, 0.5 * dl, t, b, mu, nu, out);
  const double f = vol / dl;
#pragma unroll
  for (int q = 0; q < 6; ++q) out[q] *= f;
}

__device__ __forceinline__ V3 offset_pos(const CoefGeom &g, int i, int j, int k) {
  return v3((double)i * g.h[0], (double)j * g.h[1], (double)k * g.h[2]);
}

// Near-field coefficient: the term of subcell difference index q of the
// (2m-1)^3 lattice, times its multiplicity.
__device__ __forceinline__ double near_term(const CoefGeom &g, V3 base, int q, V3 t, V3 b,
                                            double out[6]) {
  const int Dx = 2 * g.m[0] - 1, Dy = 2 * g.m[1] - 1;
  const int dx = q % Dx - (g.m[0] - 1);
  const int dy = (q / Dx) % Dy - (g.m[1] - 1);
  const int dz = q / (Dx * Dy) - (g.m[2] - 1);
  const double mult = (double)((g.m[0] - abs(dx)) * (g.m[1] - abs(dy)) * (g.m[2] - abs(dz)));
  const V3 r = base + v3(dx * g.hs[0], dy * g.hs[1], dz * g.hs[2]);
  box_coef(r, g.hs, t, b, g.mu, g.nu, out);
  return mult;
}

// Near field: |(i dx, j dy, k dz)|^2 < rn2, as ((x*x + y*y) + z*z) in round-to-nearest
// double without contraction (the same decision as the plain IEEE expression).
__device__ __forceinline__ bool near_dev(const CoefGeom &g, int i, int j, int k) {
  const double x = __dmul_rn((double)i, g.h[0]), y = __dmul_rn((double)j, g.h[1]), z = __dmul_rn((double)k, g.h[2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)) < g.rn2;
}

// Coefficient of one source cell at cell offset (i, j, k): subdivided near the target
// (mean over target subcells of the sum over source subcells), one segment otherwise.
__device__ void coef_cell(const CoefGeom &g, int i, int j, int k, V3 t, V3 b, double out[6]) {
  const V3 base = offset_pos(g, i, j, k);
  if (!near_dev(g, i, j, k)) {
    box_coef(base, g.h, t, b, g.mu, g.nu, out);
    return;
  }
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int D = (2 * g.m[0] - 1) * (2 * g.m[1] - 1) * (2 * g.m[2] - 1);
  for (int d = 0; d < D; ++d) {
    double s[6];
    const double mult = near_term(g, base, d, t, b, s);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += mult * s[c];
  }
  const double iM = 1.0 / (double)(g.m[0] * g.m[1] * g.m[2]);
#pragma unroll
  for (int c = 0; c < 6; ++c) out[c] = acc[c] * iM;
}

// With periodic boundary conditions (Sec. 4, Eq. 13): the sum over the replicas of the
// source cell, r_i + (k Lx, l Ly, 0), |k|, |l| <= n_shells.
// Replica sum of Eq. 13 around in-plane offset (i, j): images (i + kk nx, j + ll ny).
__device__ void coef_replicas(const CoefGeom &g, int i, int j, int k, V3 t, V3 b, double w, double acc[6]) {
  for (int kk = -g.n_shells; kk <= g.n_shells; ++kk)
    for (int ll = -g.n_shells; ll <= g.n_shells; ++ll) {
      double s[6];
      coef_cell(g, i + kk * g.nx, j + ll * g.ny, k, t, b, s);
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c] += w * s[c];
    }
}

// Minimal image of offset i for period n, in (-n/2, n/2]; at the tie n/2 (n even) also
// -n/2, each with weight 1/2.  Returns the number of images (1 or 2).
__device__ __forceinline__ int min_images(int i, int n, int r[2], double w[2]) {
  int m = i % n;
  if (m < 0) m += n;
  w[0] = 1.0;
  if (2 * m < n) { r[0] = m; return 1; }
  if (2 * m > n) { r[0] = m - n; return 1; }
  r[0] = m;
  r[1] = -m;
  w[0] = w[1] = 0.5;
  return 2;
}

__device__ void coef_any(const CoefGeom &g, int i, int j, int k, V3 t, V3 b, double out[6]) {
  if (g.n_shells <= 0) {
    coef_cell(g, i, j, k, t, b, out);
    return;
  }
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (!g.periodic) {
    coef_replicas(g, i, j, k, t, b, 1.0, acc);
  } else {             // shells centred on the minimal image, ties averaged (odd, periodic)
    int rx[2], ry[2];
    double wx[2], wy[2];
    const int nxr = min_images(i, g.nx, rx, wx), nyr = min_images(j, g.ny, ry, wy);
    for (int a = 0; a < nxr; ++a)
      for (int c2 = 0; c2 < nyr; ++c2) coef_replicas(g, rx[a], ry[c2], k, t, b, wx[a] * wy[c2], acc);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) out[c] = acc[c];
}

// ---- coefficients at listed offsets (parity queries) ------------------------
__global__ void k_table_at(CoefGeom g, V3 t, V3 b, long n, const int *ijk, double *out) {
  const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  double acc[6];
  coef_any(g, ijk[3 * q], ijk[3 * q + 1], ijk[3 * q + 2], t, b, acc);
#pragma unroll
  for (int c = 0; c < 6; ++c) out[6 * q + c] = acc[c];
}

// ---- padded table: far formula everywhere, gaps zero -------------------------
// tab[c][kz][ky][kx], kx < px.  Offset D maps to index D mod P; indices with no
// offset of magnitude < n (the padding gap) hold 0.
__global__ void k_table_far(CoefGeom g, V3 t, V3 b, int nx, int ny, int nz, int px, int py, int pz,
                            double *tab) {
  const long P = (long)px * py * pz;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= P) return;
  const int ix = (int)(idx % px), iy = (int)((idx / px) % py), iz = (int)(idx / ((long)px * py));
  const int i = ix < nx ? ix : ix - px;
  const int j = iy < ny ? iy : iy - py;
  const int k = iz < nz ? iz : iz - pz;
  double s[6] = {0, 0, 0, 0, 0, 0};
  if (i > -nx && j > -ny && k > -nz) {
    if (g.n_shells > 0) coef_any(g, i, j, k, t, b, s);     // replica sums include the near field
    else box_coef(offset_pos(g, i, j, k), g.h, t, b, g.mu, g.nu, s);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) tab[c * P + idx] = s[c];
}

// One block per near offset: reduce the subcell-difference lattice and overwrite.
__global__ void k_table_near(CoefGeom g, V3 t, V3 b, int px, int py, int pz, const int *ijk,
                             double *tab) {
  const int q = blockIdx.x;
  const int i = ijk[3 * q], j = ijk[3 * q + 1], k = ijk[3 * q + 2];
  const V3 base = offset_pos(g, i, j, k);
  const int D = (2 * g.m[0] - 1) * (2 * g.m[1] - 1) * (2 * g.m[2] - 1);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    double s[6];
    const double mult = near_term(g, base, d, t, b, s);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += mult * s[c];
  }
  __shared__ double red[32][6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    const long P = (long)px * py * pz;
    const int ix = i >= 0 ? i : i + px, iy = j >= 0 ? j : j + py, iz = k >= 0 ? k : k + pz;
    const long idx = ((long)iz * py + iy) * px + ix;
    tab[threadIdx.x * P + idx] = v / (double)(g.m[0] * g.m[1] * g.m[2]);
  }
}

// ---- FP64 FFT of the padded table -----------------------------------------
// R2C along x: lines of 2M reals -> M+1 complex (row pitch M+1).
template <int M>
__global__ void __launch_bounds__(128) k_r2c_lines_d(const double *in, long nlines, double2 *out,
                                                     const double2 *tw) {
  constexpr int W = 4, LD = W + 1, NT = 128;
  extern __shared__ double2 sm_d[];
  double2 *buf = sm_d;
  const long l0 = (long)blockIdx.x * W;
  const int tid = threadIdx.x;
  for (int e = tid; e < W * M; e += NT) {
    const int w = e / M, n = e % M;
    double2 z = make_double2(0.0, 0.0);
    if (l0 + w < nlines) {
      const double *src = in + (l0 + w) * (2L * M) + 2 * n;
      z = make_double2(src[0], src[1]);
    }
    buf[n * LD + w] = z;
  }
  __syncthreads();
  fft_tile<M, W, LD, NT, false, false, false>(buf, tw + tw_offset(M), tid);
  const double2 *tw2 = tw + tw_offset(2 * M);
  for (int e = tid; e < W * (M + 1); e += NT) {
    const int w = e / (M + 1), k = e % (M + 1);
    if (l0 + w >= nlines) continue;
    const double2 a = buf[(k % M) * LD + w];
    const double2 c = buf[((M - k) % M) * LD + w];
    // E = (Z[k] + conj Z[M-k]) / 2,  O = (Z[k] - conj Z[M-k]) / 2i,  X = E + W^k O
    const double2 E = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
    const double2 O = make_double2(0.5 * (a.y + c.y), -0.5 * (a.x - c.x));
    const double2 wk = (k < M) ? tw2[k] : make_double2(-1.0, 0.0);
    const double2 X = make_double2(E.x + wk.x * O.x - wk.y * O.y, E.y + wk.x * O.y + wk.y * O.x);
    out[(l0 + w) * (M + 1) + k] = X;
  }
}

// C2C along a strided axis: element n of column c of batch o at
// data[o * os + n * rs + c], c < ncols; tiles of W adjacent columns.
template <int P, int W>
__global__ void __launch_bounds__(256) k_cols_d(double2 *data, long os, long rs, long ncols,
                                                const double2 *tw) {
  constexpr int LD = W, NT = 256;
  extern __shared__ double2 sm_d[];
  double2 *buf = sm_d;
  const long tiles = (ncols + W - 1) / W;
  const long o = blockIdx.x / tiles;
  const long c0 = (blockIdx.x % tiles) * W;
  double2 *base = data + o * os + c0;
  const int tid = threadIdx.x;
  for (int e = tid; e < P * W; e += NT) {
    const int n = e / W, w = e % W;
    buf[n * LD + w] = (c0 + w < ncols) ? base[n * rs + w] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  fft_tile<P, W, LD, NT, false, false, false>(buf, tw + tw_offset(P), tid);
  for (int e = tid; e < P * W; e += NT) {
    const int n = e / W, w = e % W;
    if (c0 + w < ncols) base[n * rs + w] = buf[n * LD + w];
  }
}

// Imaginary part of the spectrum of component c of field e, scaled, into the layout
// the fused z pass reads:
//   shared-memory variant (zg = 0): kspec[tile][6][fe][pz][wz], tiles of wz columns;
//   register variant (zg = G > 0):  kspec[warp tile][6][fe][lane][E], E = pz / G, warp
//     tiles of 32/G columns, lane g * (32/G) + w holding kz = k1 + E bitrev_G(g), k1 < E;
//   three-stage variant (k_extract_four): see there.
// Main tiles cover (ky, kx < M) row by row; the Nyquist tiles (kx = M) follow.
__device__ __forceinline__ void store_val(float *p, double v) { *p = (float)v; }
__device__ __forceinline__ void store_val(__half *p, double v) { *p = __float2half_rn((float)v); }

// Largest |Im| of one spectrum (for the FP16 scale); bit patterns of non-negative
// doubles order like unsigned integers.
__global__ void k_absmax_imag(const double2 *spec, long n, unsigned long long *out) {
  double m = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(spec[i].y));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// FP16 scale of (component c, field e): the largest |value| after the FFT scaling.
__global__ void k_store_scale(const unsigned long long *amax, double scale, float *kscale, int idx) {
  const double m = __longlong_as_double((long long)*amax) * scale;
  kscale[idx] = m > 0.0 ? (float)m : 1.0f;
}

template <typename OT>
__global__ void k_extract(const double2 *spec, int M, int py, int pz, int wz, int zg, int fe, int e, int c,
                          double scale, const unsigned long long *amax, OT *kspec) {
  const int cw = zg > 0 ? 32 / zg : wz;                  // columns per tile
  const int E = zg > 0 ? pz / zg : 0;                     // registers per lane
  const long per_tile = zg > 0 ? 32L * E : (long)pz * wz;
  const long tiles_main = (long)py * (M / cw);
  const long tiles = tiles_main + py / cw;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= tiles * per_tile) return;
  const long tau = idx / per_tile;
  const int r = (int)(idx % per_tile);
  int kz, w;
  const long dst = ((tau * 6 + c) * fe + e) * per_tile + r;
  if (zg > 0) {
    const int lane = r / E, k1 = r % E, g = lane / cw;
    const int gb = zg == 4 ? (((g & 1) << 1) | (g >> 1))
                 : zg == 8 ? (((g & 1) << 2) | (g & 2) | (g >> 2)) : g;
    w = lane % cw;
    kz = k1 + E * gb;
  } else {
    kz = r / wz;
    w = r % wz;
  }
  int kx, ky;
  if (tau < tiles_main) {
    ky = (int)(tau / (M / cw));
    kx = (int)(tau % (M / cw)) * cw + w;
  } else {
    ky = (int)(tau - tiles_main) * cw + w;
    kx = M;
  }
  double v = spec[((long)kz * py + ky) * (M + 1) + kx].y * scale;
  if (amax != nullptr) {                 // FP16 storage: values relative to the largest
    const double m = __longlong_as_double((long long)*amax) * scale;
    if (m > 0.0) v /= m;
  }
  store_val(&kspec[dst], v);
}

// Imaginary part of the spectrum of component c of field e, scaled, into the layout
// the three-stage z pass reads (pz = 8 R1, tiles of W = wz columns): per stored tile s
// and component c, 16-byte chunks [j][thread t = k1 W + w], the value of
// (e, kz = k1 + R1 k2) at position (8 e + k2) % V of chunk j = (8 e + k2) / V, V values
// per chunk.  Stored tiles: the main tiles (ky, kx tile) row by row -- all of them, or
// those with ky <= py/2 when every field has the x-mirror parity (ZSym::xall) -- then
// the Nyquist tiles (kx = M).
template <typename OT>
__global__ void k_extract_four(const double2 *spec, Shape sh, int e, int c, double scale,
                               const unsigned long long *amax, OT *kspec) {
  constexpr int V = 16 / (int)sizeof(OT);
  const int W = sh.wz, R1 = sh.pz / 8, M = sh.M, py = sh.py, fe = sh.fe;
  const long per_tile = (long)sh.pz * W;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= zf_stored_tiles(sh) * per_tile) return;
  const long s = idx / per_tile;
  const int r = (int)(idx - s * per_tile), t = r / 8, k2 = r % 8, k1 = t / W, w = t % W, q = 8 * e + k2;
  const long ktiles = M / W;
  const long main_tiles = (long)(sh.zs.xall ? py / 2 + 1 : py) * ktiles;
  int kx, ky;
  if (s < main_tiles) {
    ky = (int)(s / ktiles);
    kx = (int)(s % ktiles) * W + w;
  } else {
    ky = (int)(s - main_tiles) * W + w;
    kx = M;
  }
  double v = spec[((long)(k1 + R1 * k2) * py + ky) * (M + 1) + kx].y * scale;
  if (amax != nullptr) {                 // FP16 storage: values relative to the largest
    const double m = __longlong_as_double((long long)*amax) * scale;
    if (m > 0.0) v /= m;
  }
  const size_t dst = (size_t)(s * 6 + c) * fe * per_tile + ((size_t)(q / V) * (R1 * W) + t) * V + q % V;
  store_val(&kspec[dst], v);
}

template <int M>
cudaError_t r2c_lines(const double *in, long nlines, double2 *out, const double2 *tw, cudaStream_t s) {
  const size_t smem = sizeof(double2) * M * 5;
  cudaError_t err = cudaFuncSetAttribute(k_r2c_lines_d<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  k_r2c_lines_d<M><<<(unsigned)((nlines + 3) / 4), 128, smem, s>>>(in, nlines, out, tw);
  return cudaGetLastError();
}

template <int P>
cudaError_t cols_fft(double2 *data, long nbatch, long os, long rs, long ncols, const double2 *tw,
                     cudaStream_t s) {
  constexpr int W = P >= 512 ? 4 : 8;
  const size_t smem = sizeof(double2) * P * W;
  cudaError_t err = cudaFuncSetAttribute(k_cols_d<P, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  const long tiles = (ncols + W - 1) / W;
  k_cols_d<P, W><<<(unsigned)(tiles * nbatch), 256, smem, s>>>(data, os, rs, ncols, tw);
  return cudaGetLastError();
}

cudaError_t r2c_dispatch(int M, const double *in, long nlines, double2 *out, const double2 *tw,
                         cudaStream_t s) {
  switch (M) {
    case 16: return r2c_lines<16>(in, nlines, out, tw, s);
    case 32: return r2c_lines<32>(in, nlines, out, tw, s);
    case 64: return r2c_lines<64>(in, nlines, out, tw, s);
    case 128: return r2c_lines<128>(in, nlines, out, tw, s);
    case 256: return r2c_lines<256>(in, nlines, out, tw, s);
    case 512: return r2c_lines<512>(in, nlines, out, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t cols_dispatch(int P, double2 *data, long nbatch, long os, long rs, long ncols,
                          const double2 *tw, cudaStream_t s) {
  switch (P) {
    case 16: return cols_fft<16>(data, nbatch, os, rs, ncols, tw, s);
    case 32: return cols_fft<32>(data, nbatch, os, rs, ncols, tw, s);
    case 64: return cols_fft<64>(data, nbatch, os, rs, ncols, tw, s);
    case 128: return cols_fft<128>(data, nbatch, os, rs, ncols, tw, s);
    case 256: return cols_fft<256>(data, nbatch, os, rs, ncols, tw, s);
    case 512: return cols_fft<512>(data, nbatch, os, rs, ncols, tw, s);
    case 1024: return cols_fft<1024>(data, nbatch, os, rs, ncols, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

CoefGeom coef_geom(const dds_ctx *ctx) {
  CoefGeom g;
  for (int a = 0; a < 3; ++a) g.h[a] = ctx->h[a];
  subcell_counts(ctx->h, g.m);
  for (int a = 0; a < 3; ++a) g.hs[a] = ctx->h[a] / (double)g.m[a];
  g.mu = ctx->mu;
  g.nu = ctx->nu;
  const double hmax = fmax(ctx->h[0], fmax(ctx->h[1], ctx->h[2]));
  const double rn = ctx->n_near * hmax;
  g.rn2 = rn * rn;
  g.nx = ctx->nx;
  g.ny = ctx->ny;
  g.n_shells = ctx->n_shells;
  g.periodic = ctx->pbc_periodic ? 1 : 0;
  return g;
}

}  // namespace

// -------------------------------------------------------------------------------
cudaError_t launch_table_at(const CoefGeom &g, const double t[3], const double b[3], long n,
                            const int *d_ijk, double *d_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nt = 128;
  k_table_at<<<(unsigned)((n + nt - 1) / nt), nt, 0, s>>>(g, v3(t[0], t[1], t[2]), v3(b[0], b[1], b[2]),
                                                           n, d_ijk, d_out);
  return cudaGetLastError();
}

CoefGeom make_coef_geom(const dds_ctx *ctx) { return coef_geom(ctx); }

int build_spectra(dds_ctx *ctx, cudaStream_t s) {
  const Shape &sh = ctx->shape;
  const int px = 2 * sh.M, py = sh.py, pz = sh.pz, M = sh.M;
  const long P = (long)px * py * pz;
  const long nspec = (long)(M + 1) * py * pz;
  const CoefGeom g = coef_geom(ctx);

  // near offsets (decided on the host, same expression as the definition)
  std::vector<int> near;                 // with replica shells the table kernel handles them
  if (ctx->n_near > 0.0 && ctx->n_shells == 0) {
    double hmax = fmax(ctx->h[0], fmax(ctx->h[1], ctx->h[2]));
    int lim[3] = {ctx->nx - 1, ctx->ny - 1, ctx->nz - 1};
    for (int a = 0; a < 3; ++a) {
      const double c = ceil(ctx->n_near * hmax / ctx->h[a]) + 1.0;
      if (c < lim[a]) lim[a] = (int)c;
    }
    for (int k = -lim[2]; k <= lim[2]; ++k)
      for (int j = -lim[1]; j <= lim[1]; ++j)
        for (int i = -lim[0]; i <= lim[0]; ++i)
          if (is_near(ctx->h, ctx->n_near, i, j, k)) {
            near.push_back(i);
            near.push_back(j);
            near.push_back(k);
          }
  }
  const int n_near = (int)(near.size() / 3);

  double *tab = nullptr;
  double2 *spec = nullptr;
  int *d_near = nullptr;
  unsigned long long *d_amax = nullptr;
  cudaError_t err = cudaMallocAsync(&tab, sizeof(double) * 6 * P, s);
  if (err == cudaSuccess) err = cudaMallocAsync(&d_amax, sizeof(unsigned long long), s);
  if (err == cudaSuccess) err = cudaMallocAsync(&spec, sizeof(double2) * nspec, s);
  if (err == cudaSuccess && n_near > 0) err = cudaMallocAsync(&d_near, sizeof(int) * 3 * n_near, s);
  if (err != cudaSuccess) {
    cudaFreeAsync(tab, s);
    cudaFreeAsync(spec, s);
    cudaFreeAsync(d_near, s);
    cudaFreeAsync(d_amax, s);
    cudaGetLastError();
    return fail(ctx, DDS_ERR_OOM, "build_kernels: cannot allocate %.2f GB of FP64 table workspace: %s",
                (sizeof(double) * 6.0 * P + sizeof(double2) * (double)nspec) / 1e9, cudaGetErrorString(err));
  }
  if (n_near > 0)
    err = cudaMemcpyAsync(d_near, near.data(), sizeof(int) * 3 * n_near, cudaMemcpyHostToDevice, s);

  const double scale = 1.0 / ((double)px * (double)py * (double)pz);
  for (int e = 0; e < ctx->fe && err == cudaSuccess; ++e) {
    const V3 t = v3(ctx->field_t[3 * e], ctx->field_t[3 * e + 1], ctx->field_t[3 * e + 2]);
    const V3 b = v3(ctx->field_b[3 * e], ctx->field_b[3 * e + 1], ctx->field_b[3 * e + 2]);
    k_table_far<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(g, t, b, ctx->nx, ctx->ny, ctx->nz, px, py,
                                                             pz, tab);
    err = cudaGetLastError();
    if (err == cudaSuccess && n_near > 0) {
      k_table_near<<<n_near, 128, 0, s>>>(g, t, b, px, py, pz, d_near, tab);
      err = cudaGetLastError();
    }
    for (int c = 0; c < 6 && err == cudaSuccess; ++c) {
      err = r2c_dispatch(M, tab + c * P, (long)py * pz, spec, ctx->tw.f64, s);
      if (err == cudaSuccess)   // y: batches kz, rows ky (pitch M+1), columns kx
        err = cols_dispatch(py, spec, pz, (long)py * (M + 1), M + 1, M + 1, ctx->tw.f64, s);
      if (err == cudaSuccess)   // z: one batch, rows kz, columns (ky, kx)
        err = cols_dispatch(pz, spec, 1, 0, (long)py * (M + 1), (long)py * (M + 1), ctx->tw.f64, s);
      if (err == cudaSuccess) {
        const long n = sh.zfour ? zf_stored_tiles(sh) * pz * sh.wz : (long)py * (M + 1) * pz;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        if (ctx->spectra_fp16) {
          err = cudaMemsetAsync(d_amax, 0, sizeof(unsigned long long), s);
          if (err == cudaSuccess) {
            k_absmax_imag<<<1024, 256, 0, s>>>(spec, nspec, d_amax);
            k_store_scale<<<1, 1, 0, s>>>(d_amax, scale, ctx->kscale, c * sh.fe + e);
            __half *out = static_cast<__half *>(ctx->kspec);
            if (sh.zfour) k_extract_four<__half><<<blocks, 256, 0, s>>>(spec, sh, e, c, scale, d_amax, out);
            else k_extract<__half><<<blocks, 256, 0, s>>>(spec, M, py, pz, sh.wz, sh.zreg_g, sh.fe, e, c, scale,
                                                          d_amax, out);
            err = cudaGetLastError();
          }
        } else {
          float *out = static_cast<float *>(ctx->kspec);
          if (sh.zfour) k_extract_four<float><<<blocks, 256, 0, s>>>(spec, sh, e, c, scale, nullptr, out);
          else k_extract<float><<<blocks, 256, 0, s>>>(spec, M, py, pz, sh.wz, sh.zreg_g, sh.fe, e, c, scale,
                                                       nullptr, out);
          err = cudaGetLastError();
        }
      }
    }
  }
  cudaFreeAsync(tab, s);
  cudaFreeAsync(spec, s);
  cudaFreeAsync(d_near, s);
  cudaFreeAsync(d_amax, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return fail(ctx, DDS_ERR_CUDA, "build_kernels: %s", cudaGetErrorString(err));
  return DDS_OK;
}

}  // namespace dds
