/*
 * FP64 CPU oracle for the dislocation-density stress evaluation
 * (Berkov & Gorn, "Dislocation-induced stress in polycrystalline materials").
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow definition of what the GPU path
 * computes.  It is loaded by the tests, the smoke check and the CPU-baseline
 * leg of the benchmark, never by the product path, and it shares no code with
 * the CUDA sources.
 *
 * What it computes, step by step, in the paper's order:
 *   1. the stress of a straight dislocation segment, Eq. 6 with Eq. 7a/7b
 *      (and, as an independent cross-check for t = z, Eq. 4a-4c with Eq. 5);
 *   2. the interaction coefficient per unit density, Eq. 9b applied to a segment
 *      threading the source cell through its centre, times the cell volume
 *      (Eq. 2, Eq. 10): G = (dV / dl) * sigma^AB;
 *   3. near cells (Sec. 2.3): target and source cells split into near-cubic
 *      subcells, G = mean over target subcells of the sum over source subcells;
 *   4. the self pair (observer at the source segment's midpoint) contributes 0
 *      (Sec. 2.3, last remark);
 *   5. Eq. 10 summed over families (Eq. 3b) by direct summation over all cells.
 *
 * Readings of points the paper leaves open (each one listed in the design notes):
 *   - offsets are observer minus source (Eq. 10, Sec. 2.1);
 *   - Eq. 6 is evaluated from each endpoint, with the mu/pi prefactor as printed;
 *     the vector R may be taken either way between observer and line point, the
 *     two forms differing by a constant per endpoint exactly like the region sets
 *     of Eq. 4 (Sec. 2.2); one form is used for both endpoints of a segment and it
 *     is the one whose R + R.t stays away from zero;
 *   - dl of Eq. 9b is the chord of the (sub)cell through its centre along t;
 *   - subcell counts: per axis the integer m >= 1 minimising |ln((h/m)/h_min)|,
 *     ties to the larger m; near cells: |offset| < n_near * max(h);
 *   - the near-field coefficient is the mean over target subcells of the sum over
 *     source subcells.
 *
 * Compiled without fast-math and without floating-point contraction.
 * "Parity unpinned": none — every function here is pinned by tests against
 * closed forms, identities or brute force (see tests/test_oracle_pins.py).
 */
#include "dds_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Eq. 4a-4c: vertical semi-infinite dislocation ending at z', observer below  */
/* ------------------------------------------------------------------------- */
static void eq4_semi_infinite(const double obs[3], double zp, const double b[3],
                              double mu, double nu, double s[6]) {
  const double x = obs[0], y = obs[1], z = obs[2];
  const double lam = zp - z;                                  /* Eq. 4b */
  const double R = sqrt(x * x + y * y + (z - zp) * (z - zp));
  const double R3 = R * R * R;
  const double Rl2 = R * (R + lam);                           /* R_{lambda+}^2 */
  const double Sx = x * x / (R * R) + x * x / Rl2;            /* Eq. 4c */
  const double Sy = y * y / (R * R) + y * y / Rl2;
  const double s0 = mu / (4.0 * PI * (1.0 - nu));
  const double bx = b[0], by = b[1], bz = b[2];
  double xx = bx * y / Rl2 * (1.0 + Sx) + by * x / Rl2 * (1.0 - Sx);
  double yy = -bx * y / Rl2 * (1.0 - Sy) - by * x / Rl2 * (1.0 + Sy);
  double zz = (bx * y - by * x) * (2.0 * nu / Rl2 + lam / R3);
  double xy = -bx * x / Rl2 * (1.0 - Sy) + by * y / Rl2 * (1.0 - Sx);
  double xz = -bx * x * y / R3 - by * (nu / R - x * x / R3) + bz * y * (1.0 - nu) / Rl2;
  double yz = bx * (nu / R - y * y / R3) + by * x * y / R3 - bz * x * (1.0 - nu) / Rl2;
  s[0] = s0 * xx; s[1] = s0 * yy; s[2] = s0 * zz;
  s[3] = s0 * xy; s[4] = s0 * xz; s[5] = s0 * yz;
}

void orc_segment_eq4(const double obs[3], double zA, double zB, const double b[3],
                     double mu, double nu, double out[6]) {
  double sA[6], sB[6];
  eq4_semi_infinite(obs, zA, b, mu, nu, sA);
  eq4_semi_infinite(obs, zB, b, mu, nu, sB);
  for (int c = 0; c < 6; ++c) out[c] = sB[c] - sA[c];         /* Eq. 5 */
}

/* ------------------------------------------------------------------------- */
/* Eq. 6 / 7a / 7b: general straight segment                                  */
/* ------------------------------------------------------------------------- */
static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* The bracket of Eq. 6 for one endpoint, divided by R_t^2 (the mu/pi factor is
 * applied by the caller).  R: vector between observer and the endpoint. */
static void eq6_endpoint(const double R[3], const double t[3], const double b[3],
                         double nu, double S[3][3]) {
  const double Rn = sqrt(dot3(R, R));
  const double L = dot3(R, t);
  double Rt[3], rho[3];
  for (int a = 0; a < 3; ++a) {
    Rt[a] = R[a] + Rn * t[a];
    rho[a] = R[a] - L * t[a];
  }
  const double Rt2 = dot3(Rt, Rt);
  double bxRt[3], bxt[3], Rtxt[3];
  cross3(b, Rt, bxRt);
  cross3(b, t, bxt);
  cross3(Rt, t, Rtxt);
  const double trip = dot3(b, Rtxt);                          /* (b, R_t, t), Eq. 7b */
  const double k1 = 1.0 / (1.0 - nu);
  const double k2 = trip / (2.0 * (1.0 - nu));
  for (int a = 0; a < 3; ++a) {
    for (int c = 0; c < 3; ++c) {
      const double sym1 = 0.5 * (bxRt[a] * t[c] + bxRt[c] * t[a]);   /* [b R_t t]^sym */
      const double sym2 = 0.5 * (bxt[a] * Rt[c] + bxt[c] * Rt[a]);   /* [b t R_t]^sym */
      const double phi = (2.0 / Rt2) *
                         (rho[a] * Rt[c] + rho[c] * Rt[a] + (L / Rn) * Rt[a] * Rt[c]); /* Eq. 7a */
      const double delta = (a == c) ? 1.0 : 0.0;
      S[a][c] = (sym1 - k1 * sym2 - k2 * (delta + t[a] * t[c] + phi)) / Rt2;
    }
  }
}

int orc_segment_eq6(const double obs[3], const double A[3], const double B[3],
                    const double t[3], const double b[3], double mu, double nu,
                    int form, double out[6]) {
  double RA[3], RB[3];
  for (int a = 0; a < 3; ++a) {
    RA[a] = A[a] - obs[a];
    RB[a] = B[a] - obs[a];
  }
  const double nA = sqrt(dot3(RA, RA)), nB = sqrt(dot3(RB, RB));
  if (nA == 0.0 || nB == 0.0) {            /* observer at an endpoint: no finite value */
    for (int c = 0; c < 6; ++c) out[c] = 0.0;
    return 1;
  }
  double mid[3];
  for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (A[a] + B[a]) - obs[a];
  if (mid[0] == 0.0 && mid[1] == 0.0 && mid[2] == 0.0) {   /* self pair */
    for (int c = 0; c < 6; ++c) out[c] = 0.0;
    return 1;
  }
  if (form == 0) {
    /* R = (point - observer) is regular unless the observer lies ahead of the
     * point along t; then the other form is used (cosines summed over both ends). */
    const double cA = dot3(RA, t) / nA, cB = dot3(RB, t) / nB;
    form = (cA + cB >= 0.0) ? -1 : +1;
  }
  if (form == +1) {                           /* R from the line point to the observer */
    for (int a = 0; a < 3; ++a) { RA[a] = -RA[a]; RB[a] = -RB[a]; }
  }
  double SA[3][3], SB[3][3];
  eq6_endpoint(RA, t, b, nu, SA);
  eq6_endpoint(RB, t, b, nu, SB);
  const double pref = mu / PI;
  out[0] = pref * (SB[0][0] - SA[0][0]);
  out[1] = pref * (SB[1][1] - SA[1][1]);
  out[2] = pref * (SB[2][2] - SA[2][2]);
  out[3] = pref * (SB[0][1] - SA[0][1]);
  out[4] = pref * (SB[0][2] - SA[0][2]);
  out[5] = pref * (SB[1][2] - SA[1][2]);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2.3: subcells, chord, interaction coefficient                          */
/* ------------------------------------------------------------------------- */
void orc_subcells(const double h[3], int m[3]) {
  double hmin = h[0];
  if (h[1] < hmin) hmin = h[1];
  if (h[2] < hmin) hmin = h[2];
  for (int a = 0; a < 3; ++a) {
    /* minimise |ln((h/m)/hmin)| over integers m >= 1; ties -> larger m */
    int best = 1;
    double bestv = fabs(log((h[a] / 1.0) / hmin));
    for (int mm = 2; mm <= 4096; ++mm) {
      const double v = fabs(log((h[a] / (double)mm) / hmin));
      if (v <= bestv) { best = mm; bestv = v; }
      if ((h[a] / (double)mm) < hmin * 0.25) break;
    }
    m[a] = best;
  }
}

double orc_chord(const double h[3], const double t[3]) {
  double dl = INFINITY;
  for (int a = 0; a < 3; ++a) {
    if (t[a] != 0.0) {
      const double v = h[a] / fabs(t[a]);
      if (v < dl) dl = v;
    }
  }
  return dl;
}

/* Eq. 9b times the cell volume: stress at observer offset r from the centre of a box
 * of edges hb threaded through its centre by one segment along t, per unit density. */
static void box_coefficient(const double r[3], const double hb[3], const double t[3],
                            const double b[3], double mu, double nu, double out[6]) {
  const double dl = orc_chord(hb, t);
  const double vol = hb[0] * hb[1] * hb[2];
  double A[3], B[3];
  for (int a = 0; a < 3; ++a) {
    A[a] = -0.5 * dl * t[a];
    B[a] = 0.5 * dl * t[a];
  }
  double s[6];
  orc_segment_eq6(r, A, B, t, b, mu, nu, 0, s);
  for (int c = 0; c < 6; ++c) out[c] = (vol / dl) * s[c];
}

void orc_interaction(const orc_geom *g, int i, int j, int k, const double t[3],
                     const double b[3], double out[6]) {
  const double *h = g->h;
  const double d[3] = {(double)i * h[0], (double)j * h[1], (double)k * h[2]};
  double hmax = h[0];
  if (h[1] > hmax) hmax = h[1];
  if (h[2] > hmax) hmax = h[2];
  const double rn = g->n_near * hmax;
  const int near = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < rn * rn;
  if (!near) {
    box_coefficient(d, h, t, b, g->mu, g->nu, out);
    return;
  }
  int m[3];
  orc_subcells(h, m);
  const double hs[3] = {h[0] / m[0], h[1] / m[1], h[2] / m[2]};
  const int M = m[0] * m[1] * m[2];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  /* every target subcell u, every source subcell v */
  for (int uz = 0; uz < m[2]; ++uz)
  for (int uy = 0; uy < m[1]; ++uy)
  for (int ux = 0; ux < m[0]; ++ux) {
    const double u[3] = {(ux + 0.5) * hs[0] - 0.5 * h[0], (uy + 0.5) * hs[1] - 0.5 * h[1],
                         (uz + 0.5) * hs[2] - 0.5 * h[2]};
    for (int vz = 0; vz < m[2]; ++vz)
    for (int vy = 0; vy < m[1]; ++vy)
    for (int vx = 0; vx < m[0]; ++vx) {
      const double v[3] = {(vx + 0.5) * hs[0] - 0.5 * h[0], (vy + 0.5) * hs[1] - 0.5 * h[1],
                           (vz + 0.5) * hs[2] - 0.5 * h[2]};
      const double r[3] = {d[0] + u[0] - v[0], d[1] + u[1] - v[1], d[2] + u[2] - v[2]};
      double s[6];
      box_coefficient(r, hs, t, b, g->mu, g->nu, s);
      for (int c = 0; c < 6; ++c) acc[c] += s[c];
    }
  }
  for (int c = 0; c < 6; ++c) out[c] = acc[c] / (double)M;
}

/* Sec. 4, Eq. 12 and Eq. 13: every replica of the source cell, r_i + (k Lx, l Ly, 0),
 * contributes its coefficient at its own separation from the target. */
void orc_interaction_pbc(const orc_geom *g, int i, int j, int k, const double t[3], const double b[3],
                         double out[6]) {
  const int n = g->n_shells;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int kk = -n; kk <= n; ++kk)
    for (int ll = -n; ll <= n; ++ll) {
      double s[6];
      orc_interaction(g, i + kk * g->nx, j + ll * g->ny, k, t, b, s);
      for (int c = 0; c < 6; ++c) acc[c] += s[c];
    }
  for (int c = 0; c < 6; ++c) out[c] = acc[c];
}

/* Images of the offset along one axis of period n: the minimal image r in (-n/2, n/2]
 * and, at the tie r = n/2 (n even), also -n/2 with weight 1/2 each. */
static int minimal_images(int i, int n, int r[2], double w[2]) {
  int m = i % n;
  if (m < 0) m += n;
  if (2 * m < n) {
    r[0] = m;
  } else if (2 * m > n) {
    r[0] = m - n;
  } else {
    r[0] = m;
    r[1] = -m;
    w[0] = w[1] = 0.5;
    return 2;
  }
  w[0] = 1.0;
  return 1;
}

void orc_interaction_periodic(const orc_geom *g, int i, int j, int k, const double t[3], const double b[3],
                              double out[6]) {
  int rx[2], ry[2];
  double wx[2], wy[2];
  const int nxr = minimal_images(i, g->nx, rx, wx), nyr = minimal_images(j, g->ny, ry, wy);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < nxr; ++a)
    for (int c2 = 0; c2 < nyr; ++c2) {
      double s[6];
      orc_interaction_pbc(g, rx[a], ry[c2], k, t, b, s);
      for (int c = 0; c < 6; ++c) acc[c] += wx[a] * wy[c2] * s[c];
    }
  for (int c = 0; c < 6; ++c) out[c] = acc[c];
}

static void coefficient(const orc_geom *g, int i, int j, int k, const double t[3], const double b[3],
                        double out[6]) {
  if (g->n_shells > 0 && g->periodic) orc_interaction_periodic(g, i, j, k, t, b, out);
  else if (g->n_shells > 0) orc_interaction_pbc(g, i, j, k, t, b, out);
  else orc_interaction(g, i, j, k, t, b, out);
}

void orc_gtable(const orc_geom *g, const double t[3], const double b[3], double *out) {
  const int Ix = 2 * g->nx - 1, Iy = 2 * g->ny - 1, Iz = 2 * g->nz - 1;
  const long n = (long)Ix * Iy * Iz;
#pragma omp parallel for schedule(dynamic, 64)
  for (long q = 0; q < n; ++q) {
    const int i = (int)(q % Ix) - (g->nx - 1);
    const int j = (int)((q / Ix) % Iy) - (g->ny - 1);
    const int k = (int)(q / ((long)Ix * Iy)) - (g->nz - 1);
    coefficient(g, i, j, k, t, b, out + 6 * q);
  }
}

/* ------------------------------------------------------------------------- */
/* Eq. 10 + Eq. 3b: direct summation                                          */
/* ------------------------------------------------------------------------- */
void orc_stress_direct(const orc_geom *g, int F, const double *t, const double *b,
                       const double *rho, long ntargets, const long *targets,
                       int use_table, double *out) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const long N = (long)nx * ny * nz;
  const int Ix = 2 * nx - 1, Iy = 2 * ny - 1;
  memset(out, 0, sizeof(double) * 6 * (size_t)ntargets);
  double *table = NULL;
  if (use_table) {
    table = (double *)malloc(sizeof(double) * 6 * (size_t)Ix * Iy * (2 * nz - 1));
  }
  for (int f = 0; f < F; ++f) {
    const double *tf = t + 3 * f, *bf = b + 3 * f;
    const double *rf = rho + (size_t)f * N;
    if (table) orc_gtable(g, tf, bf, table);
    const int by_target = ntargets >= 4L * orc_num_threads();
    if (by_target) {
#pragma omp parallel for schedule(dynamic, 1)
      for (long q = 0; q < ntargets; ++q) {
        const long tq = targets[q];
        const int ti = (int)(tq % nx), tj = (int)((tq / nx) % ny), tk = (int)(tq / ((long)nx * ny));
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (long s = 0; s < N; ++s) {
          const double dens = rf[s];
          if (dens == 0.0) continue;
          const int si = (int)(s % nx), sj = (int)((s / nx) % ny), sk = (int)(s / ((long)nx * ny));
          double G[6];
          if (table) {
            const long o = ((long)(tk - sk + nz - 1) * Iy + (tj - sj + ny - 1)) * Ix + (ti - si + nx - 1);
            for (int c = 0; c < 6; ++c) G[c] = table[6 * o + c];
          } else {
            coefficient(g, ti - si, tj - sj, tk - sk, tf, bf, G);
          }
          for (int c = 0; c < 6; ++c) acc[c] += G[c] * dens;
        }
        for (int c = 0; c < 6; ++c) out[6 * q + c] += acc[c];
      }
    } else {
      for (long q = 0; q < ntargets; ++q) {
        const long tq = targets[q];
        const int ti = (int)(tq % nx), tj = (int)((tq / nx) % ny), tk = (int)(tq / ((long)nx * ny));
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : a0, a1, a2, a3, a4, a5)
        for (long s = 0; s < N; ++s) {
          const double dens = rf[s];
          if (dens == 0.0) continue;
          const int si = (int)(s % nx), sj = (int)((s / nx) % ny), sk = (int)(s / ((long)nx * ny));
          double G[6];
          if (table) {
            const long o = ((long)(tk - sk + nz - 1) * Iy + (tj - sj + ny - 1)) * Ix + (ti - si + nx - 1);
            for (int c = 0; c < 6; ++c) G[c] = table[6 * o + c];
          } else {
            coefficient(g, ti - si, tj - sj, tk - sk, tf, bf, G);
          }
          a0 += G[0] * dens; a1 += G[1] * dens; a2 += G[2] * dens;
          a3 += G[3] * dens; a4 += G[4] * dens; a5 += G[5] * dens;
        }
        out[6 * q + 0] += a0; out[6 * q + 1] += a1; out[6 * q + 2] += a2;
        out[6 * q + 3] += a3; out[6 * q + 4] += a4; out[6 * q + 5] += a5;
      }
    }
  }
  free(table);
}
