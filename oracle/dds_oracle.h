/*
 * FP64 CPU oracle for the dislocation-density stress evaluation
 * (Berkov & Gorn, "Dislocation-induced stress in polycrystalline materials").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and the CUDA path never calls it.
 *
 * Conventions: SI units; stress components ordered xx, yy, zz, xy, xz, yz;
 * density fields rho[f][k][j][i] (x fastest) in lines per m^2; cell (i,j,k)
 * centred at ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz).
 */
#ifndef DDS_ORACLE_H
#define DDS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;
  double h[3];     /* cell edge lengths dx, dy, dz (m) */
  double mu, nu;   /* shear modulus (Pa), Poisson ratio */
  double n_near;   /* near field: |offset| < n_near * max(h) is subdivided (Sec. 2.3) */
  int n_shells;    /* in-plane periodic boundary conditions with replica shells |k|,|l| <= n_shells
                      (Sec. 4, Eq. 12-13); 0: open boundary */
  int periodic;    /* with n_shells > 0: 1 = the replica shells are centred on each source's
                      minimal image (periodic reading, see orc_interaction_periodic); 0 = on
                      the in-system offset (orc_interaction_pbc) */
} orc_geom;

/* Eq. 4a-4c with Eq. 5: stress of a segment parallel to z from (0,0,zA) to
 * (0,0,zB), Burgers vector b, observer obs (must be off the z axis).  out[6]. */
void orc_segment_eq4(const double obs[3], double zA, double zB, const double b[3],
                     double mu, double nu, double out[6]);

/* Eq. 6 / 7a / 7b: stress of a straight segment A->B with unit line direction t
 * and Burgers vector b.  form = +1 takes R from the line point to the observer,
 * form = -1 from the observer to the line point; form = 0 chooses per segment the
 * form whose R + R.t stays away from zero at both ends (Eq. 6 evaluated |_A^B).  Returns 1 (and zeros) if the
 * observer coincides with the segment midpoint, else 0. */
int orc_segment_eq6(const double obs[3], const double A[3], const double B[3],
                    const double t[3], const double b[3], double mu, double nu,
                    int form, double out[6]);

/* Subcell counts per axis (Sec. 2.3: subcells as close to cubic as possible). */
void orc_subcells(const double h[3], int m[3]);

/* Chord of a box of edges h through its centre along unit t. */
double orc_chord(const double h[3], const double t[3]);

/* Interaction coefficient G(Delta) for one family (t, b): the stress at the centre of
 * cell r0 per unit density (m^-2) in a source cell r_i with r0 - r_i = (i dx, j dy,
 * k dz) (Eq. 9b, Eq. 10; near cells subdivided, Sec. 2.3).  out[6]. */
void orc_interaction(const orc_geom *g, int i, int j, int k, const double t[3],
                     const double b[3], double out[6]);

/* Periodic boundary conditions in x and y (Sec. 4): F(Delta) = sum over replicas of the
 * source cell, Eq. 13, |k|, |l| <= n_shells: sum_{k,l} G(i + k nx, j + l ny, k_z).  out[6]. */
void orc_interaction_pbc(const orc_geom *g, int i, int j, int k, const double t[3], const double b[3],
                         double out[6]);

/* Full table over offsets i in [-(nx-1), nx-1] (same for j, k), layout
 * out[((k + nz-1) * (2ny-1) + (j + ny-1)) * (2nx-1) + (i + nx-1)][6]. */
void orc_gtable(const orc_geom *g, const double t[3], const double b[3], double *out);

/* Periodic reading of Sec. 4's replica sum: for the in-plane offset (i, j) taken modulo
 * (nx, ny), the images of the source column nearest to the target -- the minimal image
 * i* in (-nx/2, nx/2] shifted by m nx, |m| <= n_shells, and likewise in y -- summed;
 * where the offset is exactly half a period (nx even, i* = nx/2) the two image sets
 * starting at +nx/2 and -nx/2 are averaged, so the coefficients stay odd.  Exactly
 * periodic in i and j; the same n_shells -> infinity limit as orc_interaction_pbc.
 * out[6]. */
void orc_interaction_periodic(const orc_geom *g, int i, int j, int k, const double t[3], const double b[3],
                              double out[6]);

/* Eq. 10 summed over families (Eq. 12 with n_shells > 0): sigma at the listed target cells (linear index
 * (k*ny + j)*nx + i) by direct summation over all source cells.
 * rho: [F][nz][ny][nx]; out: [ntargets][6].  use_table != 0 builds each family's
 * full table first (small grids), else coefficients are evaluated per pair. */
void orc_stress_direct(const orc_geom *g, int F, const double *t, const double *b,
                       const double *rho, long ntargets, const long *targets,
                       int use_table, double *out);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
