/*
 * dds.h — C ABI of the GB300 dislocation-density stress library (libdds.so).
 *
 * Computes the stress created by site-dependent densities of straight
 * dislocations on a rectangular grid of (possibly strongly shape-anisotropic)
 * cells, following Berkov & Gorn, "Dislocation-induced stress in polycrystalline
 * materials: mesoscopic simulations in the dislocation density formalism":
 *
 *   sigma_c(r0) = sum_f sum_i G_c^f(r0 - r_i) rho_f(r_i)              (Eq. 10, Eq. 3b)
 *
 * over all cells r_i of the grid (open boundary: the sample is embedded in an
 * infinite elastic continuum, Sec. 3).  G_c^f is the stress at r0 per unit
 * density of family f = (line direction t, Burgers vector b) in the cell at r_i:
 * (cell volume / dl) times the stress of one straight segment of length dl
 * threading that cell through its centre (Eq. 9b with Eq. 6/7), and for cells
 * closer than the near-field radius the mean over near-cubic target subcells of
 * the sum over source subcells (Sec. 2.3).  The sum is evaluated as a
 * zero-padded FFT convolution (Sec. 2.3, first remark on Eq. 10).
 *
 * Conventions (all entry points):
 *   - SI units: lengths in m, moduli in Pa, densities in dislocation lines per m^2
 *     (1 cm^-2 = 1e4 m^-2), stress in Pa.
 *   - Grids are C-ordered [nz][ny][nx], x fastest; cell (i,j,k) is centred at
 *     ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz).
 *   - Stress components are ordered xx, yy, zz, xy, xz, yz.
 *   - The library never aborts and never prints.  Every entry point returns
 *     DDS_OK (0) or a negative DDS_ERR_* code; dds_last_error() then holds a
 *     one-line message.  A context is not thread-safe: use one context per host
 *     thread, and at most one stress evaluation in flight per context.
 *   - Device pointers are CUDA device memory on the context's device (for
 *     example torch tensors' data_ptr()); the caller owns them.  The library
 *     owns everything it allocates and frees it in dds_destroy().
 */
#ifndef DDS_H
#define DDS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dds_ctx dds_ctx;

enum {
  DDS_OK = 0,
  DDS_ERR_INVALID_ARG = -1,   /* bad pointer, size, direction or option value      */
  DDS_ERR_NOT_READY = -2,     /* geometry/families missing or kernels not built   */
  DDS_ERR_OOM = -3,           /* device allocation failed                          */
  DDS_ERR_CUDA = -4,          /* a CUDA runtime call or kernel launch failed       */
  DDS_ERR_TIMEOUT = -5,       /* a bounded device wait gave up                     */
  DDS_ERR_UNSUPPORTED = -6    /* valid request outside the library's limits        */
};

/* Density element types accepted by dds_stress. */
enum { DDS_F32 = 0, DDS_BF16 = 1 };

/* Option keys for dds_set_option. */
enum {
  DDS_OPT_NEAR_RADIUS = 1, /* near-field radius in units of the largest cell edge
                              (Sec. 2.3 "several nearest-neighbour shells"); default 3;
                              0 disables subdivision.  Invalidates built kernels. */
  DDS_OPT_Z_LANES = 2,     /* schedule of the fused z pass: 0 = automatic (default);
                              -1 = shared-memory tiles; -2 = three-stage register kernel
                              (padded z size 128 or 256, <= 6 combined fields; the
                              automatic choice there); 1, 2, 4, 8 = register-only kernel
                              with that many lanes per (kx, ky) column (needs padded
                              z size <= 64 and <= 4 combined fields).  Same result up to
                              rounding; a tuning knob.  A schedule the grid cannot take
                              fails dds_build_kernels with DDS_ERR_UNSUPPORTED.
                              Invalidates built kernels. */
  DDS_OPT_PBC_SHELLS = 4,  /* in-plane periodic boundary conditions (Sec. 4): n > 0 makes
                              every coefficient the sum over the replicas of the source
                              cell, r_i + (k Lx, l Ly, 0) with |k|, |l| <= n (Eq. 12-13;
                              the paper finds 15-20 shells accurate to 3%); the table
                              build costs (2n + 1)^2 times more.  0 (default): open
                              boundary.  Invalidates built kernels. */
  DDS_OPT_PBC_PERIODIC = 5,/* with DDS_OPT_PBC_SHELLS = n > 0: 1 centres the replica shells
                              of Sec. 4 on each source's minimal image (the in-plane offset
                              taken modulo the period; at exactly half a period the two
                              image sets averaged), so sigma is a cyclic convolution in x and
                              y; the FFT is then unpadded in y (ny must be a power of two
                              >= 32), which halves the y and z passes' work.  0 (default):
                              shells centred on the in-system offset, zero-padded FFT.  Both
                              readings share the n -> infinity limit.  Invalidates built
                              kernels. */
  DDS_OPT_YX_FUSED = 6,    /* 1: run the inverse y and x transforms as one pass, one
                              thread-block cluster per output plane (c, z) exchanging the
                              plane through distributed shared memory, where the plane
                              fits (zero-padded y, padded sizes py x px/2 of 256 x 128,
                              512 x 128, 256 x 256 or 512 x 256) and the device can hold
                              the cluster; elsewhere two separate passes.  It moves 44%
                              fewer bytes but is slower on GB300 (GaN layer 256x256x128:
                              0.51 ms against 0.37 for the two passes).  0 (default):
                              separate passes.  Same result up to rounding.  Invalidates
                              built kernels. */
  DDS_OPT_SPECTRA_FP16 = 3,/* 1: store the cached kernel spectra as FP16 with one FP32
                              scale per (component, field) -- half the bytes of the
                              dominant pass; arithmetic stays FP32.  Error: about 1e-4
                              relative L2 against the FP64 sum (tested bound 5e-4)
                              instead of 1e-5.  0 (default): FP32.  Invalidates built
                              kernels. */
};

/* Compile-time limits of the library. */
#define DDS_MAX_NXY 512        /* nx, ny <= 512 (zero-padded FFT sizes <= 1024)      */
#define DDS_MAX_NZ 256         /* nz <= 256 (zero-padded FFT size <= 512)            */
#define DDS_MAX_FAMILIES 64    /* families per context                               */
#define DDS_MAX_FIELDS 12      /* effective fields after collapsing families         */

/* Create a context bound to CUDA device `cuda_device`: the holder of one problem of
 * Sec. 2.1 (a grid of cells, the elastic medium, the dislocation families) and of its
 * interaction coefficients, which the paper computes once per geometry and reuses
 * for every density (Sec. 2.3, remark on the coefficient table).  *out receives the
 * handle (NULL on failure).  Errors: INVALID_ARG (out NULL or no such device), CUDA
 * (the device cannot be made current), OOM. */
int dds_create(dds_ctx **out, int cuda_device);

/* Grid shape and cell edges (m), shear modulus mu (Pa) and Poisson ratio nu of the
 * isotropic medium (Eq. 4: sigma_0 = mu / 4 pi (1 - nu)).  1 <= nx, ny <= DDS_MAX_NXY,
 * 1 <= nz <= DDS_MAX_NZ,
 * cell edges > 0, mu > 0, -1 < nu < 0.5.  Invalidates built kernels. */
int dds_set_geometry(dds_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                     double mu, double nu);

/* F dislocation families (Eq. 3b): t[3f..3f+2] the line direction (normalised
 * here; must be non-zero), b[3f..3f+2] the Burgers vector in m.  Host pointers,
 * copied.  1 <= F <= DDS_MAX_FAMILIES.  Families sharing a line direction are
 * combined internally through the linearity of the coefficients in b (Sec. 2.1);
 * more than DDS_MAX_FIELDS combined fields gives UNSUPPORTED.  Invalidates built
 * kernels. */
int dds_set_families(dds_ctx *ctx, int F, const double *t, const double *b);

/* Set an option (see DDS_OPT_*).  INVALID_ARG for an unknown key or bad value. */
int dds_set_option(dds_ctx *ctx, int key, double value);

/* Build the interaction coefficients in FP64 on the device (Eq. 9b, Eq. 6/7,
 * Sec. 2.3 near field) and their FP32 Fourier spectra, and size the work buffers.
 * Done once per geometry and family set (Sec. 2.3); later calls with nothing
 * changed return at once.  Runs on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream) and synchronises it before returning. */
int dds_build_kernels(dds_ctx *ctx, void *cuda_stream);

/* Autotuner (no counterpart in the paper; a schedule choice).  Call after
 * dds_set_geometry / dds_set_families and before dds_build_kernels: times one full
 * evaluation (synthetic densities and spectra; the schedule does not change the
 * arithmetic's result beyond rounding) for every fused-z-pass schedule that applies
 * -- the register kernel with each valid number of lanes per (kx, ky) column, the
 * three-stage register kernel and the shared-memory kernel with each valid tile
 * width -- on the median of five trials, each after a 256 MB write that empties L2,
 * and keeps the fastest for the build that follows.  Allocates temporary device memory and synchronises the
 * stream.  *best_ms (host, may be NULL) receives the fastest evaluation time.
 * DDS_OPT_Z_LANES set later overrides the choice. */
int dds_autotune(dds_ctx *ctx, void *cuda_stream, float *best_ms);

/* sigma = sum over families of G * rho (Eq. 10).  rho: device, [F][nz][ny][nx] in
 * m^-2, element type rho_dtype (DDS_F32; DDS_BF16 stores the density as bfloat16,
 * arithmetic stays FP32).  sigma: device, [6][nz][ny][nx] float32, Pa.  Both must be
 * 16-byte aligned.  Enqueued on `cuda_stream`; returns without synchronising.
 * NOT_READY before dds_build_kernels. */
int dds_stress(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, void *cuda_stream);

/* nb density sets on one context (same geometry and families), evaluated together:
 * rho [nb][F][nz][ny][nx], sigma [nb][6][nz][ny][nx], both contiguous.  The result for
 * each set is that of dds_stress; the cached kernel spectra are read from HBM once per
 * call and shared by all sets (each column tile processes the sets back to back), so
 * the per-set cost drops below that of nb separate calls.  The work buffers grow to
 * hold nb sets on first use (that call synchronises the device and allocates); later
 * calls with up to that many sets allocate nothing.  1 <= nb <= 4096. */
int dds_stress_multi(dds_ctx *ctx, int nb, const void *rho, int rho_dtype, float *sigma, void *cuda_stream);

/* Evaluation with the per-height statistics of Eq. 20 fused into its last pass: as
 * dds_stress_multi (nb >= 1 sets; nb = 1 is one dds_stress), and s_out (device,
 * float32, [nb][6][nz]) receives s_c(h_k) = sqrt((1/(nx ny)) sum_{i,j}
 * sigma_c(x_i, y_j, h_k)^2), the in-plane RMS of every component at every height.
 * The sums are accumulated in FP64 by atomic additions, so their rounding depends
 * on the order of the additions.  Sizes its work buffers like dds_stress_multi. */
int dds_stress_stats(dds_ctx *ctx, int nb, const void *rho, int rho_dtype, float *sigma, float *s_out,
                     void *cuda_stream);

/* As dds_stress for n contexts (each built), inputs rho[i] -> sigma[i], all enqueued
 * on one stream in order. */
int dds_stress_batched(dds_ctx **ctxs, int n, const void **rho, const int *rho_dtype,
                       float **sigma, void *cuda_stream);

/* Captured batches (CUDA graphs).  Many density sets on many grids become one
 * graph launch: dds_graph_capture records, for every entry i, the passes of
 * dds_stress_multi(ctxs[i], nb[i], rho[i], rho_dtype[i], sigma[i]) into one CUDA
 * graph; dds_graph_launch replays them all with a single launch call on any stream.
 * The graph holds the device pointers it was captured with: refill rho[i] in place
 * between launches and read sigma[i] after.  Capture first sizes each context's
 * work buffers for its batch (may synchronise the device) and runs every entry once
 * on `cuda_stream` (this writes sigma and completes the library's one-time set-up),
 * then records on a private stream.  Contexts must be built, on one device, with
 * per-pass profiling off; while a graph exists, do not change or destroy its
 * contexts, and do not run other evaluations on them concurrently with a launch
 * (they share the work buffers).  rho_dtype may be NULL (all DDS_F32).  The batch
 * sweep of Sec. 6.4-style realisations is the intended use. */
typedef struct dds_graph dds_graph;
int dds_graph_capture(dds_ctx **ctxs, int n, const int *nb, const void **rho, const int *rho_dtype, float **sigma,
                      void *cuda_stream, dds_graph **out);
int dds_graph_launch(dds_graph *graph, void *cuda_stream);
/* Number of nodes (kernels and memsets) in the captured graph. */
int dds_graph_nodes(const dds_graph *graph);
void dds_graph_destroy(dds_graph *graph);

/* Size of the fixed device work area used by dds_stress_noalloc (32 MiB). */
#define DDS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Evaluation that allocates nothing.  The paper has no counterpart: this is an
 * interface for callers that cannot call cudaMalloc while they run -- for example
 * code whose device memory is wholly owned by another allocator (a framework's
 * caching pool that must account for every byte) or a loop that may not allocate
 * once it has started.  Same inputs, outputs and result as dds_stress (the context
 * must be built by dds_build_kernels during set-up), but the work buffers between
 * the passes come from one fixed area of DDS_NOALLOC_SCRATCH_BYTES that the library
 * declares as device memory.  dds_build_kernels, a set-up step, places the area on the
 * context's device (under lazy module loading this is when the device memory is taken)
 * and looks up its device address, once per device; from then on the device holds the
 * area until the process exits, and dds_stress_noalloc itself allocates nothing.  (The
 * CUDA driver still loads the code of the evaluation kernels at their first launch
 * under lazy module loading: a caller that may not allocate at all makes one call
 * during set-up, or runs with CUDA_MODULE_LOADING=EAGER.)  All calls, from any
 * context or stream, share the one area and its contents persist between calls:
 * calls whose executions overlap on the GPU race, so serialise them (one stream, or
 * events).  No part of the area needs to start at
 * zero: every element a pass reads was written earlier in the same call.  Grids
 * whose work space exceeds the area (about 64x64x32 cells with 4 combined fields
 * fits) are rejected with DDS_ERR_UNSUPPORTED and a message giving the size
 * needed.  Enqueued on `cuda_stream`; returns without synchronising. */
int dds_stress_noalloc(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma, void *cuda_stream);

/* Evaluation for a subset of the context's families.  Eq. 3b sums the stress over the
 * families present, and the coefficients are linear in b (Sec. 2.1), so one built
 * context -- one set of kernel spectra per geometry (Sec. 2.3) -- serves any subset of
 * its families: rho holds only the n families fam[0..n-1] (distinct indices into the
 * families given to dds_set_families), the others count as zero density.  rho: device,
 * [nb][n][nz][ny][nx] (F32 or BF16); sigma: device, [nb][6][nz][ny][nx] FP32; fam: host.
 * 1 <= nb <= 4096, 1 <= n <= F.  The result equals dds_stress_multi with the absent
 * families' densities set to zero (same arithmetic, fewer density reads).  Errors:
 * INVALID_ARG (bad index, repeated index, sizes, alignment), NOT_READY, OOM, CUDA. */
int dds_stress_subset(dds_ctx *ctx, int nb, int n, const int *fam, const void *rho, int rho_dtype, float *sigma,
                      void *cuda_stream);

/* End-to-end variants with HOST buffers (Eq. 10 evaluated as dds_stress, with the
 * densities coming from and the stresses going to host memory).
 *
 * dds_stress_host_async: enqueues the copy of rho_host (float32, [F][nz][ny][nx]) to
 * the device, the evaluation on `cuda_stream`, and the copy of the result to sigma_host
 * (float32, [6][nz][ny][nx]); returns without waiting.  The copies run on two streams
 * of the context and consecutive calls use two staging sets in turn, so one call's
 * copies overlap the previous or next call's evaluation.  rho_host may be reused and
 * sigma_host read only after dds_stress_host_sync; use pinned host memory for the
 * copies to overlap.  Device staging buffers (two sets) are owned by the context.
 * dds_stress_host_sync: waits for every call enqueued so far.
 * dds_stress_host: one call and its sync. */
int dds_stress_host_async(dds_ctx *ctx, const float *rho_host, float *sigma_host, void *cuda_stream);
int dds_stress_host_sync(dds_ctx *ctx);
int dds_stress_host(dds_ctx *ctx, const float *rho_host, float *sigma_host, void *cuda_stream);

/* FP64 interaction coefficients of one family (t, b) under the current geometry
 * and options, evaluated on the device by the same code that builds the kernels:
 * out_host[6q..6q+5] = G(i, j, k) for offsets ijk_host[3q..3q+2] (observer cell
 * minus source cell, |i| < nx, |j| < ny, |k| < nz), q < n.  Host pointers;
 * synchronous.  For parity tests. */
int dds_table_at(dds_ctx *ctx, const double t[3], const double b[3], long n,
                 const int *ijk_host, double *out_host);

/* Sizes: number of effective fields after collapsing families, padded FFT sizes. */
int dds_query(const dds_ctx *ctx, int *n_fields, int *px, int *py, int *pz);

/* Bytes of the cached kernel spectra of a built context (FP32 or FP16 values).  The
 * fused z pass reads them once per evaluation; where the coefficient table has the
 * x-mirror parity for every effective field (Sec. 3 discusses these symmetries of the
 * straight-dislocation field), only the spectra of ky <= py/2 are stored.  *bytes
 * receives the size.  Errors: INVALID_ARG (NULL), NOT_READY (not built). */
int dds_spectra_bytes(const dds_ctx *ctx, unsigned long long *bytes);

/* Device bytes that dds_build_kernels will hold for this geometry and family set --
 * the kernel spectra (the per-geometry coefficients of Sec. 2.3, in Fourier space) and
 * the work buffers for nb density sets -- computed from the plan without allocating
 * (set geometry and families first).  For admission control before a build.  Errors:
 * INVALID_ARG, NOT_READY, UNSUPPORTED (no z-pass schedule for the grid). */
int dds_footprint(dds_ctx *ctx, int nb, unsigned long long *bytes);

/* The contraction of Eq. 10 in Fourier space (Sec. 2.3: the convolution becomes a
 * product of spectra, summed over the fields as in Eq. 3b) as a separate kernel, for
 * timing a library-FFT pipeline against the fused passes; dds_stress never calls it.
 *   sigma_hat[c][k] = sum_e (i g[c][e][k]) rho_hat[e][k],  c < 6, e < fe, k < nk.
 * rho_hat: device, complex FP32 (interleaved re, im), [fe][nk]; g: device, FP32 real
 * (the imaginary parts of purely imaginary kernel spectra), [6][fe][nk]; sigma_hat:
 * device, complex FP32, [6][nk], written.  1 <= fe <= 8.  Needs no context; enqueued
 * on cuda_stream.  Errors: INVALID_ARG, CUDA. */
int dds_contract_spectra(const void *rho_hat, int fe, const float *g, void *sigma_hat, long long nk,
                         void *cuda_stream);

/* Number of kernel launches one dds_stress call issues. */
int dds_launches_per_stress(const dds_ctx *ctx);

/* CTAs per cluster of the fused inverse y + x pass that a built context runs (see
 * DDS_OPT_YX_FUSED), or 0 when it runs the two inverse passes separately.  Negative:
 * INVALID_ARG (NULL) or NOT_READY (not built). */
int dds_yx_cluster(const dds_ctx *ctx);

/* Per-pass timing.  While enabled, every dds_stress on this context records CUDA
 * events on its stream before the first pass and after each pass (the passes are
 * x forward, y forward, fused z, y inverse, x inverse; with the fused inverse pass
 * of DDS_OPT_YX_FUSED the y-inverse interval is empty and the x-inverse interval
 * holds the fused pass).  Timing only; results are unchanged.  Enabling clears
 * earlier records. */
int dds_profile_enable(dds_ctx *ctx, int enable);

/* Synchronise the recorded events and return their durations: ms_out (host,
 * [max_steps][5]) gets per-pass milliseconds of the first min(recorded, max_steps)
 * evaluations since enabling; *n_steps and *n_passes receive the counts.  Clears
 * the records. */
int dds_profile_read(dds_ctx *ctx, int max_steps, float *ms_out, int *n_steps, int *n_passes);

/* Free-surface relaxation (Sec. 5, Eqs. 14-18).  The stress sigma_dis of the
 * dislocations in an infinite medium (for instance the output of dds_stress)
 * loads a film whose top and bottom faces (the centres of the first and last
 * layers) are free and whose sides are periodic.  The displacement u relaxes by
 * n_steps explicit steps of Eq. 17,
 *     u <- u + dt (A grad div u - B rot rot u + f),  f_a = sum_b d sigma_dis_ab / db,
 * A = E(1-nu)/((1+nu)(1-2nu)), B = E/(2(1+nu)), dt = min(dx,dy,dz)^2 / (5A - 3B),
 * with the traction-free conditions of Eq. 16c held by ghost layers (Eq. 18b).
 * Central differences; d sigma_dis/dz one-sided (second order) on the surface
 * layers.  Arithmetic in FP32.
 *   sigma_dis  device, [6][nz][ny][nx] FP32, Pa (xx, yy, zz, xy, xz, yz); read only.
 *   u          device, [3][nz][ny][nx] FP32, metres (x, y, z); the starting state
 *              (zeros for a fresh relaxation), overwritten by the state after
 *              n_steps, so calls continue where the last one stopped.
 *   sigma_tot  device, [6][nz][ny][nx] FP32, or NULL: sigma_dis + sigma(u), the
 *              stress of the free film (Hooke's law on central differences).
 * Needs only the geometry (dds_set_geometry), nz >= 2 (DDS_ERR_UNSUPPORTED
 * otherwise); n_steps >= 0.  Allocates 6 nx ny nz + 6 nx ny floats of work space
 * on first use (DDS_ERR_OOM).  Asynchronous on `cuda_stream`. */
int dds_relax(dds_ctx *ctx, const float *sigma_dis, float *u, int n_steps, float *sigma_tot, void *cuda_stream);

/* Bounded device waits (no counterpart in the paper).  The passes that stage their
 * input with bulk asynchronous copies wait for each copy on a shared-memory
 * barrier; a wait that has not completed after one second of device time gives
 * up, the kernel skips its remaining work (its output is then incomplete) and
 * records the event in a status word of the device.  This returns DDS_OK if no
 * wait has given up on `cuda_device` since the last reset, DDS_ERR_TIMEOUT if
 * one has, DDS_ERR_INVALID_ARG for a bad device, DDS_ERR_CUDA if the word cannot
 * be read.  It reads the word with a synchronous copy, so it sees the kernels that
 * have finished: synchronise the streams of interest first.  reset != 0 clears
 * the word after reading it.  Needs no context. */
int dds_device_status(int cuda_device, int reset);

/* Last error message of this context (never NULL; "" if none). */
const char *dds_last_error(const dds_ctx *ctx);

/* Free everything the context owns: its FP64-derived kernel spectra (the per-geometry
 * coefficients of Sec. 2.3), work buffers and staging buffers.  NULL is a no-op. */
void dds_destroy(dds_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DDS_H */
