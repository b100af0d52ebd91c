/*
 * swense.h — C ABI of the GB300 (sm_103a) incident-wave reconstruction library.
 *
 * The library evaluates the incident-wave fields of the two-phase SWENSE method (free-surface
 * elevation eta, velocity u, v, w, and the dynamic pressure or dphi/dt) from spectral (HOS)
 * modal amplitudes onto arbitrary CFD points, in the two stages of the paper's reconstruction
 * section ("Reconstruction of incident wave information on the CFD mesh"):
 *   1. inverse transforms of the modes onto a uniform horizontal grid at arbitrary vertical
 *      levels, refined by zero-padding the spectrum (subsection "Improvement of the
 *      interpolation accuracy");
 *   2. space-time interpolation of the grid fields onto cell and face centres.
 * It also computes the finite-volume divergence used as the reconstruction-error measure
 * (subsection "Reconstruction error: velocity divergence").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers documented "device" must be CUDA device (or managed) memory of the current device;
 *   "host" pointers are read before the call returns. The caller owns every buffer it passes.
 *   The library keeps a per-device scratch workspace (allocated with cudaMalloc on first use,
 *   grown on demand, freed by swense_release); entry points that may grow it must not be
 *   called for the first time inside a CUDA stream capture.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). All device work
 *   is enqueued on it; calls return before it runs unless documented otherwise.
 * - Calls that overlap on the GPU (different streams, no ordering) race on the library's scratch
 *   workspace: order them on one stream.
 * - Return value: SWENSE_OK (0) or a negative SWENSE_ERR_* code; swense_last_error() gives a
 *   one-line description for the calling thread. Invalid arguments launch nothing.
 * - Modal amplitudes use the one-sided half-spectrum layout: complex64 stored as interleaved
 *   (re, im) float pairs, index [row][m] with m = 0..nx/2 (nx/2+1 columns) and rows in FFT order
 *   (row r holds n = r for r < ny/2 and n = r - ny otherwise). Mode (m, n) has wavenumber
 *   k = (2 pi m / Lx, 2 pi n / Ly). A real field is f(x) = sum_{m >= 0} c_m Re(sum_n F_{m,n}
 *   e^{i k.x}) with c_0 = 1 and c_m = 2 otherwise. The Nyquist column m = nx/2 and row r = ny/2
 *   are ignored. For a 2-D (x, z) problem ny = 1 and y is ignored everywhere.
 * - Fields follow the paper's spectral decomposition (Eqs. whatIsSpectralMethod1 and
 *   whatIsSpectralMethod) and the velocity sums of its "analytical evaluation":
 *     eta  = sum A^eta e^{ik.x}
 *     u    = sum i kx A^phi F(z) e^{ik.x},   v = sum i ky A^phi F(z) e^{ik.x}
 *     w    = sum |k| A^phi S(z) e^{ik.x},    dphi/dt = sum A^phit F(z) e^{ik.x}
 *   with F = cosh(|k|(z+h))/cosh(|k|h), S = sinh(|k|(z+h))/cosh(|k|h), or F = S = e^{|k|z} in
 *   deep water, evaluated unchanged above z = 0 (section "Extension of incident wave solution
 *   in the air"). Pressure (Bernoulli): p_dyn = -rho (dphi/dt + |u|^2/2).
 */
#ifndef SWENSE_H
#define SWENSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWENSE_VERSION 100
#define SWENSE_MAX_LEVELS 256   /* vertical levels per grid */
#define SWENSE_MAX_FFT 8192     /* refined nodes per horizontal axis (pad_n * nx, pad_n * ny) */
#define SWENSE_MAX_TL 4         /* time levels per interpolation */

enum swense_status {
  SWENSE_OK = 0,
  SWENSE_ERR_ARG = -1,          /* NULL pointer, bad enum, non-finite or inconsistent value */
  SWENSE_ERR_SIZE = -2,         /* size not a power of two or above a SWENSE_MAX_* limit */
  SWENSE_ERR_LEVELS = -3,       /* vertical levels not strictly increasing / too few / too many */
  SWENSE_ERR_OOM = -4,          /* scratch workspace allocation failed */
  SWENSE_ERR_CUDA = -5,         /* a CUDA runtime call failed (see swense_last_error) */
  SWENSE_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
  SWENSE_ERR_UNSUPPORTED = -7,  /* valid request this build does not implement */
  SWENSE_ERR_CONVERGENCE = -8   /* a host-side nonlinear solve did not converge */
};

enum swense_p_mode {
  SWENSE_P_DYN = 0,    /* p = -rho (dphi/dt + |u|^2 / 2) */
  SWENSE_P_PHIT = 1,   /* p = dphi/dt */
  SWENSE_P_TOTAL = 2   /* p = -rho (dphi/dt + |u|^2 / 2) - rho g z */
};

/* Horizontal interpolation scheme of the grid (vertical and time: Lagrange in both). */
enum swense_scheme {
  SWENSE_LAGRANGE3 = 0,  /* grid holds node values; 4-point Lagrange in x and y */
  SWENSE_SPLINE3 = 1     /* the paper's "cubic spline": grid holds periodic cubic B-spline
                            coefficients (modes divided by the B-spline symbol before the
                            transforms) and the gather uses cubic B-spline weights in x and y */
};

/* Spectral modal amplitudes of one sea state (paper: A^eta_i, A^phi_i of Eqs.
 * whatIsSpectralMethod1 / whatIsSpectralMethod; A^phit their time derivative's modes). */
typedef struct swense_modes {
  int32_t nx, ny;        /* mode counts: nx power of two in [4, SWENSE_MAX_FFT]; ny = 1 (2-D) or
                            a power of two in [4, SWENSE_MAX_FFT] */
  double Lx, Ly;         /* periodic domain lengths [m]; Ly ignored when ny = 1 */
  double depth;          /* water depth h > 0 [m]; <= 0 means deep water */
  int32_t n_snap;        /* snapshots stored in A_* (see swense_fields_on_grid) */
  const float* A_eta;    /* device complex64 [n_snap][ny][nx/2+1] (interleaved re, im) */
  const float* A_phi;    /* device complex64 [n_snap][ny][nx/2+1]: volume potential at z = 0 */
  const float* A_phit;   /* device complex64 [n_snap][ny][nx/2+1]: dphi/dt at z = 0 */
  const double* omega;   /* device [ny][nx/2+1] angular frequency of each slot, or NULL */
  double t_ref;          /* time at which the single snapshot holds (used with omega only) */
} swense_modes;

/* The reconstruction ("HOS") grid: nx_r = pad_n*nx by ny_r = pad_n*ny (ny_r = 1 in 2-D)
 * uniform nodes x_i = i Lx/nx_r, y_j = j Ly/ny_r, at nz arbitrary levels. */
typedef struct swense_grid_desc {
  int32_t pad_n;           /* zero-padding factor, 1..8 (the paper asks for an integer) */
  int32_t nz;              /* number of levels, 4 <= nz <= SWENSE_MAX_LEVELS */
  const float* z_levels;   /* host [nz], strictly increasing */
  int32_t scheme;          /* enum swense_scheme */
} swense_grid_desc;

/*
 * swense_fields_on_grid — stage 1: modes -> grid (paper: reconstruction section, step "IFFT",
 * one inverse transform per vertical level, and the zero-padding refinement of subsection
 * "Improvement of the interpolation accuracy"; levels above z = 0 per the extension into air).
 *
 * Time levels: if modes->omega is NULL, modes->n_snap must equal n_tl and time level l uses
 * snapshot l (t may be NULL). Otherwise modes->n_snap must be 1 and time level l uses
 * A * exp(-i omega (t[l] - t_ref)), the phase reduced in FP64 (t: host [n_tl]).
 *
 * Outputs (device, caller-allocated, 16-byte aligned):
 *   nodes  float [n_tl][nz][ny_r][nx_r][4] = (u, v, w, dphi/dt) per node
 *   eta    float [n_tl][ny_r][nx_r]
 * Padding factors that are not powers of two (3, 5, 6, 7; the paper only requires an integer):
 * with pad_n = q p2, q odd, the node x_{qJ+s} is the p2-padded node x_J moved by s Lx/nx_r, so
 * the grid is built from q^2 (q in 2-D) power-of-two transforms of the modes times
 * e^{i k.shift} (the shift theorem), each scattered to every q-th node. The workspace then also
 * holds one such sub-grid. swense_fields_on_grid_noalloc and swense_autotune_grid take
 * power-of-two factors only (SWENSE_ERR_UNSUPPORTED otherwise); the tuned launch shape of the
 * factor p2 is used.
 * Arithmetic: FP32 transforms, FP32 depth factors with a compensated |k| z product.
 * Uses the scratch workspace (4 * ny_r * (nx/2 + 1) complex64 per level of a level chunk, each
 * row padded to whole 128-byte lines; twice that for transform variant 5) when ny > 1. When
 * ny > 1 the eta transform runs on a second, library-owned stream, forked from `stream` and
 * joined back before the call returns, so it overlaps the level transforms. The workspace, the
 * twiddle table and the library's streams are created by the first call on a device, which must
 * not be inside a stream capture. Errors: ARG, SIZE, LEVELS, OOM, CUDA.
 */
int swense_fields_on_grid(const swense_modes* modes, int32_t n_tl, const double* t,
                          const swense_grid_desc* desc, float* nodes, float* eta, void* stream);

/*
 * swense_fields_on_grid_noalloc — swense_fields_on_grid for callers that cannot allocate device
 * memory (the paper has no counterpart; this is a property of the library, not of the method).
 *
 * Some callers must not allocate while their time loop runs: a CFD solver that reserves all
 * device memory up front in its own pool, a plugin whose host forbids allocations outside set-up,
 * or code that cannot afford the implicit device synchronisation a cudaMalloc/cudaFree may do.
 * This entry point takes the same arguments and produces the same grid as swense_fields_on_grid,
 * with the same transform kernels and launch shape (the tuned one, else the default), except that
 * the two-stream variant 5 runs as variant 2 and the eta transform stays on `stream` (no library
 * stream is used); but it allocates nothing: it calls no cudaMalloc, cudaFree or allocating
 * library routine. Its
 * scratch (the transformed levels between the two passes, and the propagated modes) lives in a
 * fixed array of SWENSE_NOALLOC_SCRATCH_BYTES inside the library's device image, which every GPU
 * that loads the library holds until the process exits.
 *   - Requests whose scratch for one vertical level (plus the propagated modes and the eta
 *     transform) exceeds SWENSE_NOALLOC_SCRATCH_BYTES are rejected with SWENSE_ERR_SIZE before
 *     anything is launched; larger requests use swense_fields_on_grid. Within the limit, levels
 *     are processed in as many chunks as the array requires.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current) and fills the shared twiddle table; make that first call before
 *     any stream capture.
 *   - Every call on a device uses the same array and leaves its contents behind. Nothing in it
 *     has to start at zero (each call writes every scratch value before reading it), but calls
 *     that overlap on the GPU (different streams without ordering) race on it: order them.
 * Errors: as swense_fields_on_grid, with SWENSE_ERR_SIZE for the scratch limit and never
 * SWENSE_ERR_OOM.
 */
#define SWENSE_NOALLOC_SCRATCH_BYTES (16u << 20)
int swense_fields_on_grid_noalloc(const swense_modes* modes, int32_t n_tl, const double* t,
                                  const swense_grid_desc* desc, float* nodes, float* eta,
                                  void* stream);

/*
 * swense_autotune_grid — choose the launch shape of swense_fields_on_grid for this grid shape
 * (the transform path: warp-register kernels with 1, 2 or 4 levels per column-transform block,
 * or the shared-memory kernels; the level-chunk size among 16, 32, 64, 96, 128, 256 MB; and, for
 * 256- to 1024-point rows, whether one row-transform block handles both field pairs or one) by
 * timing each candidate five times on `stream` (best of five, each from a cold L2: the
 * workspace, grown to at least 256 MB, is overwritten before each repetition); the choice is
 * cached per (nx, ny, pad_n, nz)
 * and used by later calls. No counterpart in the paper. Writes the grid (same outputs as
 * swense_fields_on_grid), synchronises the stream, must not be captured. 2-D grids have a
 * single path (nothing to tune; *lpc_out = -1).
 * lpc_out (0 = shared-memory path), chunk_bytes_out, row_variant_out (0 = both field pairs per
 * warp, 1 = one field pair per block, 2 = transposed intermediate: the row pass reads its inputs
 * straight from memory; both lengths in 256..1024; 3 = as 2 with one transform per warp;
 * 4 = as 2 with each warp's rows staged in shared memory by bulk asynchronous copies; 5 = as 2
 * with chunk c's row pass on a library-internal second stream while chunk c+1's column pass
 * runs on `stream`, two intermediate buffers, joined back before the call's work ends), plus 16
 * when the transposed pair's column pass runs one modal field per block (four times the blocks
 * per level, half the registers; the untuned default for 1024-point columns):
 * host, may be NULL. Errors: as swense_fields_on_grid.
 */
int swense_autotune_grid(const swense_modes* modes, int32_t n_tl, const double* t,
                         const swense_grid_desc* desc, float* nodes, float* eta,
                         int32_t* lpc_out, int64_t* chunk_bytes_out, int32_t* row_variant_out,
                         void* stream);

/*
 * swense_set_grid_tune — set the launch shape that swense_fields_on_grid uses for grids of shape
 * (nx, ny, pad_n, nz), e.g. a choice that swense_autotune_grid returned in an earlier process.
 * lpc: -1 (forget any choice: untuned defaults again), 0 (shared-memory path), 1, 2 or 4 levels
 * per column block;
 * chunk_bytes in [1 MiB, 1 GiB] (L2-resident level chunk); row_variant 0..5, plus 16 for the
 * one-field column pass (as returned by swense_autotune_grid). Results do not depend on the choice beyond FP32 rounding. No
 * counterpart in the paper. Errors: SWENSE_ERR_ARG for values outside those sets.
 */
int swense_set_grid_tune(int32_t nx, int32_t ny, int32_t pad_n, int32_t nz, int32_t lpc,
                         int64_t chunk_bytes, int32_t row_variant);

/* Grid fields at n_tl time levels as written by swense_fields_on_grid. */
typedef struct swense_grid {
  const float* nodes;       /* device float [n_tl][nz][ny_r][nx_r][4] */
  const float* eta;         /* device float [n_tl][ny_r][nx_r] */
  int32_t nx_r, ny_r, nz;   /* nx_r, ny_r powers of two <= SWENSE_MAX_FFT (ny_r = 1 in 2-D) */
  int32_t n_tl;             /* 1..SWENSE_MAX_TL */
  double Lx, Ly;            /* domain lengths (Ly ignored when ny_r = 1) */
  const float* z_levels;    /* host [nz], strictly increasing */
  const double* t_levels;   /* host [n_tl], strictly increasing */
  int32_t scheme;           /* enum swense_scheme the grid was built with */
} swense_grid;

/*
 * swense_interp — stage 2: grid -> points (paper: reconstruction section, step
 * "Interpolation"). Tensor-product 4-point Lagrange interpolation: periodic uniform nodes
 * i0-1..i0+2 in x and y around the point's cell; in z the 4 levels around the bracketing
 * interval [z_j, z_j+1], shifted inside [0, nz-1] at the ends; Lagrange over the n_tl time
 * levels at time t (linear for 2, cubic for 4; the paper states no time scheme).
 *
 * pts: device float [np][3] (x, y, z) in the grid's frame; x and y wrap periodically.
 * Outputs: device float [np] each, any may be NULL. Points with z outside
 * [z_levels[0], z_levels[nz-1]] get NaN u, v, w, p (eta stays valid) and are counted.
 * n_out_of_range: host pointer or NULL; when non-NULL the call synchronises the stream and
 * stores the count. p_mode: enum swense_p_mode; rho, g used by P_DYN / P_TOTAL.
 * Points are taken in 1024-point chunks; a chunk whose points all have the same z (bitwise; a
 * layer of cell or face centres of an extruded mesh) is interpolated in z once per grid column
 * and then in x and y per point, which is the same tensor-product sum in another order.
 * Errors: ARG, SIZE, LEVELS, CUDA.
 */
int swense_interp(const swense_grid* grid, double t, const float* pts, int64_t np,
                  float* eta, float* u, float* v, float* w, float* p,
                  int32_t p_mode, double rho, double g, int64_t* n_out_of_range,
                  void* stream);

/*
 * Reusable gather plans (no counterpart in the paper). swense_interp first cuts the points into
 * 1024-point chunks and finds each chunk's stencil bounding box on the grid; that plan depends
 * only on the points and the grid geometry (nx_r, ny_r, Lx, Ly, z_levels), not on the time or
 * the field values, so a solver whose mesh and grid do not change can make it once:
 *   swense_interp_plan_bytes(np)      bytes of device memory a plan for np points needs
 *                                     (16 per chunk; 0 for np <= 0);
 *   swense_interp_plan(grid, pts, np, plan, stream)
 *                                     writes the plan into `plan` (device, caller-owned,
 *                                     16-byte aligned, swense_interp_plan_bytes(np) bytes;
 *                                     the size is not checked). The grid's field arrays are not
 *                                     read; its geometry and level list are;
 *   swense_interp_with_plan(...)      swense_interp with that plan (the plan kernel is skipped).
 * A plan made for other points or another grid geometry gives wrong results (reads stay inside
 * the shared-memory box and the grid: offsets are clamped, levels checked). Errors: as swense_interp; SWENSE_ERR_ARG for a
 * NULL or misaligned plan.
 */
int64_t swense_interp_plan_bytes(int64_t np);
int swense_interp_plan(const swense_grid* grid, const float* pts, int64_t np, void* plan,
                       void* stream);
int swense_interp_with_plan(const swense_grid* grid, double t, const float* pts, int64_t np,
                            const void* plan, float* eta, float* u, float* v, float* w, float* p,
                            int32_t p_mode, double rho, double g, int64_t* n_out_of_range,
                            void* stream);

/*
 * swense_bin_points — point binning for scattered point sets (no counterpart in the paper,
 * whose CFD points arrive in mesh order). Counting sort of the points by grid tile (4 x 4 cells
 * horizontally, one 4-level stencil vertically, x fastest) so that consecutive points share
 * stencils; the grid geometry comes from `grid` (nodes/eta/t_levels are not read).
 *   perm: device int32 [np], out: perm[k] = caller index of the k-th sorted point
 *   pts_sorted: device float [np][3], out: the points in sorted order
 * The order inside one tile is unspecified; results of the interpolation do not depend on it.
 * Uses the scratch workspace (4 B per point and per tile). Errors: ARG, SIZE, LEVELS, OOM, CUDA.
 */
int swense_bin_points(const swense_grid* grid, const float* pts, int64_t np, int32_t* perm,
                      float* pts_sorted, void* stream);

/* swense_interp on points sorted by swense_bin_points: reads pts_sorted in order and writes
 * every output at its caller index perm[k]. Same arguments and rules as swense_interp. */
int swense_interp_permuted(const swense_grid* grid, double t, const float* pts_sorted,
                           const int32_t* perm, int64_t np, float* eta, float* u, float* v,
                           float* w, float* p, int32_t p_mode, double rho, double g,
                           int64_t* n_out_of_range, void* stream);

/* One independent sea state of a batch: modes -> grid (own buffers) -> its own points. */
typedef struct swense_instance {
  swense_modes modes;
  swense_grid_desc desc;
  int32_t n_tl;
  const double* t_levels;   /* host [n_tl]: grid time levels (propagation times with omega) */
  float* nodes;             /* device [n_tl][nz][ny_r][nx_r][4] */
  float* eta;               /* device [n_tl][ny_r][nx_r] */
  const float* pts;         /* device [np][3]; sorted by swense_bin_points when perm != NULL */
  const int32_t* perm;      /* device [np] from swense_bin_points, or NULL */
  int64_t np;
  double t;                 /* query time of the gather */
  float *out_eta, *out_u, *out_v, *out_w, *out_p;   /* device [np] each, may be NULL */
} swense_instance;

/*
 * swense_batch_run — many independent sea states of uneven sizes in one call (no counterpart
 * in the paper): every instance's grid (as swense_fields_on_grid, with its tuned launch shape)
 * and then every instance's gather (as swense_interp, or swense_interp_permuted when perm is
 * set). The reconstructions run concurrently on four library streams forked from `stream`
 * (largest instance first, round robin, each stream in its own part of the workspace); after
 * they are joined back, one launch plans the point chunks of all instances and one persistent
 * launch gathers them, its CTAs taking chunks from a device queue. Fork and join are events,
 * so one call can be captured as a single CUDA graph and replayed as one launch. The first call
 * with a given set of instances must be made outside any capture: it sizes the workspace and
 * uploads the gather tables (arguments and level tables of every instance; a captured call
 * whose tables differ from the last uploaded ones fails with SWENSE_ERR_ARG). Power-of-two
 * padding factors only. Errors: those of the per-instance calls, UNSUPPORTED, OOM, CUDA.
 */
int swense_batch_run(const swense_instance* instances, int32_t n_instances, int32_t p_mode,
                     double rho, double g, void* stream);

enum swense_direct_precision {
  SWENSE_DIRECT_FP32 = 0,              /* FP32 arithmetic, exact integer-turn phases */
  SWENSE_DIRECT_SPLIT_BF16 = 1,        /* tcgen05 split-BF16 contraction, FP32 accumulation */
  SWENSE_DIRECT_SPLIT_BF16_PAIRWISE = 2 /* per-pair split-BF16 mma.sync kernel (comparison) */
};

/*
 * swense_direct — direct ("analytical") evaluation of the modal sums at arbitrary points
 * (paper: reconstruction section, analytical evaluation of u_I and w_I by substituting the
 * coordinates into the sums; its cost is proportional to the number of Fourier components per
 * point). No grid, no interpolation error: used for small mode counts (regular waves) and for
 * near-body points. Same field definitions as swense_fields_on_grid; pressure by Bernoulli.
 *
 * modes: one snapshot (n_snap = 1); with omega non-NULL it is propagated to time t
 *   (A e^{-i omega (t - t_ref)}, phase reduced in FP64), otherwise t is ignored.
 * pts: device float [np][3]; outputs device float [np] each, any may be NULL.
 * precision:
 *   SWENSE_DIRECT_FP32: one thread per point, every mode in FP32 (the phase m x/Lx + n y/Ly is
 *     an exact 32-bit fraction of a turn, so accuracy does not degrade with |k x|).
 *   SWENSE_DIRECT_SPLIT_BF16: the sums as a dense contraction on the tcgen05 tensor cores. The
 *     points are sorted by z (a counting sort into 65536 buckets between their min and max z)
 *     and cut into tiles of 128, two tiles per cluster of two CTAs (cta_group::2); the phase
 *     is separated, e^{i(kx x + ky y)} = X_m(x) Y_n(y), and the depth factor is expanded about
 *     the tile pair's middle z0 to second order in z - z0 (exact derivatives d/dz F = |k| S,
 *     d/dz S = |k| F); rows n and -n are paired (Y_-n = conj Y_n); per group of 8 row pairs and
 *     64 modes, a [256 points x 128] x [128 x 208] product (Re(T_n + T_-n), Im(T_n - T_-n) of
 *     u, v, w, dphi/dt at three orders, and eta) in split BF16 (hi.hi + hi.lo + lo.hi; the
 *     order-2 columns without their lo half, so hi.lo spans the other 144), FP32 accumulation
 *     in tensor memory, then
 *     Re sum_n Y_n (...) and sum_j (z - z0)^j in FP32. A tile pair whose max|k| x half-range of
 *     z exceeds 0.02 (the dropped third-order term would exceed 2e-6) is evaluated by the
 *     per-pair kernel instead. Accuracy: about 1e-5 of each field's maximum (bar 1e-3).
 *     Points with nearly equal z are ordered by atomics, so a tile's z0, and with it the last
 *     digits of the split products' rounding, can differ from call to call.
 *   SWENSE_DIRECT_SPLIT_BF16_PAIRWISE: per (point, mode) pair the operand e^{i k.x} f(z) is
 *     generated in registers and split into BF16 hi + lo for legacy mma.sync m16n8k16 products
 *     (the same accuracy; kept for comparison and for tiles the tensor-core path leaves).
 * Uses the scratch workspace (FP32: 64 B per mode slot; SPLIT_BF16: 32 B per mode slot, 20 B
 * per point and 256 KB; PAIRWISE: 80 B per mode). Errors: ARG, SIZE, UNSUPPORTED, OOM, CUDA;
 * the tensor-core kernel's bounded waits report through swense_async_status.
 */
int swense_direct(const swense_modes* modes, double t, const float* pts, int64_t np,
                  float* eta, float* u, float* v, float* w, float* p, int32_t p_mode,
                  double rho, double g, int32_t precision, void* stream);

/*
 * Learned interpolation correction (no counterpart in the paper, which interpolates with a
 * plain scheme; this is an optional refinement of its interpolation step, judged by the same
 * modal-sum reference and the same divergence measure). One multilayer perceptron is shared by
 * the fields f in (u, v, w, dphi/dt):
 *   x = [stencil_f / s_f (64 time-blended 4x4x4 node values, x fastest, then y, then z),
 *        dx, dy, dz, 0],  s_f = max |stencil_f| + 1e-30 (row of SWENSE_MLP_XLD floats),
 *   67 -> 64 -> 64 -> 4 with tanh-form GELU on the hidden layers; output y[f];
 *   corrected f = lagrange_f + s_f y[f]; pressure from the corrected fields (Bernoulli).
 * Parameters: FP32, SWENSE_MLP_NPARAM values packed as W1[64][67], b1[64], W2[64][64], b2[64],
 * W3[4][64], b3[4] (row = output unit). The kernels read a BF16 "packed" copy
 * (SWENSE_MLP_PACKED_BYTES, 16-byte aligned device buffer) written by swense_mlp_pack or by
 * each training step. Tensor cores: BF16 MMA with FP32 accumulation (inference splits inputs
 * and activations into BF16 hi + lo; training uses plain BF16).
 */
#define SWENSE_MLP_NPARAM 8772
#define SWENSE_MLP_PACKED_BYTES 32768
#define SWENSE_MLP_XLD 68

/* params (device FP32 [SWENSE_MLP_NPARAM]) -> packed (device, SWENSE_MLP_PACKED_BYTES), with
 * the inference output multiplier out_scale (> 0; training targets are divided by it so the
 * network works on O(1) values). Synchronises the stream (out_scale is copied from the host).
 * Training steps refresh the weights of packed and keep its out_scale. */
int swense_mlp_pack(const float* params, float out_scale, void* packed, void* stream);

/* Network rows of features: y[r] = out_scale * net(x[r])[r % 4] (rows point-major, fields
 * u, v, w, phit).
 * x: device float [rows][SWENSE_MLP_XLD]; y: device float [rows]. */
int swense_mlp_forward(const void* packed, const float* x, int64_t rows, float* y, void* stream);

/* Features of points on a 3-D grid: x [4 np][SWENSE_MLP_XLD], scale [4 np] (s_f), lagrange
 * [4 np] (plain interpolated f), eta [np] (plain, may be NULL); same grid rules as
 * swense_interp. Errors: ARG, SIZE, LEVELS, UNSUPPORTED (2-D grid), CUDA. */
int swense_mlp_features(const swense_grid* grid, double t, const float* pts, int64_t np,
                        float* x, float* scale, float* lagrange, float* eta, void* stream);

/* Gradient of the mean squared error of y[field[r]] against target[r] over the rows
 * batch[0 .. B-1] of x (all device; batch holds row indices). grad: device FP32
 * [SWENSE_MLP_NPARAM] (overwritten); loss: device scalar or NULL. Uses the workspace. */
int swense_mlp_grad(const void* packed, const float* x, const int32_t* field, const float* target,
                    const int32_t* batch, int32_t B, float* grad, float* loss, void* stream);

/* One Adam step (Kingma & Ba; bias-corrected, step >= 1) of the FP32 params with moments
 * adam_m, adam_v (device FP32 [SWENSE_MLP_NPARAM]) on the batch, then refreshes packed.
 * Uses the workspace. Errors: ARG, OOM, CUDA. */
int swense_mlp_train_step(float* params, float* adam_m, float* adam_v, void* packed, int64_t step,
                          const float* x, const int32_t* field, const float* target,
                          const int32_t* batch, int32_t B, float lr, float beta1, float beta2,
                          float eps, float* loss, void* stream);

/* Training targets of the learned correction from the method's own data: for point i and field
 * f (u, v, w, dphi/dt), row 4 i + f gets target = (exact_f - lagrange_f) / scale_f and field = f,
 * with exact_* device float [np] (swense_direct, p_mode PHIT), lagrange and scale device float
 * [4 np] (swense_mlp_features). target device float [4 np], field device int32 [4 np].
 * Errors: ARG, CUDA. */
int swense_mlp_targets(const float* exact_u, const float* exact_v, const float* exact_w,
                       const float* exact_phit, const float* lagrange, const float* scale,
                       int64_t np, float* target, int32_t* field, void* stream);

/* A network and its training state. The caller owns the device buffers (params, adam_m, adam_v:
 * FP32 [SWENSE_MLP_NPARAM]; packed: SWENSE_MLP_PACKED_BYTES, 16-byte aligned); step, seed and
 * out_scale are host values that the calls below read and update. */
typedef struct {
  float* params;
  float* adam_m;
  float* adam_v;
  void* packed;
  int64_t step;       /* Adam steps taken so far */
  uint64_t seed;      /* mini-batch generator seed */
  float out_scale;    /* inference output multiplier; <= 0: set by the next swense_mlp_train */
} swense_mlp;

/* `steps` Adam steps (the loop runs in the library) on mini-batches of B rows of the dataset
 * (x [n_rows][SWENSE_MLP_XLD], field [n_rows], target [n_rows], device). Batch s (s = mlp->step,
 * 0-based) holds rows SplitMix64(seed + s 2^32 + i) mod n_rows, i < B, so a run can be split
 * and resumed (swense_mlp_save / swense_mlp_load) with bit-identical parameters; gradients are
 * summed in a fixed order. Learning rate lr x (1 + cos(pi min(s, schedule_steps) /
 * schedule_steps)) / 2 (constant lr when schedule_steps <= 0). The network learns
 * target / out_scale; if mlp->out_scale <= 0 it is first set to the RMS of the targets (one
 * device reduction, synchronising) and packed. losses: device float [steps] (mean squared error
 * of each step in scaled units) or NULL. Uses the workspace. Errors: ARG, OOM, CUDA. */
int swense_mlp_train(swense_mlp* mlp, const float* x, const int32_t* field, const float* target,
                     int64_t n_rows, int32_t steps, int32_t B, float lr, int64_t schedule_steps,
                     float beta1, float beta2, float eps, float* losses, void* stream);

/* Checkpoint (little-endian file): "SWMLP002", int64 step, uint64 seed, int64 nparam (must be
 * SWENSE_MLP_NPARAM), float64 out_scale, then params, adam_m, adam_v as float32. save
 * synchronises the stream; load fills the caller's buffers and mlp's host fields and repacks
 * (synchronising). Errors: ARG (file cannot be opened, written or read, wrong header or size),
 * CUDA. */
int swense_mlp_save(const swense_mlp* mlp, const char* path, void* stream);
int swense_mlp_load(swense_mlp* mlp, const char* path, void* stream);

/* swense_interp with the learned correction applied to u, v, w and dphi/dt (eta plain).
 * Same arguments and out-of-range rules as swense_interp plus the packed weights; 3-D grids
 * only. Uses the workspace (about 0.6 GB for the largest point chunk). */
int swense_interp_learned(const swense_grid* grid, double t, const float* pts, int64_t np,
                          float* eta, float* u, float* v, float* w, float* p, int32_t p_mode,
                          double rho, double g, const void* packed, int64_t* n_out_of_range,
                          void* stream);

/*
 * swense_fv_divergence — the finite-volume divergence of the reconstruction-error subsection:
 * div_c = sum_f s_cf (u_f . A_f) / V_c with the face-centre velocity standing for the face
 * average (error source 1 of that subsection).
 *   u_face, v_face, w_face : device float [n_faces]  velocity at face centres
 *   area                   : device float [n_faces][3] face area vectors
 *   cell_faces             : device int32 [n_cells][6] signed face references, +(f+1) when
 *                            A_f points out of the cell, -(f+1) when it points in
 *   cell_volume            : device float [n_cells]
 *   div                    : device float [n_cells] output
 * Face references are not range-checked on the device; the caller guarantees
 * 1 <= |ref| <= n_faces. Errors: ARG, CUDA.
 */
int swense_fv_divergence(const float* u_face, const float* v_face, const float* w_face,
                         int64_t n_faces, const float* area, const int32_t* cell_faces,
                         const float* cell_volume, int64_t n_cells, float* div, void* stream);

/*
 * swense_tank_modes — wave-tank modes (paper: the HOS-NWT solver reproduces a rectangular tank
 * with perfectly reflective walls, so the basis functions psi_i become cosine modes) onto the
 * periodic pipeline. Tank fields:
 *   eta = sum_{m,n} A^eta_mn cos(m pi x / Lx) cos(n pi y / Ly), phi likewise with the depth
 *   factor F(|k|, z) of swense_fields_on_grid, dphi/dt likewise; u, v, w the derivatives of phi.
 * A cosine series on the tank is the Fourier series of its even extension over 2 Lx x 2 Ly, so
 * each real amplitude is written as its one or two half-spectrum coefficients of that doubled
 * periodic domain (A for m = n = 0, A/2 on an axis, A/4 at each of (m, +n) and (m, -n)).
 *   A_eta, A_phi, A_phit: device float [n_snap][ny_t][nx_t] real amplitudes, m = 0..nx_t-1
 *       along x, n = 0..ny_t-1 along y (ny_t = 1: a 2-D tank)
 *   nx_t: 2 (nx_t - 1) a power of two in [4, SWENSE_MAX_FFT]; ny_t = 1 or likewise
 *   n_snap: 1..SWENSE_MAX_TL time snapshots; Lx, Ly: tank lengths; depth (<= 0: deep)
 *   out_eta, out_phi, out_phit: device complex64 [n_snap][ny][nx/2+1] (8-byte aligned), filled
 *   out: host; set to nx = 2 (nx_t - 1), ny = 2 (ny_t - 1) (1 in 2-D), Lx' = 2 Lx, Ly' = 2 Ly,
 *        the depth, n_snap, omega = NULL and the three output tables.
 * Passing *out to swense_fields_on_grid (n_tl = n_snap, the snapshots' times) gives the grid of
 * the doubled domain. Its nodes i <= nx_t - 1 (j <= ny_t - 1) are the tank nodes
 * x_i = i Lx / (nx_t - 1). swense_interp then evaluates points inside the tank; near a wall its
 * stencil reads the mirrored nodes, which hold the extension the wall imposes. The highest mode
 * of each axis (m = nx_t - 1, n = ny_t - 1) is that grid's Nyquist mode, and it is dropped like
 * every Nyquist mode. Errors: ARG, SIZE, CUDA.
 */
int swense_tank_modes(const float* A_eta, const float* A_phi, const float* A_phit, int32_t nx_t,
                      int32_t ny_t, int32_t n_snap, double Lx, double Ly, double depth,
                      float* out_eta, float* out_phi, float* out_phit, swense_modes* out,
                      void* stream);

/*
 * Stream-function regular waves (paper: subsection on regular waves by stream-function theory,
 * after Rienecker & Fenton; the "analytical evaluation" subsection: with N ~ 10 components,
 * ka = 0.24 converging with N = 9, the fields are summed directly at the cells).
 *
 * A 2-D periodic wave of period T and height H travelling in +x over depth h, steady in the
 * frame moving at its phase speed c. In that frame (crest at X = 0, z up from the mean level):
 *   psi = -ubar (z + h) + sum_{j=1..N} B_j sinh(j k (z + h)) / cosh(j k h) cos(j k X)
 *   eta = sum_{j=0..N} E_j cos(j k X)
 * with U = dpsi/dz, W = -dpsi/dX. Found by collocation at X_m = m pi / (N k), m = 0..N: psi = -Q
 * and (U^2 + W^2)/2 + g eta = R on the surface, zero mean level, crest-to-trough height H, and
 * no mean Eulerian current (c = ubar = 2 pi / (k T)).
 */
#define SWENSE_STREAM_MAX_N 32

typedef struct {
  int32_t n;                              /* number of components N */
  double k, c, ubar;                      /* wavenumber, phase speed, mean speed in the wave frame */
  double Q, R;                            /* volume flux and Bernoulli constant (wave frame) */
  double depth, g, period, height;
  double B[SWENSE_STREAM_MAX_N];          /* B_1..B_N */
  double E[SWENSE_STREAM_MAX_N + 1];      /* E_0..E_N, cosine coefficients of the surface */
  double eta_m[SWENSE_STREAM_MAX_N + 1];  /* surface at the collocation points */
} swense_stream_wave;

/*
 * swense_stream_solve — host only (no GPU needed): the wave's coefficients by Newton's method
 * in FP64 with the analytic Jacobian, the height raised from the linear wave in height_steps
 * equal steps (4 is plenty below ~80 % of the breaking height). period, height, depth, g > 0;
 * 1 <= n <= SWENSE_STREAM_MAX_N; out: host, caller-owned.
 * Errors: ARG, SIZE, CONVERGENCE (too steep for n or too few steps).
 */
int swense_stream_solve(double period, double height, double depth, double g, int32_t n,
                        int32_t height_steps, swense_stream_wave* out);

/*
 * swense_stream_eval — the incident fields of a solved wave at points, fixed frame, time t, the
 * crest at x = x0 at t = 0: X = x - x0 - c t,
 *   u = c - ubar + sum_j j k B_j C_j cos(j k X),  v = 0,  w = sum_j j k B_j S_j sin(j k X),
 *   eta = sum_j E_j cos(j k X) (at the point's x),
 * C_j, S_j the cosh and sinh ratios at the point's z (written without overflow); pressure by
 * Bernoulli in the wave frame with p = 0 on the surface: P_TOTAL rho (R - g z - (U^2 + W^2)/2),
 * P_DYN that + rho g z, P_PHIT -p_dyn / rho - |u|^2 / 2, U = u - c.
 *   pts: device float [np][3] (x, y, z); y is not used. Outputs: device float [np], any NULL.
 * The phase is reduced in FP64 on the host and formed per point from a compensated x k product;
 * the sums are FP32 (cos/sin and the depth ratios of the harmonics by recurrence).
 * Errors: ARG, SIZE, CUDA.
 */
int swense_stream_eval(const swense_stream_wave* wave, double t, double x0, const float* pts,
                       int64_t np, float* eta, float* u, float* v, float* w, float* p,
                       int32_t p_mode, double rho, void* stream);

/*
 * Relaxation zones and the incident VOF fraction (paper: subsection on the prevention of wave
 * reflections with the relaxation zone technique, Eqs. relaxationZone, weightFunction,
 * swUcRelax and swVOFRelax; alpha_I reconstructed from eta_I, reconstruction section,
 * interpolation step).
 *
 * A zone is a slab along x or y, or a ring about the vertical axis through (cx, cy). For a cell
 * centre with coordinate s in it (x, y, or the horizontal distance from the axis), the
 * non-dimensional distance is x = clamp((s - inner) / (outer - inner), 0, 1): 0 at the inner
 * boundary (the pure CFD side), 1 at the outer one, so a zone may run in either direction. The
 * weight is w = -2x^3 + 3x^2, the largest over the zones where they overlap, 0 outside all.
 */
enum swense_zone_kind { SWENSE_ZONE_X = 0, SWENSE_ZONE_Y = 1, SWENSE_ZONE_RADIAL = 2 };
#define SWENSE_MAX_ZONES 8

typedef struct {
  int32_t kind;    /* enum swense_zone_kind */
  float inner;     /* coordinate (x, y or radius) of the inner boundary, weight 0 */
  float outer;     /* coordinate of the outer boundary, weight 1; finite, != inner */
  float cx, cy;    /* axis of a ring zone (unused by slabs) */
} swense_relax_zone;

/*
 * swense_relax_cells — per CFD cell: the incident VOF fraction, the relaxation weight and the
 * blends applied at the end of a CFD time step.
 *   cell_xyz  device float [nc][3] cell centres (x and y are read)
 *   cell_zext device float [nc][2] (z_lo, z_hi), the cell's vertical extent, z_lo < z_hi;
 *             8-byte aligned
 *   eta_c     device float [nc] incident elevation at the cell centres (swense_interp's eta)
 *   zones     host [n_zones], 0 <= n_zones <= SWENSE_MAX_ZONES
 * Outputs (device, any may be NULL):
 *   alpha_i   float [nc]  alpha_I = clamp((eta - z_lo) / (z_hi - z_lo), 0, 1): the part of the
 *             cell's height below a surface taken as horizontal across the cell (the paper
 *             states no formula); NaN eta gives NaN
 *   weight    float [nc]  w
 *   alpha     float [nc]  in place: w alpha_I + (1 - w) alpha            (Eq. swVOFRelax)
 *   u_c       float [nc][3] in place: (1 - w) u_c, the target being 0   (Eq. swUcRelax)
 * Cells with w = 0 keep alpha and u_c unchanged and are not written. FP32 arithmetic.
 * Errors: ARG (bad sizes, zone kind or boundaries, NULL inputs), CUDA.
 */
int swense_relax_cells(const float* cell_xyz, const float* cell_zext, const float* eta_c,
                       int64_t nc, const swense_relax_zone* zones, int32_t n_zones,
                       float* alpha_i, float* alpha, float* u_c, float* weight, void* stream);

/*
 * swense_async_status — errors of bounded device-side waits (no passage of the paper: library
 * housekeeping). Kernels that wait on asynchronous copies (the staged row pass of
 * swense_fields_on_grid, row variant 4) give every wait an iteration limit; a wait that runs
 * out sets a per-device flag and its warp returns without writing its grid rows, so the call
 * that launched it has already returned SWENSE_OK. This call synchronises `stream`, reads the
 * flag of the current device and, when reset != 0, clears it.
 * Returns SWENSE_ERR_TIMEOUT if a wait gave up since the flag was last cleared (the grid of that
 * call is incomplete), else SWENSE_OK; CUDA on a failed copy.
 */
int swense_async_status(int32_t reset, void* stream);

/*
 * swense_selftest_wait_timeout — self-test of the bounded-wait path above: launches the staged
 * row pass on a tiny dummy problem with its copies withheld and a limit of a few polls, so every
 * wait runs out; nothing is read or written but the flag. Afterwards swense_async_status must
 * return SWENSE_ERR_TIMEOUT and the context stays usable. Uses (and may grow) the workspace.
 * Errors: CUDA.
 */
int swense_selftest_wait_timeout(void* stream);

/*
 * swense_selftest_direct_wait_timeout — self-test switch of the tensor-core direct sum's bounded
 * waits (no passage of the paper: library housekeeping). While on (on != 0) for the current
 * device, every SWENSE_DIRECT_SPLIT_BF16 call runs k_direct_tc with its A-ready arrivals withheld
 * and a limit of a few polls per wait: the MMA thread's first wait runs out, the pair aborts
 * without issuing an MMA, its tiles' outputs are not written, and swense_async_status then
 * returns SWENSE_ERR_TIMEOUT. Switch it off (on = 0) before any real call. Errors: UNSUPPORTED,
 * CUDA.
 */
int swense_selftest_direct_wait_timeout(int32_t on);

/*
 * swense_direct_stats — tiles of the last SWENSE_DIRECT_SPLIT_BF16 call on the current device
 * (no passage of the paper): *tiles = tiles of 128 z-sorted points, *fallback_tiles = those whose
 * z range was too wide for the tensor-core expansion and went to the per-pair kernel (0 and 0
 * before any such call). Synchronises `stream`; valid until the workspace is reused or freed.
 * Errors: ARG, CUDA.
 */
int swense_direct_stats(int64_t* tiles, int64_t* fallback_tiles, void* stream);

/*
 * swense_selftest_tc_gemm — self-test of the tensor-core data path used by swense_direct (no
 * passage of the paper): D = A B^T with A device FP32 [128][K], B device FP32 [N][K] (both
 * rounded to BF16), D device FP32 [128][N], one tcgen05 MMA chain with A in tensor memory
 * (variant 0) or shared memory (variant 1) and B in shared memory in the K-major core-matrix
 * layout of the direct sum. N and K multiples of 16 in 16..256. Errors: ARG, CUDA.
 */
int swense_selftest_tc_gemm(const float* A, const float* B, float* D, int32_t N, int32_t K,
                            int32_t variant, void* stream);

/* Bytes of scratch workspace currently held on the current device. */
int64_t swense_workspace_bytes(void);

/* Free the scratch workspace of the current device (synchronises the device). */
int swense_release(void);

/* One-line description of the calling thread's last error ("" if none). */
const char* swense_last_error(void);

/* Static name of a status code. */
const char* swense_strerror(int status);

/* Number of kernels this process has launched through the library (all devices). */
int64_t swense_launches(void);

/* SWENSE_VERSION of the built library. */
int swense_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWENSE_H */
