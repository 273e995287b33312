/*
 * wproj.h -- C-ABI of libwproj, the GB300 (sm_103a) implementation of the
 * sparse w-projection hot path of Wolz et al. 2013 (arXiv:1307.3424).
 *
 * Model.  Phi = G . F . Z . A maps a real N x N sky image x to M complex
 * visibilities (Eq. 8 of the paper with continuous (u, v) and Kaiser-Bessel
 * gridding):
 *   A  divides pixel (p, q) by a(l_p) a(m_q), a the Fourier transform of the
 *      KB gridding kernel (W taps, oversampling 2);
 *   Z  zero-pads the image, centred, onto the G x G grid, G = 2N (the 2x
 *      band-limit doubling of Section 4.1);
 *   F  is the unitary 2-D DFT (1/G normalisation, e^{-2 pi i} sign of Eq. 1);
 *   G  holds one sparse row per visibility k: the w-modulation kernel C-hat of
 *      Eq. 8 (Section 3.1: the chirp of Eq. 4 in real space, Fourier
 *      transformed) convolved with the KB taps at the visibility's sub-grid
 *      offset, then sparsified by the adaptive energy threshold of Section 3.2
 *      (the smallest set of entries holding a fraction e of the row's energy).
 * Phi^H = A Z^H F^H G^H is its exact adjoint.  solve_bpdn solves Eq. 7 (BPDN,
 * Dirac sparsity basis, real image) by Douglas-Rachford splitting (Section 2.3).
 *
 * Geometry and units.  Field of view L (direction cosines); pixel size L/N;
 * uv cell du = 1/(2L); band limit B = N/(2L) (Section 4.1).  Baselines (u, v, w)
 * are in wavelengths; (u, v) must lie in [-B, B).  Grid arrays are G x G,
 * row-major, in natural FFT order (frequency q at index q mod G); the image
 * pixel p sits at offset p - N/2.  Column index of grid cell (qu, qv) is
 * (qu mod G) * G + (qv mod G).
 *
 * Conventions for every call:
 *   - Array arguments are device pointers owned by the caller unless stated.
 *     G, its index structures and all scratch space are owned by the plan.
 *   - Calls return a status and never throw; wproj_last_error() gives the
 *     message of the last failure on the calling thread.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless stated.  wproj_build_kernels synchronises the
 *     stream once (to size G).  A plan must not be used from two streams at
 *     the same time: calls on one plan share its scratch buffers.
 *   - Invalid sizes or parameters return WPROJ_ERR_INVALID_ARG and leave the
 *     plan unchanged; a CUDA failure returns WPROJ_ERR_CUDA; an allocation
 *     failure returns WPROJ_ERR_OOM.
 */
#ifndef WPROJ_H
#define WPROJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WPROJ_OK = 0,
  WPROJ_ERR_INVALID_ARG = 1,
  WPROJ_ERR_OOM = 2,
  WPROJ_ERR_CUDA = 3,
  WPROJ_ERR_TIMEOUT = 4,
  WPROJ_ERR_NOT_BUILT = 5,
  WPROJ_ERR_UNSUPPORTED = 6
} wproj_status;

typedef enum { WPROJ_CHIRP_EXACT = 0, WPROJ_CHIRP_LINEAR = 1 } wproj_chirp_kind;
typedef enum { WPROJ_EXT_FULL = 0, WPROJ_EXT_CLAMP = 1 } wproj_extension;
typedef enum { WPROJ_VAL_F32 = 0, WPROJ_VAL_BF16 = 1, WPROJ_VAL_F16 = 2 } wproj_value_dtype;

typedef struct wproj_plan wproj_plan;

/* Imaging geometry of a plan. */
typedef struct {
  int32_t n;            /* image side N: even, 8 <= N <= 2048; the grid is G = 2N */
  int32_t kb_support;   /* W = 4, 6 or 8 KB taps per axis; 1 = delta-gridding (single
                           tap at floor(u/du), a == 1; exact only for on-grid u) */
  double fov;           /* L, planar field of view in direction cosines, 0 < L, 2L^2 < 1 */
  int32_t chirp;        /* wproj_chirp_kind: exact Eq. 4, or linear Eq. 5 (sign +) */
  int32_t extension;    /* wproj_extension: chirp outside the field of view evaluated
                           as is (full) or with l, m clamped to [-L/2, L/2] (clamp) */
  int32_t box;          /* kernel box side S: 0 = rule S(w) = min(G, pow2 >= 4h+W+16),
                           h = |w| L^2 the chirp half-band in cells; else a fixed power
                           of two with 16 <= S <= G (S = G is exact) */
  int32_t value_dtype;  /* wproj_value_dtype of the stored G values; bf16/f16 values are
                           scaled per row by 1 / max|G[k,:]| (row_scale holds max|G[k,:]|) */
  int32_t index_format; /* wproj_index_format: how the columns of G are stored */
  int32_t upsampling;   /* 0: the model above (image-space zero-padding Z, KB correction A,
                           grid cells 1/(2L)).  1: the paper's own operator (Section 2.2,
                           Eq. 8): Phi = C-hat F U with U the upsampling that zero-pads the
                           image's spectrum onto the 2N x 2N grid (an isometry), the chirp
                           sampled on the upsampled image (2N pixels of L/2N), grid cells
                           1/L, (u, v) in [-N/L, N/L); needs kb_support = 1 (visibilities
                           on the grid: the cell is floor(u L)) and n >= 16 */
} wproj_grid_desc;

/* Storage of G.  The entries of a row are grouped by 32 x 32 grid tile (tiles
 * ascending) and ordered row-major inside a tile; a (row, tile) pair with
 * entries is a segment.  Two formats:
 *   COLUMNS      CSR: row_ptr, int32 column indices (4 B per entry) and values,
 *                row after row;
 *   TILE_MASK    a tile stream: for every tile (ascending) and every row with
 *                entries in it (rows ascending), one record, 16-byte aligned:
 *                  int32 row, int32 count, int32 segment id, int32 0   (16 B)
 *                  32 uint32 mask words, bit l of word r = cell (r, l) stored
 *                  32 uint16 prefixes: entries stored in tile rows 0 .. r-1
 *                  count values in row-major cell order, zero-padded to 16 B
 *                (192 B of mask and prefixes per segment instead of 4 B per
 *                entry, and each tile's records contiguous for streaming).
 *   TILE_RUNS    run lengths, for plans whose kernel boxes are at most 64 x 64
 *                cells (a small kernel keeps one contiguous run of cells per
 *                grid row).  Every run is stored padded to an even length by one
 *                zero value.  Two copies of the values:
 *                  row-major, for the degridding: per row its window origin
 *                  (j0 - S/2) mod G per axis, its runs in window order as uint32
 *                  (window row | window column << 6 | (length - 1) << 12) and
 *                  its values run after run;
 *                  tile-major records, for the gridding: for every tile
 *                  (ascending) and every row with entries in it (rows
 *                  ascending), 16-byte aligned: int32 row, uint16 stored count,
 *                  uint16 runs; the runs as uint16 (tile column | (length - 1)
 *                  << 5 | tile row << 10), zero-padded to 16 B; the values
 *                  (CSR order with the pads), zero-padded to 16 B.
 *                (about 4 B per run instead of 4 B per entry).
 * AUTO picks TILE_RUNS when every box is at most 64 x 64 cells (and the grid is
 * at least 32 x 32) and the values are F32 (or there are more than 2^22 rows),
 * else TILE_MASK when segments average >= 256 entries (dense rows), else
 * COLUMNS.  Requesting TILE_RUNS for larger boxes makes
 * wproj_build_kernels return WPROJ_ERR_UNSUPPORTED.  wproj_csr_rows exports any
 * rows in CSR order from every format. */
typedef enum {
  WPROJ_INDEX_AUTO = 0,
  WPROJ_INDEX_COLUMNS = 1,
  WPROJ_INDEX_TILE_MASK = 2,
  WPROJ_INDEX_TILE_RUNS = 3
} wproj_index_format;

/* View of G held by a plan (device pointers owned by the plan; valid until the
 * next build or the plan's destruction). */
typedef struct {
  int64_t m;                /* rows (visibilities) */
  int64_t nnz;              /* stored entries */
  int64_t n_cols;           /* G * G */
  const int64_t *row_ptr;   /* m + 1 offsets of each row's entries in CSR order (both formats) */
  const int32_t *col;       /* COLUMNS: nnz column indices; TILE_MASK: NULL */
  const void *val;          /* COLUMNS: nnz complex values in CSR order, float2 or (bf16, bf16) /
                               (f16, f16) pairs; TILE_MASK: NULL */
  const float *row_scale;   /* m scales (bf16/f16: G[k, q] = row_scale[k] * stored value),
                               NULL for f32 */
  int32_t value_dtype;
  int32_t index_format;     /* WPROJ_INDEX_COLUMNS, WPROJ_INDEX_TILE_MASK or WPROJ_INDEX_TILE_RUNS */
  int64_t n_seg;            /* (row, tile) segments */
  const void *stream;       /* TILE_MASK / TILE_RUNS: the tile-major records; else NULL */
  int64_t stream_bytes;     /* their size in bytes (0 for COLUMNS) */
} wproj_csr;

/* Entries of rows [k0, k1) of G in CSR order, whatever the index format:
 * col_out (int32, device) receives their column indices and val_out (device)
 * their stored values (the plan's value dtype, unscaled), each
 * row_ptr[k1] - row_ptr[k0] long; either may be NULL.  Synchronises `stream`
 * once (to read the range).  0 <= k0 <= k1 <= m, else WPROJ_ERR_INVALID_ARG. */
wproj_status wproj_csr_rows(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                            void *stream);

/* Douglas-Rachford parameters (the paper states none; these are the defaults
 * used by the oracle and the benchmarks). */
typedef struct {
  int32_t iters;        /* outer DR iterations T */
  int32_t inner_iters;  /* dual forward-backward iterations per projection (10) */
  double gamma_frac;    /* gamma = gamma_frac * max|Re Phi^H y| (1e-2) */
  double lambda;        /* relaxation lambda (1.0) */
  double phi_norm2;     /* ||Phi||^2; <= 0: estimate by power iteration */
  int32_t power_iters;  /* power iterations when phi_norm2 <= 0 (100) */
  int32_t resume;       /* 1: continue from the plan's current DR state (z, u, gamma,
                           ||Phi||^2) left by the previous solve or wproj_dr_state_set;
                           0: start from z = Re Phi^H y, u = 0 */
  int32_t psi;          /* sparsity basis Psi of Eq. 7: 0 = Dirac (x itself is sparse),
                           p in 1..WPROJ_DAUB_MAX_P = periodic orthonormal Daubechies
                           wavelets with p vanishing moments (8: the paper's Db8) */
  int32_t psi_levels;   /* dyadic levels of the wavelet transform (N divisible by
                           2^levels); ignored for psi = 0 */
} wproj_dr_params;

typedef struct {
  int32_t iters_done;
  double phi_norm2;     /* value used for the dual step mu = 1/||Phi||^2 */
  double gamma;
  double final_resid;   /* ||y - Phi x||_2 of the returned x */
  double final_l1;      /* ||x||_1 */
} wproj_solve_info;

/* Counters of a plan, for reporting. */
typedef struct {
  int64_t m, nnz;
  int32_t box_min, box_max;  /* smallest / largest kernel box used by the last build */
  int64_t segments;          /* (row, grid tile) segments of G */
  int64_t degrid_pieces;     /* row pieces of the degridding SpMV */
  int64_t grid_chunks;       /* tile chunks of the gridding */
  double build_ms;           /* wall time of the last wproj_build_kernels */
  /* accumulated device time (ms) and launches per step when timing is on */
  double t_fft_ms, t_degrid_ms, t_grid_ms, t_reduce_ms, t_solver_ms;
  int64_t n_fft, n_degrid, n_grid, n_reduce, n_solver;
  int64_t launches;          /* kernels launched by Phi, Phi^H and the solver since the last reset */
  int64_t runs_bytes;        /* TILE_RUNS: bytes of the row-major copy the degridding reads (values,
                                runs, per-row offsets and origins); 0 for the other formats */
  /* device time (ms) of the builds since the last reset when timing is on: box
     tables and FFTs (both passes), selection and per-tile counts, emission */
  double t_build_fft_ms, t_build_select_ms, t_build_emit_ms;
  int64_t n_build_fft;       /* box batches transformed (each pass counts) */
} wproj_stats;

/* ---- plan ---------------------------------------------------------------- */

/* Create a plan for the geometry *g on the current CUDA device.  Allocates the
 * grid work buffers (a few G x G complex arrays).  *out receives the plan. */
wproj_status wproj_plan_create(wproj_plan **out, const wproj_grid_desc *g);

/* Free the plan and everything it owns (synchronises the device). */
wproj_status wproj_plan_destroy(wproj_plan *p);

/* ---- Part I: sparse w-kernels (Sections 3.1-3.2) -------------------------- */

/* Build G for M visibilities.  uvw: device, M x 3 float64 (u, v, w in
 * wavelengths, row-major).  e in (0, 1]: kept fraction of each row's energy
 * (Section 3.2); each row keeps the smallest set of entries, largest moduli
 * first, whose energy reaches (e + 1e-5) E_k, E_k the row's total (the margin
 * covers FP32 rounding so that the kept energy reaches e E_k in exact
 * arithmetic; e + 1e-5 >= 1 keeps the whole box).  Rejects non-finite uvw,
 * (u, v) outside [-B, B) and m < 1 with WPROJ_ERR_INVALID_ARG (detected on the
 * device; the plan keeps no G then).  Replaces any previous G.  Returns after
 * the build has finished.  out (nullable) receives a view of G. */
wproj_status wproj_build_kernels(wproj_plan *p, const double *uvw, int64_t m, double e,
                                 void *stream, wproj_csr *out);

/* Direction-dependent effects (Section 3.2: the per-row threshold assumes nothing
 * about a row's structure, so it applies to any image-space modulation, not only
 * the w-chirp).  A screen A(l, m) multiplies the chirp of every row it is
 * attached to before the FFT: row k is FFT(chirp_k x A_{screen_id[k]}), convolved
 * with the gridding taps and thresholded like any other row.
 * wproj_set_screens: n_screens screens, complex64 [n_screens][G][G] row-major
 * (host or device; copied into the plan), sample (a, b) at the chirp's sample
 * points l = (a - G/2) d, m = (b - G/2) d over the padded field of view, d = L/N
 * (image pixel (p, q) at (p + N/2, q + N/2)); with upsampling = 1, d = L/(2N),
 * the pixels of the upsampled image.  n_screens = 0 drops them.  Non-finite
 * samples -> WPROJ_ERR_INVALID_ARG.  Invalidates the current G.  Synchronous.
 * wproj_build_kernels_dde: as wproj_build_kernels with screen_id (device int32[m],
 * each in [0, n_screens), else WPROJ_ERR_INVALID_ARG) naming every row's screen.
 * Needs a plan with the full kernel box (box = G; else WPROJ_ERR_UNSUPPORTED),
 * as a screen is sampled at the full box's points. */
wproj_status wproj_set_screens(wproj_plan *p, const void *screens, int32_t n_screens, void *stream);
wproj_status wproj_build_kernels_dde(wproj_plan *p, const double *uvw, int64_t m, const int32_t *screen_id,
                                     double e, void *stream);

/* View of the current G (WPROJ_ERR_NOT_BUILT before the first build). */
wproj_status wproj_get_csr(const wproj_plan *p, wproj_csr *out);

/* ---- Part II: measurement operator (Eq. 8) -------------------------------- */

/* y = Phi x.  x: device N x N float32 (row-major, pixel (p, q) at p*N + q);
 * y: device M complex (float2). */
wproj_status wproj_phi(wproj_plan *p, const float *x, void *y, void *stream);

/* Phi^H y.  y: device M float2.  x_re (nullable): N x N float32 receives
 * Re(Phi^H y); x_cplx (nullable): N x N float2 receives the complex adjoint. */
wproj_status wproj_phi_adj(wproj_plan *p, const void *y, float *x_re, void *x_cplx,
                           void *stream);

/* y = Phi x, like wproj_phi, but the call allocates no device memory and uses
 * none of the plan's work buffers.  (The paper has no counterpart: this is a
 * deployment variant.)  It is for callers that cannot call cudaMalloc while
 * they run: programs whose device memory is reserved up front by another
 * runtime or pool allocator (a cudaMalloc there fails or escapes the pool's
 * accounting), and loops that cannot afford the device-wide synchronisation
 * cudaMalloc and cudaFree imply.  Its scratch lives in one fixed array of
 * 16 MiB that every GPU loading this part of the library holds until the
 * process exits.  The scratch a plan needs is N*G + G*G complex values (FFT
 * intermediate and padded spectrum) plus its degridding partial sums: one
 * complex value per row piece of <= 16384 entries (COLUMNS) or four per
 * (row, tile) segment (TILE_MASK), each part rounded up to 256 bytes; a plan
 * whose total exceeds 16 MiB is rejected with WPROJ_ERR_INVALID_ARG.  So
 * N = 512 fits up to 524,288 partial sums and N = 256 up to 1.7 million, while
 * N = 256 with M = 32768 dense rows (8.4 million tile-stream segments) and any
 * N >= 1024 are refused.  The first call on a device looks up that array's
 * device address and keeps it for the process (a cudaDeviceReset invalidates
 * it, as it invalidates every plan); make that first call before any stream
 * capture.  All calls share the one array and leave their data in it: calls
 * that overlap on the GPU (other streams, other threads, other plans) race and
 * must be serialised by the caller.  Timing statistics (wproj_set_timing) are
 * kept in the plan's host state, so two host threads calling on one plan with
 * timing on race there too.  x, y and the built G as for wproj_phi. */
wproj_status wproj_phi_noalloc(wproj_plan *p, const float *x, void *y, void *stream);

/* Complex-image forward operator (for the adjoint identity): x_cplx N x N float2. */
wproj_status wproj_phi_cplx(wproj_plan *p, const void *x_cplx, void *y, void *stream);

/* ---- Part III: BPDN by Douglas-Rachford (Eq. 7) --------------------------- */

/* Solve min ||alpha||_1 s.t. ||y - Phi Psi alpha||_2 <= eps over real alpha and
 * return the image x = Psi alpha (Psi = identity for psi = 0).  y: device M
 * float2; x_out: device N x N float32.  prm NULL = defaults (T = 50, 10 inner
 * iterations, gamma_frac 1e-2, lambda 1, power iteration 100, Dirac basis).
 * info (nullable) makes the call synchronous and fills the summary (final_l1 =
 * ||alpha||_1); with info NULL the call is asynchronous.
 * With a wavelet Psi the DR variable z lives in coefficient space and the
 * projection onto {alpha : ||y - Phi Psi alpha|| <= eps} is taken in image space
 * as Psi^T P(Psi z), which is exact because Psi is orthonormal: one synthesis
 * and one analysis per outer iteration, none inside the inner loop. */
wproj_status wproj_solve_bpdn(wproj_plan *p, const void *y, double eps,
                              const wproj_dr_params *prm, float *x_out,
                              wproj_solve_info *info, void *stream);

/* ||Phi||^2 of the real-image operator by `iters` power iterations from the
 * unit impulse at the image centre (synchronous). */
wproj_status wproj_power_norm2(wproj_plan *p, int32_t iters, double *out, void *stream);

/* Checkpoint / resume of the Douglas-Rachford state: z (N x N float32; wavelet
 * coefficients when the solve used a wavelet Psi, which resume must use again), the dual
 * variable u (M float2, one per visibility of the current G), gamma and ||Phi||^2.
 * Pointers may be host or device memory (copied with cudaMemcpyDefault, then the
 * stream is synchronised).  get needs a previous solve (WPROJ_ERR_NOT_BUILT
 * otherwise); set makes the next solve with resume = 1 continue from the given
 * state, which reproduces the saved run's next iterate exactly on the same GPU. */
wproj_status wproj_dr_state_get(wproj_plan *p, float *z, void *u, double *gamma, double *phi_norm2,
                                void *stream);
wproj_status wproj_dr_state_set(wproj_plan *p, const float *z, const void *u, double gamma,
                                double phi_norm2, void *stream);

/* ---- utilities ------------------------------------------------------------ */

/* Unnormalised 2-D DFT of `batch` n x n complex arrays (n a power of two,
 * 16 <= n <= 4096): out[k] = sum_j in[j] exp(sign 2 pi i k.j / n), sign -1
 * (inverse = 0) or +1 (inverse = 1).  in and out: device float2, may alias. */
wproj_status wproj_fft2d(const void *in, void *out, int32_t n, int32_t batch, int32_t inverse,
                         void *stream);

/* The Daubechies sparsity basis (Eq. 7; Db8 in the paper's experiments).
 * Taps: the low-pass analysis filter of the extremal-phase Daubechies wavelet with
 * p vanishing moments (1 <= p <= WPROJ_DAUB_MAX_P), 2p doubles into h_out (host),
 * from Daubechies' spectral factorisation; the high-pass is g_k = (-1)^k h_{2p-1-k}.
 * One periodic level on an even length n: a_i = sum_k h_k x_{(2i+k) mod n},
 * d_i = sum_k g_k x_{(2i+k) mod n}.  In 2-D a level filters the fast axis, then
 * the slow axis, and stores the Mallat layout: [0,h)x[0,h) low-low, [0,h)x[h,n)
 * low (slow) / high (fast), [h,n)x[0,h) high / low, [h,n)x[h,n) high-high; the
 * next level transforms the low-low block.
 * wproj_dwt2: alpha = Psi^T x; wproj_idwt2: x = Psi alpha.  x, alpha: device
 * n x n float32, row-major, must not alias; work: device scratch of n*n/2
 * floats; n divisible by 2^levels, levels >= 1.  Asynchronous on `stream`. */
#define WPROJ_DAUB_MAX_P 10
wproj_status wproj_daubechies_taps(int32_t p, double *h_out);
wproj_status wproj_dwt2(int32_t n, int32_t levels, int32_t p, const float *x, float *alpha, float *work,
                        void *stream);
wproj_status wproj_idwt2(int32_t n, int32_t levels, int32_t p, const float *alpha, float *x, float *work,
                         void *stream);

/* Per-kernel device timing with CUDA events (0 = off, default). */
wproj_status wproj_set_timing(wproj_plan *p, int32_t enable);
wproj_status wproj_get_stats(wproj_plan *p, wproj_stats *out);   /* synchronises */
wproj_status wproj_reset_stats(wproj_plan *p);

/* Default DR parameters. */
void wproj_dr_defaults(wproj_dr_params *prm);

const char *wproj_last_error(void);
const char *wproj_version(void);

/* ---- dense BF16 GEMM on the tensor cores ------------------------------------------
 * C[m x n] = A[m x k] B[n x k]^T (+ bias[n]): A, B row-major BF16, C row-major FP32
 * (out_bf16 = 0) or BF16, FP32 accumulation, on the tcgen05 tensor cores.  The
 * dense contraction of the learned-kernel MLP, exported for testing.
 * m, n multiples of 128, k a multiple of 64, else WPROJ_ERR_INVALID_ARG.
 * bias may be NULL.  Synchronous; WPROJ_ERR_TIMEOUT if a tensor-core wait ran out. */
/* Test hook of the GEMM's bounded waits (no counterpart in the paper; failure
 * detection).  wait_on_unset_barrier != 0 makes every later wproj_gemm_bf16 CTA
 * first wait on an mbarrier that nothing arrives on, for at most limit_ns
 * nanoseconds (0 = the normal limit of 2 s): the call then returns
 * WPROJ_ERR_TIMEOUT after each CTA has drained its committed MMAs and freed its
 * tensor memory, and the context stays usable.  (0, 0) restores normal
 * operation.  Affects the current device; synchronous. */
wproj_status wproj_gemm_test_hook(int32_t wait_on_unset_barrier, uint64_t limit_ns);
wproj_status wproj_gemm_bf16(int32_t m, int32_t n, int32_t k, const void *a, const void *b, const float *bias,
                             void *c, int32_t out_bf16, void *stream);

/* ---- learned kernels ----------------------------------------------------------
 * An MLP mapping a visibility's (w, sub-grid offset) to its w-kernel on a fixed
 * 32 x 32 window of grid cells plus a support mask, trained on kernels of the
 * plain build (which stays the reference and the fallback):
 *   x0 = (w_c/2 - 1, 2 du - 1, 2 dv - 1), w_c = |w| L^2 / 2 grid cells, (du, dv)
 *        the sub-grid offset of (u, v) / du_cell;
 *   h1 = GELU(W1 x0 + b1), h2 = GELU(W2 h1 + b2), h3 = GELU(W3 h2 + b3)  (256 each)
 *   y  = W4 h3 + b4  (3072): y[2(32a+b)], y[2(32a+b)+1] the real and imaginary
 *        parts of the kernel at window cell (a, b) = grid cell (j0 - 16 + a,
 *        j0 - 16 + b) mod G scaled by 1/sqrt(E_kb) (E_kb = prod over axes of
 *        sum_t kb(delta - t)^2), y[2048 + 32a + b] the logit of (a, b) being in
 *        the support;
 *   loss = mean over values of (y - t)^2 + mask_weight * mean BCE(logit, mask).
 * GELU is the erf form.  Layers 2-4 and their gradients run as BF16 GEMMs on the
 * tensor cores with FP32 accumulation; parameters, Adam and reductions are FP32.
 * Parameters are one flat FP32 vector: W1 (256x3), b1, W2 (256x256), b2, W3, b3,
 * W4 (3072x256), b4, matrices row-major [out][in]. */
typedef struct wproj_mlp wproj_mlp;
int64_t wproj_mlp_num_params(void);
wproj_status wproj_mlp_create(wproj_mlp **out);   /* parameters zero until set */
wproj_status wproj_mlp_destroy(wproj_mlp *n);
/* params: wproj_mlp_num_params() floats, host or device; set resets Adam. */
wproj_status wproj_mlp_set_params(wproj_mlp *n, const float *params, void *stream);
wproj_status wproj_mlp_get_params(const wproj_mlp *n, float *params, void *stream);
/* Training data from a built plan (complex64, column indices), rows of uvw
 * (device, m x 3 as given to wproj_build_kernels): x0 (m x 3), tval (m x 2048),
 * tmask (m x 1024), device FP32. */
wproj_status wproj_mlp_targets(const wproj_plan *p, const double *uvw, float *x0, float *tval, float *tmask,
                               void *stream);
/* y (m x 3072) = network(x0) for m rows, m a multiple of 128.  Synchronous. */
wproj_status wproj_mlp_forward(wproj_mlp *n, const float *x0, int64_t m, float *y, void *stream);
/* loss (host) and, when grad (device or host, num_params floats) is given, the
 * gradient of the loss over the m rows (a multiple of 128, <= 65536).  Synchronous. */
wproj_status wproj_mlp_gradients(wproj_mlp *n, const float *x0, const float *tval, const float *tmask, int64_t m,
                                 double mask_weight, double *loss, float *grad, void *stream);
/* steps of Adam (beta 0.9, 0.999, eps 1e-8, learning rate lr) on batches of
 * `batch` consecutive rows, cycling through m rows (batch | m); losses (host,
 * steps floats, may be NULL) receives each step's loss.  Synchronous. */
wproj_status wproj_mlp_train(wproj_mlp *n, const float *x0, const float *tval, const float *tmask, int64_t m,
                             int32_t batch, int32_t steps, double lr, double mask_weight, float *losses,
                             void *stream);

/* Learned build: G by the plain build (COLUMNS, complex64 plans), then every
 * row's kernel predicted by the network and judged against the plain one on the
 * 32 x 32 window: a row takes the predicted values on its support only when the
 * relative L2 error over the window is <= rel_l2_max, the predicted support
 * holds >= e of the kernel energy and no plain entry lies outside the window;
 * every other row keeps the plain kernel (the fallback).  row_err (device, m
 * floats, may be NULL) receives each row's relative L2 error.  Synchronous. */
typedef struct {
  int64_t rows;
  int64_t learned;        /* rows that took the predicted kernel */
  double rel_l2_mean;     /* mean relative L2 error of the predictions */
  double plain_ms;        /* wall time of the plain build */
  double learned_ms;      /* wall time of inference and judging */
} wproj_learned_info;
wproj_status wproj_build_kernels_learned(wproj_plan *p, wproj_mlp *n, const double *uvw, int64_t m, double e,
                                         double rel_l2_max, float *row_err, wproj_learned_info *info,
                                         void *stream);

/* ---- batches of independent problems ------------------------------------------
 * Many imaging problems of uneven N and M (each a full Eq. 7 problem with its own
 * Phi, Section 3) held in one object.  Every stage of Phi, Phi^H and the
 * Douglas-Rachford iteration runs as one launch for all problems, and one DR
 * iteration is captured as a CUDA graph and replayed.  Batches store G with
 * column indices in complex64 (value_dtype F32; index_format AUTO or COLUMNS).
 *
 * Concatenated layouts (problems in order p = 0 .. n-1):
 *   images        x_p is N_p x N_p floats at offset sum_{q<p} N_q^2
 *   visibilities  y_p is m_p complex64 at offset sum_{q<p} m_q
 *   uvw           m_p x 3 doubles at offset 3 sum_{q<p} m_q
 * All arrays are caller-owned device pointers unless stated. */
typedef struct wproj_batch wproj_batch;

/* Work split of the batch operators: degridding row pieces of <= piece entries,
 * each taken by lanes_per_piece lanes of a warp (32, 16, 8 or 4: 32 / lanes pieces
 * per warp),
 * gridding chunks of about chunk entries of one grid tile. */
typedef struct {
  int64_t piece;
  int64_t chunk;
  double degrid_ms;     /* wproj_batch_tune: measured time of the chosen schedules */
  double grid_ms;
  int32_t lanes_per_piece;
} wproj_batch_schedule;

typedef struct {
  int32_t n_problems;
  int64_t m;            /* visibilities of all problems */
  int64_t pixels;       /* image pixels of all problems */
  int64_t nnz;          /* stored entries of all G */
  int64_t n_pieces, n_chunks, piece, chunk;
  int64_t launches;     /* kernels launched by batch operator and solver calls */
  int64_t iter_launches;  /* kernels in one captured Douglas-Rachford iteration */
  int32_t lanes_per_piece;  /* degridding lanes per row piece (32, 16, 8 or 4) */
} wproj_batch_info;

/* n problems (1 <= n <= 65535) with geometries descs[n] (host); each is validated
 * as by wproj_plan_create.  Other value dtypes or TILE_MASK: WPROJ_ERR_UNSUPPORTED. */
wproj_status wproj_batch_create(wproj_batch **out, int32_t n, const wproj_grid_desc *descs);
wproj_status wproj_batch_destroy(wproj_batch *b);

/* Part I for every problem: uvw concatenated as above (device), m[n] rows per
 * problem (host), energy fraction e as in wproj_build_kernels.  Synchronous.
 * Sets a default schedule (piece 1024, chunk 8192). */
wproj_status wproj_batch_build(wproj_batch *b, const double *uvw, const int64_t *m, double e, void *stream);

/* Times candidate schedules on this batch (pieces 64 .. 16384 entries taken by
 * 32, 16, 8 or 4 lanes, chunks 2048 .. 65536 entries), keeps the fastest of each; out
 * (host) may be NULL.  Synchronous. */
wproj_status wproj_batch_tune(wproj_batch *b, wproj_batch_schedule *out, void *stream);
/* Sets a schedule explicitly (piece, chunk >= 32; lanes_per_piece 32, 16, 8 or 4, 0
 * keeps the current one; anything else is WPROJ_ERR_INVALID_ARG).  Synchronous. */
wproj_status wproj_batch_set_schedule(wproj_batch *b, int64_t piece, int64_t chunk, int32_t lanes_per_piece,
                                      void *stream);

/* y = Phi x and x_re = Re Phi^H y for every problem (layouts above). */
wproj_status wproj_batch_phi(wproj_batch *b, const float *x, void *y, void *stream);
wproj_status wproj_batch_phi_adj(wproj_batch *b, const void *y, float *x_re, void *stream);

/* Eq. 7 for every problem by Douglas-Rachford as wproj_solve_bpdn, with eps[n]
 * (host) per problem and one parameter set; ||Phi_p||^2 is always estimated per
 * problem by prm->power_iters power iterations (prm->phi_norm2 is ignored).
 * prm->resume continues the batch's state.  The iterations replay a captured
 * CUDA graph (recaptured when y, inner_iters, lambda or the basis change).
 * x_out: all images, concatenated.  prm->psi selects the sparsity basis as for
 * wproj_solve_bpdn (0 Dirac, p Daubechies-p over prm->psi_levels levels; every
 * side must be divisible by 2^levels, else WPROJ_ERR_INVALID_ARG). */
wproj_status wproj_batch_solve_bpdn(wproj_batch *b, const void *y, const double *eps, const wproj_dr_params *prm,
                                    float *x_out, void *stream);
wproj_status wproj_batch_get_info(const wproj_batch *b, wproj_batch_info *out);

#ifdef __cplusplus
}
#endif

#endif /* WPROJ_H */
