// Internal state of a libwproj plan (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace wproj {

// Owning device allocation.
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  wproj_status alloc(size_t n);           // exact size, contents undefined
  wproj_status ensure(size_t n);          // grow (contents discarded)
  template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// One (row, tile) segment of G as the gridding reads it: entries [off, off+cnt)
// of row `row`, all inside one grid tile.
struct __align__(16) SegMeta {
  unsigned long long off_cnt;   // first entry (low 40 bits) | entry count << 40
  int seg;                      // segment id (row-major segment order)
  int row;
};
__host__ __device__ __forceinline__ long long meta_off(const SegMeta &m) {
  return (long long)(m.off_cnt & ((1ull << 40) - 1));
}
__host__ __device__ __forceinline__ int meta_cnt(const SegMeta &m) { return (int)(m.off_cnt >> 40); }

// One problem of a batch (wproj_batch): its geometry and where its arrays sit in
// the batch's concatenated buffers.
struct BProb {
  int N, G, logG, nT;
  int64_t m;
  int64_t img_off;     // images: N*N floats
  int64_t vis_off;     // visibilities
  int64_t grid_off;    // grids: G*G complex; also added to the stored columns
  int64_t inter_off;   // FFT intermediates: N*G complex
  int64_t inva_off;    // 1/a(l) tables: N floats
  int64_t tile_off;    // first of its nT*nT grid tiles in the batch's tile order
};

// The column-format operator arrays of a batch (concatenated over problems).
struct BatchOps {
  int64_t m = 0, n_pieces = 0, n_chunks = 0, n_tiles = 0;
  int lpp = 32;                          // degridding lanes per row piece (32, 16, 8 or 4)
  const int32_t *col = nullptr;          // columns + the problem's grid_off
  const void *val = nullptr;             // complex64
  const int32_t *piece_row = nullptr, *piece_len = nullptr, *row_piece_ptr = nullptr;
  const int64_t *piece_lo = nullptr;
  const int32_t *chunk_tile = nullptr, *chunk_prob = nullptr, *tile_chunk_ptr = nullptr, *tile_prob = nullptr;
  const int64_t *chunk_lo = nullptr, *chunk_hi = nullptr;
  const SegMeta *meta = nullptr;         // tile order, entry offsets and rows of the batch
  const BProb *tab = nullptr;
  // cell-major copy (rows local to their problem); null when absent
  const int64_t *tile_ent = nullptr;
  const uint32_t *cell_ent = nullptr;
  const void *cell_val = nullptr;
};

// Timing accumulator for one class of kernels.
// (TC_B*: the kernel build: box tables + box FFTs, selection + counts, emission)
enum TimerClass { TC_FFT = 0, TC_DEGRID, TC_GRID, TC_REDUCE, TC_SOLVER, TC_BFFT, TC_BSEL, TC_BEMIT, TC_COUNT };

struct EventTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  size_t used = 0;
  double ms[TC_COUNT] = {0};
  int64_t count[TC_COUNT] = {0};
  ~EventTimer();
  cudaEvent_t get();
};

struct GridGeom {
  int N, G, W;
  double L, du, B, beta;
  int chirp, extension, box;
  int value_dtype;
  int index_format;   // requested wproj_index_format
  int upsampling;     // 1: the paper's Fourier-space upsampling U instead of Z A
  int nT;        // tiles per axis = G / tile
  int tile;      // tile side (min(32, G))
};

}  // namespace wproj

struct wproj_plan {
  wproj::GridGeom g;
  int device = 0;

  // constant tables
  wproj::DevBuf twiddle;     // float2[kTwiddleLen]
  wproj::DevBuf inv_a;       // float[N]: 1 / a(l_p)

  // G
  bool built = false;
  int64_t m = 0, nnz = 0;
  int box_min = 0, box_max = 0;
  wproj::DevBuf row_ptr;     // int64[m+1]
  wproj::DevBuf col;         // int32[nnz]
  wproj::DevBuf val;         // float2 or 2x16-bit [nnz]
  wproj::DevBuf row_scale;   // float[m]
  int fmt = WPROJ_INDEX_COLUMNS;   // index format of the built G
  wproj::DevBuf stream;      // tile-stream records (TILE_MASK format), stream_bytes long
  int64_t stream_bytes = 0;
  wproj::DevBuf seg_rec;     // int64[n_seg] byte offset of each segment's record (TILE_MASK)
  wproj::DevBuf rec_off;     // int64[n_seg+1] byte offset of the records in stream order (TILE_MASK)
  wproj::DevBuf seg_tile;    // int32[n_seg] tile index of each segment
  // TILE_RUNS: the row-major copy of the degridding (runs padded to even lengths);
  // the tile-major records of the gridding live in `stream` / `rec_off` / `seg_rec`
  int64_t rm_runs = 0, rm_vals = 0;
  wproj::DevBuf rm_vptr;     // int64[m+1] first stored value of each row
  wproj::DevBuf rm_rptr;     // int64[m+1] first run of each row
  wproj::DevBuf rm_org;      // uint32[m] window origin (j0 - S/2) mod G: u | v << 16
  wproj::DevBuf rm_run;      // uint32[rm_runs] window row | window column << 6 | (length - 1) << 12
  wproj::DevBuf rm_val;      // values[rm_vals]
  wproj::DevBuf seg_base;    // int64[m+1] first segment of each row

  // segments: one per (row, touched tile), ordered by row then tile
  int64_t n_seg = 0;
  wproj::DevBuf seg_off;     // int64[n_seg]  first entry in col/val
  wproj::DevBuf seg_cnt;     // int32[n_seg]
  wproj::DevBuf seg_row;     // int32[n_seg]
  // gridding: segments sorted by tile (rows ascending), chunked by nnz
  wproj::DevBuf seg_meta;    // SegMeta[n_seg] in tile-sorted order (COLUMNS)
  // cell-major copy for the gridding (COLUMNS, m <= 2^22): per tile its entries
  // sorted by cell then row, packed (row << 10 | cell) with their values
  bool has_cells = false;
  wproj::DevBuf tile_ent;    // int64[nT*nT+1] first entry of each tile
  wproj::DevBuf cell_ent;    // uint32[nnz]
  wproj::DevBuf cell_val;    // values[nnz]
  int cell_parts = 1;        // blocks per tile of the cell-major gridding (small grids)
  wproj::DevBuf cell_partial;    // float2[nT*nT*cell_parts*1024] when cell_parts > 1
  int64_t n_chunks = 0;
  wproj::DevBuf chunk_tile;  // int32[n_chunks]
  wproj::DevBuf chunk_lo;    // int64[n_chunks]  first position in the tile order (seg_meta /
                             //                  stream records)
  wproj::DevBuf chunk_hi;    // int64[n_chunks]  end of the range
  wproj::DevBuf tile_chunk_ptr;  // int32[nT*nT+1]
  // degridding pieces: column format -> entry ranges; tile-mask format -> segment ranges
  int64_t n_pieces = 0;
  wproj::DevBuf piece_row;   // int32[n_pieces]
  wproj::DevBuf piece_lo;    // int64[n_pieces]  first entry / first segment
  wproj::DevBuf piece_len;   // int32[n_pieces]  entries / segments
  wproj::DevBuf row_piece_ptr;   // int32[m+1]

  // work buffers
  wproj::DevBuf Xt;          // float2[G*G]  F Z A x
  wproj::DevBuf Xt2;         // float2[G*G]  G^H y
  wproj::DevBuf inter;       // float2[N*G]  between FFT passes
  wproj::DevBuf grid_partial;    // float2[n_chunks * tile^2]
  wproj::DevBuf piece_partial;   // float2[degrid_partials]: per row piece (columns) or segment (mask)
  wproj::DevBuf xtmp;        // float[N*N]
  wproj::DevBuf ytmp;        // float2[m]
  // solver buffers
  wproj::DevBuf s_z, s_x, s_u, s_r, s_scal;   // scal: double scratch for reductions
  wproj::DevBuf s_zi, s_alpha, s_wwork;       // wavelet Psi: Psi z, Psi^T x, transform scratch
  // direction-dependent screens: float2[n_screens][G][G] (centred) and max |A|^2 of each
  int n_screens = 0;
  wproj::DevBuf screens, screen_max2;

  // Douglas-Rachford state kept for resume / checkpoint
  bool dr_valid = false;
  double dr_phi_norm2 = 0;

  double build_ms = 0;
  int64_t launches = 0;     // kernels launched by Phi, Phi^H and the solver
  bool timing = false;
  wproj::EventTimer timer;
};

namespace wproj {

// timing helpers (no-ops when timing is off)
struct ScopedTimer {
  wproj_plan *p;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  ScopedTimer(wproj_plan *p_, int cls_, cudaStream_t s_);
  ~ScopedTimer();
  void stop();   // end the interval now (the destructor then does nothing)
};

// fft.cu
wproj_status init_twiddles(wproj_plan *p, cudaStream_t s);
wproj_status make_twiddles(DevBuf &tw, cudaStream_t s);
wproj_status phi_forward_fft(wproj_plan *p, const float *x, const float2 *xc, float2 *Xt, cudaStream_t s);
// mode 0: x_re = Re(...), x_cplx optional; mode 1: x_re = z - Re(...)
wproj_status phi_adjoint_fft(wproj_plan *p, const float2 *Xt2, float *x_re, float2 *x_cplx,
                             const float *z, int mode, cudaStream_t s);
wproj_status fft2d_generic(const float2 *in, float2 *out, int n, int batch, int inverse,
                           const float2 *twiddle, cudaStream_t s);
// box FFT for the kernel build: nb boxes of S x S, in place; tables per box
struct BoxBatch;
wproj_status box_fft(wproj_plan *p, const BoxBatch &bb, cudaStream_t s);

wproj_status phi_forward_fft_into(wproj_plan *p, const float *x, float2 *inter, float2 *Xt, cudaStream_t s);
// batches: F Z A and A Z^H F^H for the np problems plist (device) of one grid size 2^logG
wproj_status batch_phi_fwd(int logG, int np, const int32_t *plist, const BProb *tab, const float *x,
                           const float *inv_a, float2 *inter, float2 *Xt, const float2 *tw, cudaStream_t s);
wproj_status batch_phi_adj(int logG, int np, const int32_t *plist, const BProb *tab, const float2 *Xt2,
                           const float *inv_a, float2 *inter, float *x_re, const float *z, int mode,
                           const float2 *tw, cudaStream_t s);

// build.cu: G from (u, v, w); sid (device, nullable): a screen per row (needs box = G)
wproj_status build_kernels_impl(wproj_plan *p, const double *uvw, int64_t m, double e, cudaStream_t s,
                                const int32_t *sid = nullptr);
wproj_status set_screens_impl(wproj_plan *p, const float2 *screens, int n, cudaStream_t s);

// wavelet.cu: the Daubechies basis; work holds N*N/2 floats
wproj_status daubechies_taps_impl(int p, double *h_out);
wproj_status dwt2_impl(int N, int levels, int p, const float *x, float *alpha, float *work, int64_t *launches,
                       cudaStream_t s);
wproj_status idwt2_impl(int N, int levels, int p, const float *alpha, float *x, float *work, int64_t *launches,
                        cudaStream_t s);
// every problem of a batch (tab[np] on the device, images at img_off); work: sum N^2/2 floats
wproj_status batch_dwt2(const BProb *tab, int np, int maxN, int levels, int p, const float *x, float *alpha,
                        float *work, int64_t *launches, cudaStream_t s);
wproj_status batch_idwt2(const BProb *tab, int np, int maxN, int levels, int p, const float *alpha, float *x,
                         float *work, int64_t *launches, cudaStream_t s);

// ops.cu
wproj_status degrid(wproj_plan *p, const float2 *Xt, float2 *y, cudaStream_t s);
wproj_status degrid_into(wproj_plan *p, const float2 *Xt, float2 *partial, float2 *y, cudaStream_t s);
wproj_status csr_rows(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                      cudaStream_t s);
int64_t degrid_partials(const wproj_plan *p);   // partial sums degridding needs

// cells.cu: cell-major gridding of the column format
constexpr int64_t kCellPad = 4;   // entries of padding after the cell-major copy
wproj_status build_cells(wproj_plan *p, const int64_t *tptr, const int64_t *cum, int64_t n_seg, cudaStream_t s);
wproj_status grid_cells(wproj_plan *p, const float2 *y, float2 *Xt2, cudaStream_t s);
wproj_status rebuild_cells(wproj_plan *p, cudaStream_t s);
wproj_status batch_grid_cells(const BatchOps &b, const float2 *y, float2 *Xt2, cudaStream_t s);

// gemm.cu: C = A B^T (+ bias) on the tcgen05 tensor cores, BF16 in, FP32 accumulate
wproj_status gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
                          void *C, bool out_bf16, int *err, cudaStream_t s);

// mlp.cu: the learned-kernel network
int64_t mlp_num_params();
wproj_status build_learned_impl(wproj_plan *p, wproj_mlp *n, const double *uvw, int64_t m, double e, double relmax,
                                float *row_err, wproj_learned_info *info, cudaStream_t s);

// batches (column format)
wproj_status batch_degrid(const BatchOps &b, const float2 *Xt, float2 *partial, float2 *y, cudaStream_t s);
wproj_status batch_grid(const BatchOps &b, const float2 *y, float2 *partial, float2 *Xt2, cudaStream_t s);

// tiles.cu (tile-stream records, TILE_MASK format)
int64_t degrid_stream_partials(const wproj_plan *p);
wproj_status degrid_stream(wproj_plan *p, const float2 *Xt, float2 *partial, cudaStream_t s);
wproj_status degrid_stream_reduce(wproj_plan *p, const float2 *partial, float2 *y, cudaStream_t s);
wproj_status grid_stream(wproj_plan *p, const float2 *y, cudaStream_t s);
wproj_status stream_export(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                           cudaStream_t s);
wproj_status grid(wproj_plan *p, const float2 *y, float2 *Xt2, cudaStream_t s);
wproj_status apply_phi(wproj_plan *p, const float *x, const float2 *xc, float2 *y, cudaStream_t s);
wproj_status apply_phi_adj(wproj_plan *p, const float2 *y, float *x_re, float2 *x_cplx,
                           const float *z, int mode, cudaStream_t s);

// runs.cu (TILE_RUNS format): both copies from the column form in col / val, which
// is then released; tile_seg / tptr = segments in tile order, compacted in place
// to the n_rec segments that hold entries
wproj_status build_runs(wproj_plan *p, const int2 *j0, const int32_t *Sk, int32_t *tile_seg, int64_t *tptr,
                        int64_t *n_rec, cudaStream_t s);
wproj_status degrid_runs(wproj_plan *p, const float2 *Xt, float2 *y, cudaStream_t s);
wproj_status grid_runs(wproj_plan *p, const float2 *y, float2 *Xt2, int *launches, cudaStream_t s);
wproj_status runs_export(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                         cudaStream_t s);

// build.cu: work units shared by plans and batches
// row pieces of <= piece entries (m rows, row_ptr[m+1])
wproj_status make_row_pieces(int64_t m, const int64_t *row_ptr, int64_t piece, DevBuf &piece_row, DevBuf &piece_lo,
                             DevBuf &piece_len, DevBuf &row_piece_ptr, int64_t *n_pieces, cudaStream_t s);
// chunks of about `chunk` entries of each tile's segments [tptr[t], tptr[t+1]) (cum = entry prefix)
wproj_status make_tile_chunks(int n_tiles, const int64_t *tptr, const int64_t *cum, int64_t n_seg, int64_t nnz,
                              int64_t chunk, DevBuf &chunk_tile, DevBuf &chunk_lo, DevBuf &chunk_hi,
                              DevBuf &tile_chunk_ptr, int64_t *n_chunks, cudaStream_t s);

// scan.cu
wproj_status exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
wproj_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// stable counting sort of ids [0, n) by key[i] in [0, n_bins): out_ids, bin_ptr[n_bins+1]
wproj_status stable_bin_sort(const int32_t *key, int64_t n, int n_bins, int32_t *out_ids,
                             int64_t *bin_ptr, cudaStream_t s);

}  // namespace wproj
