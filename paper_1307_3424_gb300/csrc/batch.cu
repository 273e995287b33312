// Batches of independent imaging problems of uneven size (wproj_batch_*).
//
// Each problem is built by the plan builder (Part I, column format, complex64)
// and then concatenated into one set of arrays: images, visibilities, grids,
// G (columns offset by the problem's grid offset, so one gather array serves
// all problems), the tile-ordered segment list and the 1/a tables.  Every stage
// of Phi, Phi^H and the Douglas-Rachford iteration (Section 2.3) then runs as
// one launch for the whole batch: the FFT passes once per grid size (blockIdx.y
// = problem), the degridding over all row pieces, the gridding over all tile
// chunks, and the solver's per-problem reductions as (blocks, problem) grids.
// One DR iteration is captured as a CUDA graph and replayed.  The row-piece
// size of the degridding and the chunk size of the gridding are picked by
// timing candidate schedules on the batch (batch_tune).
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fft.cuh"
#include "plan.h"

namespace wproj {
}

struct wproj_batch {
  int np = 0;
  std::vector<wproj_grid_desc> desc;
  std::vector<wproj::BProb> prob;
  wproj::DevBuf tab;   // BProb[np]
  struct Cls {
    int logG = 0, np = 0;
    wproj::DevBuf plist;
  };
  Cls cls[wproj::kMaxLogN + 1];   // problems by grid size 2^logG (np = 0: none)
  int64_t m = 0, img = 0, grid = 0, inter = 0, inva = 0, nnz = 0, nseg = 0, tiles = 0;
  int64_t max_m = 0, max_img = 0;
  wproj::DevBuf twiddle, inv_a;
  // G of all problems
  bool built = false;
  wproj::DevBuf row_ptr, col, val, meta, tptr, cum, tile_prob;
  bool has_cells = false;   // cell-major copy for the gridding (every problem has one)
  wproj::DevBuf tile_ent, cell_ent, cell_val;
  // schedule
  int64_t piece = 0, chunk = 0, n_pieces = 0, n_chunks = 0;
  int lpp = 32;   // degridding lanes per row piece (32, 16, 8 or 4: the row-split schedule)
  wproj::DevBuf piece_row, piece_lo, piece_len, row_piece_ptr;
  wproj::DevBuf chunk_tile, chunk_lo, chunk_hi, chunk_prob, tile_chunk_ptr;
  wproj::DevBuf piece_partial, grid_partial;
  // work buffers and Douglas-Rachford state
  wproj::DevBuf Xt, Xt2, interb, x, z, u, r, xtmp, scal, part, eps, mu;
  wproj::DevBuf zi, alpha, wwork;   // wavelet Psi: Psi z, Psi^T x, transform scratch
  int max_n = 0;                    // largest image side
  int pow2_div = 0;                 // largest power of two dividing every side
  bool dr_valid = false;
  // one DR iteration captured as a graph
  cudaStream_t cap = nullptr;
  cudaGraphExec_t dr_exec = nullptr;
  const void *graph_y = nullptr;
  int graph_inner = -1;
  double graph_lambda = 0;
  int graph_psi = -1, graph_levels = -1;
  int64_t iter_launches = 0;   // kernels in the captured iteration
  int64_t launches = 0;        // kernels launched by operator and solver calls
  ~wproj_batch() {
    if (dr_exec) cudaGraphExecDestroy(dr_exec);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace wproj {

namespace {

constexpr int kBT = 256;          // threads of the per-problem passes
constexpr int kScal = 8;          // doubles of per-problem solver scalars
// scal[8p + 0] ball scale * mu, 1 ||d||, 2 gamma, 3 power-iteration sum

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

int nbx_for(int64_t n) { return (int)std::min<int64_t>(64, std::max<int64_t>(1, ceil_div(n, kBT))); }

// ---- concatenation ----------------------------------------------------------------

__global__ void k_add_i32(int64_t n, const int32_t *__restrict__ src, int32_t add, int32_t *__restrict__ dst) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i] + add;
}
__global__ void k_add_i64(int64_t n, const int64_t *__restrict__ src, int64_t add, int64_t *__restrict__ dst) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i] + add;
}
__global__ void k_cat_meta(int64_t n, const SegMeta *__restrict__ src, int64_t ent_add, int row_add,
                           SegMeta *__restrict__ dst) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    SegMeta m = src[i];
    m.off_cnt = (unsigned long long)(meta_off(m) + ent_add) | ((unsigned long long)meta_cnt(m) << 40);
    m.row += row_add;
    dst[i] = m;
  }
}
// first segment of every tile of one problem, from its chunk list
__global__ void k_cat_tptr(int n_tiles, const int64_t *__restrict__ chunk_lo, const int32_t *__restrict__ tile_chunk_ptr,
                           int64_t seg_add, int prob, int64_t *__restrict__ tptr, int32_t *__restrict__ tile_prob) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  tptr[t] = seg_add + chunk_lo[tile_chunk_ptr[t]];
  tile_prob[t] = prob;
}
__global__ void k_meta_cnt(int64_t n, const SegMeta *__restrict__ meta, int32_t *__restrict__ cnt) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    cnt[i] = meta_cnt(meta[i]);
}
// batch tile index -> problem and local tile
__global__ void k_chunk_prob(int64_t n, const int32_t *__restrict__ tile_prob, const BProb *__restrict__ tab,
                             int32_t *__restrict__ chunk_tile, int32_t *__restrict__ chunk_prob) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int t = chunk_tile[c];
  const int p = tile_prob[t];
  chunk_prob[c] = p;
  chunk_tile[c] = t - int(tab[p].tile_off);
}

// ---- per-problem solver passes (blockIdx.y = problem) ---------------------------------

__global__ void __launch_bounds__(kBT)
k_bs_dual_residual(const BProb *__restrict__ tab, const float2 *__restrict__ u, float2 *__restrict__ r,
                   const float2 *__restrict__ y, const double *__restrict__ mu, double *__restrict__ part) {
  const BProb P = tab[blockIdx.y];
  const float inv_mu = float(1.0 / mu[blockIdx.y]);
  double acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.m; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = P.vis_off + i;
    const float2 uu = u[k], rr = r[k], yy = y[k];
    const float2 d = make_float2(uu.x * inv_mu + rr.x - yy.x, uu.y * inv_mu + rr.y - yy.y);
    r[k] = d;
    acc += double(d.x) * d.x + double(d.y) * d.y;
  }
  const double t = block_sum_d<kBT>(acc);
  if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

// thread per problem: scal[0] = max(0, 1 - eps/||d||) mu, scal[1] = ||d||
__global__ void k_bs_ball_scale(int np, int nbx, const double *__restrict__ part, const double *__restrict__ eps,
                                const double *__restrict__ mu, double *__restrict__ scal) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double s = 0;
  for (int i = 0; i < nbx; ++i) s += part[int64_t(p) * nbx + i];
  const double nd = sqrt(s);
  const double f = (nd > 0) ? fmax(0.0, 1.0 - eps[p] / nd) : 0.0;
  scal[p * kScal + 0] = f * mu[p];
  scal[p * kScal + 1] = nd;
}

__global__ void k_bs_dual_update(const BProb *__restrict__ tab, const float2 *__restrict__ d,
                                 const double *__restrict__ scal, float2 *__restrict__ u) {
  const BProb P = tab[blockIdx.y];
  const float f = float(scal[blockIdx.y * kScal + 0]);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P.m; i += int64_t(gridDim.x) * blockDim.x)
    u[P.vis_off + i] = cscale(d[P.vis_off + i], f);
}

// z = z + lambda (soft(2x - z, gamma) - x)
__global__ void k_bs_dr_update(const BProb *__restrict__ tab, const float *__restrict__ x, float *__restrict__ z,
                               float lambda, const double *__restrict__ scal) {
  const BProb P = tab[blockIdx.y];
  const float gamma = float(scal[blockIdx.y * kScal + 2]);
  const int64_t n = int64_t(P.N) * P.N;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t o = P.img_off + i;
    const float xi = x[o], zi = z[o];
    const float a = 2.f * xi - zi;
    const float sa = copysignf(fmaxf(fabsf(a) - gamma, 0.f), a);
    z[o] = zi + lambda * (sa - xi);
  }
}

// per problem: max |x| (MODE 0) or sum x^2 (MODE 1) over its image, block partials
template <int MODE>
__global__ void __launch_bounds__(kBT)
k_bs_image_part(const BProb *__restrict__ tab, const float *__restrict__ x, double *__restrict__ part) {
  const BProb P = tab[blockIdx.y];
  const int64_t n = int64_t(P.N) * P.N;
  double acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = x[P.img_off + i];
    acc = MODE == 0 ? fmax(acc, fabs(v)) : acc + v * v;
  }
  if (MODE == 0) {
    for (int o = 16; o; o >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __shared__ double red[kBT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int i = 0; i < kBT / 32; ++i) t = fmax(t, red[i]);
      part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
  } else {
    const double t = block_sum_d<kBT>(acc);
    if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

// thread per problem: MODE 0: scal[2] = frac * max(part); MODE 1: scal[3] = sum(part)
template <int MODE>
__global__ void k_bs_image_scalar(int np, int nbx, const double *__restrict__ part, double frac,
                                  double *__restrict__ scal) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double v = 0;
  for (int i = 0; i < nbx; ++i) v = MODE == 0 ? fmax(v, part[int64_t(p) * nbx + i]) : v + part[int64_t(p) * nbx + i];
  if (MODE == 0) scal[p * kScal + 2] = frac * v;
  else scal[p * kScal + 3] = v;
}

// x = z / sqrt(scal[3]) (power iteration), or the unit impulse at the image centre
// (start) when scal is null
__global__ void k_bs_scale_image(const BProb *__restrict__ tab, const float *__restrict__ z,
                                 const double *__restrict__ scal, float *__restrict__ x) {
  const BProb P = tab[blockIdx.y];
  const int64_t n = int64_t(P.N) * P.N;
  const float f = scal ? float(1.0 / sqrt(scal[blockIdx.y * kScal + 3])) : 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[P.img_off + i] = scal ? z[P.img_off + i] * f : (i == int64_t(P.N / 2) * P.N + P.N / 2 ? 1.f : 0.f);
}

// ||Phi||^2 = sqrt(sum) of the last power iteration; mu = 1 / ||Phi||^2
__global__ void k_bs_mu(int np, const double *__restrict__ scal, double *__restrict__ mu) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) mu[p] = 1.0 / sqrt(scal[p * kScal + 3]);
}

// ---- the batch operators ------------------------------------------------------------

BatchOps ops_of(const wproj_batch *b) {
  BatchOps o;
  o.m = b->m;
  o.n_pieces = b->n_pieces;
  o.n_chunks = b->n_chunks;
  o.lpp = b->lpp;
  o.n_tiles = b->tiles;
  o.col = b->col.as<int32_t>();
  o.val = b->val.ptr;
  o.piece_row = b->piece_row.as<int32_t>();
  o.piece_len = b->piece_len.as<int32_t>();
  o.row_piece_ptr = b->row_piece_ptr.as<int32_t>();
  o.piece_lo = b->piece_lo.as<int64_t>();
  o.chunk_tile = b->chunk_tile.as<int32_t>();
  o.chunk_prob = b->chunk_prob.as<int32_t>();
  o.tile_chunk_ptr = b->tile_chunk_ptr.as<int32_t>();
  o.tile_prob = b->tile_prob.as<int32_t>();
  o.chunk_lo = b->chunk_lo.as<int64_t>();
  o.chunk_hi = b->chunk_hi.as<int64_t>();
  o.meta = b->meta.as<SegMeta>();
  o.tab = b->tab.as<BProb>();
  if (b->has_cells) {
    o.tile_ent = b->tile_ent.as<int64_t>();
    o.cell_ent = b->cell_ent.as<uint32_t>();
    o.cell_val = b->cell_val.ptr;
  }
  return o;
}

wproj_status bphi(wproj_batch *b, const float *x, float2 *y, cudaStream_t s) {
  for (auto &c : b->cls) {
    if (c.np == 0) continue;
    WPROJ_TRY(batch_phi_fwd(c.logG, c.np, c.plist.as<int32_t>(), b->tab.as<BProb>(), x, b->inv_a.as<float>(),
                            b->interb.as<float2>(), b->Xt.as<float2>(), b->twiddle.as<float2>(), s));
    b->launches += 2;
  }
  b->launches += 2;
  return batch_degrid(ops_of(b), b->Xt.as<float2>(), b->piece_partial.as<float2>(), y, s);
}

// mode 0: x_re = Re Phi^H y; mode 1: x_re = z - Re Phi^H y
wproj_status bphi_adj(wproj_batch *b, const float2 *y, float *x_re, const float *z, int mode, cudaStream_t s) {
  WPROJ_TRY(batch_grid(ops_of(b), y, b->grid_partial.as<float2>(), b->Xt2.as<float2>(), s));
  b->launches += 2;
  for (auto &c : b->cls) {
    if (c.np == 0) continue;
    WPROJ_TRY(batch_phi_adj(c.logG, c.np, c.plist.as<int32_t>(), b->tab.as<BProb>(), b->Xt2.as<float2>(),
                            b->inv_a.as<float>(), b->interb.as<float2>(), x_re, z, mode, b->twiddle.as<float2>(), s));
    b->launches += 2;
  }
  return WPROJ_OK;
}

wproj_status set_pieces(wproj_batch *b, int64_t piece, cudaStream_t s) {
  WPROJ_TRY(make_row_pieces(b->m, b->row_ptr.as<int64_t>(), piece, b->piece_row, b->piece_lo, b->piece_len,
                            b->row_piece_ptr, &b->n_pieces, s));
  WPROJ_TRY(b->piece_partial.alloc(sizeof(float2) * std::max<int64_t>(1, b->n_pieces)));
  b->piece = piece;
  if (b->dr_exec) {   // the captured iteration holds the old buffers
    cudaGraphExecDestroy(b->dr_exec);
    b->dr_exec = nullptr;
  }
  return WPROJ_OK;
}

wproj_status set_chunks(wproj_batch *b, int64_t chunk, cudaStream_t s) {
  WPROJ_TRY(make_tile_chunks((int)b->tiles, b->tptr.as<int64_t>(), b->cum.as<int64_t>(), b->nseg, b->nnz, chunk,
                             b->chunk_tile, b->chunk_lo, b->chunk_hi, b->tile_chunk_ptr, &b->n_chunks, s));
  WPROJ_TRY(b->chunk_prob.alloc(sizeof(int32_t) * std::max<int64_t>(1, b->n_chunks)));
  k_chunk_prob<<<ceil_div(b->n_chunks, 256), 256, 0, s>>>(b->n_chunks, b->tile_prob.as<int32_t>(),
                                                          b->tab.as<BProb>(), b->chunk_tile.as<int32_t>(),
                                                          b->chunk_prob.as<int32_t>());
  WPROJ_CHECK_LAUNCH("chunk problems");
  WPROJ_TRY(b->grid_partial.alloc(sizeof(float2) * size_t(std::max<int64_t>(1, b->n_chunks)) * kTile * kTile));
  b->chunk = chunk;
  if (b->dr_exec) {   // the captured iteration holds the old buffers
    cudaGraphExecDestroy(b->dr_exec);
    b->dr_exec = nullptr;
  }
  return WPROJ_OK;
}

wproj_status ensure_solver(wproj_batch *b) {
  WPROJ_TRY(b->x.ensure(sizeof(float) * b->img));
  WPROJ_TRY(b->z.ensure(sizeof(float) * b->img));
  WPROJ_TRY(b->xtmp.ensure(sizeof(float) * b->img));
  WPROJ_TRY(b->u.ensure(sizeof(float2) * std::max<int64_t>(1, b->m)));
  WPROJ_TRY(b->r.ensure(sizeof(float2) * std::max<int64_t>(1, b->m)));
  WPROJ_TRY(b->scal.ensure(sizeof(double) * kScal * b->np));
  WPROJ_TRY(b->part.ensure(sizeof(double) * 64 * b->np));
  WPROJ_TRY(b->eps.ensure(sizeof(double) * b->np));
  WPROJ_TRY(b->mu.ensure(sizeof(double) * b->np));
  return WPROJ_OK;
}

// One Douglas-Rachford iteration of every problem (launches only: graph-capturable).
// psi > 0: z holds Daubechies-psi coefficients; the projection runs on zi = Psi z
// and its result is analysed again before the update (exact: Psi is orthonormal).
wproj_status dr_iteration(wproj_batch *b, const float2 *y, int inner, float lambda, int psi, int levels,
                          cudaStream_t s) {
  const BProb *tab = b->tab.as<BProb>();
  float *zc = b->z.as<float>(), *x = b->x.as<float>();
  float *z = psi ? b->zi.as<float>() : zc;   // the image the projection starts from
  if (psi) WPROJ_TRY(batch_idwt2(tab, b->np, b->max_n, levels, psi, zc, z, b->wwork.as<float>(), &b->launches, s));
  float2 *u = b->u.as<float2>(), *r = b->r.as<float2>();
  double *scal = b->scal.as<double>(), *part = b->part.as<double>();
  const int nbm = nbx_for(b->max_m), nbn = nbx_for(b->max_img);
  for (int j = 0; j < inner; ++j) {
    WPROJ_TRY(bphi_adj(b, u, x, z, 1, s));   // x = z - Re Phi^H u
    WPROJ_TRY(bphi(b, x, r, s));             // r = Phi x
    k_bs_dual_residual<<<dim3(nbm, b->np), kBT, 0, s>>>(tab, u, r, y, b->mu.as<double>(), part);
    k_bs_ball_scale<<<ceil_div(b->np, 128), 128, 0, s>>>(b->np, nbm, part, b->eps.as<double>(), b->mu.as<double>(),
                                                         scal);
    k_bs_dual_update<<<dim3(nbm, b->np), kBT, 0, s>>>(tab, r, scal, u);
    WPROJ_CHECK_LAUNCH("batch dual step");
    b->launches += 3;
  }
  WPROJ_TRY(bphi_adj(b, u, x, z, 1, s));     // x = P_B(z)
  float *px = x;
  if (psi) {
    px = b->alpha.as<float>();
    WPROJ_TRY(batch_dwt2(tab, b->np, b->max_n, levels, psi, x, px, b->wwork.as<float>(), &b->launches, s));
  }
  k_bs_dr_update<<<dim3(nbn, b->np), kBT, 0, s>>>(tab, px, zc, lambda, scal);
  WPROJ_CHECK_LAUNCH("batch dr update");
  b->launches += 1;
  return WPROJ_OK;
}

// ||Phi_p||^2 of every problem by power iteration from the centre impulse, then mu_p
wproj_status power_mu(wproj_batch *b, int iters, cudaStream_t s) {
  const BProb *tab = b->tab.as<BProb>();
  float *x = b->xtmp.as<float>(), *z = b->x.as<float>();
  float2 *r = b->r.as<float2>();
  double *scal = b->scal.as<double>(), *part = b->part.as<double>();
  const int nbn = nbx_for(b->max_img);
  k_bs_scale_image<<<dim3(nbn, b->np), kBT, 0, s>>>(tab, nullptr, nullptr, x);
  WPROJ_CHECK_LAUNCH("batch power start");
  for (int it = 0; it < iters; ++it) {
    WPROJ_TRY(bphi(b, x, r, s));
    WPROJ_TRY(bphi_adj(b, r, z, nullptr, 0, s));
    k_bs_image_part<1><<<dim3(nbn, b->np), kBT, 0, s>>>(tab, z, part);
    k_bs_image_scalar<1><<<ceil_div(b->np, 128), 128, 0, s>>>(b->np, nbn, part, 0.0, scal);
    k_bs_scale_image<<<dim3(nbn, b->np), kBT, 0, s>>>(tab, z, scal, x);
    WPROJ_CHECK_LAUNCH("batch power iteration");
  }
  k_bs_mu<<<ceil_div(b->np, 128), 128, 0, s>>>(b->np, scal, b->mu.as<double>());
  WPROJ_CHECK_LAUNCH("batch mu");
  return WPROJ_OK;
}

template <class F>
wproj_status time_ms(F &&f, int reps, cudaStream_t s, double *ms) {
  cudaEvent_t a, c;
  WPROJ_CUDA(cudaEventCreate(&a));
  WPROJ_CUDA(cudaEventCreate(&c));
  wproj_status st = f();   // warm-up
  if (st == WPROJ_OK) {
    cudaEventRecord(a, s);
    for (int i = 0; i < reps && st == WPROJ_OK; ++i) st = f();
    cudaEventRecord(c, s);
    cudaEventSynchronize(c);
    float t = 0;
    cudaEventElapsedTime(&t, a, c);
    *ms = t / reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(c);
  return st;
}

}  // namespace

wproj_status batch_build_impl(wproj_batch *b, const double *uvw, const int64_t *m, double e, cudaStream_t s) {
  b->built = false;
  b->dr_valid = false;
  if (b->dr_exec) {
    cudaGraphExecDestroy(b->dr_exec);
    b->dr_exec = nullptr;
  }
  const int np = b->np;
  // ---- build every problem with the plan builder
  std::vector<wproj_plan *> plans(np, nullptr);
  struct Guard {
    std::vector<wproj_plan *> &v;
    ~Guard() {
      for (auto *p : v) if (p) wproj_plan_destroy(p);
    }
  } guard{plans};
  int64_t vis = 0;
  for (int p = 0; p < np; ++p) {
    wproj_grid_desc d = b->desc[p];
    d.index_format = WPROJ_INDEX_COLUMNS;
    WPROJ_TRY(wproj_plan_create(&plans[p], &d));
    WPROJ_TRY(build_kernels_impl(plans[p], uvw + 3 * vis, m[p], e, s));
    vis += m[p];
  }
  // ---- offsets
  b->prob.assign(np, BProb{});
  int64_t img = 0, grid = 0, inter = 0, inva = 0, nnz = 0, nseg = 0, tiles = 0;
  vis = 0;
  b->max_m = b->max_img = 0;
  b->max_n = 0;
  b->pow2_div = 1 << 30;
  for (int p = 0; p < np; ++p) {
    const wproj_plan *pl = plans[p];
    BProb &P = b->prob[p];
    P.N = pl->g.N;
    P.G = pl->g.G;
    P.logG = ilog2(P.G);
    P.nT = pl->g.nT;
    P.m = pl->m;
    P.img_off = img;
    P.vis_off = vis;
    P.grid_off = grid;
    P.inter_off = inter;
    P.inva_off = inva;
    P.tile_off = tiles;
    img += int64_t(P.N) * P.N;
    vis += P.m;
    grid += int64_t(P.G) * P.G;
    inter += int64_t(P.N) * P.G;
    inva += P.N;
    nnz += pl->nnz;
    nseg += pl->n_seg;
    tiles += int64_t(P.nT) * P.nT;
    b->max_m = std::max(b->max_m, P.m);
    b->max_img = std::max<int64_t>(b->max_img, int64_t(P.N) * P.N);
    b->max_n = std::max(b->max_n, P.N);
    b->pow2_div = std::min(b->pow2_div, P.N & -P.N);
  }
  if (grid >= (int64_t(1) << 31)) return fail(WPROJ_ERR_UNSUPPORTED, "batch: grids exceed 2^31 cells in total");
  b->m = vis;
  b->img = img;
  b->grid = grid;
  b->inter = inter;
  b->inva = inva;
  b->nnz = nnz;
  b->nseg = nseg;
  b->tiles = tiles;
  WPROJ_TRY(b->tab.alloc(sizeof(BProb) * np));
  WPROJ_CUDA(cudaMemcpyAsync(b->tab.ptr, b->prob.data(), sizeof(BProb) * np, cudaMemcpyHostToDevice, s));
  // ---- concatenate G and the per-problem tables
  WPROJ_TRY(b->row_ptr.alloc(sizeof(int64_t) * (vis + 1)));
  WPROJ_TRY(b->col.alloc(sizeof(int32_t) * std::max<int64_t>(1, nnz)));
  WPROJ_TRY(b->val.alloc(sizeof(float2) * std::max<int64_t>(1, nnz)));
  WPROJ_TRY(b->meta.alloc(sizeof(SegMeta) * std::max<int64_t>(1, nseg)));
  WPROJ_TRY(b->tptr.alloc(sizeof(int64_t) * (tiles + 1)));
  WPROJ_TRY(b->tile_prob.alloc(sizeof(int32_t) * tiles));
  WPROJ_TRY(b->inv_a.alloc(sizeof(float) * inva));
  b->has_cells = true;
  for (auto *pl : plans) b->has_cells = b->has_cells && pl->has_cells;
  if (b->has_cells) {
    WPROJ_TRY(b->tile_ent.alloc(sizeof(int64_t) * (tiles + 1)));
    // 4 entries of padding: the gridding reads whole 16-byte words of 4 entries
    WPROJ_TRY(b->cell_ent.alloc(sizeof(uint32_t) * (nnz + kCellPad)));
    WPROJ_TRY(b->cell_val.alloc(sizeof(float2) * (nnz + kCellPad)));
  } else {
    b->tile_ent.release();
    b->cell_ent.release();
    b->cell_val.release();
  }
  int64_t ent = 0, sg = 0;
  for (int p = 0; p < np; ++p) {
    wproj_plan *pl = plans[p];
    const BProb &P = b->prob[p];
    const int nt = P.nT * P.nT;
    if (pl->nnz > 0) {
      k_add_i32<<<std::min(ceil_div(pl->nnz, 256), 152 * 8), 256, 0, s>>>(pl->nnz, pl->col.as<int32_t>(),
                                                                          int32_t(P.grid_off), b->col.as<int32_t>() + ent);
      WPROJ_CUDA(cudaMemcpyAsync(b->val.as<float2>() + ent, pl->val.ptr, sizeof(float2) * pl->nnz,
                                 cudaMemcpyDeviceToDevice, s));
    }
    k_add_i64<<<std::max(1, std::min(ceil_div(P.m, 256), 152 * 8)), 256, 0, s>>>(
        P.m, pl->row_ptr.as<int64_t>(), ent, b->row_ptr.as<int64_t>() + P.vis_off);
    if (pl->n_seg > 0)
      k_cat_meta<<<std::min(ceil_div(pl->n_seg, 256), 152 * 8), 256, 0, s>>>(
          pl->n_seg, pl->seg_meta.as<SegMeta>(), ent, int(P.vis_off), b->meta.as<SegMeta>() + sg);
    k_cat_tptr<<<ceil_div(nt, 256), 256, 0, s>>>(nt, pl->chunk_lo.as<int64_t>(), pl->tile_chunk_ptr.as<int32_t>(), sg,
                                                 p, b->tptr.as<int64_t>() + P.tile_off,
                                                 b->tile_prob.as<int32_t>() + P.tile_off);
    WPROJ_CHECK_LAUNCH("batch concatenation");
    WPROJ_CUDA(cudaMemcpyAsync(b->inv_a.as<float>() + P.inva_off, pl->inv_a.ptr, sizeof(float) * P.N,
                               cudaMemcpyDeviceToDevice, s));
    if (b->has_cells) {   // rows stay local to the problem; tiles and entries shift
      k_add_i64<<<ceil_div(nt, 256), 256, 0, s>>>(nt, pl->tile_ent.as<int64_t>(), ent,
                                                  b->tile_ent.as<int64_t>() + P.tile_off);
      if (pl->nnz > 0) {
        WPROJ_CUDA(cudaMemcpyAsync(b->cell_ent.as<uint32_t>() + ent, pl->cell_ent.ptr, sizeof(uint32_t) * pl->nnz,
                                   cudaMemcpyDeviceToDevice, s));
        WPROJ_CUDA(cudaMemcpyAsync(b->cell_val.as<float2>() + ent, pl->cell_val.ptr, sizeof(float2) * pl->nnz,
                                   cudaMemcpyDeviceToDevice, s));
      }
      WPROJ_CHECK_LAUNCH("batch cell concatenation");
    }
    ent += pl->nnz;
    sg += pl->n_seg;
  }
  WPROJ_CUDA(cudaMemcpyAsync(b->row_ptr.as<int64_t>() + vis, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  WPROJ_CUDA(cudaMemcpyAsync(b->tptr.as<int64_t>() + tiles, &nseg, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  if (b->has_cells)
    WPROJ_CUDA(cudaMemcpyAsync(b->tile_ent.as<int64_t>() + tiles, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  // entry prefix over the tile-ordered segments (chunk balancing)
  {
    DevBuf cnt;
    WPROJ_TRY(cnt.alloc(sizeof(int32_t) * std::max<int64_t>(1, nseg)));
    WPROJ_TRY(b->cum.alloc(sizeof(int64_t) * std::max<int64_t>(1, nseg)));
    if (nseg > 0) {
      k_meta_cnt<<<std::min(ceil_div(nseg, 256), 152 * 8), 256, 0, s>>>(nseg, b->meta.as<SegMeta>(), cnt.as<int32_t>());
      WPROJ_CHECK_LAUNCH("batch segment counts");
      WPROJ_TRY(exclusive_scan_i32_to_i64(cnt.as<int32_t>(), b->cum.as<int64_t>(), nseg, s));
    }
    WPROJ_CUDA(cudaStreamSynchronize(s));
  }
  // the plans' G is no longer needed
  for (auto *&p : plans) {
    wproj_plan_destroy(p);
    p = nullptr;
  }
  // ---- size classes, work buffers, a default schedule
  for (int lg = 0; lg <= kMaxLogN; ++lg) {
    wproj_batch::Cls &c = b->cls[lg];
    c.np = 0;
    c.plist.release();
    std::vector<int32_t> ids;
    for (int p = 0; p < np; ++p)
      if (b->prob[p].logG == lg) ids.push_back(p);
    if (ids.empty()) continue;
    c.logG = lg;
    c.np = (int)ids.size();
    WPROJ_TRY(c.plist.alloc(sizeof(int32_t) * ids.size()));
    WPROJ_CUDA(cudaMemcpy(c.plist.ptr, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice));
  }
  WPROJ_TRY(b->Xt.alloc(sizeof(float2) * grid));
  WPROJ_TRY(b->Xt2.alloc(sizeof(float2) * grid));
  WPROJ_TRY(b->interb.alloc(sizeof(float2) * inter));
  WPROJ_TRY(ensure_solver(b));
  WPROJ_TRY(set_pieces(b, 1024, s));
  WPROJ_TRY(set_chunks(b, 8192, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  b->built = true;
  return WPROJ_OK;
}

wproj_status batch_tune_impl(wproj_batch *b, wproj_batch_schedule *out, cudaStream_t s) {
  static const int64_t pieces[] = {64, 256, 512, 1024, 2048, 4096, 16384};
  static const int lanes[] = {32, 16, 8, 4};
  static const int64_t chunks[] = {2048, 4096, 8192, 16384, 65536};
  double best = 1e30;
  int64_t bp = b->piece;
  int bl = b->lpp;
  WPROJ_CUDA(cudaMemsetAsync(b->Xt.ptr, 0, sizeof(float2) * b->grid, s));
  WPROJ_CUDA(cudaMemsetAsync(b->u.ptr, 0, sizeof(float2) * b->m, s));
  // row split: pieces of at most `piece` entries, each taken by 32, 16, 8 or 4 lanes
  for (int64_t pc : pieces) {
    WPROJ_TRY(set_pieces(b, pc, s));
    for (int l : lanes) {
      b->lpp = l;
      double ms = 0;
      WPROJ_TRY(time_ms([&] { return batch_degrid(ops_of(b), b->Xt.as<float2>(), b->piece_partial.as<float2>(),
                                                  b->r.as<float2>(), s); }, 5, s, &ms));
      if (ms < best) { best = ms; bp = pc; bl = l; }
    }
  }
  const double deg_ms = best;
  b->lpp = bl;
  WPROJ_TRY(set_pieces(b, bp, s));
  best = 1e30;
  int64_t bc = b->chunk;
  for (int64_t ch : chunks) {
    WPROJ_TRY(set_chunks(b, ch, s));
    double ms = 0;
    WPROJ_TRY(time_ms([&] { return batch_grid(ops_of(b), b->u.as<float2>(), b->grid_partial.as<float2>(),
                                              b->Xt2.as<float2>(), s); }, 5, s, &ms));
    if (ms < best) { best = ms; bc = ch; }
  }
  WPROJ_TRY(set_chunks(b, bc, s));
  if (out) {
    out->piece = bp;
    out->lanes_per_piece = bl;
    out->chunk = bc;
    out->degrid_ms = deg_ms;
    out->grid_ms = best;
  }
  return WPROJ_OK;
}

wproj_status batch_solve_impl(wproj_batch *b, const float2 *y, const double *eps, const wproj_dr_params &prm,
                              float *x_out, cudaStream_t s) {
  const bool resume = prm.resume && b->dr_valid;
  WPROJ_TRY(ensure_solver(b));
  WPROJ_CUDA(cudaMemcpyAsync(b->eps.ptr, eps, sizeof(double) * b->np, cudaMemcpyHostToDevice, s));
  const BProb *tab = b->tab.as<BProb>();
  const int nbn = nbx_for(b->max_img);
  const int psi = prm.psi, lev = prm.psi_levels;
  if (psi) {
    WPROJ_TRY(b->zi.ensure(sizeof(float) * b->img));
    WPROJ_TRY(b->alpha.ensure(sizeof(float) * b->img));
    WPROJ_TRY(b->wwork.ensure(sizeof(float) * (b->img / 2 + 1)));
  }
  if (!resume) {
    WPROJ_TRY(power_mu(b, prm.power_iters, s));
    // z0 = Psi^T Re Phi^H y, gamma = frac max|z0|, u = 0
    if (psi) {
      WPROJ_TRY(bphi_adj(b, y, b->x.as<float>(), nullptr, 0, s));
      WPROJ_TRY(batch_dwt2(tab, b->np, b->max_n, lev, psi, b->x.as<float>(), b->z.as<float>(),
                           b->wwork.as<float>(), &b->launches, s));
    } else {
      WPROJ_TRY(bphi_adj(b, y, b->z.as<float>(), nullptr, 0, s));
    }
    k_bs_image_part<0><<<dim3(nbn, b->np), kBT, 0, s>>>(tab, b->z.as<float>(), b->part.as<double>());
    k_bs_image_scalar<0><<<ceil_div(b->np, 128), 128, 0, s>>>(b->np, nbn, b->part.as<double>(), prm.gamma_frac,
                                                              b->scal.as<double>());
    WPROJ_CHECK_LAUNCH("batch dr init");
    WPROJ_CUDA(cudaMemsetAsync(b->u.ptr, 0, sizeof(float2) * b->m, s));
  }
  b->dr_valid = true;
  if (prm.iters > 0) {
    if (!b->dr_exec || b->graph_y != y || b->graph_inner != prm.inner_iters || b->graph_lambda != prm.lambda ||
        b->graph_psi != psi || b->graph_levels != lev) {
      if (b->dr_exec) cudaGraphExecDestroy(b->dr_exec);
      b->dr_exec = nullptr;
      if (!b->cap) WPROJ_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      WPROJ_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
      const int64_t l0 = b->launches;
      wproj_status st = dr_iteration(b, y, prm.inner_iters, float(prm.lambda), psi, lev, b->cap);
      const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
      if (st != WPROJ_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "batch: capture of the DR iteration");
      const cudaError_t ie = cudaGraphInstantiate(&b->dr_exec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) return cuda_fail(ie, "batch: graph instantiation");
      b->graph_y = y;
      b->graph_inner = prm.inner_iters;
      b->graph_lambda = prm.lambda;
      b->graph_psi = psi;
      b->graph_levels = lev;
      b->iter_launches = b->launches - l0;   // kernels per replay
      b->launches = l0;
    }
    for (int t = 0; t < prm.iters; ++t) WPROJ_CUDA(cudaGraphLaunch(b->dr_exec, s));
    b->launches += b->iter_launches * prm.iters;
  }
  float *src = prm.iters > 0 ? b->x.as<float>() : b->z.as<float>();
  if (prm.iters == 0 && psi) {   // x = Psi z0
    WPROJ_TRY(batch_idwt2(tab, b->np, b->max_n, lev, psi, b->z.as<float>(), b->x.as<float>(), b->wwork.as<float>(),
                          &b->launches, s));
    src = b->x.as<float>();
  }
  WPROJ_CUDA(cudaMemcpyAsync(x_out, src, sizeof(float) * b->img, cudaMemcpyDeviceToDevice, s));
  return WPROJ_OK;
}

}  // namespace wproj

// ---- C-ABI ------------------------------------------------------------------------

using namespace wproj;

extern "C" {

wproj_status wproj_batch_create(wproj_batch **out, int32_t n, const wproj_grid_desc *descs) {
  if (!out || !descs) return fail(WPROJ_ERR_INVALID_ARG, "batch_create: null argument");
  *out = nullptr;
  if (n < 1 || n > 65535) return fail(WPROJ_ERR_INVALID_ARG, "batch_create: need 1 <= n <= 65535 problems");
  for (int p = 0; p < n; ++p) {
    if (descs[p].value_dtype != WPROJ_VAL_F32)
      return fail(WPROJ_ERR_UNSUPPORTED, "batch_create: batches store G in complex64");
    if (descs[p].index_format != WPROJ_INDEX_AUTO && descs[p].index_format != WPROJ_INDEX_COLUMNS)
      return fail(WPROJ_ERR_UNSUPPORTED, "batch_create: batches store G with column indices");
    wproj_plan *probe = nullptr;   // validates the geometry
    wproj_status st = wproj_plan_create(&probe, &descs[p]);
    if (st != WPROJ_OK) return st;
    wproj_plan_destroy(probe);
  }
  auto *b = new (std::nothrow) wproj_batch();
  if (!b) return fail(WPROJ_ERR_OOM, "batch_create: host allocation");
  b->np = n;
  b->desc.assign(descs, descs + n);
  wproj_status st = make_twiddles(b->twiddle, nullptr);
  if (st == WPROJ_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(WPROJ_ERR_CUDA, "batch_create: twiddles");
  if (st != WPROJ_OK) {
    delete b;
    return st;
  }
  *out = b;
  return WPROJ_OK;
}

wproj_status wproj_batch_destroy(wproj_batch *b) {
  delete b;
  return WPROJ_OK;
}

wproj_status wproj_batch_build(wproj_batch *b, const double *uvw, const int64_t *m, double e, void *stream) {
  if (!b || !uvw || !m) return fail(WPROJ_ERR_INVALID_ARG, "batch_build: null argument");
  if (!(e > 0.0 && e <= 1.0)) return fail(WPROJ_ERR_INVALID_ARG, "batch_build: e must lie in (0, 1]");
  for (int p = 0; p < b->np; ++p)
    if (m[p] < 1) return fail(WPROJ_ERR_INVALID_ARG, "batch_build: every problem needs m >= 1");
  return batch_build_impl(b, uvw, m, e, as_stream(stream));
}

wproj_status wproj_batch_tune(wproj_batch *b, wproj_batch_schedule *out, void *stream) {
  if (!b || !b->built) return fail(WPROJ_ERR_NOT_BUILT, "batch_tune: build the batch first");
  return batch_tune_impl(b, out, as_stream(stream));
}

wproj_status wproj_batch_set_schedule(wproj_batch *b, int64_t piece, int64_t chunk, int32_t lanes_per_piece,
                                      void *stream) {
  if (!b || !b->built) return fail(WPROJ_ERR_NOT_BUILT, "batch_set_schedule: build the batch first");
  if (piece < 32 || chunk < 32) return fail(WPROJ_ERR_INVALID_ARG, "batch_set_schedule: piece and chunk >= 32");
  if (lanes_per_piece != 0 && lanes_per_piece != 4 && lanes_per_piece != 8 && lanes_per_piece != 16 &&
      lanes_per_piece != 32)
    return fail(WPROJ_ERR_INVALID_ARG, "batch_set_schedule: lanes_per_piece is 32, 16, 8 or 4");
  if (lanes_per_piece) b->lpp = lanes_per_piece;
  WPROJ_TRY(set_pieces(b, piece, as_stream(stream)));
  return set_chunks(b, chunk, as_stream(stream));
}

wproj_status wproj_batch_phi(wproj_batch *b, const float *x, void *y, void *stream) {
  if (!b || !b->built) return fail(WPROJ_ERR_NOT_BUILT, "batch_phi: build the batch first");
  if (!x || !y) return fail(WPROJ_ERR_INVALID_ARG, "batch_phi: null argument");
  return bphi(b, x, static_cast<float2 *>(y), as_stream(stream));
}

wproj_status wproj_batch_phi_adj(wproj_batch *b, const void *y, float *x_re, void *stream) {
  if (!b || !b->built) return fail(WPROJ_ERR_NOT_BUILT, "batch_phi_adj: build the batch first");
  if (!x_re || !y) return fail(WPROJ_ERR_INVALID_ARG, "batch_phi_adj: null argument");
  return bphi_adj(b, static_cast<const float2 *>(y), x_re, nullptr, 0, as_stream(stream));
}

wproj_status wproj_batch_solve_bpdn(wproj_batch *b, const void *y, const double *eps, const wproj_dr_params *prm,
                                    float *x_out, void *stream) {
  if (!b || !b->built) return fail(WPROJ_ERR_NOT_BUILT, "batch_solve_bpdn: build the batch first");
  if (!y || !eps || !x_out) return fail(WPROJ_ERR_INVALID_ARG, "batch_solve_bpdn: null argument");
  wproj_dr_params q;
  wproj_dr_defaults(&q);
  if (prm) q = *prm;
  if (q.iters < 0 || q.inner_iters < 1 || q.power_iters < 1 || !(q.lambda > 0.0 && q.lambda < 2.0) ||
      !(q.gamma_frac >= 0.0))
    return fail(WPROJ_ERR_INVALID_ARG, "batch_solve_bpdn: invalid parameters");
  if (q.psi < 0 || q.psi > WPROJ_DAUB_MAX_P) return fail(WPROJ_ERR_INVALID_ARG, "batch_solve_bpdn: psi");
  if (q.psi && (q.psi_levels < 1 || q.psi_levels > 29 || b->pow2_div % (1 << q.psi_levels) != 0))
    return fail(WPROJ_ERR_INVALID_ARG, "batch_solve_bpdn: every N must be divisible by 2^psi_levels");
  for (int p = 0; p < b->np; ++p)
    if (!(eps[p] >= 0.0) || !isfinite(eps[p]))
      return fail(WPROJ_ERR_INVALID_ARG, "batch_solve_bpdn: eps must be finite and >= 0");
  return batch_solve_impl(b, static_cast<const float2 *>(y), eps, q, x_out, as_stream(stream));
}

wproj_status wproj_batch_get_info(const wproj_batch *b, wproj_batch_info *out) {
  if (!b || !out) return fail(WPROJ_ERR_INVALID_ARG, "batch_get_info: null argument");
  out->n_problems = b->np;
  out->m = b->m;
  out->pixels = b->img;
  out->nnz = b->nnz;
  out->n_pieces = b->n_pieces;
  out->n_chunks = b->n_chunks;
  out->piece = b->piece;
  out->chunk = b->chunk;
  out->lanes_per_piece = b->lpp;
  out->launches = b->launches;
  out->iter_launches = b->iter_launches;
  return WPROJ_OK;
}

}  // extern "C"
