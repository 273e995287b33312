// C-ABI entry points of libwproj (include/wproj.h): plan management, argument
// checks, error reporting and timing.  All computation happens in the kernels of
// fft.cu, build.cu, ops.cu, solve.cu and wavelet.cu.
#include <math.h>

#include <algorithm>
#include <string>

#include "plan.h"

namespace wproj {

wproj_status power_norm2_impl(wproj_plan *p, int iters, double *out, cudaStream_t s);
wproj_status solve_bpdn_impl(wproj_plan *p, const float2 *y, double eps, const wproj_dr_params &prm,
                             float *x_out, wproj_solve_info *info, cudaStream_t s);
wproj_status dr_state_get(wproj_plan *p, float *z, void *u, double *gamma, double *phi_norm2, cudaStream_t s);
wproj_status dr_state_set(wproj_plan *p, const float *z, const void *u, double gamma, double phi_norm2,
                          cudaStream_t s);

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
wproj_status fail(wproj_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}
wproj_status cuda_fail(cudaError_t err, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
  return err == cudaErrorMemoryAllocation ? WPROJ_ERR_OOM : WPROJ_ERR_CUDA;
}

wproj_status DevBuf::alloc(size_t n) {
  release();
  if (n == 0) n = 16;
  cudaError_t err = cudaMalloc(&ptr, n);
  if (err != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    return fail(err == cudaErrorMemoryAllocation ? WPROJ_ERR_OOM : WPROJ_ERR_CUDA,
                "cudaMalloc(" + std::to_string(n) + " bytes): " + cudaGetErrorString(err));
  }
  bytes = n;
  return WPROJ_OK;
}
wproj_status DevBuf::ensure(size_t n) {
  if (ptr && bytes >= n) return WPROJ_OK;
  return alloc(n);
}

EventTimer::~EventTimer() {
  for (auto e : pool) cudaEventDestroy(e);
}
cudaEvent_t EventTimer::get() {
  if (used == pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
  }
  return pool[used++];
}

static void fold_timer(wproj_plan *p) {
  EventTimer &t = p->timer;
  for (auto &pr : t.pending) {
    float ms = 0;
    cudaEventSynchronize(pr.second.second);
    if (cudaEventElapsedTime(&ms, pr.second.first, pr.second.second) == cudaSuccess) {
      t.ms[pr.first] += ms;
      t.count[pr.first] += 1;
    }
  }
  t.pending.clear();
  t.used = 0;
}

ScopedTimer::ScopedTimer(wproj_plan *p_, int cls_, cudaStream_t s_) : p(p_), cls(cls_), s(s_) {
  if (!p->timing) return;
  if (p->timer.pending.size() >= 4096) fold_timer(p);
  a = p->timer.get();
  b = p->timer.get();
  if (a && b) cudaEventRecord(a, s);
}
ScopedTimer::~ScopedTimer() { stop(); }
void ScopedTimer::stop() {
  if (!p->timing || !a || !b) return;
  cudaEventRecord(b, s);
  p->timer.pending.push_back({cls, {a, b}});
  a = b = nullptr;
}

namespace {

__global__ void k_inv_a(int N, int W, double beta, float *__restrict__ inv_a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (W == 1) { inv_a[i] = 1.f; return; }
  // a(l_p) = continuous Fourier transform of the KB kernel at nu = l_p du = (p - N/2) / (2N)
  const double nu = double(i - N / 2) / (2.0 * N);
  const double z2 = beta * beta - (M_PI * W * nu) * (M_PI * W * nu);
  double a;
  if (z2 > 0) { const double z = sqrt(z2); a = W * sinh(z) / z; }
  else if (z2 < 0) { const double z = sqrt(-z2); a = W * sin(z) / z; }
  else a = W;
  inv_a[i] = float(1.0 / a);
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

wproj_status check_built(const wproj_plan *p) {
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  if (!p->built) return fail(WPROJ_ERR_NOT_BUILT, "G has not been built (call wproj_build_kernels)");
  return WPROJ_OK;
}

}  // namespace
}  // namespace wproj

using namespace wproj;

extern "C" {

const char *wproj_last_error(void) { return g_last_error.c_str(); }
const char *wproj_version(void) { return "wproj 0.1 (sm_103a)"; }

void wproj_dr_defaults(wproj_dr_params *prm) {
  if (!prm) return;
  prm->iters = 50;
  prm->inner_iters = 10;
  prm->gamma_frac = 1e-2;
  prm->lambda = 1.0;
  prm->phi_norm2 = 0.0;
  prm->power_iters = 100;
  prm->resume = 0;
  prm->psi = 0;
  prm->psi_levels = 4;
}

wproj_status wproj_plan_create(wproj_plan **out, const wproj_grid_desc *d) {
  if (!out || !d) return fail(WPROJ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (d->n < 8 || d->n > 2048 || (d->n & 1) || !is_pow2(d->n))
    return fail(WPROJ_ERR_INVALID_ARG, "n must be a power of two in [8, 2048]");
  if (!(d->kb_support == 1 || d->kb_support == 4 || d->kb_support == 6 || d->kb_support == 8))
    return fail(WPROJ_ERR_INVALID_ARG, "kb_support must be 1, 4, 6 or 8");
  if (!(d->fov > 0) || !isfinite(d->fov)) return fail(WPROJ_ERR_INVALID_ARG, "fov must be positive");
  if (d->chirp != WPROJ_CHIRP_EXACT && d->chirp != WPROJ_CHIRP_LINEAR)
    return fail(WPROJ_ERR_INVALID_ARG, "chirp must be 0 (exact) or 1 (linear)");
  if (d->extension != WPROJ_EXT_FULL && d->extension != WPROJ_EXT_CLAMP)
    return fail(WPROJ_ERR_INVALID_ARG, "extension must be 0 (full) or 1 (clamp)");
  const int G = 2 * d->n;
  if (d->box != 0 && (!is_pow2(d->box) || d->box < 16 || d->box > G))
    return fail(WPROJ_ERR_INVALID_ARG, "box must be 0 or a power of two in [16, 2N]");
  if (d->value_dtype < 0 || d->value_dtype > 2) return fail(WPROJ_ERR_INVALID_ARG, "value_dtype must be 0, 1 or 2");
  if (d->index_format < 0 || d->index_format > 3) return fail(WPROJ_ERR_INVALID_ARG, "index_format must be 0, 1, 2 or 3");
  if (d->upsampling != 0 && d->upsampling != 1) return fail(WPROJ_ERR_INVALID_ARG, "upsampling must be 0 or 1");
  if (d->upsampling == 1 && d->kb_support != 1)
    return fail(WPROJ_ERR_INVALID_ARG, "upsampling = 1 (visibilities on the grid) needs kb_support = 1");
  if (d->upsampling == 1 && d->n < 16) return fail(WPROJ_ERR_INVALID_ARG, "upsampling = 1 needs n >= 16");
  const double lmax = d->extension == WPROJ_EXT_CLAMP ? 0.5 * d->fov : d->fov;
  if (d->chirp == WPROJ_CHIRP_EXACT && 2.0 * lmax * lmax >= 1.0)
    return fail(WPROJ_ERR_INVALID_ARG, "1 - l^2 - m^2 < 0 on the sampled box (fov too large)");

  wproj_plan *p = new wproj_plan();
  GridGeom &g = p->g;
  g.N = d->n;
  g.G = G;
  g.W = d->kb_support;
  // the kernel geometry: with upsampling the chirp is sampled on the upsampled
  // image, i.e. on a box spanning [-L/2, L/2), and the grid cell is 1/L
  const double Lk = d->upsampling ? 0.5 * d->fov : d->fov;
  g.L = Lk;
  g.du = 1.0 / (2.0 * Lk);
  g.B = d->n / (2.0 * Lk);
  g.upsampling = d->upsampling;
  g.beta = (g.W > 1) ? M_PI * sqrt((g.W / 2.0) * (g.W / 2.0) * 1.5 * 1.5 - 0.8) : 0.0;
  g.chirp = d->chirp;
  g.extension = d->extension;
  g.box = d->box;
  g.value_dtype = d->value_dtype;
  g.index_format = d->index_format;
  g.tile = G < kTile ? G : kTile;
  g.nT = G / g.tile;
  cudaGetDevice(&p->device);
  cudaStream_t s = 0;
  wproj_status st = WPROJ_OK;
  auto chk = [&](wproj_status x) { if (st == WPROJ_OK) st = x; };
  chk(init_twiddles(p, s));
  chk(p->inv_a.alloc(sizeof(float) * g.N));
  chk(p->Xt.alloc(sizeof(float2) * size_t(G) * G));
  chk(p->Xt2.alloc(sizeof(float2) * size_t(G) * G));
  chk(p->inter.alloc(sizeof(float2) * size_t(g.N) * G));
  chk(p->xtmp.alloc(sizeof(float) * size_t(g.N) * g.N));
  if (st == WPROJ_OK) {
    k_inv_a<<<ceil_div(g.N, 256), 256, 0, s>>>(g.N, g.W, g.beta, p->inv_a.as<float>());
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) st = cuda_fail(err, "plan init");
  }
  if (st != WPROJ_OK) {
    delete p;
    return st;
  }
  *out = p;
  return WPROJ_OK;
}

wproj_status wproj_plan_destroy(wproj_plan *p) {
  if (!p) return WPROJ_OK;
  cudaDeviceSynchronize();
  delete p;
  return WPROJ_OK;
}

wproj_status wproj_build_kernels(wproj_plan *p, const double *uvw, int64_t m, double e, void *stream,
                                 wproj_csr *out) {
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  if (!uvw) return fail(WPROJ_ERR_INVALID_ARG, "null uvw");
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(WPROJ_ERR_INVALID_ARG, "m must be in [1, 2^31)");
  if (!(e > 0.0 && e <= 1.0)) return fail(WPROJ_ERR_INVALID_ARG, "e must be in (0, 1]");
  wproj_status st = build_kernels_impl(p, uvw, m, e, as_stream(stream));
  if (st != WPROJ_OK) {
    p->built = false;
    return st;
  }
  if (out) return wproj_get_csr(p, out);
  return WPROJ_OK;
}

wproj_status wproj_set_screens(wproj_plan *p, const void *screens, int32_t n_screens, void *stream) {
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  if (n_screens < 0 || (n_screens > 0 && !screens)) return fail(WPROJ_ERR_INVALID_ARG, "set_screens: bad arguments");
  return set_screens_impl(p, static_cast<const float2 *>(screens), n_screens, as_stream(stream));
}

wproj_status wproj_build_kernels_dde(wproj_plan *p, const double *uvw, int64_t m, const int32_t *screen_id,
                                     double e, void *stream) {
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  if (!uvw || !screen_id) return fail(WPROJ_ERR_INVALID_ARG, "null uvw or screen_id");
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(WPROJ_ERR_INVALID_ARG, "m must be in [1, 2^31)");
  if (!(e > 0.0 && e <= 1.0)) return fail(WPROJ_ERR_INVALID_ARG, "e must be in (0, 1]");
  if (p->n_screens < 1) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels_dde: set the screens first");
  if (p->g.box != p->g.G) return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels_dde: screens need the full box (box = G)");
  wproj_status st = build_kernels_impl(p, uvw, m, e, as_stream(stream), screen_id);
  if (st != WPROJ_OK) p->built = false;
  return st;
}

wproj_status wproj_get_csr(const wproj_plan *p, wproj_csr *out) {
  WPROJ_TRY(check_built(p));
  if (!out) return fail(WPROJ_ERR_INVALID_ARG, "null out");
  out->m = p->m;
  out->nnz = p->nnz;
  out->n_cols = int64_t(p->g.G) * p->g.G;
  out->row_ptr = p->row_ptr.as<int64_t>();
  out->row_scale = p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>();
  out->value_dtype = p->g.value_dtype;
  out->index_format = p->fmt;
  out->n_seg = p->n_seg;
  const bool cols = p->fmt == WPROJ_INDEX_COLUMNS;
  out->col = cols ? p->col.as<int32_t>() : nullptr;
  out->val = cols ? p->val.ptr : nullptr;
  out->stream = cols ? nullptr : p->stream.ptr;
  out->stream_bytes = cols ? 0 : p->stream_bytes;
  return WPROJ_OK;
}

wproj_status wproj_csr_rows(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                            void *stream) {
  WPROJ_TRY(check_built(p));
  if (k0 < 0 || k1 < k0 || k1 > p->m) return fail(WPROJ_ERR_INVALID_ARG, "csr_rows: need 0 <= k0 <= k1 <= m");
  return csr_rows(p, k0, k1, col_out, val_out, as_stream(stream));
}

wproj_status wproj_phi(wproj_plan *p, const float *x, void *y, void *stream) {
  WPROJ_TRY(check_built(p));
  if (!x || !y) return fail(WPROJ_ERR_INVALID_ARG, "null x or y");
  return apply_phi(p, x, nullptr, static_cast<float2 *>(y), as_stream(stream));
}

wproj_status wproj_phi_cplx(wproj_plan *p, const void *x_cplx, void *y, void *stream) {
  WPROJ_TRY(check_built(p));
  if (!x_cplx || !y) return fail(WPROJ_ERR_INVALID_ARG, "null x or y");
  return apply_phi(p, nullptr, static_cast<const float2 *>(x_cplx), static_cast<float2 *>(y), as_stream(stream));
}

wproj_status wproj_phi_adj(wproj_plan *p, const void *y, float *x_re, void *x_cplx, void *stream) {
  WPROJ_TRY(check_built(p));
  if (!y || (!x_re && !x_cplx)) return fail(WPROJ_ERR_INVALID_ARG, "null y or outputs");
  return apply_phi_adj(p, static_cast<const float2 *>(y), x_re, static_cast<float2 *>(x_cplx), nullptr, 0,
                       as_stream(stream));
}

wproj_status wproj_solve_bpdn(wproj_plan *p, const void *y, double eps, const wproj_dr_params *prm,
                              float *x_out, wproj_solve_info *info, void *stream) {
  WPROJ_TRY(check_built(p));
  if (!y || !x_out) return fail(WPROJ_ERR_INVALID_ARG, "null y or x_out");
  if (!(eps >= 0) || !isfinite(eps)) return fail(WPROJ_ERR_INVALID_ARG, "eps must be finite and >= 0");
  wproj_dr_params q;
  wproj_dr_defaults(&q);
  if (prm) q = *prm;
  if (q.iters < 0 || q.inner_iters < 1 || !(q.gamma_frac >= 0) || !(q.lambda > 0 && q.lambda < 2) ||
      q.power_iters < 1)
    return fail(WPROJ_ERR_INVALID_ARG, "invalid DR parameters");
  if (q.psi < 0 || q.psi > WPROJ_DAUB_MAX_P) return fail(WPROJ_ERR_INVALID_ARG, "psi: 0 or a Daubechies order");
  if (q.psi && (q.psi_levels < 1 || p->g.N % (1 << std::min(q.psi_levels, 30)) != 0))
    return fail(WPROJ_ERR_INVALID_ARG, "psi_levels: N must be divisible by 2^levels");
  return solve_bpdn_impl(p, static_cast<const float2 *>(y), eps, q, x_out, info, as_stream(stream));
}

wproj_status wproj_dr_state_get(wproj_plan *p, float *z, void *u, double *gamma, double *phi_norm2,
                                void *stream) {
  WPROJ_TRY(check_built(p));
  return dr_state_get(p, z, u, gamma, phi_norm2, as_stream(stream));
}

wproj_status wproj_dr_state_set(wproj_plan *p, const float *z, const void *u, double gamma,
                                double phi_norm2, void *stream) {
  WPROJ_TRY(check_built(p));
  if (!z || !u || !(phi_norm2 > 0) || !(gamma >= 0)) return fail(WPROJ_ERR_INVALID_ARG, "invalid DR state");
  return dr_state_set(p, z, u, gamma, phi_norm2, as_stream(stream));
}

wproj_status wproj_power_norm2(wproj_plan *p, int32_t iters, double *out, void *stream) {
  WPROJ_TRY(check_built(p));
  if (!out || iters < 1) return fail(WPROJ_ERR_INVALID_ARG, "invalid power iteration arguments");
  return power_norm2_impl(p, iters, out, as_stream(stream));
}

wproj_status wproj_fft2d(const void *in, void *out, int32_t n, int32_t batch, int32_t inverse, void *stream) {
  if (!in || !out) return fail(WPROJ_ERR_INVALID_ARG, "null in or out");
  if (!is_pow2(n) || n < 16 || n > 4096 || batch < 1) return fail(WPROJ_ERR_INVALID_ARG, "n must be a power of two in [16, 4096]");
  // a private twiddle table per device, built on first use
  static DevBuf tw[64];
  int dev = 0;
  WPROJ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(WPROJ_ERR_UNSUPPORTED, "device index");
  if (!tw[dev].ptr) {
    wproj_plan tmp;
    WPROJ_TRY(init_twiddles(&tmp, as_stream(stream)));
    WPROJ_CUDA(cudaStreamSynchronize(as_stream(stream)));
    tw[dev].ptr = tmp.twiddle.ptr;
    tw[dev].bytes = tmp.twiddle.bytes;
    tmp.twiddle.ptr = nullptr;
  }
  return fft2d_generic(static_cast<const float2 *>(in), static_cast<float2 *>(out), n, batch, inverse,
                       tw[dev].as<float2>(), as_stream(stream));
}

wproj_status wproj_set_timing(wproj_plan *p, int32_t enable) {
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  p->timing = enable != 0;
  return WPROJ_OK;
}

wproj_status wproj_reset_stats(wproj_plan *p) {
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  fold_timer(p);
  for (int i = 0; i < TC_COUNT; ++i) { p->timer.ms[i] = 0; p->timer.count[i] = 0; }
  p->launches = 0;
  return WPROJ_OK;
}

wproj_status wproj_get_stats(wproj_plan *p, wproj_stats *out) {
  if (!p || !out) return fail(WPROJ_ERR_INVALID_ARG, "null argument");
  fold_timer(p);
  out->m = p->m;
  out->nnz = p->nnz;
  out->box_min = p->box_min;
  out->box_max = p->box_max;
  out->segments = p->n_seg;
  out->degrid_pieces = p->n_pieces;
  out->grid_chunks = p->n_chunks;
  out->build_ms = p->build_ms;
  out->t_fft_ms = p->timer.ms[TC_FFT];
  out->t_degrid_ms = p->timer.ms[TC_DEGRID];
  out->t_grid_ms = p->timer.ms[TC_GRID];
  out->t_reduce_ms = p->timer.ms[TC_REDUCE];
  out->t_solver_ms = p->timer.ms[TC_SOLVER];
  out->n_fft = p->timer.count[TC_FFT];
  out->n_degrid = p->timer.count[TC_DEGRID];
  out->n_grid = p->timer.count[TC_GRID];
  out->n_reduce = p->timer.count[TC_REDUCE];
  out->n_solver = p->timer.count[TC_SOLVER];
  out->launches = p->launches;
  out->t_build_fft_ms = p->timer.ms[TC_BFFT];
  out->t_build_select_ms = p->timer.ms[TC_BSEL];
  out->t_build_emit_ms = p->timer.ms[TC_BEMIT];
  out->n_build_fft = p->timer.count[TC_BFFT];
  out->runs_bytes = p->fmt == WPROJ_INDEX_TILE_RUNS
                        ? p->rm_vals * (p->g.value_dtype == WPROJ_VAL_F32 ? 8 : 4) + p->rm_runs * 4 + p->m * 20
                        : 0;
  return WPROJ_OK;
}

}  // extern "C"
