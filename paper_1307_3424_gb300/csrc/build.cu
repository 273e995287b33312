// Part I: construction of the sparse w-kernel matrix G (Sections 3.1-3.2).
//
// For every visibility k with grid coordinate g = (u, v)/du, j0 = floor(g),
// delta = g - j0, its kernel on an S x S box of cells j0 + s, s in [-S/2, S/2)^2:
//
//   K_k[s] = (1/S^2) sum_P c_k(l_P) tau_k(P) exp(+2 pi i s.P / S)
//
// c_k the chirp of Eq. 4 (or Eq. 5) sampled at l_P = P (2L/S), tau_k(P) =
// sum_t kb(delta - t) exp(-2 pi i t.P / S) the image-space polynomial of the
// KB taps.  This equals (1/S) sum_t kb kb C-hat_k[t - s], the circular
// convolution of the row of C-hat (Eq. 8: FFT of the real-space chirp) with
// the gridding taps.  Each row keeps the smallest set of entries, largest
// modulus first, that holds a fraction e of the row energy (Section 3.2).
//
// Pipeline (boxes processed in batches sized to stay in L2):
//   plan rows -> per-box tables -> 2 FFT passes -> 3-level energy-weighted
//   radix select (exact integer prefix) -> per-tile counts  [phase 1]
//   scan counts -> allocate G exactly -> tables + FFT again -> emit  [phase 2]
//   -> tile lists for gridding, row pieces for degridding.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "build.cuh"
#include "plan.h"

namespace wproj {

namespace {

__host__ __device__ __forceinline__ int64_t i64max(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int64_t i64min(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr size_t kBuildBatchBytes = size_t(128) << 20;   // kernel boxes in flight
// (32 MB batches of 512^2 boxes, which stay in L2 between the passes, measured
// slower: 866 against 638 ms for 32768 boxes; the selection's histogram
// launches lose more parallelism than the L2 residency gains)
size_t batch_bytes(int) { return kBuildBatchBytes; }
constexpr int kMaxBatchBoxes = 16384;     // grid.y limit for per-box launches
constexpr int kHistBins = 2048;
constexpr int kSelChunk = 8192;          // entries per histogram block
constexpr int kRun = 8;   // consecutive samples a thread takes in the histogram and tile counts (16: slower)
// Work units of the operators, sized from nnz so that small problems still
// fill the GPU and large ones keep the partial sums small.
int64_t degrid_piece(int64_t nnz) { return std::min<int64_t>(16384, std::max<int64_t>(512, nnz / (152 * 64))); }
int64_t grid_chunk(int64_t nnz) { return std::min<int64_t>(262144, std::max<int64_t>(4096, nnz / (152 * 16))); }

enum : int { ERR_NONFINITE = 1, ERR_BAND = 2, ERR_EMIT = 4, ERR_SCREEN = 8 };

// ---- per-axis tile geometry of a box -----------------------------------------
// The box covers cells (j0 - S/2 + d) mod G, d in [0, S).  Its touched tiles
// are listed in ascending tile index.
struct AxisTiles {
  int a;        // first cell (j0 - S/2) mod G
  int nt;       // number of touched tiles
  int kind;     // 0: all tiles; 1: contiguous t0..; 2: wrapped {0..t1} U {t0..nT-1}
  int t0, t1;
};

__host__ __device__ __forceinline__ AxisTiles axis_tiles(int j0, int S, int G, int TS) {
  AxisTiles r;
  const int nT = G / TS;
  r.a = ((j0 - S / 2) % G + G) % G;
  r.t0 = r.a / TS;
  const int last = (r.a + S - 1) % G;
  r.t1 = last / TS;
  if (S >= G || nT == 1) {
    r.kind = 0; r.nt = nT; r.t0 = 0;
  } else if (r.a + S <= G) {
    r.kind = 1; r.nt = r.t1 - r.t0 + 1;
  } else if (r.t1 >= r.t0 - 1) {
    r.kind = 0; r.nt = nT; r.t0 = 0;
  } else {
    r.kind = 2; r.nt = (r.t1 + 1) + (nT - r.t0);
  }
  return r;
}
__host__ __device__ __forceinline__ int axis_tile_at(const AxisTiles &t, int i, int nT) {
  if (t.kind == 0) return i;
  if (t.kind == 1) return t.t0 + i;
  return (i <= t.t1) ? i : t.t0 + (i - t.t1 - 1);
}
__host__ __device__ __forceinline__ int axis_tile_pos(const AxisTiles &t, int tile) {
  if (t.kind == 0) return tile;
  if (t.kind == 1) return tile - t.t0;
  return (tile <= t.t1) ? tile : tile - t.t0 + t.t1 + 1;
}

// Upper bound of the tiles one S x S box touches: all of them when S = G, else
// at most ceil(S/tile) + 1 per axis.
int box_tiles(int S, const GridGeom &g) {
  if (S >= g.G) return g.nT * g.nT;
  const int per = std::min(g.nT, (S + g.tile - 1) / g.tile + 1);
  return per * per;
}

// ---- row plan -------------------------------------------------------------------

__global__ void k_row_plan(const double *__restrict__ uvw, int64_t m, GridGeom g,
                           int2 *__restrict__ j0, double2 *__restrict__ delta,
                           int32_t *__restrict__ Sk, int32_t *__restrict__ ntile,
                           int32_t *__restrict__ sclass, int *__restrict__ err) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
  int e = 0;
  if (!isfinite(u) || !isfinite(v) || !isfinite(w)) e |= ERR_NONFINITE;
  else if (u < -g.B || u >= g.B || v < -g.B || v >= g.B) e |= ERR_BAND;
  if (e) {
    atomicOr(err, e);
    j0[k] = make_int2(0, 0); delta[k] = make_double2(0, 0); Sk[k] = 16; ntile[k] = 0; sclass[k] = 0;
    return;
  }
  const double gu = u / g.du, gv = v / g.du;
  double fu = floor(gu), fv = floor(gv);
  int iu = int(fu), iv = int(fv);
  // u < B keeps iu < N = G/2; guard rounding at the edge
  if (iu >= g.G / 2) { iu = g.G / 2 - 1; fu = iu; }
  if (iv >= g.G / 2) { iv = g.G / 2 - 1; fv = iv; }
  j0[k] = make_int2(iu, iv);
  delta[k] = make_double2(gu - fu, gv - fv);
  int S;
  if (g.box > 0) {
    S = g.box;
  } else {
    const double h = fabs(w) * g.L * g.L;
    const double need = 4.0 * h + g.W + 16.0;
    S = 16;
    while (S < need && S < g.G) S <<= 1;
    if (S > g.G) S = g.G;
  }
  Sk[k] = S;
  int lg = 0;
  while ((1 << lg) < S) ++lg;
  sclass[k] = lg - 4;
  const AxisTiles tu = axis_tiles(iu, S, g.G, g.tile);
  const AxisTiles tv = axis_tiles(iv, S, g.G, g.tile);
  ntile[k] = tu.nt * tv.nt;
}

__global__ void k_seg_fill(int64_t m, GridGeom g, const int2 *__restrict__ j0,
                           const int32_t *__restrict__ Sk, const int64_t *__restrict__ seg_base,
                           int32_t *__restrict__ seg_row, int32_t *__restrict__ seg_tile) {
  const int64_t k = blockIdx.x;
  if (k >= m) return;
  const int S = Sk[k];
  const AxisTiles tu = axis_tiles(j0[k].x, S, g.G, g.tile);
  const AxisTiles tv = axis_tiles(j0[k].y, S, g.G, g.tile);
  const int n = tu.nt * tv.nt;
  const int64_t base = seg_base[k];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int a = i / tv.nt, b = i % tv.nt;
    seg_row[base + i] = int32_t(k);
    seg_tile[base + i] = axis_tile_at(tu, a, g.nT) * g.nT + axis_tile_at(tv, b, g.nT);
  }
}

// ---- direction-dependent screens ---------------------------------------------------

// every screen id in [0, n)
__global__ void k_check_sid(int64_t m, const int32_t *__restrict__ sid, int n, int *__restrict__ err) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < m && (sid[k] < 0 || sid[k] >= n)) atomicOr(err, ERR_SCREEN);
}

// max |A|^2 of each screen (one block per screen); non-finite samples flag err
__global__ void __launch_bounds__(256)
k_screen_max(const float2 *__restrict__ scr, int64_t per, float *__restrict__ max2, int *__restrict__ err) {
  const float2 *a = scr + int64_t(blockIdx.x) * per;
  float mx = 0.f;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < per; i += blockDim.x) {
    const float2 v = a[i];
    if (!isfinite(v.x) || !isfinite(v.y)) bad = true;
    else mx = fmaxf(mx, v.x * v.x + v.y * v.y);
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  if (bad) atomicOr(err, ERR_NONFINITE);
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t = fmaxf(t, red[i]);
    max2[blockIdx.x] = t > 0.f ? t : 1.f;   // an all-zero screen keeps the unit scale
  }
}

// ---- per-box tables ----------------------------------------------------------------

__global__ void k_coord_tables(int S, double L, int clamp, double *__restrict__ lcoord,
                               float *__restrict__ lsq) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= S) return;
  const int off = (P < S / 2) ? P : P - S;
  double l = double(off) * (2.0 * L / S);
  if (clamp) l = fmin(fmax(l, -0.5 * L), 0.5 * L);
  lcoord[P] = l;
  lsq[P] = float(l * l);
}

struct SelState {
  unsigned long long target, q_above, q_tot;
  int32_t qexp;         // fixed-point scale 2^qexp: the largest power of two <= 2^62 / E_closed
  uint32_t prefix;
  uint32_t maxkey;
  int32_t n_above;
  int32_t done;
  int32_t all;
  uint32_t thr_key;
  int32_t n_tie;
};

__global__ void k_box_tables(const int32_t *__restrict__ ids, const double *__restrict__ uvw,
                             const double2 *__restrict__ delta, GridGeom g, int S,
                             const double *__restrict__ lcoord, float2 *__restrict__ Au,
                             float2 *__restrict__ Av, int8_t *__restrict__ mode,
                             float *__restrict__ wf, double *__restrict__ wd,
                             SelState *__restrict__ sel, const int32_t *__restrict__ sid,
                             const float *__restrict__ scr_max2, int32_t *__restrict__ bsid) {
  const int b = blockIdx.x;
  const int k = ids[b];
  const double w = uvw[3 * int64_t(k) + 2];
  const double2 dl = delta[k];
  __shared__ double tapu[8], tapv[8];
  __shared__ int md;
  const int W = g.W;
  const int ntap = (W == 1) ? 1 : W;
  if (threadIdx.x < ntap) {
    const int t = (W == 1) ? 0 : int(threadIdx.x) - W / 2 + 1;
    tapu[threadIdx.x] = (W == 1) ? 1.0 : kb_dev(dl.x - t, W, g.beta);
    tapv[threadIdx.x] = (W == 1) ? 1.0 : kb_dev(dl.y - t, W, g.beta);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double eu = 0, ev = 0;
    for (int i = 0; i < ntap; ++i) { eu += tapu[i] * tapu[i]; ev += tapv[i] * tapv[i]; }
    int m_ = 0;
    if (g.chirp == WPROJ_CHIRP_EXACT) {
      const double lmax = g.extension == WPROJ_EXT_CLAMP ? 0.5 * g.L : g.L;
      const double x = 2.0 * lmax * lmax;
      const double d = 1.0 + sqrt(1.0 - x);
      const double gmax = x * x / (2.0 * d * d);
      m_ = (fabs(w) * gmax <= 0.25) ? 1 : 2;
    }
    md = m_;
    mode[b] = int8_t(m_);
    wf[b] = float(w);
    wd[b] = w;
    SelState s = {};
    // 2^62 / E: fixed-point energies; with a screen the row energy is at most
    // E_kb max|A|^2 (Parseval), which keeps the integer sums below 2^62.  The
    // scale is rounded down to a power of two, so that a sample's fixed-point
    // energy is its FP32 value shifted (exact, no FP64 arithmetic per sample)
    double escale = eu * ev;
    if (sid) {
      escale *= double(scr_max2[sid[k]]);
      bsid[b] = sid[k];
    }
    int ex = 0;
    frexp(4611686018427387904.0 / escale, &ex);   // 2^(ex - 1) <= 2^62 / E < 2^ex
    s.qexp = ex - 1;
    sel[b] = s;
  }
  __syncthreads();
  const int m_ = md;
  for (int P = threadIdx.x; P < S; P += blockDim.x) {
    const int off = (P < S / 2) ? P : P - S;
    float2 tu = make_float2(0.f, 0.f), tv = make_float2(0.f, 0.f);
    for (int i = 0; i < ntap; ++i) {
      const int t = (W == 1) ? 0 : i - W / 2 + 1;
      float sn, cs;
      sincospif(-2.0f * float(t * off) / float(S), &sn, &cs);
      tu.x += float(tapu[i]) * cs; tu.y += float(tapu[i]) * sn;
      tv.x += float(tapv[i]) * cs; tv.y += float(tapv[i]) * sn;
    }
    if (m_ != 2) {
      // separable phase w l^2 / 2 in FP64, reduced mod 1
      const double l = lcoord[P];
      const double ph = 0.5 * w * l * l;
      const float fr = float(ph - floor(ph));
      float sn, cs;
      sincospif(2.f * fr, &sn, &cs);
      const float2 e = make_float2(cs, sn);
      tu = cmul(tu, e);
      tv = cmul(tv, e);
    }
    Au[int64_t(b) * S + P] = tu;
    Av[int64_t(b) * S + P] = tv;
  }
}

// ---- energy-weighted radix select ------------------------------------------------
// Keys are the FP32 bit patterns of |K|^2 (non-negative, so integer order is
// value order).  Energies are fixed point q = floor(|K|^2 2^qexp), 2^qexp the
// largest power of two <= 2^62 / E_closed, and summed as integers, so the
// prefix is exact and independent of order.

__host__ __device__ constexpr int lvl_shift(int L) { return L == 0 ? 20 : (L == 1 ? 9 : 0); }

// floor(a2 2^qexp) for a non-negative finite float a2, by integer shifts of its
// significand (exact; capped below 2^63)
__device__ __forceinline__ unsigned long long fixed_energy(float a2, int qexp) {
  const unsigned bits = __float_as_uint(a2);
  int e8 = int(bits >> 23);
  unsigned long long m = bits & 0x7fffffu;
  if (e8) m |= 0x800000u;
  else e8 = 1;                      // subnormal: m 2^(1 - 150)
  const int sh = e8 - 150 + qexp;   // a2 = m 2^(e8 - 150)
  if (sh >= 0) return m << (sh < 39 ? sh : 39);
  return sh > -64 ? (m >> -sh) : 0ull;
}
__host__ __device__ constexpr int lvl_bits(int L) { return L == 2 ? 9 : 11; }

template <int LEVEL>
__global__ void __launch_bounds__(256)
k_sel_hist(const float2 *__restrict__ K, int S, SelState *__restrict__ sel,
           unsigned *__restrict__ hcnt, unsigned long long *__restrict__ hq) {
  __shared__ unsigned scnt[kHistBins];
  __shared__ unsigned long long sq[kHistBins];
  __shared__ unsigned smax;
  const int b = blockIdx.y;
  const SelState st = sel[b];
  if (st.done) return;
  constexpr int nb = 1 << lvl_bits(LEVEL);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) { scnt[i] = 0; sq[i] = 0; }
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  const int64_t n = int64_t(S) * S;
  const int64_t lo = int64_t(blockIdx.x) * kSelChunk;
  const int64_t hi = min(n, lo + kSelChunk);
  const float2 *Kb = K + int64_t(b) * n;
  unsigned lmax = 0;
  // A thread takes kRun consecutive samples (16-byte loads; S^2 and the
  // chunk bounds are multiples of kRun) and adds a run of samples in one bin with
  // one pair of atomics: neighbouring samples of a kernel have similar
  // magnitudes, so runs are common and same-bin conflicts between the lanes of
  // a warp fall.  The sums are integers, so the histogram does not depend on
  // the grouping.  (Grouping lanes by bin with match / reduce before the
  // atomics measured slower: 389 against 210 ms of selection per paper-scale
  // build.)
  for (int64_t i0 = lo + kRun * int64_t(threadIdx.x); i0 < hi; i0 += kRun * int64_t(blockDim.x)) {
    float4 pk[kRun / 2];
#pragma unroll
    for (int h = 0; h < kRun / 2; ++h) pk[h] = __ldg(reinterpret_cast<const float4 *>(Kb + i0) + h);
    unsigned rbin = 0xffffffffu, rcnt = 0;
    unsigned long long rq = 0;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const float4 &v = pk[j >> 1];
      const float a2 = abs2_rn((j & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y));
      const unsigned key = __float_as_uint(a2);
      if (LEVEL == 0) lmax = max(lmax, key);
      if (LEVEL > 0 && (key >> lvl_shift(LEVEL - 1)) != st.prefix) continue;
      const unsigned bin = (key >> lvl_shift(LEVEL)) & (nb - 1);
      const unsigned long long q = fixed_energy(a2, st.qexp);
      if (bin != rbin) {
        if (rcnt) {
          atomicAdd(&scnt[rbin], rcnt);
          atomicAdd(&sq[rbin], rq);
        }
        rbin = bin;
        rcnt = 0;
        rq = 0;
      }
      rcnt += 1;
      rq += q;
    }
    if (rcnt) {
      atomicAdd(&scnt[rbin], rcnt);
      atomicAdd(&sq[rbin], rq);
    }
  }
  if (LEVEL == 0) {
    for (int o = 16; o; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, lmax);
  }
  __syncthreads();
  unsigned *gc = hcnt + int64_t(b) * kHistBins;
  unsigned long long *gq = hq + int64_t(b) * kHistBins;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    if (scnt[i]) {
      atomicAdd(&gc[i], scnt[i]);
      atomicAdd(&gq[i], sq[i]);
    }
  }
  if (LEVEL == 0 && threadIdx.x == 0) atomicMax(&sel[b].maxkey, smax);
}

template <class T>
__device__ __forceinline__ T block_sum256(T v, T *red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 8; ++i) t += red[i];
    red[8] = t;
  }
  __syncthreads();
  t = red[8];
  __syncthreads();
  return t;
}

// inclusive prefix over 256 threads (one value each)
__device__ __forceinline__ unsigned long long block_incl_scan256(unsigned long long v,
                                                                 unsigned long long *wt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) wt[wid] = v;
  __syncthreads();
  unsigned long long off = 0;
  for (int i = 0; i < wid; ++i) off += wt[i];
  __syncthreads();
  return v + off;
}

template <int LEVEL>
__global__ void __launch_bounds__(256)
k_sel_find(SelState *__restrict__ sel, const unsigned *__restrict__ hcnt,
           const unsigned long long *__restrict__ hq, double e_target) {
  __shared__ unsigned long long red[9];
  __shared__ unsigned long long wt[8];
  __shared__ long long redc[9];
  const int b = blockIdx.x;
  SelState st = sel[b];
  if (st.done) return;
  constexpr int nb = 1 << lvl_bits(LEVEL);
  constexpr int PER = nb / 256;
  const unsigned *gc = hcnt + int64_t(b) * kHistBins;
  const unsigned long long *gq = hq + int64_t(b) * kHistBins;
  // thread t holds the reversed bins j = t*PER .. t*PER+PER-1 (bin = nb-1-j)
  unsigned long long q[PER];
  unsigned c[PER];
  unsigned long long tq = 0;
  for (int i = 0; i < PER; ++i) {
    const int bin = nb - 1 - (threadIdx.x * PER + i);
    q[i] = gq[bin];
    c[i] = gc[bin];
    tq += q[i];
  }
  if (LEVEL == 0) {
    const unsigned long long tot = block_sum256<unsigned long long>(tq, red);
    st.q_tot = tot;
    const double tgt = e_target * double(tot);
    if (!(tgt < double(tot))) {
      st.all = 1; st.done = 1; st.thr_key = 0; st.n_tie = 0x7fffffff;
      if (threadIdx.x == 0) sel[b] = st;
      return;
    }
    unsigned long long t = (unsigned long long)ceil(tgt);
    if (t < 1) t = 1;
    st.target = t;
  }
  // inclusive prefix of q over reversed bins
  const unsigned long long excl_thread = block_incl_scan256(tq, wt) - tq;
  // crossing index j*: number of reversed bins whose inclusive prefix stays below target
  long long below = 0;
  unsigned long long run = st.q_above + excl_thread;
  unsigned long long q_before = 0;    // q of bins above the crossing bin (this thread's share)
  long long c_before = 0;
  for (int i = 0; i < PER; ++i) {
    run += q[i];
    if (run < st.target) { ++below; q_before += q[i]; c_before += c[i]; }
  }
  const long long jstar = block_sum256<long long>(below, redc);
  const unsigned long long qb = block_sum256<unsigned long long>(q_before, red);
  const long long cb = block_sum256<long long>(c_before, redc);
  __shared__ unsigned cstar;
  if (threadIdx.x == (int)(jstar / PER) && jstar < nb) cstar = c[jstar % PER];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int binstar = nb - 1 - int(jstar);
    st.q_above += qb;
    st.n_above += int32_t(cb);
    st.prefix = (LEVEL == 0) ? unsigned(binstar) : ((st.prefix << lvl_bits(LEVEL)) | unsigned(binstar));
    if (LEVEL == 2) {
      st.thr_key = st.prefix;
      const unsigned long long qthr =
          fixed_energy(__uint_as_float(st.thr_key), st.qexp);
      const unsigned long long rem = st.target - st.q_above;
      long long nt = (qthr > 0) ? (long long)((rem + qthr - 1) / qthr) : (long long)cstar;
      if (nt > (long long)cstar) nt = cstar;
      if (nt < 0) nt = 0;
      st.n_tie = int32_t(nt);
      st.done = 1;
    }
    sel[b] = st;
  }
}

// ---- per-tile counts ------------------------------------------------------------------

__global__ void __launch_bounds__(256)
k_tile_count(const float2 *__restrict__ K, int S, const int32_t *__restrict__ ids,
             const int2 *__restrict__ j0, const int64_t *__restrict__ seg_base, GridGeom g,
             const SelState *__restrict__ sel, int32_t *__restrict__ cnt_gt,
             int32_t *__restrict__ cnt_eq, int smem_tiles) {
  extern __shared__ int32_t sc[];   // [2][smem_tiles]
  const int b = blockIdx.y;
  const int k = ids[b];
  const SelState st = sel[b];
  const AxisTiles tu = axis_tiles(j0[k].x, S, g.G, g.tile);
  const AxisTiles tv = axis_tiles(j0[k].y, S, g.G, g.tile);
  const int nt = tu.nt * tv.nt;
  const bool use_smem = nt <= smem_tiles;   // else count straight into global memory
  int32_t *gt = use_smem ? sc : cnt_gt + seg_base[k];
  int32_t *eq = use_smem ? sc + nt : cnt_eq + seg_base[k];
  if (use_smem) {
    for (int i = threadIdx.x; i < 2 * nt; i += blockDim.x) sc[i] = 0;
    __syncthreads();
  }
  const int64_t n = int64_t(S) * S;
  const int64_t lo = int64_t(blockIdx.x) * kSelChunk;
  const int64_t hi = min(n, lo + kSelChunk);
  const float2 *Kb = K + int64_t(b) * n;
  const int logS = 31 - __clz(S), logT = 31 - __clz(g.tile);
  const int Gm = g.G - 1;   // G and the tile side are powers of two
  const int2 jk = j0[k];
  // a thread takes kRun consecutive samples of one box row (S >= 16, S^2 and
  // the chunk bounds are multiples of kRun) and adds each run of samples in one tile with
  // one pair of atomics (integer counts: the grouping does not matter)
  for (int64_t i0 = lo + kRun * int64_t(threadIdx.x); i0 < hi; i0 += kRun * int64_t(blockDim.x)) {
    float4 pk[kRun / 2];
    if (!st.all) {
#pragma unroll
      for (int h = 0; h < kRun / 2; ++h) pk[h] = __ldg(reinterpret_cast<const float4 *>(Kb + i0) + h);
    }
    const int iu = int(i0 >> logS), iv0 = int(i0 & (S - 1));
    const int su = iu < S / 2 ? iu : iu - S;
    const int pu = axis_tile_pos(tu, ((jk.x + su) & Gm) >> logT) * tv.nt;
    int rpos = -1, rgt = 0, req = 0;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const int iv = iv0 + j;
      const int sv = iv < S / 2 ? iv : iv - S;
      const int pos = pu + axis_tile_pos(tv, ((jk.y + sv) & Gm) >> logT);
      int isgt = 1, iseq = 0;
      if (!st.all) {
        const float4 &v = pk[j >> 1];
        const unsigned key = __float_as_uint(abs2_rn((j & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y)));
        isgt = key > st.thr_key;
        iseq = key == st.thr_key;
      }
      if (pos != rpos) {
        if (rgt) atomicAdd(&gt[rpos], rgt);
        if (req) atomicAdd(&eq[rpos], req);
        rpos = pos;
        rgt = req = 0;
      }
      rgt += isgt;
      req += iseq;
    }
    if (rgt) atomicAdd(&gt[rpos], rgt);
    if (req) atomicAdd(&eq[rpos], req);
  }
  if (use_smem) {
    __syncthreads();
    const int64_t base = seg_base[k];
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      if (sc[i]) atomicAdd(&cnt_gt[base + i], sc[i]);
      if (sc[nt + i]) atomicAdd(&cnt_eq[base + i], sc[nt + i]);
    }
  }
}

// ties go to the earliest tiles (emission order): tile i of a box takes
// min(eq_i, n_tie - sum_{j<i} eq_j) of its threshold ties; one block per box
__global__ void __launch_bounds__(128)
k_tie_alloc(const int32_t *__restrict__ ids, const int64_t *__restrict__ seg_base,
            const int32_t *__restrict__ ntile, const SelState *__restrict__ sel,
            const int32_t *__restrict__ cnt_gt, const int32_t *__restrict__ cnt_eq,
            int32_t *__restrict__ seg_cnt, int32_t *__restrict__ seg_tieb,
            uint32_t *__restrict__ r_thr, int32_t *__restrict__ r_ntie,
            int8_t *__restrict__ r_all, float *__restrict__ r_max) {
  __shared__ int wsum[4];
  const int b = blockIdx.x;
  const int k = ids[b];
  const SelState st = sel[b];
  const int64_t base = seg_base[k];
  const int nt = ntile[k];
  const int ntie = st.all ? 0 : st.n_tie;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int carry = 0;   // ties of the tiles before this group of 128
  for (int i0 = 0; i0 < nt; i0 += 128) {
    const int i = i0 + threadIdx.x;
    const int e = (i < nt && !st.all) ? cnt_eq[base + i] : 0;
    int inc = e;
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += n;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int before = carry;
    for (int j = 0; j < w; ++j) before += wsum[j];
    const int excl = before + inc - e;
    if (i < nt) {
      const int a = min(e, max(0, ntie - excl));
      seg_tieb[base + i] = min(excl, ntie);
      seg_cnt[base + i] = cnt_gt[base + i] + a;
    }
    carry += wsum[0] + wsum[1] + wsum[2] + wsum[3];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    r_thr[k] = st.thr_key;
    r_ntie[k] = st.n_tie;
    r_all[k] = int8_t(st.all);
    r_max[k] = sqrtf(__uint_as_float(st.maxkey));
  }
}

// ---- emission -------------------------------------------------------------------------

// One warp per (box, touched tile) segment, lane = tile column: the warp walks
// the tile's rows in order, so a ballot is one row of the tile (the selection
// word of the tile-mask format) and running popcounts give each entry's place
// in the row-major compacted order and each tie's rank (ties are taken in the
// same row-major order).  No block barriers: the 8 warps of a block take 8
// segments.
__global__ void __launch_bounds__(256)
k_emit(const float2 *__restrict__ K, int S, const int32_t *__restrict__ ids,
       const int2 *__restrict__ j0, const int64_t *__restrict__ seg_base,
       const int32_t *__restrict__ ntile, GridGeom g, const int64_t *__restrict__ seg_off,
       const int32_t *__restrict__ seg_tieb, const uint32_t *__restrict__ r_thr,
       const int32_t *__restrict__ r_ntie, const int8_t *__restrict__ r_all,
       const float *__restrict__ r_max, const int32_t *__restrict__ seg_cnt,
       int32_t *__restrict__ col, int fmt, void *__restrict__ val, int vdt,
       const int64_t *__restrict__ seg_rec, unsigned char *__restrict__ stream, int *__restrict__ err) {
  const int b = blockIdx.y;
  const int k = ids[b];
  const int nt = ntile[k];
  const int TS = g.tile;
  const AxisTiles tu = axis_tiles(j0[k].x, S, g.G, TS);
  const AxisTiles tv = axis_tiles(j0[k].y, S, g.G, TS);
  const unsigned thr = r_thr[k];
  const int ntie = r_ntie[k];
  const bool all = r_all[k] != 0;
  const float inv_scale = (vdt != WPROJ_VAL_F32 && r_max[k] > 0.f) ? 1.0f / r_max[k] : 1.0f;
  const float2 *Kb = K + int64_t(b) * S * S;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const bool rec = fmt == WPROJ_INDEX_TILE_MASK;
  const int Gm = g.G - 1;   // G is a power of two
  for (int seg = blockIdx.x * 8 + w; seg < nt; seg += gridDim.x * 8) {
    const int iu_t = seg / tv.nt, iv_t = seg % tv.nt;
    const int tile_u = axis_tile_at(tu, iu_t, g.nT), tile_v = axis_tile_at(tv, iv_t, g.nT);
    const int64_t sid = seg_base[k] + seg;
    const int tie0 = seg_tieb[sid];
    const int cnt = seg_cnt[sid];
    // COLUMNS: entries at seg_off in col / val; TILE_MASK: the segment's record
    const int64_t o = rec ? 0 : seg_off[sid];
    unsigned char *rp = rec ? stream + seg_rec[sid] : nullptr;
    void *vdst = rec ? static_cast<void *>(rp + kRecValues) : val;
    const int cv = tile_v * TS + lane;
    const int dv = (cv - tv.a) & Gm;
    const bool col_in = lane < TS && dv < S;
    const int iv = (dv + S / 2) & (S - 1);
    int tie_run = 0, sel_run = 0;
    unsigned my_w = 0;    // lane r keeps row r's selection word and prefix
    int my_pre = 0;
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      bool gt = false, eq = false;
      int kidx = 0;
      if (r < TS && col_in) {
        const int du = (tile_u * TS + r - tu.a) & Gm;
        if (du < S) {
          kidx = ((du + S / 2) & (S - 1)) * S + iv;
          const unsigned key = __float_as_uint(abs2_rn(Kb[kidx]));
          gt = all || key > thr;
          eq = !all && key == thr;
        }
      }
      const unsigned tw = __ballot_sync(0xffffffffu, eq);
      const int rank = tie0 + tie_run + __popc(tw & lt);
      const bool sel = gt || (eq && rank < ntie);
      const unsigned sw = __ballot_sync(0xffffffffu, sel);
      const int pos = sel_run + __popc(sw & lt);
      if (sel && pos < cnt) {    // pos < cnt always holds when the two passes agree
        const int64_t at = o + pos;
        if (!rec) col[at] = (tile_u * TS + r) * g.G + cv;
        const float2 v = Kb[kidx];
        if (vdt == WPROJ_VAL_F32) {
          reinterpret_cast<float2 *>(vdst)[at] = v;
        } else if (vdt == WPROJ_VAL_BF16) {
          reinterpret_cast<__nv_bfloat162 *>(vdst)[at] = __floats2bfloat162_rn(v.x * inv_scale, v.y * inv_scale);
        } else {
          reinterpret_cast<__half2 *>(vdst)[at] = __floats2half2_rn(v.x * inv_scale, v.y * inv_scale);
        }
      }
      if (lane == r) {
        my_w = sw;
        my_pre = sel_run;
      }
      tie_run += __popc(tw);
      sel_run += __popc(sw);
    }
    if (lane == 0 && sel_run != cnt) atomicOr(err, ERR_EMIT);
    if (rec) {
      reinterpret_cast<uint32_t *>(rp + kRecHeader)[lane] = my_w;
      reinterpret_cast<uint16_t *>(rp + kRecPrefix)[lane] = uint16_t(my_pre);
      if (lane == 0) *reinterpret_cast<int4 *>(rp) = make_int4(k, cnt, int(sid), 0);
    }
  }
}

__global__ void k_row_ptr(int64_t m, const int64_t *__restrict__ seg_base,
                          const int64_t *__restrict__ seg_off, const int32_t *__restrict__ ntile,
                          int64_t n_seg, int64_t nnz, int64_t *__restrict__ row_ptr) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k > m) return;
  if (k == m) { row_ptr[m] = nnz; return; }
  const int64_t sb = seg_base[k];
  const int64_t start = (sb < n_seg) ? seg_off[sb] : nnz;
  const int64_t end = (k + 1 < m) ? ((seg_base[k + 1] < n_seg) ? seg_off[seg_base[k + 1]] : nnz) : nnz;
  row_ptr[k] = start;
  (void)ntile;
  (void)end;
}

__global__ void k_npieces(int64_t m, const int64_t *__restrict__ row_ptr, int64_t piece,
                          int32_t *__restrict__ npieces) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < m) npieces[k] = int32_t(i64max(1, (row_ptr[k + 1] - row_ptr[k] + piece - 1) / piece));
}

// Row pieces of the column-format degridding: ranges of <= piece entries.
__global__ void k_pieces(int64_t m, const int64_t *__restrict__ row_ptr,
                         const int64_t *__restrict__ piece_base, int32_t *__restrict__ piece_row,
                         int64_t *__restrict__ piece_lo, int32_t *__restrict__ piece_len,
                         int32_t *__restrict__ row_piece_ptr, int64_t n_pieces, int64_t piece) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k > m) return;
  if (k == m) { row_piece_ptr[m] = int32_t(n_pieces); return; }
  const int64_t pb = piece_base[k];
  row_piece_ptr[k] = int32_t(pb);
  const int64_t lo = row_ptr[k], n = row_ptr[k + 1] - lo, step = piece;
  const int np = int(i64max(1, (n + step - 1) / step));
  for (int i = 0; i < np; ++i) {
    piece_row[pb + i] = int32_t(k);
    piece_lo[pb + i] = lo + int64_t(i) * step;
    piece_len[pb + i] = int32_t(i64max(0, i64min(step, n - int64_t(i) * step)));
  }
}

// gridding: per-tile nnz (sorted segment order) and chunk counts
__global__ void k_gather_cnt(int64_t n, const int32_t *__restrict__ tile_seg,
                             const int32_t *__restrict__ seg_cnt, const int64_t *__restrict__ seg_off,
                             const int32_t *__restrict__ seg_row, int32_t *__restrict__ out,
                             SegMeta *__restrict__ meta) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sg = tile_seg[i];
  const int c = seg_cnt[sg];
  out[i] = c;
  if (!meta) return;
  SegMeta m;
  m.off_cnt = (unsigned long long)seg_off[sg] | ((unsigned long long)c << 40);
  m.seg = sg;
  m.row = seg_row[sg];
  meta[i] = m;
}

// tile-stream layout: record bytes of each segment in tile order
__global__ void k_rec_size(int64_t n, const int32_t *__restrict__ tile_seg, const int32_t *__restrict__ seg_cnt,
                           int vb, int32_t *__restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = kRecValues + ((seg_cnt[tile_seg[i]] * vb + 15) & ~15);
}

__global__ void k_rec_scatter(int64_t n, const int32_t *__restrict__ tile_seg, const int64_t *__restrict__ rec_off,
                              int64_t *__restrict__ seg_rec) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  seg_rec[tile_seg[i]] = rec_off[i];
}


__global__ void k_tile_chunks(int n_tiles, const int64_t *__restrict__ tile_ptr,
                              const int64_t *__restrict__ cum, int64_t n_seg, int64_t nnz_total,
                              int64_t chunk, int32_t *__restrict__ nch) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const int64_t a = tile_ptr[t], bq = tile_ptr[t + 1];
  const int64_t ca = (a < n_seg) ? cum[a] : nnz_total;
  const int64_t cb = (bq < n_seg) ? cum[bq] : nnz_total;
  nch[t] = int32_t(i64max(1, (cb - ca + chunk - 1) / chunk));
}

__global__ void k_chunk_fill(int n_tiles, const int64_t *__restrict__ tile_ptr,
                             const int64_t *__restrict__ cum, int64_t n_seg, int64_t nnz_total,
                             const int64_t *__restrict__ ch_base, int32_t *__restrict__ chunk_tile,
                             int64_t *__restrict__ chunk_lo, int64_t *__restrict__ chunk_hi,
                             int32_t *__restrict__ tile_chunk_ptr, int64_t n_chunks, int64_t chunk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  if (t == n_tiles) { tile_chunk_ptr[n_tiles] = int32_t(n_chunks); return; }
  const int64_t a = tile_ptr[t], bq = tile_ptr[t + 1];
  auto cumat = [&](int64_t j) { return j < n_seg ? cum[j] : nnz_total; };
  const int64_t ca = cumat(a), cb = cumat(bq);
  const int nc = int(i64max(1, (cb - ca + chunk - 1) / chunk));
  const int64_t base = ch_base[t];
  tile_chunk_ptr[t] = int32_t(base);
  int64_t lo = a;
  for (int c = 0; c < nc; ++c) {
    int64_t hi;
    if (c == nc - 1) {
      hi = bq;
    } else {
      // first position j in [lo, bq] with cum[j] - ca >= (c+1) * chunk
      const int64_t want = ca + int64_t(c + 1) * chunk;
      int64_t l = lo, r = bq;
      while (l < r) {
        const int64_t mid = (l + r) / 2;
        if (cumat(mid) >= want) r = mid; else l = mid + 1;
      }
      hi = l;
    }
    chunk_tile[base + c] = t;
    chunk_lo[base + c] = lo;
    chunk_hi[base + c] = hi;
    lo = hi;
  }
}

}  // namespace

wproj_status make_row_pieces(int64_t m, const int64_t *row_ptr, int64_t piece, DevBuf &piece_row, DevBuf &piece_lo,
                             DevBuf &piece_len, DevBuf &row_piece_ptr, int64_t *n_pieces, cudaStream_t s) {
  DevBuf npc, pbase;
  WPROJ_TRY(npc.alloc(sizeof(int32_t) * std::max<int64_t>(1, m)));
  WPROJ_TRY(pbase.alloc(sizeof(int64_t) * (m + 1)));
  k_npieces<<<ceil_div(m, 256), 256, 0, s>>>(m, row_ptr, piece, npc.as<int32_t>());
  WPROJ_CHECK_LAUNCH("piece counts");
  WPROJ_TRY(exclusive_scan_i32_to_i64(npc.as<int32_t>(), pbase.as<int64_t>(), m, s));
  int64_t lb = 0;
  int32_t ln = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&lb, pbase.as<int64_t>() + (m - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&ln, npc.as<int32_t>() + (m - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  *n_pieces = lb + ln;
  if (*n_pieces >= (int64_t(1) << 31)) return fail(WPROJ_ERR_UNSUPPORTED, "too many row pieces");
  WPROJ_TRY(piece_row.alloc(sizeof(int32_t) * *n_pieces));
  WPROJ_TRY(piece_lo.alloc(sizeof(int64_t) * *n_pieces));
  WPROJ_TRY(piece_len.alloc(sizeof(int32_t) * *n_pieces));
  WPROJ_TRY(row_piece_ptr.alloc(sizeof(int32_t) * (m + 1)));
  k_pieces<<<ceil_div(m + 1, 256), 256, 0, s>>>(m, row_ptr, pbase.as<int64_t>(), piece_row.as<int32_t>(),
                                                piece_lo.as<int64_t>(), piece_len.as<int32_t>(),
                                                row_piece_ptr.as<int32_t>(), *n_pieces, piece);
  WPROJ_CHECK_LAUNCH("pieces");
  return WPROJ_OK;
}

wproj_status make_tile_chunks(int n_tiles, const int64_t *tptr, const int64_t *cum, int64_t n_seg, int64_t nnz,
                              int64_t chunk, DevBuf &chunk_tile, DevBuf &chunk_lo, DevBuf &chunk_hi,
                              DevBuf &tile_chunk_ptr, int64_t *n_chunks, cudaStream_t s) {
  DevBuf nch, chbase;
  WPROJ_TRY(nch.alloc(sizeof(int32_t) * n_tiles));
  WPROJ_TRY(chbase.alloc(sizeof(int64_t) * (n_tiles + 1)));
  k_tile_chunks<<<ceil_div(n_tiles, 256), 256, 0, s>>>(n_tiles, tptr, cum, n_seg, nnz, chunk, nch.as<int32_t>());
  WPROJ_CHECK_LAUNCH("tile chunks");
  WPROJ_TRY(exclusive_scan_i32_to_i64(nch.as<int32_t>(), chbase.as<int64_t>(), n_tiles, s));
  int64_t lb = 0;
  int32_t ln = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&lb, chbase.as<int64_t>() + (n_tiles - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&ln, nch.as<int32_t>() + (n_tiles - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  *n_chunks = lb + ln;
  WPROJ_TRY(chunk_tile.alloc(sizeof(int32_t) * *n_chunks));
  WPROJ_TRY(chunk_lo.alloc(sizeof(int64_t) * *n_chunks));
  WPROJ_TRY(chunk_hi.alloc(sizeof(int64_t) * *n_chunks));
  WPROJ_TRY(tile_chunk_ptr.alloc(sizeof(int32_t) * (n_tiles + 1)));
  k_chunk_fill<<<ceil_div(n_tiles + 1, 256), 256, 0, s>>>(n_tiles, tptr, cum, n_seg, nnz, chbase.as<int64_t>(),
                                                          chunk_tile.as<int32_t>(), chunk_lo.as<int64_t>(),
                                                          chunk_hi.as<int64_t>(), tile_chunk_ptr.as<int32_t>(),
                                                          *n_chunks, chunk);
  WPROJ_CHECK_LAUNCH("chunk fill");
  return WPROJ_OK;
}

wproj_status set_screens_impl(wproj_plan *p, const float2 *screens, int n, cudaStream_t s) {
  p->built = false;
  p->dr_valid = false;
  p->n_screens = 0;
  if (n == 0) {
    p->screens.release();
    p->screen_max2.release();
    return WPROJ_OK;
  }
  const int64_t per = int64_t(p->g.G) * p->g.G;
  WPROJ_TRY(p->screens.alloc(sizeof(float2) * per * n));
  WPROJ_TRY(p->screen_max2.alloc(sizeof(float) * n));
  WPROJ_CUDA(cudaMemcpyAsync(p->screens.ptr, screens, sizeof(float2) * per * n, cudaMemcpyDefault, s));
  DevBuf d_err;
  WPROJ_TRY(d_err.alloc(sizeof(int)));
  WPROJ_CUDA(cudaMemsetAsync(d_err.ptr, 0, sizeof(int), s));
  k_screen_max<<<n, 256, 0, s>>>(p->screens.as<float2>(), per, p->screen_max2.as<float>(), d_err.as<int>());
  WPROJ_CHECK_LAUNCH("screen max");
  int herr = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&herr, d_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(WPROJ_ERR_INVALID_ARG, "set_screens: non-finite screen values");
  p->n_screens = n;
  return WPROJ_OK;
}

wproj_status build_kernels_impl(wproj_plan *p, const double *uvw, int64_t m, double e, cudaStream_t s,
                                const int32_t *sid) {
  auto t_start = std::chrono::steady_clock::now();
  const GridGeom &g = p->g;
  p->built = false;
  p->dr_valid = false;
  p->m = p->nnz = p->n_seg = p->n_chunks = p->n_pieces = 0;

  // ---- rows
  DevBuf d_j0, d_delta, d_Sk, d_ntile, d_sclass, d_err, d_segbase;
  WPROJ_TRY(d_j0.alloc(sizeof(int2) * m));
  WPROJ_TRY(d_delta.alloc(sizeof(double2) * m));
  WPROJ_TRY(d_Sk.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(d_ntile.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(d_sclass.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(d_err.alloc(sizeof(int)));
  WPROJ_TRY(d_segbase.alloc(sizeof(int64_t) * (m + 1)));
  WPROJ_CUDA(cudaMemsetAsync(d_err.ptr, 0, sizeof(int), s));
  k_row_plan<<<ceil_div(m, 256), 256, 0, s>>>(uvw, m, g, d_j0.as<int2>(), d_delta.as<double2>(),
                                              d_Sk.as<int32_t>(), d_ntile.as<int32_t>(),
                                              d_sclass.as<int32_t>(), d_err.as<int>());
  WPROJ_CHECK_LAUNCH("row plan");
  if (sid) {
    if (p->n_screens < 1 || g.box != g.G) return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels: screens need box = G");
    k_check_sid<<<ceil_div(m, 256), 256, 0, s>>>(m, sid, p->n_screens, d_err.as<int>());
    WPROJ_CHECK_LAUNCH("screen ids");
  }
  int herr = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&herr, d_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (herr & ERR_NONFINITE) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels: non-finite (u, v, w)");
  if (herr & ERR_BAND) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels: (u, v) outside [-B, B)");
  if (herr & ERR_SCREEN) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels: screen id out of range");

  // ---- segments (row, touched tile)
  WPROJ_TRY(exclusive_scan_i32_to_i64(d_ntile.as<int32_t>(), d_segbase.as<int64_t>(), m, s));
  int64_t last_base = 0;
  int32_t last_nt = 0;
  WPROJ_CUDA(cudaMemcpy(&last_base, d_segbase.as<int64_t>() + (m - 1), sizeof(int64_t), cudaMemcpyDeviceToHost));
  WPROJ_CUDA(cudaMemcpy(&last_nt, d_ntile.as<int32_t>() + (m - 1), sizeof(int32_t), cudaMemcpyDeviceToHost));
  const int64_t n_seg = last_base + last_nt;
  if (n_seg >= (int64_t(1) << 31)) return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels: too many (row, tile) segments");
  WPROJ_TRY(p->seg_off.alloc(sizeof(int64_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_TRY(p->seg_cnt.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_TRY(p->seg_row.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  DevBuf d_cntgt, d_cnteq, d_tieb;
  WPROJ_TRY(p->seg_tile.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_TRY(d_cntgt.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_TRY(d_cnteq.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_TRY(d_tieb.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_CUDA(cudaMemsetAsync(d_cntgt.ptr, 0, sizeof(int32_t) * n_seg, s));
  WPROJ_CUDA(cudaMemsetAsync(d_cnteq.ptr, 0, sizeof(int32_t) * n_seg, s));
  k_seg_fill<<<(unsigned)m, 128, 0, s>>>(m, g, d_j0.as<int2>(), d_Sk.as<int32_t>(), d_segbase.as<int64_t>(),
                                         p->seg_row.as<int32_t>(), p->seg_tile.as<int32_t>());
  WPROJ_CHECK_LAUNCH("seg fill");

  // ---- group rows by box size (stable: rows ascending inside a group)
  DevBuf d_ids, d_cls_ptr;
  WPROJ_TRY(d_ids.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(d_cls_ptr.alloc(sizeof(int64_t) * 10));
  WPROJ_TRY(stable_bin_sort(d_sclass.as<int32_t>(), m, 9, d_ids.as<int32_t>(), d_cls_ptr.as<int64_t>(), s));
  int64_t cls_ptr[10];
  WPROJ_CUDA(cudaMemcpy(cls_ptr, d_cls_ptr.ptr, sizeof(cls_ptr), cudaMemcpyDeviceToHost));

  // per-row selection results
  DevBuf r_thr, r_ntie, r_all, r_max;
  WPROJ_TRY(r_thr.alloc(sizeof(uint32_t) * m));
  WPROJ_TRY(r_ntie.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(r_all.alloc(sizeof(int8_t) * m));
  WPROJ_TRY(r_max.alloc(sizeof(float) * m));

  p->box_min = 1 << 30;
  p->box_max = 0;
  int max_nb = 1;
  for (int c = 0; c < 9; ++c) {
    if (cls_ptr[c + 1] <= cls_ptr[c]) continue;
    const int S = 16 << c;
    p->box_min = std::min(p->box_min, S);
    p->box_max = std::max(p->box_max, S);
    const int64_t per = int64_t(S) * S * sizeof(float2);
    max_nb = std::max<int>(max_nb, (int)std::min<int64_t>(std::min<int64_t>(cls_ptr[c + 1] - cls_ptr[c], kMaxBatchBoxes),
                                                            std::max<int64_t>(1, batch_bytes(S) / per)));
  }
  DevBuf Kbuf, Au, Av, bmode, bwf, bwd, bsel, hcnt, hq, lcoord, lsq, bsid;
  // Pass 2 needs every box's transform again.  When the device has room for all
  // of them (and, with a margin, for G, whose size is at most 1.5x theirs), pass
  // 1 keeps them and pass 2 emits without recomputing the tables and FFTs;
  // otherwise pass 2 recomputes them batch by batch.
  int64_t k_total = 0;
  for (int c = 0; c < 9; ++c) k_total += (cls_ptr[c + 1] - cls_ptr[c]) * int64_t(16 << c) * (16 << c) * int64_t(sizeof(float2));
  DevBuf Kall;
  bool keep_all = false;
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
        double(free_b) > 2.5 * double(k_total) + double(size_t(2) << 30)) {
      keep_all = Kall.alloc(size_t(k_total)) == WPROJ_OK;
      if (!keep_all) cudaGetLastError();   // fall back to recomputing
    }
  }
  if (!keep_all)
    WPROJ_TRY(Kbuf.alloc(std::max<size_t>(kBuildBatchBytes, size_t(p->box_max) * p->box_max * sizeof(float2))));
  WPROJ_TRY(Au.alloc(sizeof(float2) * size_t(max_nb) * p->box_max));
  WPROJ_TRY(Av.alloc(sizeof(float2) * size_t(max_nb) * p->box_max));
  WPROJ_TRY(bmode.alloc(max_nb));
  WPROJ_TRY(bwf.alloc(sizeof(float) * max_nb));
  WPROJ_TRY(bwd.alloc(sizeof(double) * max_nb));
  WPROJ_TRY(bsel.alloc(sizeof(SelState) * max_nb));
  if (sid) WPROJ_TRY(bsid.alloc(sizeof(int32_t) * max_nb));
  WPROJ_TRY(hcnt.alloc(sizeof(unsigned) * kHistBins * size_t(max_nb)));
  WPROJ_TRY(hq.alloc(sizeof(unsigned long long) * kHistBins * size_t(max_nb)));
  WPROJ_TRY(lcoord.alloc(sizeof(double) * p->box_max));
  WPROJ_TRY(lsq.alloc(sizeof(float) * p->box_max));

  const double e_target = e + kSelectMargin;
  const int vdt = g.value_dtype;
  const int vb = vdt == WPROJ_VAL_F32 ? 8 : 4;
  const int n_tiles = g.nT * g.nT;
  DevBuf tile_seg, tptr;
  bool want_runs = false;   // TILE_RUNS: emitted as columns, then transcoded
  int64_t n_rec = 0;        // TILE_RUNS: records (segments holding entries), tile order

  for (int phase = 1; phase <= 2; ++phase) {
    int64_t koff = 0;   // boxes transformed so far (position in Kall)
    if (phase == 2) {
      // lay out G exactly
      WPROJ_TRY(exclusive_scan_i32_to_i64(p->seg_cnt.as<int32_t>(), p->seg_off.as<int64_t>(), n_seg, s));
      int64_t lo = 0;
      int32_t lc = 0;
      if (n_seg > 0) {
        WPROJ_CUDA(cudaMemcpy(&lo, p->seg_off.as<int64_t>() + (n_seg - 1), sizeof(int64_t), cudaMemcpyDeviceToHost));
        WPROJ_CUDA(cudaMemcpy(&lc, p->seg_cnt.as<int32_t>() + (n_seg - 1), sizeof(int32_t), cudaMemcpyDeviceToHost));
      }
      p->nnz = lo + lc;
      // column storage: the tile masks pay off for dense segments (they cut 4 of
      // 12 bytes per entry), the column indices for sparse ones (the mask kernels
      // spend per-segment work on all 32 tile rows); measured at N=256/M=32768
      // (573 entries per segment: masks 1.5x faster) and N=1024/M=2^21 (41 per
      // segment: columns 5x faster)
      // boxes of at most 64 x 64 cells keep one run of cells per grid row: run
      // descriptors (TILE_RUNS) then cost a few per cent of the value bytes
      // (measured at N=1024/M=2^21: 283 entries in 16.6 runs per row).  With
      // 16-bit values the column form with its cell-major gridding copy is the
      // faster of the two there (313.9 against 279.9 Phi+Phi^H pairs/s in bf16;
      // f32: 266.4 against 291.0), when its packed rows fit (m <= 2^22)
      const bool runs_ok = p->box_max <= 64 && g.tile == 32;
      const bool cols_16 = g.value_dtype != WPROJ_VAL_F32 && m <= (int64_t(1) << 22);
      int fmt = g.index_format;
      if (fmt == WPROJ_INDEX_AUTO)
        fmt = (runs_ok && !cols_16) ? WPROJ_INDEX_TILE_RUNS
                                    : ((p->nnz >= 256 * n_seg) ? WPROJ_INDEX_TILE_MASK : WPROJ_INDEX_COLUMNS);
      if (fmt == WPROJ_INDEX_TILE_RUNS && !runs_ok)
        return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels: TILE_RUNS needs kernel boxes of at most 64 x 64 cells");
      if (g.tile != 32) fmt = WPROJ_INDEX_COLUMNS;
      want_runs = fmt == WPROJ_INDEX_TILE_RUNS;
      if (want_runs) fmt = WPROJ_INDEX_COLUMNS;
      p->fmt = fmt;
      // segments in tile order, rows ascending inside a tile: the gridding's
      // order, and the record order of the tile stream
      WPROJ_TRY(tile_seg.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
      WPROJ_TRY(tptr.alloc(sizeof(int64_t) * (n_tiles + 1)));
      WPROJ_TRY(stable_bin_sort(p->seg_tile.as<int32_t>(), n_seg, n_tiles, tile_seg.as<int32_t>(),
                                tptr.as<int64_t>(), s));
      if (fmt == WPROJ_INDEX_TILE_MASK) {
        p->col.release();
        p->val.release();
        p->seg_meta.release();
        DevBuf rsz;
        WPROJ_TRY(rsz.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
        WPROJ_TRY(p->rec_off.alloc(sizeof(int64_t) * (n_seg + 1)));
        WPROJ_TRY(p->seg_rec.alloc(sizeof(int64_t) * std::max<int64_t>(1, n_seg)));
        int64_t total = 0;
        if (n_seg > 0) {
          k_rec_size<<<ceil_div(n_seg, 256), 256, 0, s>>>(n_seg, tile_seg.as<int32_t>(), p->seg_cnt.as<int32_t>(), vb,
                                                          rsz.as<int32_t>());
          WPROJ_CHECK_LAUNCH("record sizes");
          WPROJ_TRY(exclusive_scan_i32_to_i64(rsz.as<int32_t>(), p->rec_off.as<int64_t>(), n_seg, s));
          int64_t lo2 = 0;
          int32_t lc2 = 0;
          WPROJ_CUDA(cudaMemcpy(&lo2, p->rec_off.as<int64_t>() + (n_seg - 1), sizeof(int64_t), cudaMemcpyDeviceToHost));
          WPROJ_CUDA(cudaMemcpy(&lc2, rsz.as<int32_t>() + (n_seg - 1), sizeof(int32_t), cudaMemcpyDeviceToHost));
          total = lo2 + lc2;
          k_rec_scatter<<<ceil_div(n_seg, 256), 256, 0, s>>>(n_seg, tile_seg.as<int32_t>(), p->rec_off.as<int64_t>(),
                                                             p->seg_rec.as<int64_t>());
          WPROJ_CHECK_LAUNCH("record offsets");
        }
        WPROJ_CUDA(cudaMemcpy(p->rec_off.as<int64_t>() + n_seg, &total, sizeof(int64_t), cudaMemcpyHostToDevice));
        WPROJ_TRY(p->stream.alloc(std::max<int64_t>(16, total)));
        WPROJ_CUDA(cudaMemsetAsync(p->stream.ptr, 0, std::max<int64_t>(16, total), s));   // record padding
        p->stream_bytes = total;
      } else {
        p->stream.release();
        p->seg_rec.release();
        p->rec_off.release();
        p->stream_bytes = 0;
        WPROJ_TRY(p->col.alloc(sizeof(int32_t) * std::max<int64_t>(1, p->nnz)));
        WPROJ_TRY(p->val.alloc(int64_t(vb) * std::max<int64_t>(1, p->nnz)));
      }
      WPROJ_TRY(p->row_ptr.alloc(sizeof(int64_t) * (m + 1)));
      k_row_ptr<<<ceil_div(m + 1, 256), 256, 0, s>>>(m, d_segbase.as<int64_t>(), p->seg_off.as<int64_t>(),
                                                     d_ntile.as<int32_t>(), n_seg, p->nnz, p->row_ptr.as<int64_t>());
      WPROJ_CHECK_LAUNCH("row ptr");
    }
    for (int c = 0; c < 9; ++c) {
      const int64_t glo = cls_ptr[c], ghi = cls_ptr[c + 1];
      if (ghi <= glo) continue;
      const int S = 16 << c;
      const int64_t per = int64_t(S) * S;
      const int nbmax = (int)std::min<int64_t>(std::min<int64_t>(ghi - glo, kMaxBatchBoxes),
                                               std::max<int64_t>(1, batch_bytes(S) / (per * 8)));
      k_coord_tables<<<ceil_div(S, 256), 256, 0, s>>>(S, g.L, g.extension == WPROJ_EXT_CLAMP,
                                                      lcoord.as<double>(), lsq.as<float>());
      WPROJ_CHECK_LAUNCH("coord tables");
      for (int64_t b0 = glo; b0 < ghi; b0 += nbmax) {
        const int nb = (int)std::min<int64_t>(nbmax, ghi - b0);
        const int32_t *ids = d_ids.as<int32_t>() + b0;
        float2 *Kb = keep_all ? Kall.as<float2>() + koff : Kbuf.as<float2>();
        koff += int64_t(nb) * per;
        BoxBatch bb;
        bb.S = S; bb.nb = nb;
        bb.K = Kb;
        const bool transform = phase == 1 || !keep_all;
        ScopedTimer t_fft(p, TC_BFFT, s);
        if (transform) {
          k_box_tables<<<nb, 128, 0, s>>>(ids, uvw, d_delta.as<double2>(), g, S, lcoord.as<double>(),
                                          Au.as<float2>(), Av.as<float2>(), bmode.as<int8_t>(),
                                          bwf.as<float>(), bwd.as<double>(), bsel.as<SelState>(), sid,
                                          sid ? p->screen_max2.as<float>() : nullptr, bsid.as<int32_t>());
          WPROJ_CHECK_LAUNCH("box tables");
          bb.Au = Au.as<float2>(); bb.Av = Av.as<float2>();
          bb.mode = bmode.as<int8_t>(); bb.wf = bwf.as<float>(); bb.wd = bwd.as<double>();
          bb.lsq = lsq.as<float>(); bb.lcoord = lcoord.as<double>();
          if (sid) {
            bb.screens = p->screens.as<float2>();
            bb.bsid = bsid.as<int32_t>();
          }
          WPROJ_TRY(box_fft(p, bb, s));
        }
        t_fft.stop();
        const dim3 hgrid(ceil_div(per, kSelChunk), nb);
        if (phase == 1) {
          ScopedTimer t_sel(p, TC_BSEL, s);
          WPROJ_CUDA(cudaMemsetAsync(hcnt.ptr, 0, sizeof(unsigned) * kHistBins * nb, s));
          WPROJ_CUDA(cudaMemsetAsync(hq.ptr, 0, sizeof(unsigned long long) * kHistBins * nb, s));
          k_sel_hist<0><<<hgrid, 256, 0, s>>>(bb.K, S, bsel.as<SelState>(), hcnt.as<unsigned>(), hq.as<unsigned long long>());
          k_sel_find<0><<<nb, 256, 0, s>>>(bsel.as<SelState>(), hcnt.as<unsigned>(), hq.as<unsigned long long>(), e_target);
          WPROJ_CUDA(cudaMemsetAsync(hcnt.ptr, 0, sizeof(unsigned) * kHistBins * nb, s));
          WPROJ_CUDA(cudaMemsetAsync(hq.ptr, 0, sizeof(unsigned long long) * kHistBins * nb, s));
          k_sel_hist<1><<<hgrid, 256, 0, s>>>(bb.K, S, bsel.as<SelState>(), hcnt.as<unsigned>(), hq.as<unsigned long long>());
          k_sel_find<1><<<nb, 256, 0, s>>>(bsel.as<SelState>(), hcnt.as<unsigned>(), hq.as<unsigned long long>(), e_target);
          WPROJ_CUDA(cudaMemsetAsync(hcnt.ptr, 0, sizeof(unsigned) * kHistBins * nb, s));
          WPROJ_CUDA(cudaMemsetAsync(hq.ptr, 0, sizeof(unsigned long long) * kHistBins * nb, s));
          k_sel_hist<2><<<hgrid, 256, 0, s>>>(bb.K, S, bsel.as<SelState>(), hcnt.as<unsigned>(), hq.as<unsigned long long>());
          k_sel_find<2><<<nb, 256, 0, s>>>(bsel.as<SelState>(), hcnt.as<unsigned>(), hq.as<unsigned long long>(), e_target);
          WPROJ_CHECK_LAUNCH("select");
          const int nt_box = box_tiles(S, g);
          const int smem_tiles = std::min(nt_box, 4096);
          const size_t smem = sizeof(int32_t) * 2 * smem_tiles;
          if (smem > 48 * 1024) {
            WPROJ_CUDA(cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          }
          k_tile_count<<<hgrid, 256, smem, s>>>(bb.K, S, ids, d_j0.as<int2>(), d_segbase.as<int64_t>(), g,
                                                bsel.as<SelState>(), d_cntgt.as<int32_t>(), d_cnteq.as<int32_t>(),
                                                smem_tiles);
          WPROJ_CHECK_LAUNCH("tile count");
          k_tie_alloc<<<nb, 128, 0, s>>>(ids, d_segbase.as<int64_t>(), d_ntile.as<int32_t>(),
                                                       bsel.as<SelState>(), d_cntgt.as<int32_t>(),
                                                       d_cnteq.as<int32_t>(), p->seg_cnt.as<int32_t>(),
                                                       d_tieb.as<int32_t>(), r_thr.as<uint32_t>(),
                                                       r_ntie.as<int32_t>(), r_all.as<int8_t>(), r_max.as<float>());
          WPROJ_CHECK_LAUNCH("tie alloc");
        } else {
          ScopedTimer t_emit(p, TC_BEMIT, s);
          const int gx = std::min(ceil_div(box_tiles(S, g), 8), 1024);   // 8 segments a block; strides over more
          k_emit<<<dim3(gx, nb), 256, 0, s>>>(bb.K, S, ids, d_j0.as<int2>(), d_segbase.as<int64_t>(),
                                              d_ntile.as<int32_t>(), g, p->seg_off.as<int64_t>(),
                                              d_tieb.as<int32_t>(), r_thr.as<uint32_t>(), r_ntie.as<int32_t>(),
                                              r_all.as<int8_t>(), r_max.as<float>(), p->seg_cnt.as<int32_t>(),
                                              p->col.as<int32_t>(), p->fmt, p->val.ptr, vdt,
                                              p->seg_rec.as<int64_t>(), p->stream.as<unsigned char>(),
                                              d_err.as<int>());
          WPROJ_CHECK_LAUNCH("emit");
        }
      }
    }
  }
  // row scales (max |K| per row) for the 16-bit value forms
  if (vdt != WPROJ_VAL_F32) {
    WPROJ_TRY(p->row_scale.alloc(sizeof(float) * m));
    WPROJ_CUDA(cudaMemcpyAsync(p->row_scale.ptr, r_max.ptr, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
  } else {
    p->row_scale.release();
  }
  if (want_runs) {
    p->m = m;
    p->n_seg = n_seg;
    const wproj_status st = build_runs(p, d_j0.as<int2>(), d_Sk.as<int32_t>(), tile_seg.as<int32_t>(),
                                       tptr.as<int64_t>(), &n_rec, s);
    if (st == WPROJ_OK) {
      p->fmt = WPROJ_INDEX_TILE_RUNS;
    } else if (!(st == WPROJ_ERR_UNSUPPORTED && g.index_format == WPROJ_INDEX_AUTO)) {
      return st;
    }   // AUTO: rows with more than 64 runs keep the column form
  }
  if (p->fmt != WPROJ_INDEX_TILE_RUNS) {
    p->rm_vptr.release();
    p->rm_rptr.release();
    p->rm_org.release();
    p->rm_run.release();
    p->rm_val.release();
    p->rm_runs = p->rm_vals = 0;
  }

  // ---- degridding: row pieces (COLUMNS) or one partial per (segment, warp) (TILE_MASK)
  if (p->fmt == WPROJ_INDEX_TILE_RUNS) {
    p->n_pieces = 0;
    p->piece_row.release();
    p->piece_lo.release();
    p->piece_len.release();
    p->row_piece_ptr.release();
    WPROJ_TRY(p->piece_partial.alloc(sizeof(float2)));
  } else if (p->fmt == WPROJ_INDEX_TILE_MASK) {
    p->n_pieces = 0;
    p->piece_row.release();
    p->piece_lo.release();
    p->piece_len.release();
    p->row_piece_ptr.release();
    WPROJ_TRY(p->piece_partial.alloc(sizeof(float2) * std::max<int64_t>(1, kStreamWarps * n_seg)));
  } else {
    WPROJ_TRY(make_row_pieces(m, p->row_ptr.as<int64_t>(), degrid_piece(p->nnz), p->piece_row, p->piece_lo,
                              p->piece_len, p->row_piece_ptr, &p->n_pieces, s));
    WPROJ_TRY(p->piece_partial.alloc(sizeof(float2) * std::max<int64_t>(1, p->n_pieces)));
  }

  // ---- gridding: chunks of one tile's segments (tile order), balanced by entries
  {
    const bool rec = p->fmt == WPROJ_INDEX_TILE_MASK || p->fmt == WPROJ_INDEX_TILE_RUNS;
    const int64_t chunk = grid_chunk(p->nnz);
    // the gridding's items in tile order: all segments, or the records of TILE_RUNS
    const int64_t n_items = p->fmt == WPROJ_INDEX_TILE_RUNS ? n_rec : n_seg;
    DevBuf cntsorted, cum;
    WPROJ_TRY(cntsorted.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_items)));
    WPROJ_TRY(cum.alloc(sizeof(int64_t) * std::max<int64_t>(1, n_items)));
    if (!rec) WPROJ_TRY(p->seg_meta.alloc(sizeof(SegMeta) * std::max<int64_t>(1, n_seg)));
    if (n_items > 0) {
      k_gather_cnt<<<ceil_div(n_items, 256), 256, 0, s>>>(n_items, tile_seg.as<int32_t>(), p->seg_cnt.as<int32_t>(),
                                                        p->seg_off.as<int64_t>(), p->seg_row.as<int32_t>(),
                                                        cntsorted.as<int32_t>(),
                                                        rec ? nullptr : p->seg_meta.as<SegMeta>());
      WPROJ_CHECK_LAUNCH("gather cnt");
      WPROJ_TRY(exclusive_scan_i32_to_i64(cntsorted.as<int32_t>(), cum.as<int64_t>(), n_items, s));
    }
    WPROJ_TRY(make_tile_chunks(n_tiles, tptr.as<int64_t>(), cum.as<int64_t>(), n_items, p->nnz, chunk, p->chunk_tile,
                               p->chunk_lo, p->chunk_hi, p->tile_chunk_ptr, &p->n_chunks, s));
    // column format: a cell-major copy for the gridding (packed rows need m <= 2^22)
    p->has_cells = false;
    p->tile_ent.release();
    p->cell_ent.release();
    p->cell_val.release();
    if (!rec && g.tile == 32 && m <= (int64_t(1) << 22)) {
      WPROJ_TRY(build_cells(p, tptr.as<int64_t>(), cum.as<int64_t>(), n_seg, s));
      p->has_cells = true;
    }
    WPROJ_TRY(p->grid_partial.alloc(sizeof(float2) * size_t(p->n_chunks) * g.tile * g.tile));
  }
  WPROJ_TRY(p->ytmp.alloc(sizeof(float2) * m));
  WPROJ_CUDA(cudaMemcpyAsync(&herr, d_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (herr & ERR_EMIT) return fail(WPROJ_ERR_CUDA, "build_kernels: emission pass disagrees with the counting pass");
  // first segment of every row, closed by n_seg (per-row reduction of segment partials)
  WPROJ_TRY(p->seg_base.alloc(sizeof(int64_t) * (m + 1)));
  WPROJ_CUDA(cudaMemcpy(p->seg_base.ptr, d_segbase.ptr, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice));
  WPROJ_CUDA(cudaMemcpy(p->seg_base.as<int64_t>() + m, &n_seg, sizeof(int64_t), cudaMemcpyHostToDevice));
  p->m = m;
  p->n_seg = n_seg;
  p->built = true;
  p->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return WPROJ_OK;
}

}  // namespace wproj
