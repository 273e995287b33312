// The Daubechies wavelet sparsity basis Psi of the BPDN problem (Eq. 7; the
// paper's second dictionary is Daubechies 8, Section 4): the periodic,
// orthonormal, separable 2-D transform in the Mallat layout.
//
// One dyadic level is one kernel: a CTA stages the input region of its output
// tile in shared memory (periodic wrap), filters the fast axis into two shared
// intermediates and the slow axis into the four sub-bands.  The image at this
// size lives in L2, so the levels are latency- rather than bandwidth-bound; the
// point of the fused level is one launch and one pass over global memory per
// level instead of one per axis.
//
// Conventions (one level on an even length n, h = n/2, i in [0, h)):
//   a_i = sum_k h_k x_{(2i + k) mod n},  d_i = sum_k g_k x_{(2i + k) mod n},
//   g_k = (-1)^k h_{2p-1-k}.
// The synthesis is the transpose: x_j = sum over k = j mod 2 of
//   h_k a_{((j - k)/2) mod h} + g_k d_{((j - k)/2) mod h}.
#include <complex>
#include <cmath>
#include <vector>

#include "plan.h"

namespace wproj {

constexpr int kMaxTaps = 2 * WPROJ_DAUB_MAX_P;
constexpr int kWT = 32;                       // analysis output tile (per sub-band); synthesis input tile
constexpr int kWThreads = 256;
constexpr int kWWarps = kWThreads / 32;

struct Taps {
  float h[kMaxTaps];
  float g[kMaxTaps];
  int len;
};

// ---- the taps: Daubechies' spectral factorisation, in double on the host ------

namespace {

using cd = std::complex<double>;

cd poly_eval(const std::vector<double> &c, cd z) {   // c[0] + c[1] z + ...
  cd v = 0;
  for (size_t i = c.size(); i-- > 0;) v = v * z + c[i];
  return v;
}

// all roots of c[0] + c[1] z + ... + c[d] z^d by the Weierstrass (Durand-Kerner)
// simultaneous iteration, then Newton steps on each root
std::vector<cd> poly_roots(const std::vector<double> &c) {
  const int d = int(c.size()) - 1;
  std::vector<cd> r(d);
  if (d <= 0) return r;
  const double lead = c[d];
  // start on a circle of the Cauchy bound, at angles that avoid symmetry
  double bound = 0;
  for (int i = 0; i < d; ++i) bound = std::max(bound, std::abs(c[i] / lead));
  bound = 1.0 + bound;
  for (int i = 0; i < d; ++i) r[i] = std::polar(0.5 * bound, 2.0 * M_PI * i / d + 0.4);
  for (int it = 0; it < 2000; ++it) {
    double change = 0;
    for (int i = 0; i < d; ++i) {
      cd den = lead;
      for (int j = 0; j < d; ++j)
        if (j != i) den *= (r[i] - r[j]);
      const cd step = poly_eval(c, r[i]) / den;
      r[i] -= step;
      change = std::max(change, std::abs(step) / std::max(1.0, std::abs(r[i])));
    }
    if (change < 1e-16) break;
  }
  std::vector<double> dc(d);
  for (int i = 1; i <= d; ++i) dc[i - 1] = i * c[i];
  for (int i = 0; i < d; ++i)
    for (int it = 0; it < 3; ++it) {
      const cd f = poly_eval(c, r[i]), fp = poly_eval(dc, r[i]);
      if (std::abs(fp) == 0) break;
      r[i] -= f / fp;
    }
  return r;
}

}  // namespace

// Low-pass taps of the extremal-phase Daubechies wavelet with p vanishing
// moments: |H|^2 = cos^{2p}(w/2) P_p(sin^2(w/2)), P_p(y) = sum_{k<p} C(p-1+k, k) y^k;
// every root y_k of P_p contributes the root of z^2 - (2 - 4 y_k) z + 1 inside the
// unit circle; H(z) = (1 + z)^p prod (z - z_k), scaled to sum sqrt(2), in the
// order whose partial energies are front-loaded.
wproj_status daubechies_taps_impl(int p, double *h_out) {
  if (p < 1 || p > WPROJ_DAUB_MAX_P) return fail(WPROJ_ERR_INVALID_ARG, "Daubechies order out of range");
  std::vector<double> P(p);
  double binom = 1.0;                           // C(p-1+k, k)
  for (int k = 0; k < p; ++k) {
    P[k] = binom;
    binom = binom * double(p + k) / double(k + 1);
  }
  const std::vector<cd> yk = poly_roots(P);
  std::vector<cd> poly(1, cd(1.0));             // coefficient of z^i at index i
  auto mul_linear = [&](cd root) {              // poly *= (z - root)
    std::vector<cd> out(poly.size() + 1, cd(0));
    for (size_t i = 0; i < poly.size(); ++i) {
      out[i + 1] += poly[i];
      out[i] -= root * poly[i];
    }
    poly.swap(out);
  };
  for (int i = 0; i < p; ++i) mul_linear(cd(-1.0));
  for (const cd &y : yk) {
    const cd b = 2.0 - 4.0 * y;
    const cd disc = std::sqrt(b * b - 4.0);
    const cd z1 = 0.5 * (b + disc), z2 = 0.5 * (b - disc);
    mul_linear(std::abs(z1) < 1.0 ? z1 : z2);
  }
  const int L = 2 * p;
  std::vector<double> h(L);
  double sum = 0;
  for (int i = 0; i < L; ++i) {
    h[i] = poly[i].real();
    sum += h[i];
  }
  for (int i = 0; i < L; ++i) h[i] *= std::sqrt(2.0) / sum;
  double ef = 0, er = 0, cf = 0, cr = 0;
  for (int i = 0; i < L; ++i) {
    cf += h[i] * h[i];
    cr += h[L - 1 - i] * h[L - 1 - i];
    ef += cf;
    er += cr;
  }
  for (int i = 0; i < L; ++i) h_out[i] = er > ef ? h[L - 1 - i] : h[i];
  return WPROJ_OK;
}

namespace {

Taps make_taps(const double *h, int L) {
  Taps t{};
  t.len = L;
  for (int k = 0; k < L; ++k) {
    t.h[k] = float(h[k]);
    t.g[k] = float(((k & 1) ? -1.0 : 1.0) * h[L - 1 - k]);
  }
  return t;
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// global -> shared copy of one float without a register round trip, so that all
// of a CTA's staging copies are in flight together
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// i in [0, 2n) when n >= the staged span (one subtraction), else a full wrap
__device__ __forceinline__ int wrap_up(int i, int n, bool big) {
  if (big) return i >= n ? i - n : i;
  return i % n;
}

// One analysis level: src (n x n, row stride lds) -> the four sub-bands; the
// low-low band to ll (row stride ldl), the three others into the Mallat blocks of
// coef (row stride ldc).  A CTA makes a 32 x 32 tile of each band from the
// (64 + L - 2)^2 input region, wrapped periodically.  Each filtering task keeps
// the inputs of 8 consecutive outputs in registers (two shared-memory loads per
// output instead of L), the tap count L = 2p a compile-time constant.
template <int L>
__device__ __forceinline__ void dwt_level_body(const float *__restrict__ src, int lds, int n, const Taps &t,
                                               float *__restrict__ ll, int ldl, float *__restrict__ coef, int ldc) {
  constexpr int span = 2 * kWT + L - 2;
  constexpr int SEG = 8, NW = 2 * SEG + L - 2;      // outputs per task, inputs per task
  __shared__ float in[span][span + 1];
  __shared__ float lo[span][kWT + 1], hi[span][kWT + 1];
  const int h = n / 2;
  const int i0 = blockIdx.y * kWT, c0 = blockIdx.x * kWT;
  const bool big = n >= span;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float hk[L], gk[L];
#pragma unroll
  for (int k = 0; k < L; ++k) { hk[k] = t.h[k]; gk[k] = t.g[k]; }
  for (int r = wid; r < span; r += kWWarps) {
    const float *row = src + int64_t(wrap_up(2 * i0 + r, n, big)) * lds;
    for (int c = lane; c < span; c += 32) cp_async4(&in[r][c], row + wrap_up(2 * c0 + c, n, big));
  }
  cp_async_wait_all();
  __syncthreads();
  for (int task = threadIdx.x; task < span * (kWT / SEG); task += kWThreads) {   // fast axis
    const int r = task / (kWT / SEG), q = task % (kWT / SEG);
    float v[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) v[j] = in[r][2 * SEG * q + j];
#pragma unroll
    for (int o = 0; o < SEG; ++o) {
      float a = 0.f, d = 0.f;
#pragma unroll
      for (int k = 0; k < L; ++k) {
        a = fmaf(hk[k], v[2 * o + k], a);
        d = fmaf(gk[k], v[2 * o + k], d);
      }
      lo[r][SEG * q + o] = a;
      hi[r][SEG * q + o] = d;
    }
  }
  __syncthreads();
  {                                                  // slow axis: one task per thread
    const int c = threadIdx.x & 31, sel = (threadIdx.x >> 5) & 1, q = threadIdx.x >> 6;
    float v[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) v[j] = sel ? hi[2 * SEG * q + j][c] : lo[2 * SEG * q + j][c];
    const int gc = c0 + c;
#pragma unroll
    for (int o = 0; o < SEG; ++o) {
      float a = 0.f, d = 0.f;
#pragma unroll
      for (int k = 0; k < L; ++k) {
        a = fmaf(hk[k], v[2 * o + k], a);
        d = fmaf(gk[k], v[2 * o + k], d);
      }
      const int gi = i0 + SEG * q + o;
      if (gi < h && gc < h) {
        if (sel == 0) {
          ll[int64_t(gi) * ldl + gc] = a;                  // low slow, low fast
          coef[int64_t(h + gi) * ldc + gc] = d;            // high slow, low fast
        } else {
          coef[int64_t(gi) * ldc + h + gc] = a;            // low slow, high fast
          coef[int64_t(h + gi) * ldc + h + gc] = d;        // high slow, high fast
        }
      }
    }
  }
}

// One synthesis level: the low-low band ll (row stride ldl) and the three other
// bands of coef (row stride ldc) -> dst (n x n, row stride ldd).  A CTA makes a
// 64 x 64 output tile from (32 + L/2 - 1)^2 samples of each band; each task keeps
// the band samples of 16 consecutive outputs in registers.
template <int L>
__device__ __forceinline__ void idwt_level_body(const float *__restrict__ ll, int ldl, const float *__restrict__ coef,
                                                int ldc, int n, const Taps &t, float *__restrict__ dst, int ldd) {
  constexpr int off = L / 2 - 1;                   // staged index = band index - (j0/2 - off)
  constexpr int span = kWT + off;
  constexpr int SEG = 16, NW = SEG / 2 + off;      // outputs per task, band samples per task
  __shared__ float sb[4][span][span + 1];
  __shared__ float lo[span][2 * kWT + 1], hi[span][2 * kWT + 1];
  const int h = n / 2;
  const int j10 = blockIdx.y * 2 * kWT, j20 = blockIdx.x * 2 * kWT;
  const int b1 = j10 / 2 - off, b2 = j20 / 2 - off;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float hk[L], gk[L];
#pragma unroll
  for (int k = 0; k < L; ++k) { hk[k] = t.h[k]; gk[k] = t.g[k]; }
  for (int r = wid; r < span; r += kWWarps) {
    const int gi = wrap(b1 + r, h);
    const float *lrow = ll + int64_t(gi) * ldl;
    const float *crow = coef + int64_t(gi) * ldc, *crow2 = coef + int64_t(h + gi) * ldc;
    for (int c = lane; c < span; c += 32) {
      const int gc = wrap(b2 + c, h);
      cp_async4(&sb[0][r][c], lrow + gc);
      cp_async4(&sb[1][r][c], crow + h + gc);
      cp_async4(&sb[2][r][c], crow2 + gc);
      cp_async4(&sb[3][r][c], crow2 + h + gc);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // fast axis: task (band row r, pair: 0 = (LL, LH) -> lo, 1 = (HL, HH) -> hi, segment q)
  for (int task = threadIdx.x; task < span * 2 * (2 * kWT / SEG); task += kWThreads) {
    const int q = task % (2 * kWT / SEG), pr = (task / (2 * kWT / SEG)) & 1, r = task / (4 * kWT / SEG);
    float a[NW], d[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      a[j] = sb[2 * pr][r][SEG / 2 * q + j];
      d[j] = sb[2 * pr + 1][r][SEG / 2 * q + j];
    }
    float *outr = pr ? hi[r] : lo[r];
#pragma unroll
    for (int o = 0; o < SEG; ++o) {
      float x = 0.f;
#pragma unroll
      for (int k = o & 1; k < L; k += 2) {
        const int idx = (o - k) / 2 + off;            // compile-time after unrolling
        x = fmaf(hk[k], a[idx], fmaf(gk[k], d[idx], x));
      }
      outr[SEG * q + o] = x;
    }
  }
  __syncthreads();
  {                                                  // slow axis: task (column jj, segment q)
    const int jj = threadIdx.x & (2 * kWT - 1), q = threadIdx.x / (2 * kWT);
    float a[NW], d[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      a[j] = lo[SEG / 2 * q + j][jj];
      d[j] = hi[SEG / 2 * q + j][jj];
    }
    const int g2 = j20 + jj;
#pragma unroll
    for (int o = 0; o < SEG; ++o) {
      float x = 0.f;
#pragma unroll
      for (int k = o & 1; k < L; k += 2) {
        const int idx = (o - k) / 2 + off;
        x = fmaf(hk[k], a[idx], fmaf(gk[k], d[idx], x));
      }
      const int g1 = j10 + SEG * q + o;
      if (g1 < n && g2 < n) dst[int64_t(g1) * ldd + g2] = x;
    }
  }
}

template <int L>
__global__ void __launch_bounds__(kWThreads)
k_dwt_level(const float *__restrict__ src, int lds, int n, const Taps t, float *__restrict__ ll, int ldl,
            float *__restrict__ coef, int ldc) {
  dwt_level_body<L>(src, lds, n, t, ll, ldl, coef, ldc);
}

template <int L>
__global__ void __launch_bounds__(kWThreads)
k_idwt_level(const float *__restrict__ ll, int ldl, const float *__restrict__ coef, int ldc, int n, const Taps t,
             float *__restrict__ dst, int ldd) {
  idwt_level_body<L>(ll, ldl, coef, ldc, n, t, dst, ldd);
}

// Batches: level lv of every problem (blockIdx.z) at once.  Problem p's image
// sits at img_off in x / alpha, its two ping-pong low-low bands (N^2 / 4 floats
// each) at img_off / 2 in work; the grid is sized for the largest problem and
// the other problems' surplus tiles return at once.
template <int L>
__global__ void __launch_bounds__(kWThreads)
k_bdwt_level(const BProb *__restrict__ tab, int lv, int levels, const float *__restrict__ x,
             float *__restrict__ alpha, float *__restrict__ work, const Taps t) {
  const BProb P = tab[blockIdx.z];
  const int N = P.N, n = N >> lv, h = n / 2;
  if (int(blockIdx.x) * kWT >= h || int(blockIdx.y) * kWT >= h) return;
  float *a = alpha + P.img_off;
  float *ping0 = work + P.img_off / 2, *ping1 = ping0 + int64_t(N) * N / 4;
  const float *src = lv == 0 ? x + P.img_off : (((lv - 1) & 1) ? ping1 : ping0);
  const int lds = lv == 0 ? N : n;
  const bool last = lv == levels - 1;
  dwt_level_body<L>(src, lds, n, t, last ? a : ((lv & 1) ? ping1 : ping0), last ? N : h, a, N);
}

template <int L>
__global__ void __launch_bounds__(kWThreads)
k_bidwt_level(const BProb *__restrict__ tab, int lv, int levels, const float *__restrict__ alpha,
              float *__restrict__ x, float *__restrict__ work, const Taps t) {
  const BProb P = tab[blockIdx.z];
  const int N = P.N, n = N >> lv;
  if (int(blockIdx.x) * 2 * kWT >= n || int(blockIdx.y) * 2 * kWT >= n) return;
  const float *a = alpha + P.img_off;
  float *ping0 = work + P.img_off / 2, *ping1 = ping0 + int64_t(N) * N / 4;
  const bool deepest = lv == levels - 1;
  const float *ll = deepest ? a : (((lv + 1) & 1) ? ping1 : ping0);
  const int ldl = deepest ? N : n / 2;
  float *dst = lv == 0 ? x + P.img_off : ((lv & 1) ? ping1 : ping0);
  idwt_level_body<L>(ll, ldl, a, N, n, t, dst, lv == 0 ? N : n);
}

wproj_status check_psi(int N, int levels, int p) {
  if (p < 1 || p > WPROJ_DAUB_MAX_P) return fail(WPROJ_ERR_INVALID_ARG, "Daubechies order out of range");
  if (N < 2 || levels < 1 || levels > 30 || N % (1 << levels) != 0)
    return fail(WPROJ_ERR_INVALID_ARG, "n must be divisible by 2^levels");
  return WPROJ_OK;
}

}  // namespace

// alpha = Psi^T x.  work: N*N/2 floats (two ping-pong low-low bands).
wproj_status dwt2_impl(int N, int levels, int p, const float *x, float *alpha, float *work, int64_t *launches,
                       cudaStream_t s) {
  WPROJ_TRY(check_psi(N, levels, p));
  double hd[kMaxTaps];
  WPROJ_TRY(daubechies_taps_impl(p, hd));
  const Taps t = make_taps(hd, 2 * p);
  float *ping[2] = {work, work + int64_t(N) * N / 4};
  const float *src = x;
  int lds = N, n = N;
  for (int lv = 0; lv < levels; ++lv) {
    const int h = n / 2;
    const bool last = lv == levels - 1;
    float *ll = last ? alpha : ping[lv & 1];
    const int ldl = last ? N : h;
    const dim3 grid(ceil_div(h, kWT), ceil_div(h, kWT));
    switch (t.len) {
#define DWT_CASE(L) \
  case L: k_dwt_level<L><<<grid, kWThreads, 0, s>>>(src, lds, n, t, ll, ldl, alpha, N); break;
      DWT_CASE(2) DWT_CASE(4) DWT_CASE(6) DWT_CASE(8) DWT_CASE(10)
      DWT_CASE(12) DWT_CASE(14) DWT_CASE(16) DWT_CASE(18) DWT_CASE(20)
#undef DWT_CASE
      default: return fail(WPROJ_ERR_INVALID_ARG, "Daubechies order out of range");
    }
    WPROJ_CHECK_LAUNCH("wavelet analysis level");
    src = ll;
    lds = ldl;
    n = h;
  }
  if (launches) *launches += levels;
  return WPROJ_OK;
}

// x = Psi alpha.  work: N*N/2 floats.
wproj_status idwt2_impl(int N, int levels, int p, const float *alpha, float *x, float *work, int64_t *launches,
                        cudaStream_t s) {
  WPROJ_TRY(check_psi(N, levels, p));
  double hd[kMaxTaps];
  WPROJ_TRY(daubechies_taps_impl(p, hd));
  const Taps t = make_taps(hd, 2 * p);
  float *ping[2] = {work, work + int64_t(N) * N / 4};
  const float *ll = alpha;
  int ldl = N;
  int n = N >> (levels - 1);
  for (int lv = levels - 1; lv >= 0; --lv) {
    const bool last = lv == 0;
    float *dst = last ? x : ping[lv & 1];
    const int ldd = last ? N : n;
    const dim3 grid(ceil_div(n, 2 * kWT), ceil_div(n, 2 * kWT));
    switch (t.len) {
#define IDWT_CASE(L) \
  case L: k_idwt_level<L><<<grid, kWThreads, 0, s>>>(ll, ldl, alpha, N, n, t, dst, ldd); break;
      IDWT_CASE(2) IDWT_CASE(4) IDWT_CASE(6) IDWT_CASE(8) IDWT_CASE(10)
      IDWT_CASE(12) IDWT_CASE(14) IDWT_CASE(16) IDWT_CASE(18) IDWT_CASE(20)
#undef IDWT_CASE
      default: return fail(WPROJ_ERR_INVALID_ARG, "Daubechies order out of range");
    }
    WPROJ_CHECK_LAUNCH("wavelet synthesis level");
    ll = dst;
    ldl = ldd;
    n *= 2;
  }
  if (launches) *launches += levels;
  return WPROJ_OK;
}

// Batched transforms: every problem's image (tab[np] on the device, sides up to
// maxN) through `levels` levels; work holds sum N^2 / 2 floats.
wproj_status batch_dwt2(const BProb *tab, int np, int maxN, int levels, int p, const float *x, float *alpha,
                        float *work, int64_t *launches, cudaStream_t s) {
  WPROJ_TRY(check_psi(maxN, levels, p));
  double hd[kMaxTaps];
  WPROJ_TRY(daubechies_taps_impl(p, hd));
  const Taps t = make_taps(hd, 2 * p);
  for (int lv = 0; lv < levels; ++lv) {
    const int h = (maxN >> lv) / 2;
    const dim3 grid(ceil_div(h, kWT), ceil_div(h, kWT), np);
    switch (t.len) {
#define BDWT_CASE(L) \
  case L: k_bdwt_level<L><<<grid, kWThreads, 0, s>>>(tab, lv, levels, x, alpha, work, t); break;
      BDWT_CASE(2) BDWT_CASE(4) BDWT_CASE(6) BDWT_CASE(8) BDWT_CASE(10)
      BDWT_CASE(12) BDWT_CASE(14) BDWT_CASE(16) BDWT_CASE(18) BDWT_CASE(20)
#undef BDWT_CASE
      default: return fail(WPROJ_ERR_INVALID_ARG, "Daubechies order out of range");
    }
    WPROJ_CHECK_LAUNCH("batch wavelet analysis level");
  }
  if (launches) *launches += levels;
  return WPROJ_OK;
}

wproj_status batch_idwt2(const BProb *tab, int np, int maxN, int levels, int p, const float *alpha, float *x,
                         float *work, int64_t *launches, cudaStream_t s) {
  WPROJ_TRY(check_psi(maxN, levels, p));
  double hd[kMaxTaps];
  WPROJ_TRY(daubechies_taps_impl(p, hd));
  const Taps t = make_taps(hd, 2 * p);
  for (int lv = levels - 1; lv >= 0; --lv) {
    const int n = maxN >> lv;
    const dim3 grid(ceil_div(n, 2 * kWT), ceil_div(n, 2 * kWT), np);
    switch (t.len) {
#define BIDWT_CASE(L) \
  case L: k_bidwt_level<L><<<grid, kWThreads, 0, s>>>(tab, lv, levels, alpha, x, work, t); break;
      BIDWT_CASE(2) BIDWT_CASE(4) BIDWT_CASE(6) BIDWT_CASE(8) BIDWT_CASE(10)
      BIDWT_CASE(12) BIDWT_CASE(14) BIDWT_CASE(16) BIDWT_CASE(18) BIDWT_CASE(20)
#undef BIDWT_CASE
      default: return fail(WPROJ_ERR_INVALID_ARG, "Daubechies order out of range");
    }
    WPROJ_CHECK_LAUNCH("batch wavelet synthesis level");
  }
  if (launches) *launches += levels;
  return WPROJ_OK;
}

}  // namespace wproj

using namespace wproj;

extern "C" {

wproj_status wproj_daubechies_taps(int32_t p, double *h_out) {
  if (!h_out) return fail(WPROJ_ERR_INVALID_ARG, "null output");
  return daubechies_taps_impl(p, h_out);
}

wproj_status wproj_dwt2(int32_t n, int32_t levels, int32_t p, const float *x, float *alpha, float *work,
                        void *stream) {
  if (!x || !alpha || !work) return fail(WPROJ_ERR_INVALID_ARG, "null pointer");
  if (x == alpha) return fail(WPROJ_ERR_INVALID_ARG, "x and alpha must not alias");
  return dwt2_impl(n, levels, p, x, alpha, work, nullptr, static_cast<cudaStream_t>(stream));
}

wproj_status wproj_idwt2(int32_t n, int32_t levels, int32_t p, const float *alpha, float *x, float *work,
                         void *stream) {
  if (!x || !alpha || !work) return fail(WPROJ_ERR_INVALID_ARG, "null pointer");
  if (x == alpha) return fail(WPROJ_ERR_INVALID_ARG, "x and alpha must not alias");
  return idwt2_impl(n, levels, p, alpha, x, work, nullptr, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
