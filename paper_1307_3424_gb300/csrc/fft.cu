// 2-D FFT passes of libwproj.
//
//  * Phi  (F Z A):   row pass over the N image rows with the zero-padding and
//    the KB correction 1/(a(l) a(m)) fused into the load, then a column pass
//    over all G columns that reads only the N non-zero rows.
//  * Phi^H (A Z^H F^H): column pass over the G columns that keeps only the N
//    image rows, then a row pass over those rows that keeps only the N image
//    columns, fused with the correction and Re(.) (or z - Re(.) for the
//    Douglas-Rachford dual step).
//  * The kernel build: batched S x S inverse transforms of the chirp times the
//    KB tap polynomial, with the chirp generated in the first pass's load.
#include "build.cuh"
#include "fft.cuh"
#include "plan.h"

namespace wproj {

namespace {

__global__ void k_twiddles(float2 *tw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 || i >= kTwiddleLen) return;
  const int l = 31 - __clz(i);
  const int n = 1 << l;
  const int k = i - n;
  double sn, cs;
  sincospi(-2.0 * double(k) / double(n), &sn, &cs);
  tw[i] = make_float2(float(cs), float(sn));
}

// padded index -> image index (or -1): offset p - N/2 sits at (p - N/2) mod G
__device__ __forceinline__ int pad_to_img(int P, int N, int G) {
  const int h = N >> 1;
  if (P < h) return P + h;
  if (P >= G - h) return P - G + h;
  return -1;
}
__device__ __forceinline__ int img_to_pad(int p, int N, int G) {
  const int h = N >> 1;
  return (p >= h) ? p - h : p - h + G;
}

// Block copy of TOT elements into shared memory, element idx from ld(idx) and
// stored by st(idx, v): all of a thread's loads are issued before its first
// store, so a thread keeps TOT / T loads in flight instead of one.
template <int TOT, int T, class LD, class ST>
__device__ __forceinline__ void staged_copy(LD ld, ST st) {
  constexpr int PER = (TOT + T - 1) / T;
  float2 r[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = int(threadIdx.x) + i * T;
    r[i] = (TOT % T == 0 || idx < TOT) ? ld(idx) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = int(threadIdx.x) + i * T;
    if (TOT % T == 0 || idx < TOT) st(idx, r[i]);
  }
}

// ---- Phi: F Z A --------------------------------------------------------------

// Each pass is a device body (block `blk` of one transform set) called by a
// kernel for one plan and by a kernel for a batch of same-size problems
// (blockIdx.y = problem of the size class, offsets from its BProb entry).
template <int LOGN>
__device__ __forceinline__ void phi_fwd_rows_body(const float *__restrict__ x, const float2 *__restrict__ xc,
                                                  const float *__restrict__ inv_a, int N,
                                                  float2 *__restrict__ inter, const float2 *__restrict__ tw,
                                                  int blk) {
  using Cfg = RowCfg<LOGN>;
  constexpr int G = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int p0 = blk * Cfg::C;
  staged_copy<Cfg::C * G, Cfg::T>(
      [&](int idx) {
        const int c = idx / G, Q = idx % G;
        const int p = p0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (p < N) {
          const int q = pad_to_img(Q, N, G);
          if (q >= 0) {
            const float s = inv_a[p] * inv_a[q];
            if (xc) v = cscale(xc[int64_t(p) * N + q], s);
            else v = make_float2(x[int64_t(p) * N + q] * s, 0.f);
          }
        }
        return v;
      },
      [&](int idx, float2 v) { sm[(idx / G) * Cfg::LD + idx % G] = v; });
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, -1>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * G; idx += Cfg::T) {
    const int c = idx / G, Q = idx % G;
    const int p = p0 + c;
    if (p < N) inter[int64_t(p) * G + Q] = sm[c * Cfg::LD + Q];
  }
}

template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::T)
k_phi_fwd_rows(const float *__restrict__ x, const float2 *__restrict__ xc, const float *__restrict__ inv_a, int N,
               float2 *__restrict__ inter, const float2 *__restrict__ tw) {
  phi_fwd_rows_body<LOGN>(x, xc, inv_a, N, inter, tw, blockIdx.x);
}

template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::T)
k_bphi_fwd_rows(const BProb *__restrict__ tab, const int32_t *__restrict__ plist, const float *__restrict__ x,
                const float *__restrict__ inv_a, float2 *__restrict__ inter, const float2 *__restrict__ tw) {
  const BProb P = tab[plist[blockIdx.y]];
  phi_fwd_rows_body<LOGN>(x + P.img_off, nullptr, inv_a + P.inva_off, P.N, inter + P.inter_off, tw, blockIdx.x);
}

template <int LOGN>
__device__ __forceinline__ void phi_fwd_cols_body(const float2 *__restrict__ inter, int N, float2 *__restrict__ Xt,
                                                  float scale, const float2 *__restrict__ tw, int blk) {
  using Cfg = ColCfg<LOGN>;
  constexpr int G = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int Q0 = blk * Cfg::C;
  staged_copy<Cfg::C * G, Cfg::T>(
      [&](int idx) {
        const int P = idx / Cfg::C, c = idx % Cfg::C;
        const int p = pad_to_img(P, N, G);
        return (p >= 0 && Q0 + c < G) ? inter[int64_t(p) * G + Q0 + c] : make_float2(0.f, 0.f);
      },
      [&](int idx, float2 v) { sm[(idx % Cfg::C) * Cfg::LD + idx / Cfg::C] = v; });
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, -1>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * G; idx += Cfg::T) {
    const int P = idx / Cfg::C, c = idx % Cfg::C;
    if (Q0 + c < G) Xt[int64_t(P) * G + Q0 + c] = cscale(sm[c * Cfg::LD + P], scale);
  }
}

template <int LOGN>
__global__ void __launch_bounds__(ColCfg<LOGN>::T)
k_phi_fwd_cols(const float2 *__restrict__ inter, int N, float2 *__restrict__ Xt, float scale,
               const float2 *__restrict__ tw) {
  phi_fwd_cols_body<LOGN>(inter, N, Xt, scale, tw, blockIdx.x);
}

template <int LOGN>
__global__ void __launch_bounds__(ColCfg<LOGN>::T)
k_bphi_fwd_cols(const BProb *__restrict__ tab, const int32_t *__restrict__ plist, const float2 *__restrict__ inter,
                float2 *__restrict__ Xt, const float2 *__restrict__ tw) {
  const BProb P = tab[plist[blockIdx.y]];
  phi_fwd_cols_body<LOGN>(inter + P.inter_off, P.N, Xt + P.grid_off, 1.0f / P.G, tw, blockIdx.x);
}

// ---- Phi^H: A Z^H F^H -----------------------------------------------------------

template <int LOGN>
__device__ __forceinline__ void phi_adj_cols_body(const float2 *__restrict__ Xt2, int N, float2 *__restrict__ inter,
                                                  const float2 *__restrict__ tw, int blk) {
  using Cfg = ColCfg<LOGN>;
  constexpr int G = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int Q0 = blk * Cfg::C;
  staged_copy<Cfg::C * G, Cfg::T>(
      [&](int idx) {
        const int P = idx / Cfg::C, c = idx % Cfg::C;
        return (Q0 + c < G) ? Xt2[int64_t(P) * G + Q0 + c] : make_float2(0.f, 0.f);
      },
      [&](int idx, float2 v) { sm[(idx % Cfg::C) * Cfg::LD + idx / Cfg::C] = v; });
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, +1>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * N; idx += Cfg::T) {
    const int p = idx / Cfg::C, c = idx % Cfg::C;
    if (Q0 + c < G) inter[int64_t(p) * G + Q0 + c] = sm[c * Cfg::LD + img_to_pad(p, N, G)];
  }
}

template <int LOGN>
__global__ void __launch_bounds__(ColCfg<LOGN>::T)
k_phi_adj_cols(const float2 *__restrict__ Xt2, int N, float2 *__restrict__ inter, const float2 *__restrict__ tw) {
  phi_adj_cols_body<LOGN>(Xt2, N, inter, tw, blockIdx.x);
}

template <int LOGN>
__global__ void __launch_bounds__(ColCfg<LOGN>::T)
k_bphi_adj_cols(const BProb *__restrict__ tab, const int32_t *__restrict__ plist, const float2 *__restrict__ Xt2,
                float2 *__restrict__ inter, const float2 *__restrict__ tw) {
  const BProb P = tab[plist[blockIdx.y]];
  phi_adj_cols_body<LOGN>(Xt2 + P.grid_off, P.N, inter + P.inter_off, tw, blockIdx.x);
}

// mode 0: x_re = Re(v) s (and x_c = v s when given); mode 1: x_re = z - Re(v) s
template <int LOGN>
__device__ __forceinline__ void phi_adj_rows_body(const float2 *__restrict__ inter, const float *__restrict__ inv_a,
                                                  int N, float scale, float *__restrict__ x_re,
                                                  float2 *__restrict__ x_c, const float *__restrict__ z, int mode,
                                                  const float2 *__restrict__ tw, int blk) {
  using Cfg = RowCfg<LOGN>;
  constexpr int G = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int p0 = blk * Cfg::C;
  staged_copy<Cfg::C * G, Cfg::T>(
      [&](int idx) {
        const int p = p0 + idx / G;
        return (p < N) ? inter[int64_t(p) * G + idx % G] : make_float2(0.f, 0.f);
      },
      [&](int idx, float2 v) { sm[(idx / G) * Cfg::LD + idx % G] = v; });
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, +1>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * N; idx += Cfg::T) {
    const int c = idx / N, q = idx % N;
    const int p = p0 + c;
    if (p >= N) continue;
    const float s = inv_a[p] * inv_a[q] * scale;
    const float2 v = sm[c * Cfg::LD + img_to_pad(q, N, G)];
    const int64_t o = int64_t(p) * N + q;
    if (mode == 0) {
      if (x_re) x_re[o] = v.x * s;
      if (x_c) x_c[o] = cscale(v, s);
    } else {
      x_re[o] = z[o] - v.x * s;
    }
  }
}

template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::T)
k_phi_adj_rows(const float2 *__restrict__ inter, const float *__restrict__ inv_a, int N, float scale,
               float *__restrict__ x_re, float2 *__restrict__ x_c, const float *__restrict__ z, int mode,
               const float2 *__restrict__ tw) {
  phi_adj_rows_body<LOGN>(inter, inv_a, N, scale, x_re, x_c, z, mode, tw, blockIdx.x);
}

template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::T)
k_bphi_adj_rows(const BProb *__restrict__ tab, const int32_t *__restrict__ plist, const float2 *__restrict__ inter,
                const float *__restrict__ inv_a, float *__restrict__ x_re, const float *__restrict__ z, int mode,
                const float2 *__restrict__ tw) {
  const BProb P = tab[plist[blockIdx.y]];
  phi_adj_rows_body<LOGN>(inter + P.inter_off, inv_a + P.inva_off, P.N, 1.0f / P.G, x_re + P.img_off, nullptr,
                          z ? z + P.img_off : nullptr, mode, tw, blockIdx.x);
}

// ---- generic batched 2-D FFT (rows then columns) --------------------------------

template <int LOGN, int DIR>
__global__ void __launch_bounds__(RowCfg<LOGN>::T)
k_fft_rows(const float2 *__restrict__ in, float2 *__restrict__ out, int64_t n_rows,
           const float2 *__restrict__ tw) {
  using Cfg = RowCfg<LOGN>;
  constexpr int N = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int64_t r0 = int64_t(blockIdx.x) * Cfg::C;
  staged_copy<Cfg::C * N, Cfg::T>(
      [&](int idx) {
        const int64_t r = r0 + idx / N;
        return (r < n_rows) ? in[r * N + idx % N] : make_float2(0.f, 0.f);
      },
      [&](int idx, float2 v) { sm[(idx / N) * Cfg::LD + idx % N] = v; });
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, DIR>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * N; idx += Cfg::T) {
    const int c = idx / N, i = idx % N;
    if (r0 + c < n_rows) out[(r0 + c) * N + i] = sm[c * Cfg::LD + i];
  }
}

// columns of `batch` N x N arrays, flattened as batch * N global columns
template <int LOGN, int DIR>
__global__ void __launch_bounds__(ColCfg<LOGN>::T)
k_fft_cols(const float2 *__restrict__ in, float2 *__restrict__ out, int64_t n_cols, float scale,
           const float2 *__restrict__ tw) {
  using Cfg = ColCfg<LOGN>;
  constexpr int N = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int64_t g0 = int64_t(blockIdx.x) * Cfg::C;
  staged_copy<Cfg::C * N, Cfg::T>(
      [&](int idx) {
        const int P = idx / Cfg::C;
        const int64_t gc = g0 + idx % Cfg::C;
        if (gc >= n_cols) return make_float2(0.f, 0.f);
        const int64_t b = gc >> LOGN, Q = gc & (N - 1);
        return in[(b * N + P) * N + Q];
      },
      [&](int idx, float2 v) { sm[(idx % Cfg::C) * Cfg::LD + idx / Cfg::C] = v; });
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, DIR>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * N; idx += Cfg::T) {
    const int P = idx / Cfg::C, c = idx % Cfg::C;
    const int64_t gc = g0 + c;
    if (gc < n_cols) {
      const int64_t b = gc >> LOGN, Q = gc & (N - 1);
      out[(b * N + P) * N + Q] = cscale(sm[c * Cfg::LD + P], scale);
    }
  }
}

// ---- kernel build: S x S boxes ---------------------------------------------------

// f[P][Q] = Au[P] Av[Q] e^{2 pi i w g(x)}: the chirp (Eq. 4 / Eq. 5) times the KB
// tap polynomial, at box offsets P' = P (P < S/2) or P - S; Au, Av carry the
// separable part of the phase, w (l^2 + m^2) / 2, and the taps.
__device__ __forceinline__ float2 box_value(const BoxBatch &bb, int b, int P, int Q) {
  const float2 a = bb.Au[int64_t(b) * bb.S + P];
  const float2 c = bb.Av[int64_t(b) * bb.S + Q];
  float2 f = cmul(a, c);
  const int mode = bb.mode[b];
  if (mode == 1) {
    // exact chirp: phase w (1 - n) = w x / 2 + w g(x), g = x^2 / (2 (1 + n)^2), the
    // remainder |w g| <= 1/4 cycle so FP32 keeps it to ~1e-7 cycles
    const float x = bb.lsq[P] + bb.lsq[Q];
    const float n = sqrtf(1.f - x);
    const float d = 1.f + n;
    const float g = (x * x) / (2.f * d * d);
    float sn, cs;
    sincospif(2.f * (bb.wf[b] * g), &sn, &cs);
    f = cmul(f, make_float2(cs, sn));
  } else if (mode == 2) {
    // large w: the full phase argument in FP64, reduced mod 1
    const double l = bb.lcoord[P], m = bb.lcoord[Q];
    const double x = l * l + m * m;
    const double ph = bb.wd[b] * x / (1.0 + sqrt(1.0 - x));
    const double fr = ph - floor(ph);
    float sn, cs;
    sincospif(2.f * float(fr), &sn, &cs);
    f = cmul(f, make_float2(cs, sn));
  }
  if (bb.screens) {
    const int S = bb.S, h = S / 2;
    const float2 a = bb.screens[(int64_t(bb.bsid[b]) * S + ((P + h) & (S - 1))) * S + ((Q + h) & (S - 1))];
    f = cmul(f, a);
  }
  return f;
}

template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::T)
k_box_rows(BoxBatch bb, const float2 *__restrict__ tw) {
  using Cfg = RowCfg<LOGN>;
  constexpr int S = 1 << LOGN;
  extern __shared__ float2 sm[];
  const int64_t n_rows = int64_t(bb.nb) * S;
  const int64_t r0 = int64_t(blockIdx.x) * Cfg::C;
  for (int idx = threadIdx.x; idx < Cfg::C * S; idx += Cfg::T) {
    const int c = idx / S, Q = idx % S;
    const int64_t r = r0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (r < n_rows) v = box_value(bb, int(r >> LOGN), int(r & (S - 1)), Q);
    sm[c * Cfg::LD + Q] = v;
  }
  __syncthreads();
  fft_block<LOGN, Cfg::C, Cfg::T, +1>(sm, Cfg::LD, tw);
  for (int idx = threadIdx.x; idx < Cfg::C * S; idx += Cfg::T) {
    const int c = idx / S, Q = idx % S;
    const int64_t r = r0 + c;
    if (r < n_rows) bb.K[r * S + Q] = sm[c * Cfg::LD + Q];
  }
}

// ---- separable kernel boxes (linear chirp, Eq. 5) ------------------------------------
// exp(pi i w (l^2 + m^2)) times the separable taps is an outer product Au x Av,
// so its 2-D inverse DFT is the outer product of two 1-D ones: K = (IDFT Au) x
// (IDFT Av) / S^2, two length-S transforms per box instead of an S x S one.
__global__ void k_box_outer(int nb, int S, const float2 *__restrict__ Au, const float2 *__restrict__ Av, float scale,
                            float2 *__restrict__ K) {
  const int64_t n = int64_t(nb) * S * S;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = i / (int64_t(S) * S);
    const int P = int((i / S) % S), Q = int(i % S);
    K[i] = cscale(cmul(Au[b * S + P], Av[b * S + Q]), scale);
  }
}

// ---- the paper's upsampling U (Section 2.2): spectral zero-padding -----------------
// F_G U x = P F_N x: the unitary spectrum of the image (pixel offset p - N/2 at
// index (p - N/2) mod N) placed on the G x G grid, frequency k in [-N/2, N/2)
// at index k mod G, zeros elsewhere.  Its adjoint crops and inverts.

__global__ void k_up_in(int N, const float *__restrict__ x, const float2 *__restrict__ xc, float2 *__restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(N) * N) return;
  const int p = int(i / N), q = int(i % N), h = N / 2;
  const float2 v = xc ? xc[i] : make_float2(x[i], 0.f);
  out[int64_t((p - h + N) % N) * N + (q - h + N) % N] = v;
}

__global__ void k_up_scatter(int N, int G, const float2 *__restrict__ spec, float scale, float2 *__restrict__ Xt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(G) * G) return;
  const int a = int(i / G), b = int(i % G), h = N / 2;
  const int ka = a < G / 2 ? a : a - G, kb = b < G / 2 ? b : b - G;
  float2 v = make_float2(0.f, 0.f);
  if (ka >= -h && ka < h && kb >= -h && kb < h) v = cscale(spec[int64_t((ka + N) % N) * N + (kb + N) % N], scale);
  Xt[i] = v;
}

__global__ void k_up_gather(int N, int G, const float2 *__restrict__ Xt2, float2 *__restrict__ spec) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(N) * N) return;
  const int a = int(i / N), b = int(i % N);
  const int ka = a < N / 2 ? a : a - N, kb = b < N / 2 ? b : b - N;
  spec[i] = Xt2[int64_t((ka + G) % G) * G + (kb + G) % G];
}

// mode 0: x_re = Re(v) (and x_c = v); mode 1: x_re = z - Re(v); v = scale * img
__global__ void k_up_out(int N, const float2 *__restrict__ img, float scale, float *__restrict__ x_re,
                         float2 *__restrict__ x_c, const float *__restrict__ z, int mode) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(N) * N) return;
  const int p = int(i / N), q = int(i % N), h = N / 2;
  const float2 v = cscale(img[int64_t((p - h + N) % N) * N + (q - h + N) % N], scale);
  if (mode == 0) {
    if (x_re) x_re[i] = v.x;
    if (x_c) x_c[i] = v;
  } else {
    x_re[i] = z[i] - v.x;
  }
}

// ---- dispatch ------------------------------------------------------------------

template <class K>
wproj_status set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) {
    WPROJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  return WPROJ_OK;
}

template <int LOGN>
wproj_status phi_fwd_impl(wproj_plan *p, const float *x, const float2 *xc, float2 *Xt, cudaStream_t s) {
  const int N = p->g.N, G = p->g.G;
  const float2 *tw = p->twiddle.as<float2>();
  float2 *inter = p->inter.as<float2>();
  {
    using Cfg = RowCfg<LOGN>;
    WPROJ_TRY(set_smem(k_phi_fwd_rows<LOGN>, Cfg::SMEM));
    k_phi_fwd_rows<LOGN><<<ceil_div(N, Cfg::C), Cfg::T, Cfg::SMEM, s>>>(x, xc, p->inv_a.as<float>(), N, inter, tw);
    WPROJ_CHECK_LAUNCH("phi fwd rows");
  }
  {
    using Cfg = ColCfg<LOGN>;
    WPROJ_TRY(set_smem(k_phi_fwd_cols<LOGN>, Cfg::SMEM));
    k_phi_fwd_cols<LOGN><<<ceil_div(G, Cfg::C), Cfg::T, Cfg::SMEM, s>>>(inter, N, Xt, 1.0f / G, tw);
    WPROJ_CHECK_LAUNCH("phi fwd cols");
  }
  return WPROJ_OK;
}

// The same two passes with a caller-provided intermediate buffer (N x G float2).
template <int LOGN>
wproj_status phi_fwd_into_impl(wproj_plan *p, const float *x, float2 *inter, float2 *Xt, cudaStream_t s) {
  const int N = p->g.N, G = p->g.G;
  const float2 *tw = p->twiddle.as<float2>();
  {
    using Cfg = RowCfg<LOGN>;
    WPROJ_TRY(set_smem(k_phi_fwd_rows<LOGN>, Cfg::SMEM));
    k_phi_fwd_rows<LOGN><<<ceil_div(N, Cfg::C), Cfg::T, Cfg::SMEM, s>>>(x, nullptr, p->inv_a.as<float>(), N, inter, tw);
    WPROJ_CHECK_LAUNCH("phi fwd rows");
  }
  {
    using Cfg = ColCfg<LOGN>;
    WPROJ_TRY(set_smem(k_phi_fwd_cols<LOGN>, Cfg::SMEM));
    k_phi_fwd_cols<LOGN><<<ceil_div(G, Cfg::C), Cfg::T, Cfg::SMEM, s>>>(inter, N, Xt, 1.0f / G, tw);
    WPROJ_CHECK_LAUNCH("phi fwd cols");
  }
  return WPROJ_OK;
}

template <int LOGN>
wproj_status phi_adj_impl(wproj_plan *p, const float2 *Xt2, float *x_re, float2 *x_c, const float *z,
                          int mode, cudaStream_t s) {
  const int N = p->g.N, G = p->g.G;
  const float2 *tw = p->twiddle.as<float2>();
  float2 *inter = p->inter.as<float2>();
  {
    using Cfg = ColCfg<LOGN>;
    WPROJ_TRY(set_smem(k_phi_adj_cols<LOGN>, Cfg::SMEM));
    k_phi_adj_cols<LOGN><<<ceil_div(G, Cfg::C), Cfg::T, Cfg::SMEM, s>>>(Xt2, N, inter, tw);
    WPROJ_CHECK_LAUNCH("phi adj cols");
  }
  {
    using Cfg = RowCfg<LOGN>;
    WPROJ_TRY(set_smem(k_phi_adj_rows<LOGN>, Cfg::SMEM));
    k_phi_adj_rows<LOGN><<<ceil_div(N, Cfg::C), Cfg::T, Cfg::SMEM, s>>>(
        inter, p->inv_a.as<float>(), N, 1.0f / G, x_re, x_c, z, mode, tw);
    WPROJ_CHECK_LAUNCH("phi adj rows");
  }
  return WPROJ_OK;
}

template <int LOGN>
wproj_status fft2d_impl(const float2 *in, float2 *out, int batch, int inverse, const float2 *tw,
                        cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  using RC = RowCfg<LOGN>;
  using CC = ColCfg<LOGN>;
  const int64_t rows = int64_t(batch) * N;
  if (inverse) {
    WPROJ_TRY(set_smem(k_fft_rows<LOGN, +1>, RC::SMEM));
    WPROJ_TRY(set_smem(k_fft_cols<LOGN, +1>, CC::SMEM));
    k_fft_rows<LOGN, +1><<<ceil_div(rows, RC::C), RC::T, RC::SMEM, s>>>(in, out, rows, tw);
    k_fft_cols<LOGN, +1><<<ceil_div(rows, CC::C), CC::T, CC::SMEM, s>>>(out, out, rows, 1.f, tw);
  } else {
    WPROJ_TRY(set_smem(k_fft_rows<LOGN, -1>, RC::SMEM));
    WPROJ_TRY(set_smem(k_fft_cols<LOGN, -1>, CC::SMEM));
    k_fft_rows<LOGN, -1><<<ceil_div(rows, RC::C), RC::T, RC::SMEM, s>>>(in, out, rows, tw);
    k_fft_cols<LOGN, -1><<<ceil_div(rows, CC::C), CC::T, CC::SMEM, s>>>(out, out, rows, 1.f, tw);
  }
  WPROJ_CHECK_LAUNCH("fft2d");
  return WPROJ_OK;
}

template <int LOGN>
wproj_status box_fft_impl(wproj_plan *p, const BoxBatch &bb, cudaStream_t s) {
  constexpr int S = 1 << LOGN;
  using RC = RowCfg<LOGN>;
  using CC = ColCfg<LOGN>;
  const float2 *tw = p->twiddle.as<float2>();
  const int64_t rows = int64_t(bb.nb) * S;
  WPROJ_TRY(set_smem(k_box_rows<LOGN>, RC::SMEM));
  WPROJ_TRY(set_smem(k_fft_cols<LOGN, +1>, CC::SMEM));
  k_box_rows<LOGN><<<ceil_div(rows, RC::C), RC::T, RC::SMEM, s>>>(bb, tw);
  WPROJ_CHECK_LAUNCH("box rows");
  k_fft_cols<LOGN, +1><<<ceil_div(rows, CC::C), CC::T, CC::SMEM, s>>>(
      bb.K, bb.K, rows, 1.0f / (float(S) * float(S)), tw);
  WPROJ_CHECK_LAUNCH("box cols");
  return WPROJ_OK;
}

#define WPROJ_LOGN_SWITCH(logn, CALL)                    \
  switch (logn) {                                         \
    case 4: return CALL(4);                               \
    case 5: return CALL(5);                               \
    case 6: return CALL(6);                               \
    case 7: return CALL(7);                               \
    case 8: return CALL(8);                               \
    case 9: return CALL(9);                               \
    case 10: return CALL(10);                             \
    case 11: return CALL(11);                             \
    case 12: return CALL(12);                             \
    default: return fail(WPROJ_ERR_UNSUPPORTED, "FFT size out of range"); \
  }

}  // namespace

// ---- batches: one launch per pass for all problems of a size class ---------------

template <int LOGN>
wproj_status bphi_fwd_impl(int np, const int32_t *plist, const BProb *tab, const float *x, const float *inv_a,
                           float2 *inter, float2 *Xt, const float2 *tw, cudaStream_t s) {
  constexpr int G = 1 << LOGN;
  const int N = G / 2;
  {
    using Cfg = RowCfg<LOGN>;
    WPROJ_TRY(set_smem(k_bphi_fwd_rows<LOGN>, Cfg::SMEM));
    k_bphi_fwd_rows<LOGN><<<dim3(ceil_div(N, Cfg::C), np), Cfg::T, Cfg::SMEM, s>>>(tab, plist, x, inv_a, inter, tw);
    WPROJ_CHECK_LAUNCH("batch phi fwd rows");
  }
  {
    using Cfg = ColCfg<LOGN>;
    WPROJ_TRY(set_smem(k_bphi_fwd_cols<LOGN>, Cfg::SMEM));
    k_bphi_fwd_cols<LOGN><<<dim3(ceil_div(G, Cfg::C), np), Cfg::T, Cfg::SMEM, s>>>(tab, plist, inter, Xt, tw);
    WPROJ_CHECK_LAUNCH("batch phi fwd cols");
  }
  return WPROJ_OK;
}

template <int LOGN>
wproj_status bphi_adj_impl(int np, const int32_t *plist, const BProb *tab, const float2 *Xt2, const float *inv_a,
                           float2 *inter, float *x_re, const float *z, int mode, const float2 *tw, cudaStream_t s) {
  constexpr int G = 1 << LOGN;
  const int N = G / 2;
  {
    using Cfg = ColCfg<LOGN>;
    WPROJ_TRY(set_smem(k_bphi_adj_cols<LOGN>, Cfg::SMEM));
    k_bphi_adj_cols<LOGN><<<dim3(ceil_div(G, Cfg::C), np), Cfg::T, Cfg::SMEM, s>>>(tab, plist, Xt2, inter, tw);
    WPROJ_CHECK_LAUNCH("batch phi adj cols");
  }
  {
    using Cfg = RowCfg<LOGN>;
    WPROJ_TRY(set_smem(k_bphi_adj_rows<LOGN>, Cfg::SMEM));
    k_bphi_adj_rows<LOGN><<<dim3(ceil_div(N, Cfg::C), np), Cfg::T, Cfg::SMEM, s>>>(tab, plist, inter, inv_a, x_re,
                                                                                 z, mode, tw);
    WPROJ_CHECK_LAUNCH("batch phi adj rows");
  }
  return WPROJ_OK;
}

// F U x into Xt (G x G); work: 2 N^2 complex
wproj_status up_forward(wproj_plan *p, const float *x, const float2 *xc, float2 *work, float2 *Xt, cudaStream_t s) {
  const int N = p->g.N, G = p->g.G;
  float2 *a = work, *b = work + int64_t(N) * N;
  k_up_in<<<ceil_div(int64_t(N) * N, 256), 256, 0, s>>>(N, x, xc, a);
  WPROJ_CHECK_LAUNCH("upsampling input");
  WPROJ_TRY(fft2d_generic(a, b, N, 1, 0, p->twiddle.as<float2>(), s));
  k_up_scatter<<<ceil_div(int64_t(G) * G, 256), 256, 0, s>>>(N, G, b, 1.0f / N, Xt);
  WPROJ_CHECK_LAUNCH("upsampling scatter");
  return WPROJ_OK;
}

// (F U)^H of Xt2 into the image; work: 2 N^2 complex
wproj_status up_adjoint(wproj_plan *p, const float2 *Xt2, float *x_re, float2 *x_c, const float *z, int mode,
                        float2 *work, cudaStream_t s) {
  const int N = p->g.N, G = p->g.G;
  float2 *a = work, *b = work + int64_t(N) * N;
  k_up_gather<<<ceil_div(int64_t(N) * N, 256), 256, 0, s>>>(N, G, Xt2, a);
  WPROJ_CHECK_LAUNCH("upsampling gather");
  WPROJ_TRY(fft2d_generic(a, b, N, 1, 1, p->twiddle.as<float2>(), s));
  k_up_out<<<ceil_div(int64_t(N) * N, 256), 256, 0, s>>>(N, b, 1.0f / N, x_re, x_c, z, mode);
  WPROJ_CHECK_LAUNCH("upsampling output");
  return WPROJ_OK;
}

wproj_status phi_forward_fft_into(wproj_plan *p, const float *x, float2 *inter, float2 *Xt, cudaStream_t s) {
  if (p->g.upsampling) return up_forward(p, x, nullptr, inter, Xt, s);
#define CALL(L) phi_fwd_into_impl<L>(p, x, inter, Xt, s)
  WPROJ_LOGN_SWITCH(ilog2(p->g.G), CALL)
#undef CALL
}

wproj_status make_twiddles(DevBuf &tw, cudaStream_t s) {
  WPROJ_TRY(tw.alloc(sizeof(float2) * kTwiddleLen));
  k_twiddles<<<kTwiddleLen / 256, 256, 0, s>>>(tw.as<float2>());
  WPROJ_CHECK_LAUNCH("twiddles");
  return WPROJ_OK;
}

wproj_status init_twiddles(wproj_plan *p, cudaStream_t s) { return make_twiddles(p->twiddle, s); }

wproj_status phi_forward_fft(wproj_plan *p, const float *x, const float2 *xc, float2 *Xt, cudaStream_t s) {
  ScopedTimer t(p, TC_FFT, s);
  if (p->g.upsampling) {
    p->launches += 4;
    return up_forward(p, x, xc, p->inter.as<float2>(), Xt, s);
  }
  p->launches += 2;
#define CALL(L) phi_fwd_impl<L>(p, x, xc, Xt, s)
  WPROJ_LOGN_SWITCH(ilog2(p->g.G), CALL)
#undef CALL
}

wproj_status phi_adjoint_fft(wproj_plan *p, const float2 *Xt2, float *x_re, float2 *x_cplx,
                             const float *z, int mode, cudaStream_t s) {
  ScopedTimer t(p, TC_FFT, s);
  if (p->g.upsampling) {
    p->launches += 4;
    return up_adjoint(p, Xt2, x_re, x_cplx, z, mode, p->inter.as<float2>(), s);
  }
  p->launches += 2;
#define CALL(L) phi_adj_impl<L>(p, Xt2, x_re, x_cplx, z, mode, s)
  WPROJ_LOGN_SWITCH(ilog2(p->g.G), CALL)
#undef CALL
}

wproj_status fft2d_generic(const float2 *in, float2 *out, int n, int batch, int inverse,
                           const float2 *tw, cudaStream_t s) {
#define CALL(L) fft2d_impl<L>(in, out, batch, inverse, tw, s)
  WPROJ_LOGN_SWITCH(ilog2(n), CALL)
#undef CALL
}

template <int LOGN>
wproj_status box_fft_separable_impl(wproj_plan *p, const BoxBatch &bb, cudaStream_t s) {
  constexpr int S = 1 << LOGN;
  using RC = RowCfg<LOGN>;
  const float2 *tw = p->twiddle.as<float2>();
  WPROJ_TRY(set_smem(k_fft_rows<LOGN, +1>, RC::SMEM));
  // the per-box tables are rebuilt for every batch, so they are transformed in place
  float2 *Au = const_cast<float2 *>(bb.Au), *Av = const_cast<float2 *>(bb.Av);
  k_fft_rows<LOGN, +1><<<ceil_div(bb.nb, RC::C), RC::T, RC::SMEM, s>>>(Au, Au, bb.nb, tw);
  k_fft_rows<LOGN, +1><<<ceil_div(bb.nb, RC::C), RC::T, RC::SMEM, s>>>(Av, Av, bb.nb, tw);
  const int64_t n = int64_t(bb.nb) * S * S;
  k_box_outer<<<(int)std::min<int64_t>(152 * 32, ceil_div(n, 256)), 256, 0, s>>>(bb.nb, S, Au, Av,
                                                                                1.0f / (float(S) * float(S)), bb.K);
  WPROJ_CHECK_LAUNCH("separable boxes");
  return WPROJ_OK;
}

wproj_status box_fft(wproj_plan *p, const BoxBatch &bb, cudaStream_t s) {
  if (p->g.chirp == WPROJ_CHIRP_LINEAR && !bb.screens) {   // every box is separable (mode 0)
#define CALL(L) box_fft_separable_impl<L>(p, bb, s)
    WPROJ_LOGN_SWITCH(ilog2(bb.S), CALL)
#undef CALL
  }
#define CALL(L) box_fft_impl<L>(p, bb, s)
  WPROJ_LOGN_SWITCH(ilog2(bb.S), CALL)
#undef CALL
}

wproj_status batch_phi_fwd(int logG, int np, const int32_t *plist, const BProb *tab, const float *x,
                           const float *inv_a, float2 *inter, float2 *Xt, const float2 *tw, cudaStream_t s) {
#define CALL(L) bphi_fwd_impl<L>(np, plist, tab, x, inv_a, inter, Xt, tw, s)
  WPROJ_LOGN_SWITCH(logG, CALL)
#undef CALL
}

wproj_status batch_phi_adj(int logG, int np, const int32_t *plist, const BProb *tab, const float2 *Xt2,
                           const float *inv_a, float2 *inter, float *x_re, const float *z, int mode,
                           const float2 *tw, cudaStream_t s) {
#define CALL(L) bphi_adj_impl<L>(np, plist, tab, Xt2, inv_a, inter, x_re, z, mode, tw, s)
  WPROJ_LOGN_SWITCH(logG, CALL)
#undef CALL
}

}  // namespace wproj
