// The learned-kernel network: an MLP that maps (w, sub-grid offset) to a
// visibility's w-kernel on a fixed 32 x 32 window of grid cells around its cell
// (2048 values: real and imaginary parts) plus a support mask (1024 logits).
// It is trained on kernels from the plain FFT-and-threshold build (Part I), which
// stays the reference and the fallback.
//
//   x0 = (w_c / 2 - 1, 2 du - 1, 2 dv - 1)                     w_c in grid cells
//   h1 = GELU(W1 x0 + b1)   h2 = GELU(W2 h1 + b2)   h3 = GELU(W3 h2 + b3)   (256 each)
//   y  = W4 h3 + b4                                                     (3072)
//   loss = mean_v (y_v - t_v)^2 + mask_weight * mean_m BCE(y_m, t_m)
//
// Layers 2-4 and all their gradients are BF16 GEMMs on the tcgen05 tensor cores
// (gemm.cu) with FP32 accumulation; the 3-wide first layer runs on the FP32
// cores.  Master parameters, Adam moments and all reductions are FP32 (bias
// gradients and losses are summed in a fixed order).  Activations and the
// gradients fed to GEMMs are rounded to BF16.  GELU is the erf form.
#include <math.h>

#include <chrono>
#include <new>
#include <vector>

#include "plan.h"

namespace wproj {
namespace mlpk {
constexpr int kIn = 3, kH = 256, kOutV = 2048, kOutM = 1024, kOut = kOutV + kOutM, kWin = 32;
constexpr int64_t oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
                  oB3 = oW3 + kH * kH, oW4 = oB3 + kH, oB4 = oW4 + int64_t(kOut) * kH, kParams = oB4 + kOut;
}  // namespace mlpk
}  // namespace wproj

struct wproj_mlp {
  wproj::DevBuf P, Mo, Ve, Gr;          // FP32 parameters, Adam moments, gradients (flat)
  wproj::DevBuf W2b, W3b, W4b;          // BF16 copies [out x in]
  wproj::DevBuf W2t, W3t, W4t;          // BF16 transposes [in x out]
  int64_t step = 0;
  int64_t cap = 0;                      // batch capacity of the activation buffers
  wproj::DevBuf Z1, Z2, Z3, H1, H2, H3, Y, dY, dYt, Ht, dZt, dH, dZ, dZ1, part, err;
  wproj::DevBuf csum;                   // column-sum partials and the first layer's sums
  int64_t csum_off = 0;
};

namespace wproj {

namespace {

using namespace mlpk;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// first layer on the FP32 cores: Z1 = x0 W1^T + b1, H1 = GELU(Z1)
__global__ void k_in_fwd(int64_t B, const float *__restrict__ x0, const float *__restrict__ P, float *__restrict__ Z1,
                         __nv_bfloat16 *__restrict__ H1) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= B * kH) return;
  const int64_t b = i / kH;
  const int j = int(i % kH);
  const float *W1 = P + oW1 + j * kIn;
  const float z = P[oB1 + j] + W1[0] * x0[b * 3] + W1[1] * x0[b * 3 + 1] + W1[2] * x0[b * 3 + 2];
  Z1[i] = z;
  H1[i] = __float2bfloat16_rn(gelu(z));
}

__global__ void k_gelu_fwd(int64_t n, const float *__restrict__ Z, __nv_bfloat16 *__restrict__ H) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    H[i] = __float2bfloat16_rn(gelu(Z[i]));
}

// loss partials and dY = d loss / d y (BF16); rows [0, B)
__global__ void __launch_bounds__(256)
k_loss(int64_t B, const float *__restrict__ Y, const float *__restrict__ Tv, const float *__restrict__ Tm,
       float mask_weight, __nv_bfloat16 *__restrict__ dY, double *__restrict__ part) {
  const float sv = 2.f / float(B * kOutV), sm = mask_weight / float(B * kOutM);
  double acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < B * kOut; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = i / kOut;
    const int j = int(i % kOut);
    const float y = Y[i];
    float g;
    if (j < kOutV) {
      const float d = y - Tv[b * kOutV + j];
      acc += double(d) * d / double(B * kOutV);
      g = sv * d;
    } else {
      const float t = Tm[b * kOutM + (j - kOutV)];
      // BCE with logits: max(y, 0) - t y + log(1 + e^{-|y|})
      acc += double(mask_weight) * (fmaxf(y, 0.f) - t * y + log1pf(__expf(-fabsf(y)))) / double(B * kOutM);
      g = sm * (1.f / (1.f + __expf(-y)) - t);
    }
    dY[i] = __float2bfloat16_rn(g);
  }
  const double t = block_sum_d<256>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_part_d(const double *__restrict__ part, int n, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// out[c][r] = in[r][c], R x C BF16
__global__ void k_transpose(int64_t R, int64_t C, const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int64_t r0 = int64_t(blockIdx.y) * 32, c0 = int64_t(blockIdx.x) * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y)
    if (r0 + i < R && c0 + threadIdx.x < C) t[i][threadIdx.x] = in[(r0 + i) * C + c0 + threadIdx.x];
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y)
    if (c0 + i < C && r0 + threadIdx.x < R) out[(c0 + i) * R + r0 + threadIdx.x] = t[threadIdx.x][i];
}

// Column sums in two passes with a fixed order: block (32 columns x 8 row
// groups) over rows [1024 y, 1024 (y + 1)) -> part[y][NV][col]; then k_sum_chunks.
// NV = 1: sum_r in[r][j]; NV = 4 (first layer): sum_r in[r][j] (x0[r][0..2], 1).
constexpr int kChunkRows = 1024;
template <class T, int NV>
__global__ void __launch_bounds__(256)
k_colsum_part(int64_t R, int C, const T *__restrict__ in, const float *__restrict__ x0, float *__restrict__ part) {
  __shared__ float red[8][NV][32];
  const int j = blockIdx.x * 32 + threadIdx.x, g = threadIdx.y;
  const int64_t r0 = int64_t(blockIdx.y) * kChunkRows;
  const int64_t r1 = r0 + kChunkRows < R ? r0 + kChunkRows : R;
  float acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.f;
  if (j < C) {
    for (int64_t r = r0 + g; r < r1; r += 8) {
      const float d = float(in[r * C + j]);
      if constexpr (NV == 1) {
        acc[0] += d;
      } else {
        acc[0] += d * x0[r * 3];
        acc[1] += d * x0[r * 3 + 1];
        acc[2] += d * x0[r * 3 + 2];
        acc[3] += d;
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) red[g][v][threadIdx.x] = acc[v];
  __syncthreads();
  if (g == 0 && j < C) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float t = 0.f;
      for (int q = 0; q < 8; ++q) t += red[q][v][threadIdx.x];
      part[(int64_t(blockIdx.y) * NV + v) * C + j] = t;
    }
  }
}

// out[v][j] = sum over chunks of part[chunk][v][j], chunks in order
__global__ void k_sum_chunks(int nchunk, int nv, int C, const float *__restrict__ part, float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv * C) return;
  float t = 0.f;
  for (int c = 0; c < nchunk; ++c) t += part[int64_t(c) * nv * C + i];
  out[i] = t;
}

// dZ = dH * GELU'(Z) as BF16 (next GEMM) and, when dZf is given, FP32
__global__ void k_gelu_bwd(int64_t n, const float *__restrict__ dH, const float *__restrict__ Z,
                           __nv_bfloat16 *__restrict__ dZ, float *__restrict__ dZf) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float g = dH[i] * gelu_d(Z[i]);
    if (dZ) dZ[i] = __float2bfloat16_rn(g);
    if (dZf) dZf[i] = g;
  }
}

// first layer gradients from out[v][j] of the 4-way column sums
__global__ void k_in_grad(const float *__restrict__ s4, float *__restrict__ G) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kH) return;
  G[oW1 + j * kIn] = s4[j];
  G[oW1 + j * kIn + 1] = s4[kH + j];
  G[oW1 + j * kIn + 2] = s4[2 * kH + j];
  G[oB1 + j] = s4[3 * kH + j];
}

__global__ void k_adam(int64_t n, float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                       float *__restrict__ V, float lr, float c1, float c2) {
  constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ in, __nv_bfloat16 *__restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>(152 * 16, std::max<int64_t>(1, ceil_div(n, 256))); }

// column sums of an R x C matrix (NV = 1), or the first layer's four (NV = 4)
template <class T, int NV>
wproj_status colsum(int64_t R, int C, const T *in, const float *x0, float *scratch, float *out, cudaStream_t s) {
  const int nchunk = ceil_div(R, kChunkRows);
  k_colsum_part<T, NV><<<dim3(ceil_div(C, 32), nchunk), dim3(32, 8), 0, s>>>(R, C, in, x0, scratch);
  k_sum_chunks<<<ceil_div(NV * C, 256), 256, 0, s>>>(nchunk, NV, C, scratch, out);
  WPROJ_CHECK_LAUNCH("column sums");
  return WPROJ_OK;
}

wproj_status transpose(int64_t R, int64_t C, const __nv_bfloat16 *in, __nv_bfloat16 *out, cudaStream_t s) {
  k_transpose<<<dim3(ceil_div(C, 32), ceil_div(R, 32)), dim3(32, 8), 0, s>>>(R, C, in, out);
  WPROJ_CHECK_LAUNCH("transpose");
  return WPROJ_OK;
}

// BF16 copies and transposes of W2..W4 from the master parameters
wproj_status refresh_weights(wproj_mlp *n, cudaStream_t s) {
  const float *P = n->P.as<float>();
  k_to_bf16<<<blocks_for(kH * kH), 256, 0, s>>>(kH * kH, P + oW2, n->W2b.as<__nv_bfloat16>());
  k_to_bf16<<<blocks_for(kH * kH), 256, 0, s>>>(kH * kH, P + oW3, n->W3b.as<__nv_bfloat16>());
  k_to_bf16<<<blocks_for(int64_t(kOut) * kH), 256, 0, s>>>(int64_t(kOut) * kH, P + oW4, n->W4b.as<__nv_bfloat16>());
  WPROJ_CHECK_LAUNCH("weights to bf16");
  WPROJ_TRY(transpose(kH, kH, n->W2b.as<__nv_bfloat16>(), n->W2t.as<__nv_bfloat16>(), s));
  WPROJ_TRY(transpose(kH, kH, n->W3b.as<__nv_bfloat16>(), n->W3t.as<__nv_bfloat16>(), s));
  WPROJ_TRY(transpose(kOut, kH, n->W4b.as<__nv_bfloat16>(), n->W4t.as<__nv_bfloat16>(), s));
  return WPROJ_OK;
}

wproj_status ensure_batch(wproj_mlp *n, int64_t B) {
  if (n->cap >= B) return WPROJ_OK;
  WPROJ_TRY(n->Z1.alloc(sizeof(float) * B * kH));
  WPROJ_TRY(n->Z2.alloc(sizeof(float) * B * kH));
  WPROJ_TRY(n->Z3.alloc(sizeof(float) * B * kH));
  WPROJ_TRY(n->H1.alloc(2 * B * kH));
  WPROJ_TRY(n->H2.alloc(2 * B * kH));
  WPROJ_TRY(n->H3.alloc(2 * B * kH));
  WPROJ_TRY(n->Y.alloc(sizeof(float) * B * kOut));
  WPROJ_TRY(n->dY.alloc(2 * B * kOut));
  WPROJ_TRY(n->dYt.alloc(2 * B * kOut));
  WPROJ_TRY(n->Ht.alloc(2 * B * kH));
  WPROJ_TRY(n->dZt.alloc(2 * B * kH));
  WPROJ_TRY(n->dH.alloc(sizeof(float) * B * kH));
  WPROJ_TRY(n->dZ.alloc(2 * B * kH));
  WPROJ_TRY(n->dZ1.alloc(sizeof(float) * B * kH));
  // column-sum partials: up to ceil(B / 1024) chunks x max(3072, 4 x 256) columns, then 4 x 256 results
  n->csum_off = int64_t(ceil_div(B, kChunkRows)) * kOut;
  WPROJ_TRY(n->csum.alloc(sizeof(float) * (n->csum_off + 4 * kH)));
  n->cap = B;
  return WPROJ_OK;
}

wproj_status gemm(int M, int N, int K, const void *A, const void *B, const float *bias, void *C, wproj_mlp *n,
                  cudaStream_t s) {
  return gemm_bf16_tn(M, N, K, static_cast<const __nv_bfloat16 *>(A), static_cast<const __nv_bfloat16 *>(B), bias,
                      C, false, n->err.as<int>(), s);
}

// forward of B rows (B a multiple of 128) into n->Y
wproj_status forward(wproj_mlp *n, const float *x0, int64_t B, float *Y, cudaStream_t s) {
  const float *P = n->P.as<float>();
  k_in_fwd<<<ceil_div(B * kH, 256), 256, 0, s>>>(B, x0, P, n->Z1.as<float>(), n->H1.as<__nv_bfloat16>());
  WPROJ_CHECK_LAUNCH("mlp layer 1");
  WPROJ_TRY(gemm((int)B, kH, kH, n->H1.ptr, n->W2b.ptr, P + oB2, n->Z2.ptr, n, s));
  k_gelu_fwd<<<blocks_for(B * kH), 256, 0, s>>>(B * kH, n->Z2.as<float>(), n->H2.as<__nv_bfloat16>());
  WPROJ_TRY(gemm((int)B, kH, kH, n->H2.ptr, n->W3b.ptr, P + oB3, n->Z3.ptr, n, s));
  k_gelu_fwd<<<blocks_for(B * kH), 256, 0, s>>>(B * kH, n->Z3.as<float>(), n->H3.as<__nv_bfloat16>());
  WPROJ_CHECK_LAUNCH("mlp gelu");
  return gemm((int)B, kOut, kH, n->H3.ptr, n->W4b.ptr, P + oB4, Y, n, s);
}

// loss (device double at *loss_d) and gradients into n->Gr for B rows
wproj_status backward(wproj_mlp *n, const float *x0, const float *Tv, const float *Tm, int64_t B, float mask_weight,
                      double *loss_d, cudaStream_t s) {
  float *G = n->Gr.as<float>();
  const float *Z[3] = {n->Z1.as<float>(), n->Z2.as<float>(), n->Z3.as<float>()};
  const __nv_bfloat16 *H[3] = {n->H1.as<__nv_bfloat16>(), n->H2.as<__nv_bfloat16>(), n->H3.as<__nv_bfloat16>()};
  const int nb = blocks_for(B * kOut);
  k_loss<<<nb, 256, 0, s>>>(B, n->Y.as<float>(), Tv, Tm, mask_weight, n->dY.as<__nv_bfloat16>(), n->part.as<double>());
  k_sum_part_d<<<1, 32, 0, s>>>(n->part.as<double>(), nb, loss_d);
  WPROJ_CHECK_LAUNCH("mlp loss");
  // layer 4
  WPROJ_TRY(transpose(B, kOut, n->dY.as<__nv_bfloat16>(), n->dYt.as<__nv_bfloat16>(), s));
  WPROJ_TRY(transpose(B, kH, H[2], n->Ht.as<__nv_bfloat16>(), s));
  WPROJ_TRY(gemm(kOut, kH, (int)B, n->dYt.ptr, n->Ht.ptr, nullptr, G + oW4, n, s));
  WPROJ_TRY((colsum<__nv_bfloat16, 1>(B, kOut, n->dY.as<__nv_bfloat16>(), nullptr, n->csum.as<float>(), G + oB4, s)));
  WPROJ_TRY(gemm((int)B, kH, kOut, n->dY.ptr, n->W4t.ptr, nullptr, n->dH.ptr, n, s));
  // layers 3 and 2
  const __nv_bfloat16 *Wt[2] = {n->W3t.as<__nv_bfloat16>(), n->W2t.as<__nv_bfloat16>()};
  const int64_t oW[2] = {oW3, oW2}, oB[2] = {oB3, oB2};
  for (int l = 0; l < 2; ++l) {
    const int zi = 2 - l;   // Z3 then Z2
    k_gelu_bwd<<<blocks_for(B * kH), 256, 0, s>>>(B * kH, n->dH.as<float>(), Z[zi], n->dZ.as<__nv_bfloat16>(), nullptr);
    WPROJ_CHECK_LAUNCH("mlp gelu backward");
    WPROJ_TRY(transpose(B, kH, n->dZ.as<__nv_bfloat16>(), n->dZt.as<__nv_bfloat16>(), s));
    WPROJ_TRY(transpose(B, kH, H[zi - 1], n->Ht.as<__nv_bfloat16>(), s));
    WPROJ_TRY(gemm(kH, kH, (int)B, n->dZt.ptr, n->Ht.ptr, nullptr, G + oW[l], n, s));
    WPROJ_TRY((colsum<__nv_bfloat16, 1>(B, kH, n->dZ.as<__nv_bfloat16>(), nullptr, n->csum.as<float>(), G + oB[l], s)));
    WPROJ_TRY(gemm((int)B, kH, kH, n->dZ.ptr, Wt[l], nullptr, n->dH.ptr, n, s));
  }
  // layer 1
  k_gelu_bwd<<<blocks_for(B * kH), 256, 0, s>>>(B * kH, n->dH.as<float>(), Z[0], nullptr, n->dZ1.as<float>());
  WPROJ_TRY((colsum<float, 4>(B, kH, n->dZ1.as<float>(), x0, n->csum.as<float>(), n->csum.as<float>() + n->csum_off, s)));
  k_in_grad<<<1, kH, 0, s>>>(n->csum.as<float>() + n->csum_off, G);
  WPROJ_CHECK_LAUNCH("mlp layer 1 backward");
  return WPROJ_OK;
}

wproj_status check_err(wproj_mlp *n, cudaStream_t s) {
  int h = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&h, n->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(WPROJ_ERR_TIMEOUT, "mlp: a tensor-core wait ran out");
  return WPROJ_OK;
}

// Training targets from a built plan: window cell (a, b) <-> grid cell
// (j0 - 16 + a, j0 - 16 + b) mod G; values scaled by 1 / sqrt(E_kb), E_kb =
// prod_axes sum_t kb(delta - t)^2 over the W taps.
__global__ void k_targets(int64_t m, const double *__restrict__ uvw, const int64_t *__restrict__ row_ptr,
                          const int32_t *__restrict__ col, const float2 *__restrict__ val, int G, double du,
                          double L, int W, double beta, float *__restrict__ x0, float *__restrict__ Tv,
                          float *__restrict__ Tm) {
  const int64_t k = blockIdx.x;
  if (k >= m) return;
  const double gu = uvw[3 * k] / du, gv = uvw[3 * k + 1] / du;
  const double fu = floor(gu), fv = floor(gv);
  const int ju = int(fu), jv = int(fv);
  const double dlu = gu - fu, dlv = gv - fv;
  for (int i = threadIdx.x; i < kOutV; i += blockDim.x) Tv[k * kOutV + i] = 0.f;
  for (int i = threadIdx.x; i < kOutM; i += blockDim.x) Tm[k * kOutM + i] = 0.f;
  double eu = 0, ev = 0;
  for (int t = -W / 2 + 1; t <= W / 2; ++t) {
    const double a = kb_dev(dlu - t, W, beta), b = kb_dev(dlv - t, W, beta);
    eu += a * a;
    ev += b * b;
  }
  const float inv = float(1.0 / sqrt(eu * ev));
  if (threadIdx.x == 0) {
    const double wc = fabs(uvw[3 * k + 2]) * L * L / 2.0;   // h = |w| L^2 = 2 w_c
    x0[k * 3] = float(wc / 2.0 - 1.0);
    x0[k * 3 + 1] = float(2.0 * dlu - 1.0);
    x0[k * 3 + 2] = float(2.0 * dlv - 1.0);
  }
  __syncthreads();
  const int ou = ((ju - kWin / 2) % G + G) % G, ov = ((jv - kWin / 2) % G + G) % G;
  for (int64_t i = row_ptr[k] + threadIdx.x; i < row_ptr[k + 1]; i += blockDim.x) {
    const int q = col[i];
    const int a = ((q / G - ou) % G + G) % G, b = ((q % G - ov) % G + G) % G;
    if (a < kWin && b < kWin) {
      const float2 v = val[i];
      Tv[k * kOutV + 2 * (a * kWin + b)] = v.x * inv;
      Tv[k * kOutV + 2 * (a * kWin + b) + 1] = v.y * inv;
      Tm[k * kOutM + a * kWin + b] = 1.f;
    }
  }
}

// Network input of every row (the x0 of k_targets).
__global__ void k_features(int64_t m, const double *__restrict__ uvw, double du, double L, float *__restrict__ x0) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const double gu = uvw[3 * k] / du, gv = uvw[3 * k + 1] / du;
  const double wc = fabs(uvw[3 * k + 2]) * L * L / 2.0;
  x0[k * 3] = float(wc / 2.0 - 1.0);
  x0[k * 3 + 1] = float(2.0 * (gu - floor(gu)) - 1.0);
  x0[k * 3 + 2] = float(2.0 * (gv - floor(gv)) - 1.0);
}

// Judge the predicted kernels of rows [r0, r0 + nr) against the plain ones and
// take the predicted values where they pass: rel. L2 over the window <= relmax,
// the predicted support holding >= e of the kernel energy (measured on the
// plain kernel), and no plain entry outside the window.  Block per row.
__global__ void __launch_bounds__(256)
k_judge(int64_t r0, const double *__restrict__ uvw, const int64_t *__restrict__ row_ptr,
        const int32_t *__restrict__ col, float2 *__restrict__ val, const float *__restrict__ Y, int G, double du,
        int W, double beta, double e, double relmax, float *__restrict__ row_err, int8_t *__restrict__ pass) {
  __shared__ float2 T[kWin * kWin];
  __shared__ int outside;
  const int64_t k = r0 + blockIdx.x;
  const float *y = Y + int64_t(blockIdx.x) * kOut;
  const double gu = uvw[3 * k] / du, gv = uvw[3 * k + 1] / du;
  const double fu = floor(gu), fv = floor(gv);
  const double dlu = gu - fu, dlv = gv - fv;
  double eu = 0, ev = 0;
  for (int t = -W / 2 + 1; t <= W / 2; ++t) {
    const double a = kb_dev(dlu - t, W, beta), b = kb_dev(dlv - t, W, beta);
    eu += a * a;
    ev += b * b;
  }
  const double ekb = eu * ev;
  const float sc = float(sqrt(ekb));
  for (int i = threadIdx.x; i < kWin * kWin; i += blockDim.x) T[i] = make_float2(0.f, 0.f);
  if (threadIdx.x == 0) outside = 0;
  __syncthreads();
  const int ou = ((int(fu) - kWin / 2) % G + G) % G, ov = ((int(fv) - kWin / 2) % G + G) % G;
  const int64_t lo = row_ptr[k], hi = row_ptr[k + 1];
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int q = col[i];
    const int a = ((q / G - ou) % G + G) % G, b = ((q % G - ov) % G + G) % G;
    if (a < kWin && b < kWin) T[a * kWin + b] = val[i];
    else outside = 1;
  }
  __syncthreads();
  double d2 = 0, t2 = 0, sup = 0;
  for (int i = threadIdx.x; i < kWin * kWin; i += blockDim.x) {
    const float2 t = T[i];
    const float px = y[2 * i] * sc, py = y[2 * i + 1] * sc;
    d2 += double(px - t.x) * (px - t.x) + double(py - t.y) * (py - t.y);
    const double tt = double(t.x) * t.x + double(t.y) * t.y;
    t2 += tt;
    if (y[kOutV + i] > 0.f) sup += tt;
  }
  d2 = block_sum_d<256>(d2);
  t2 = block_sum_d<256>(t2);
  sup = block_sum_d<256>(sup);
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const double r = t2 > 0 ? sqrt(d2 / t2) : 1.0;
    ok = (!outside && r <= relmax && sup >= e * ekb) ? 1 : 0;
    if (row_err) row_err[k] = float(r);
    pass[k] = int8_t(ok);
  }
  __syncthreads();
  if (!ok) return;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int q = col[i];
    const int a = ((q / G - ou) % G + G) % G, b = ((q % G - ov) % G + G) % G;
    const int c = a * kWin + b;
    val[i] = make_float2(y[2 * c] * sc, y[2 * c + 1] * sc);
  }
}

__global__ void k_count_pass(int64_t m, const int8_t *__restrict__ pass, const float *__restrict__ err,
                             unsigned long long *__restrict__ n, double *__restrict__ esum) {
  __shared__ double es[256];
  __shared__ unsigned long long ns[256];
  double a = 0;
  unsigned long long c = 0;
  for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
    c += pass[k];
    a += err[k];
  }
  es[threadIdx.x] = a;
  ns[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    unsigned long long u = 0;
    for (int i = 0; i < 256; ++i) { t += es[i]; u += ns[i]; }
    *n = u;
    *esum = t;
  }
}

}  // namespace

int64_t mlp_num_params() { return kParams; }

wproj_status build_learned_impl(wproj_plan *p, wproj_mlp *n, const double *uvw, int64_t m, double e, double relmax,
                                float *row_err, wproj_learned_info *info, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  WPROJ_TRY(build_kernels_impl(p, uvw, m, e, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  if (p->fmt != WPROJ_INDEX_COLUMNS || p->g.value_dtype != WPROJ_VAL_F32)
    return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels_learned: needs complex64 values and column indices");
  const int64_t chunk = 65536;
  DevBuf x0, Y, err, pass, cnt;
  WPROJ_TRY(x0.alloc(sizeof(float) * 3 * (m + 128)));
  WPROJ_TRY(Y.alloc(sizeof(float) * chunk * kOut));
  WPROJ_TRY(pass.alloc(m));
  WPROJ_TRY(cnt.alloc(sizeof(double) * 2));
  float *err_p = row_err;
  if (!err_p) {
    WPROJ_TRY(err.alloc(sizeof(float) * m));
    err_p = err.as<float>();
  }
  WPROJ_CUDA(cudaMemsetAsync(x0.ptr, 0, sizeof(float) * 3 * (m + 128), s));
  k_features<<<ceil_div(m, 256), 256, 0, s>>>(m, uvw, p->g.du, p->g.L, x0.as<float>());
  WPROJ_CHECK_LAUNCH("mlp features");
  WPROJ_TRY(ensure_batch(n, chunk));
  for (int64_t r = 0; r < m; r += chunk) {
    const int64_t nr = std::min(chunk, m - r);
    const int64_t B = (nr + 127) / 128 * 128;   // padded rows read zero features
    WPROJ_TRY(forward(n, x0.as<float>() + 3 * r, B, Y.as<float>(), s));
    k_judge<<<(unsigned)nr, 256, 0, s>>>(r, uvw, p->row_ptr.as<int64_t>(), p->col.as<int32_t>(), p->val.as<float2>(),
                                         Y.as<float>(), p->g.G, p->g.du, p->g.W, p->g.beta, e, relmax, err_p,
                                         pass.as<int8_t>());
    WPROJ_CHECK_LAUNCH("mlp judge");
  }
  WPROJ_TRY(check_err(n, s));
  WPROJ_TRY(rebuild_cells(p, s));
  k_count_pass<<<1, 256, 0, s>>>(m, pass.as<int8_t>(), err_p, cnt.as<unsigned long long>(), cnt.as<double>() + 1);
  WPROJ_CHECK_LAUNCH("mlp pass count");
  unsigned long long np_ = 0;
  double es = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&np_, cnt.ptr, sizeof(np_), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&es, cnt.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  auto t2 = std::chrono::steady_clock::now();
  p->dr_valid = false;
  if (info) {
    info->rows = m;
    info->learned = int64_t(np_);
    info->rel_l2_mean = es / double(m);
    info->plain_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->learned_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
  }
  return WPROJ_OK;
}

wproj_status mlp_create(wproj_mlp *n) {
  WPROJ_TRY(n->P.alloc(sizeof(float) * kParams));
  WPROJ_TRY(n->Mo.alloc(sizeof(float) * kParams));
  WPROJ_TRY(n->Ve.alloc(sizeof(float) * kParams));
  WPROJ_TRY(n->Gr.alloc(sizeof(float) * kParams));
  WPROJ_TRY(n->W2b.alloc(2 * kH * kH));
  WPROJ_TRY(n->W3b.alloc(2 * kH * kH));
  WPROJ_TRY(n->W4b.alloc(2 * int64_t(kOut) * kH));
  WPROJ_TRY(n->W2t.alloc(2 * kH * kH));
  WPROJ_TRY(n->W3t.alloc(2 * kH * kH));
  WPROJ_TRY(n->W4t.alloc(2 * int64_t(kOut) * kH));
  WPROJ_TRY(n->part.alloc(sizeof(double) * (152 * 16 + 8)));
  WPROJ_TRY(n->err.alloc(sizeof(int)));
  WPROJ_CUDA(cudaMemset(n->P.ptr, 0, sizeof(float) * kParams));
  WPROJ_CUDA(cudaMemset(n->Mo.ptr, 0, sizeof(float) * kParams));
  WPROJ_CUDA(cudaMemset(n->Ve.ptr, 0, sizeof(float) * kParams));
  WPROJ_CUDA(cudaMemset(n->err.ptr, 0, sizeof(int)));
  return WPROJ_OK;
}

wproj_status mlp_set_params(wproj_mlp *n, const float *p, cudaStream_t s) {
  WPROJ_CUDA(cudaMemcpyAsync(n->P.ptr, p, sizeof(float) * kParams, cudaMemcpyDefault, s));
  WPROJ_CUDA(cudaMemsetAsync(n->Mo.ptr, 0, sizeof(float) * kParams, s));
  WPROJ_CUDA(cudaMemsetAsync(n->Ve.ptr, 0, sizeof(float) * kParams, s));
  n->step = 0;
  WPROJ_TRY(refresh_weights(n, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  return WPROJ_OK;
}

wproj_status mlp_get_params(const wproj_mlp *n, float *p, cudaStream_t s) {
  WPROJ_CUDA(cudaMemcpyAsync(p, n->P.ptr, sizeof(float) * kParams, cudaMemcpyDefault, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  return WPROJ_OK;
}

wproj_status mlp_forward(wproj_mlp *n, const float *x0, int64_t m, float *y, int64_t chunk, cudaStream_t s) {
  WPROJ_TRY(ensure_batch(n, chunk));
  for (int64_t r = 0; r < m; r += chunk) {
    const int64_t B = std::min<int64_t>(chunk, m - r);
    WPROJ_TRY(forward(n, x0 + 3 * r, B, y + r * kOut, s));
  }
  return check_err(n, s);
}

wproj_status mlp_gradients(wproj_mlp *n, const float *x0, const float *Tv, const float *Tm, int64_t B,
                           double mask_weight, double *loss, float *grad, cudaStream_t s) {
  WPROJ_TRY(ensure_batch(n, B));
  WPROJ_TRY(forward(n, x0, B, n->Y.as<float>(), s));
  WPROJ_TRY(backward(n, x0, Tv, Tm, B, float(mask_weight), n->part.as<double>() + 152 * 16, s));
  WPROJ_CUDA(cudaMemcpyAsync(loss, n->part.as<double>() + 152 * 16, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad) WPROJ_CUDA(cudaMemcpyAsync(grad, n->Gr.ptr, sizeof(float) * kParams, cudaMemcpyDefault, s));
  return check_err(n, s);
}

wproj_status mlp_train(wproj_mlp *n, const float *x0, const float *Tv, const float *Tm, int64_t m, int B, int steps,
                       double lr, double mask_weight, float *losses, cudaStream_t s) {
  WPROJ_TRY(ensure_batch(n, B));
  std::vector<double> hl(steps);
  DevBuf dl;
  WPROJ_TRY(dl.alloc(sizeof(double) * std::max(1, steps)));
  const int64_t nbatch = m / B;
  for (int it = 0; it < steps; ++it) {
    const int64_t r = (it % nbatch) * B;
    WPROJ_TRY(forward(n, x0 + 3 * r, B, n->Y.as<float>(), s));
    WPROJ_TRY(backward(n, x0 + 3 * r, Tv + r * kOutV, Tm + r * kOutM, B, float(mask_weight), dl.as<double>() + it, s));
    n->step += 1;
    const float c1 = 1.f - powf(0.9f, float(n->step)), c2 = 1.f - powf(0.999f, float(n->step));
    k_adam<<<blocks_for(kParams), 256, 0, s>>>(kParams, n->P.as<float>(), n->Gr.as<float>(), n->Mo.as<float>(),
                                               n->Ve.as<float>(), float(lr), c1, c2);
    WPROJ_CHECK_LAUNCH("adam");
    WPROJ_TRY(refresh_weights(n, s));
  }
  WPROJ_CUDA(cudaMemcpyAsync(hl.data(), dl.ptr, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
  WPROJ_TRY(check_err(n, s));
  if (losses)
    for (int i = 0; i < steps; ++i) losses[i] = float(hl[i]);
  return WPROJ_OK;
}

wproj_status mlp_targets(const wproj_plan *p, const double *uvw, float *x0, float *Tv, float *Tm, cudaStream_t s) {
  if (p->fmt != WPROJ_INDEX_COLUMNS || p->g.value_dtype != WPROJ_VAL_F32)
    return fail(WPROJ_ERR_UNSUPPORTED, "mlp_targets: needs a complex64 plan with column indices");
  k_targets<<<(unsigned)p->m, 128, 0, s>>>(p->m, uvw, p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
                                           p->val.as<float2>(), p->g.G, p->g.du, p->g.L, p->g.W, p->g.beta, x0, Tv,
                                           Tm);
  WPROJ_CHECK_LAUNCH("mlp targets");
  return WPROJ_OK;
}

}  // namespace wproj

// ---- C-ABI ------------------------------------------------------------------------

using namespace wproj;

extern "C" {

int64_t wproj_mlp_num_params(void) { return mlp_num_params(); }

wproj_status wproj_mlp_create(wproj_mlp **out) {
  if (!out) return fail(WPROJ_ERR_INVALID_ARG, "mlp_create: null out");
  *out = nullptr;
  auto *n = new (std::nothrow) wproj_mlp();
  if (!n) return fail(WPROJ_ERR_OOM, "mlp_create: host allocation");
  wproj_status st = mlp_create(n);
  if (st != WPROJ_OK) {
    delete n;
    return st;
  }
  *out = n;
  return WPROJ_OK;
}

wproj_status wproj_mlp_destroy(wproj_mlp *n) {
  delete n;
  return WPROJ_OK;
}

wproj_status wproj_mlp_set_params(wproj_mlp *n, const float *params, void *stream) {
  if (!n || !params) return fail(WPROJ_ERR_INVALID_ARG, "mlp_set_params: null argument");
  return mlp_set_params(n, params, static_cast<cudaStream_t>(stream));
}

wproj_status wproj_mlp_get_params(const wproj_mlp *n, float *params, void *stream) {
  if (!n || !params) return fail(WPROJ_ERR_INVALID_ARG, "mlp_get_params: null argument");
  return mlp_get_params(n, params, static_cast<cudaStream_t>(stream));
}

wproj_status wproj_mlp_targets(const wproj_plan *p, const double *uvw, float *x0, float *tval, float *tmask,
                               void *stream) {
  if (!p || !p->built) return fail(WPROJ_ERR_NOT_BUILT, "mlp_targets: build the plan first");
  if (!uvw || !x0 || !tval || !tmask) return fail(WPROJ_ERR_INVALID_ARG, "mlp_targets: null argument");
  return mlp_targets(p, uvw, x0, tval, tmask, static_cast<cudaStream_t>(stream));
}

wproj_status wproj_mlp_forward(wproj_mlp *n, const float *x0, int64_t m, float *y, void *stream) {
  if (!n || !x0 || !y) return fail(WPROJ_ERR_INVALID_ARG, "mlp_forward: null argument");
  if (m < 128 || m % 128) return fail(WPROJ_ERR_INVALID_ARG, "mlp_forward: m must be a positive multiple of 128");
  return mlp_forward(n, x0, m, y, std::min<int64_t>(m, 65536), static_cast<cudaStream_t>(stream));
}

wproj_status wproj_mlp_gradients(wproj_mlp *n, const float *x0, const float *tval, const float *tmask, int64_t m,
                                 double mask_weight, double *loss, float *grad, void *stream) {
  if (!n || !x0 || !tval || !tmask || !loss) return fail(WPROJ_ERR_INVALID_ARG, "mlp_gradients: null argument");
  if (m < 128 || m % 128 || m > 65536)
    return fail(WPROJ_ERR_INVALID_ARG, "mlp_gradients: m must be a multiple of 128 up to 65536");
  return mlp_gradients(n, x0, tval, tmask, m, mask_weight, loss, grad, static_cast<cudaStream_t>(stream));
}

wproj_status wproj_build_kernels_learned(wproj_plan *p, wproj_mlp *n, const double *uvw, int64_t m, double e,
                                         double rel_l2_max, float *row_err, wproj_learned_info *info, void *stream) {
  if (!p || !n || !uvw) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels_learned: null argument");
  if (m < 1) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels_learned: m >= 1");
  if (!(e > 0.0 && e <= 1.0)) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels_learned: e must lie in (0, 1]");
  if (!(rel_l2_max >= 0.0)) return fail(WPROJ_ERR_INVALID_ARG, "build_kernels_learned: rel_l2_max >= 0");
  return build_learned_impl(p, n, uvw, m, e, rel_l2_max, row_err, info, static_cast<cudaStream_t>(stream));
}

wproj_status wproj_mlp_train(wproj_mlp *n, const float *x0, const float *tval, const float *tmask, int64_t m,
                             int32_t batch, int32_t steps, double lr, double mask_weight, float *losses,
                             void *stream) {
  if (!n || !x0 || !tval || !tmask) return fail(WPROJ_ERR_INVALID_ARG, "mlp_train: null argument");
  if (batch < 128 || batch % 128 || batch > 65536 || m < batch || m % batch || steps < 0 || !(lr > 0))
    return fail(WPROJ_ERR_INVALID_ARG, "mlp_train: batch a multiple of 128 (<= 65536) dividing m, lr > 0");
  return mlp_train(n, x0, tval, tmask, m, batch, steps, lr, mask_weight, losses, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
