// Shared device helpers of libwproj (product code only).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

#include "wproj.h"

namespace wproj {

constexpr int kTile = 32;          // side of the grid tiles used for gridding and CSR order
constexpr double kSelectMargin = 1e-5;   // extra kept energy fraction (covers FP32 error)
// tile-stream records (TILE_MASK format): 16-byte header (row, count, segment
// id, 0), 32 mask words, 32 uint16 row prefixes (entries before each tile row),
// then the values from kRecValues on
constexpr int kRecHeader = 16;
constexpr int kRecPrefix = kRecHeader + 32 * 4;
constexpr int kRecValues = kRecPrefix + 32 * 2;
// consumer warps of the tile-stream kernels: the degridding leaves one partial
// sum per (record, warp)
constexpr int kStreamWarps = 4;

// ---- complex helpers --------------------------------------------------------
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
  return make_float2(a.x * s, a.y * s);
}

// |z|^2 with a fixed rounding sequence (no FMA contraction), so every kernel
// that recomputes a selection key gets the same bits.
__device__ __forceinline__ float abs2_rn(float2 z) {
  return __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y));
}

// Kaiser-Bessel gridding kernel of support W (unnormalised), t in cells
__device__ __forceinline__ double kb_dev(double t, int W, double beta) {
  const double r = 2.0 * t / W;
  const double arg = 1.0 - r * r;
  if (arg < 0.0) return 0.0;
  return cyl_bessel_i0(beta * sqrt(arg));
}

// ---- FP64 block reductions (fixed order: bit-reproducible) ---------------------
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over a block of T threads; the result is valid in thread 0
template <int T>
__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red[T / 32];
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < T / 32) ? red[threadIdx.x] : 0.0;
    t = warp_sum_d(t);
  }
  __syncthreads();
  return t;
}

// ---- error state ------------------------------------------------------------
void set_error(const std::string &msg);
wproj_status fail(wproj_status st, const std::string &msg);
wproj_status cuda_fail(cudaError_t err, const char *what);

#define WPROJ_CUDA(call)                                    \
  do {                                                      \
    cudaError_t err__ = (call);                             \
    if (err__ != cudaSuccess) return ::wproj::cuda_fail(err__, #call); \
  } while (0)

#define WPROJ_CHECK_LAUNCH(what)                            \
  do {                                                      \
    cudaError_t err__ = cudaGetLastError();                 \
    if (err__ != cudaSuccess) return ::wproj::cuda_fail(err__, what); \
  } while (0)

#define WPROJ_TRY(expr)                                     \
  do {                                                      \
    wproj_status st__ = (expr);                             \
    if (st__ != WPROJ_OK) return st__;                      \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int ilog2(int64_t n) { int l = 0; while ((int64_t(1) << l) < n) ++l; return l; }
inline bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace wproj
