// Device prefix sums and a stable counting sort, used to lay out G.
#include "plan.h"

namespace wproj {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

// Exclusive block scan of one value per thread; returns the prefix and the block total.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = kScanThreads / 32;
    T w = (lane < NW) ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T n = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += n;
    }
    if (lane < NW) warp_tot[lane] = wi - w;   // exclusive prefix of the warp totals
    if (lane == NW - 1) *total = wi;
  }
  __syncthreads();
  T res = warp_tot[wid] + inc - v;
  __syncthreads();
  return res;
}

template <class Tin, class Tout>
__global__ void k_block_sums(const Tin *__restrict__ in, int64_t n, Tout *__restrict__ sums) {
  __shared__ Tout tot;
  const int64_t base = int64_t(blockIdx.x) * kScanTile + threadIdx.x * kScanPer;
  Tout s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i)
    if (base + i < n) s += Tout(in[base + i]);
  Tout pre = block_exclusive_scan<Tout>(s, &tot);
  (void)pre;
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single-block exclusive scan of `n` values in place (sequential over tiles).
template <class T>
__global__ void k_scan_single(T *__restrict__ a, int64_t n, T *__restrict__ total) {
  __shared__ T tot;
  T carry = 0;
  for (int64_t t0 = 0; t0 < n; t0 += kScanTile) {
    const int64_t base = t0 + threadIdx.x * kScanPer;
    T v[kScanPer];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      v[i] = (base + i < n) ? a[base + i] : T(0);
      s += v[i];
    }
    T pre = block_exclusive_scan<T>(s, &tot) + carry;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      if (base + i < n) a[base + i] = pre;
      pre += v[i];
    }
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <class Tin, class Tout>
__global__ void k_scan_apply(const Tin *__restrict__ in, int64_t n, const Tout *__restrict__ offs,
                             Tout *__restrict__ out) {
  __shared__ Tout tot;
  const int64_t base = int64_t(blockIdx.x) * kScanTile + threadIdx.x * kScanPer;
  Tout v[kScanPer];
  Tout s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = (base + i < n) ? Tout(in[base + i]) : Tout(0);
    s += v[i];
  }
  Tout pre = block_exclusive_scan<Tout>(s, &tot) + offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    if (base + i < n) out[base + i] = pre;
    pre += v[i];
  }
}

template <class Tin, class Tout>
wproj_status exclusive_scan(const Tin *in, Tout *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return WPROJ_OK;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  DevBuf sums;
  WPROJ_TRY(sums.alloc(sizeof(Tout) * (nb + 1)));
  k_block_sums<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.as<Tout>());
  WPROJ_CHECK_LAUNCH("scan block sums");
  k_scan_single<Tout><<<1, kScanThreads, 0, s>>>(sums.as<Tout>(), nb, sums.as<Tout>() + nb);
  WPROJ_CHECK_LAUNCH("scan sums");
  k_scan_apply<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.as<Tout>(), out);
  WPROJ_CHECK_LAUNCH("scan apply");
  // the temporary is freed at scope exit; make sure the kernels are done with it
  WPROJ_CUDA(cudaStreamSynchronize(s));
  return WPROJ_OK;
}

// ---- stable counting sort ---------------------------------------------------

__global__ void k_bin_hist(const int32_t *__restrict__ key, int64_t n, int64_t chunk, int n_bins,
                           int n_blocks, int32_t *__restrict__ hist) {
  extern __shared__ int32_t h[];
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const int64_t lo = int64_t(blockIdx.x) * chunk;
  const int64_t hi = min(n, lo + chunk);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[key[i]], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
    hist[int64_t(b) * n_blocks + blockIdx.x] = h[b];
}

// One warp per block walks its chunk in order; ties inside a group of 32 are
// ranked by lane, so the sort is stable.
__global__ void k_bin_scatter(const int32_t *__restrict__ key, int64_t n, int64_t chunk, int n_bins,
                              int n_blocks, const int64_t *__restrict__ offs,
                              int32_t *__restrict__ out_ids) {
  extern __shared__ int32_t run[];
  for (int b = threadIdx.x; b < n_bins; b += 32) run[b] = int32_t(offs[int64_t(b) * n_blocks + blockIdx.x]);
  __syncwarp();
  const int lane = threadIdx.x;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t lo = int64_t(blockIdx.x) * chunk;
  const int64_t hi = min(n, lo + chunk);
  for (int64_t g = lo; g < hi; g += 32) {
    const int64_t i = g + lane;
    const bool act = i < hi;
    const int k = act ? key[i] : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    const int rank = __popc(peers & lt);
    int base = 0;
    if (act) base = run[k];
    __syncwarp();
    if (act) {
      out_ids[base + rank] = int32_t(i);
      const int leader = 31 - __clz(peers);
      if (lane == leader) run[k] = base + __popc(peers);
    }
    __syncwarp();
  }
}

__global__ void k_bin_ptr(const int64_t *__restrict__ offs, int n_bins, int n_blocks, int64_t n,
                          int64_t *__restrict__ bin_ptr) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_bins) bin_ptr[b] = offs[int64_t(b) * n_blocks];
  if (b == n_bins) bin_ptr[b] = n;
}

}  // namespace

wproj_status exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  return exclusive_scan<int32_t, int64_t>(in, out, n, s);
}
wproj_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  return exclusive_scan<int64_t, int64_t>(in, out, n, s);
}

wproj_status stable_bin_sort(const int32_t *key, int64_t n, int n_bins, int32_t *out_ids,
                             int64_t *bin_ptr, cudaStream_t s) {
  if (n >= (int64_t(1) << 31)) return fail(WPROJ_ERR_UNSUPPORTED, "stable_bin_sort: too many items");
  if (n_bins > 16384) return fail(WPROJ_ERR_UNSUPPORTED, "stable_bin_sort: too many bins");
  int n_blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (n + 4095) / 4096));
  int64_t chunk = (n + n_blocks - 1) / n_blocks;
  chunk = std::max<int64_t>(32, (chunk + 31) / 32 * 32);
  n_blocks = (int)std::max<int64_t>(1, (n + chunk - 1) / chunk);
  DevBuf hist, offs;
  const int64_t nh = int64_t(n_bins) * n_blocks;
  WPROJ_TRY(hist.alloc(sizeof(int32_t) * nh));
  WPROJ_TRY(offs.alloc(sizeof(int64_t) * nh));
  const size_t smem = sizeof(int32_t) * n_bins;
  if (smem > 48 * 1024) {
    WPROJ_CUDA(cudaFuncSetAttribute(k_bin_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    WPROJ_CUDA(cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  if (n > 0) {
    k_bin_hist<<<n_blocks, 256, smem, s>>>(key, n, chunk, n_bins, n_blocks, hist.as<int32_t>());
    WPROJ_CHECK_LAUNCH("bin hist");
  } else {
    WPROJ_CUDA(cudaMemsetAsync(hist.ptr, 0, sizeof(int32_t) * nh, s));
  }
  WPROJ_TRY(exclusive_scan_i32_to_i64(hist.as<int32_t>(), offs.as<int64_t>(), nh, s));
  if (n > 0) {
    k_bin_scatter<<<n_blocks, 32, smem, s>>>(key, n, chunk, n_bins, n_blocks, offs.as<int64_t>(), out_ids);
    WPROJ_CHECK_LAUNCH("bin scatter");
  }
  k_bin_ptr<<<(n_bins + 1 + 255) / 256, 256, 0, s>>>(offs.as<int64_t>(), n_bins, n_blocks, n, bin_ptr);
  WPROJ_CHECK_LAUNCH("bin ptr");
  WPROJ_CUDA(cudaStreamSynchronize(s));
  return WPROJ_OK;
}

}  // namespace wproj
