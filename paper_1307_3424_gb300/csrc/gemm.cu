// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory:  C[M x N] = A[M x K] . B[N x K]^T  (+ bias[N]),
// A and B row-major ("K-major"), C row-major FP32 (or BF16).  This is the dense
// contraction of the learned-kernel MLP (its layers X W^T and their gradients).
//
// A CTA of 128 threads owns a 128 x 128 tile of C.  For every 64-wide K slice
// the threads copy the A and B slices into shared memory in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices, K-adjacent core
// matrices 128 B apart, row-adjacent ones 1 KB apart), one thread issues four
// tcgen05.mma (K = 16 each) accumulating into a 128 x 128 FP32 tile in tensor
// memory, and tcgen05.commit signals an mbarrier when they have read the
// slice.  Slices are copied with cp.async, two in flight per CTA and three
// CTAs per SM; a stage is refilled once the MMAs that
// read it have completed.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = rows of C), transposes each 32 x 32
// block through shared memory so that stores are row-contiguous, adds the bias
// and stores.
//
// Shapes: M, N multiples of 128, K a multiple of 64 (the callers pad).  Waits
// are bounded; a wait that runs out sets *err, and the CTA still frees its
// tensor memory before it exits.
#include "plan.h"

namespace wproj {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kSliceA = kBM * kBK * 2;   // bytes of one A slice (16 KB)
constexpr int kSliceB = kBN * kBK * 2;
constexpr int kStages = 2;   // slices in flight (3 CTAs fit on an SM)
constexpr unsigned long long kGemmWaitNs = 2000000000ull;

// Test hook (wproj_gemm_test_hook): when g_gemm_unset_wait is nonzero every CTA
// first waits on an mbarrier that nothing ever arrives on, bounded by
// g_gemm_wait_ns, so the timeout path (error word, drain of the committed MMAs,
// tensor memory freed) runs without any fault.
__device__ int g_gemm_unset_wait = 0;
__device__ unsigned long long g_gemm_wait_ns = kGemmWaitNs;

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ unsigned long long gns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity,
                                                  unsigned long long limit_ns = kGemmWaitNs) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = gns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_test(b, parity)) return true;
    if ((it & 63u) == 63u && gns() - t0 > limit_ns) return false;
  }
  return false;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (row-group) byte offsets >> 4, the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, N and M.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// asynchronous copy (cp.async, 16 B per request) of a rows x 64 bf16 slice
// (row stride ld elements) into the core-matrix layout
__device__ __forceinline__ void stage_slice(const __nv_bfloat16 *__restrict__ g, int64_t ld, int rows,
                                            unsigned char *s) {
  for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
    const int r = i >> 3, c = i & 7;   // row, 16-byte chunk along K
    const void *src = reinterpret_cast<const uint4 *>(g + int64_t(r) * ld) + c;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(s + ((r >> 3) * 8 + c) * 128 + (r & 7) * 16)),
                 "l"(src)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <bool OUT_BF16>
__global__ void __launch_bounds__(128)
k_gemm_tn(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
          const float *__restrict__ bias, void *__restrict__ C, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sa = smem;                              // kStages A slices
  unsigned char *sb = smem + kStages * kSliceA;          // kStages B slices
  __shared__ __align__(8) uint64_t done[kStages];        // MMAs of a stage finished reading it
  __shared__ __align__(8) uint64_t never;                // test hook: nothing arrives on it
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(kBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done[i])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&never)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc(kBM, kBN);
  const int nk = K / kBK;
  bool ok = true;
  if (g_gemm_unset_wait) ok = __syncthreads_and(mbar_wait_bounded(&never, 0, g_gemm_wait_ns));
  int k_issued = -1;   // last K slice whose MMAs were committed
  // every thread commits one copy group per slice (empty past the end), so
  // slice k's group is complete once at most kStages - 1 younger groups pend
  for (int k = 0; k < kStages; ++k) {
    if (k < nk) {
      stage_slice(A + int64_t(m0) * K + int64_t(k) * kBK, K, kBM, sa + k * kSliceA);
      stage_slice(B + int64_t(n0) * K + int64_t(k) * kBK, K, kBN, sb + k * kSliceB);
    }
    cp_commit();
  }
  for (int k = 0; k < nk && ok; ++k) {
    const int st = k % kStages;
    cp_wait<kStages - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // copies -> async proxy (tcgen05)
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = su32(sa + st * kSliceA), b0 = su32(sb + st * kSliceB);
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j) {   // K = 16 per MMA: two core matrices along K
        const uint64_t ad = smem_desc(a0 + j * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + j * 256, 128, 1024);
        const uint32_t acc = (k > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&done[st]))
                   : "memory");
    }
    k_issued = k;
    // refill this stage with slice k + kStages once its MMAs have read it
    const int nx = k + kStages;
    if (nx < nk) {
      ok = __syncthreads_and(mbar_wait_bounded(&done[st], (k / kStages) & 1));
      if (ok) {
        stage_slice(A + int64_t(m0) * K + int64_t(nx) * kBK, K, kBM, sa + st * kSliceA);
        stage_slice(B + int64_t(n0) * K + int64_t(nx) * kBK, K, kBN, sb + st * kSliceB);
      }
    }
    cp_commit();
  }
  cp_wait<0>();
  // all MMAs done: the last commit covers every earlier MMA.  After a timeout
  // the committed MMAs are still drained (normal limit) before the tensor
  // memory is freed.
  if (k_issued >= 0) {
    const bool drained = __syncthreads_and(mbar_wait_bounded(&done[k_issued % kStages], (k_issued / kStages) & 1));
    ok = ok && drained && k_issued == nk - 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // warp w reads TMEM lanes 32w.. (rows m0 + 32w + lane), 32 columns at a time
#pragma unroll 1
    for (int c0 = 0; c0 < kBN; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // transpose the warp's 32 x 32 block through shared memory (the staging
      // area is free now), so that each store instruction writes one row
      float *blk = reinterpret_cast<float *>(smem) + warp * 32 * 33;
#pragma unroll
      for (int i = 0; i < 32; ++i) blk[lane * 33 + i] = __uint_as_float(r[i]);
      __syncwarp();
      const int col = n0 + c0 + lane;
      const float bv = bias ? __ldg(bias + col) : 0.f;
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        const int rr = m0 + warp * 32 + i;
        const float v = blk[i * 33 + lane] + bv;
        if (rr < M) {
          if (OUT_BF16) reinterpret_cast<__nv_bfloat16 *>(C)[int64_t(rr) * N + col] = __float2bfloat16_rn(v);
          else reinterpret_cast<float *>(C)[int64_t(rr) * N + col] = v;
        }
      }
      __syncwarp();
    }
  } else if (threadIdx.x == 0) {
    atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN) : "memory");
}

}  // namespace

size_t gemm_smem_bytes() { return size_t(kStages) * (kSliceA + kSliceB) + 1024; }

// C = A B^T (+ bias); M, N multiples of 128, K a multiple of 64; err: device int
wproj_status gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
                          void *C, bool out_bf16, int *err, cudaStream_t s) {
  if (M % kBM || N % kBN || K % kBK || M <= 0 || N <= 0 || K <= 0)
    return fail(WPROJ_ERR_INVALID_ARG, "gemm: M, N must be multiples of 128 and K of 64");
  const size_t smem = gemm_smem_bytes();
  const dim3 grid(M / kBM, N / kBN);
  if (out_bf16) {
    WPROJ_CUDA(cudaFuncSetAttribute(k_gemm_tn<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gemm_tn<true><<<grid, 128, smem, s>>>(M, N, K, A, B, bias, C, err);
  } else {
    WPROJ_CUDA(cudaFuncSetAttribute(k_gemm_tn<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gemm_tn<false><<<grid, 128, smem, s>>>(M, N, K, A, B, bias, C, err);
  }
  WPROJ_CHECK_LAUNCH("gemm");
  return WPROJ_OK;
}

}  // namespace wproj

// ---- C-ABI ------------------------------------------------------------------------

namespace {
__device__ int g_gemm_err;   // timeouts of wproj_gemm_bf16 calls
}

extern "C" wproj_status wproj_gemm_test_hook(int32_t wait_on_unset_barrier, uint64_t limit_ns) {
  using namespace wproj;
  const int flag = wait_on_unset_barrier ? 1 : 0;
  const unsigned long long lim = limit_ns ? (unsigned long long)limit_ns : kGemmWaitNs;
  WPROJ_CUDA(cudaMemcpyToSymbol(g_gemm_unset_wait, &flag, sizeof(flag)));
  WPROJ_CUDA(cudaMemcpyToSymbol(g_gemm_wait_ns, &lim, sizeof(lim)));
  return WPROJ_OK;
}

extern "C" wproj_status wproj_gemm_bf16(int32_t m, int32_t n, int32_t k, const void *a, const void *b,
                                        const float *bias, void *c, int32_t out_bf16, void *stream) {
  using namespace wproj;
  if (!a || !b || !c) return fail(WPROJ_ERR_INVALID_ARG, "gemm: null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int *err = nullptr;
  WPROJ_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_gemm_err));
  WPROJ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  WPROJ_TRY(gemm_bf16_tn(m, n, k, static_cast<const __nv_bfloat16 *>(a), static_cast<const __nv_bfloat16 *>(b), bias,
                         c, out_bf16 != 0, err, s));
  int h = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(WPROJ_ERR_TIMEOUT, "gemm: a tensor-core wait ran out");
  return WPROJ_OK;
}
