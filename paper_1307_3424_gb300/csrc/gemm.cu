// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory:  C[M x N] = A[M x K] . B[N x K]^T  (+ bias[N]),
// A and B row-major ("K-major"), C row-major FP32 (or BF16).  This is the dense
// contraction of the learned-kernel MLP (its layers X W^T and their gradients).
//
// Persistent and warp-specialised: one CTA per SM walks the 128 x BN tiles of
// C (BN = 256 when N allows, else 128; tile t = CTA, CTA + grid, ...; tiles of
// one row block of A are adjacent, so concurrent CTAs share A rows and B in
// L2).  Six warps:
//   warp 0   TMA producer: for every 64-wide K slice of a tile, waits for a free
//            stage, arms its `full` mbarrier with the slice's bytes and issues
//            two cp.async.bulk.tensor loads (A: 128 rows, B: BN rows, x 64 bf16,
//            128-byte swizzled) that complete on that barrier;
//   warp 1   MMA issuer: allocates 2 BN tensor-memory columns (two 128 x BN FP32
//            accumulators), and for every tile waits for a free accumulator,
//            issues four tcgen05.mma (kind::f16, K = 16) per slice from
//            128B-swizzle K-major shared-memory descriptors, commits each slice
//            to its stage's `empty` barrier and the tile to `acc_full`;
//   warps 2-5  epilogue: wait for `acc_full`, read the accumulator with
//            tcgen05.ld (warp w reads tensor-memory lanes 32 (w mod 4) ..), add
//            the bias, transpose each 32 x 32 block through shared memory so that
//            stores are row-contiguous, store, and release the accumulator.
// So the loads of tile i + 1 and the MMAs of tile i + 1 overlap the epilogue of
// tile i.  Four stages of 48 KB (BN = 256); 1 CTA per SM.
//
// Shapes: M, N multiples of 128, K a multiple of 64 (the callers pad).  Every
// wait is bounded (2 s); a wait that runs out sets *err and its role stops, the
// other roles run out of their own waits, the MMA warp waits (bounded) for its
// committed MMAs, and the tensor memory is freed before the CTA exits.
#include <cuda.h>

#include <mutex>

#include "plan.h"

namespace wproj {

namespace {

constexpr int kBM = 128, kBK = 64;      // tile rows; K slice (64 bf16 = one 128-byte swizzle row)
constexpr int kSliceA = kBM * kBK * 2;   // bytes of one A slice: 16 KB
constexpr int kStages = 4;
constexpr int kThreads = 192;            // 6 warps
constexpr unsigned long long kGemmWaitNs = 2000000000ull;

// Test hook (wproj_gemm_test_hook): when g_gemm_unset_wait is nonzero every
// warp of every CTA first waits on an mbarrier that nothing ever arrives on,
// bounded by g_gemm_wait_ns, so the timeout path (error word, no work issued,
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

// waits for the phase of parity `parity` to complete; false after limit_ns
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

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

// 2-D tiled TMA load of box (x = K element, y = row) into shared memory,
// completing `bytes` on the mbarrier
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05) of a K-major operand in the
// 128-byte-swizzled layout TMA writes: start address >> 4, leading byte offset
// (unused for swizzled K-major; 1), stride byte offset 1024 (8 rows of 128 B),
// the fixed 0b001 at bits 46-48, swizzle mode 2 (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, N and M.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// BN: tile columns (128 or 256); a tile's accumulator takes BN tensor-memory
// columns, two of them 2 BN (512 at most: the whole tensor memory).
template <int BN>
struct GemmSmem {
  unsigned char a[kStages][kSliceA];     // 1024-byte aligned (swizzle atoms)
  unsigned char b[kStages][BN * kBK * 2];
  float epi[4][32 * 33];                 // epilogue transposes, one block per warp
  uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2], never;
  uint32_t tmem_base;
};

template <int BN, bool OUT_BF16>
__global__ void __launch_bounds__(kThreads, 1)
k_gemm_ws(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
          const float *__restrict__ bias, void *__restrict__ C, int *__restrict__ err) {
  constexpr int kAccCols = BN;
  constexpr int kSliceB = BN * kBK * 2;
  extern __shared__ unsigned char smem_raw[];
  GemmSmem<BN> &sm =
      *reinterpret_cast<GemmSmem<BN> *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nN = N / BN, n_tiles = (M / kBM) * nN, nk = K / kBK;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sm.full[i], 1);    // the producer's arrive.expect_tx
      mbar_init(&sm.empty[i], 1);   // one tcgen05.commit
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sm.acc_full[i], 1);    // one tcgen05.commit
      mbar_init(&sm.acc_empty[i], 4);   // one arrive per epilogue warp
    }
    mbar_init(&sm.never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem_base)),
                 "r"(2 * kAccCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem_base;
  bool ok = true;
  if (g_gemm_unset_wait) ok = mbar_wait_bounded(&sm.never, 0, g_gemm_wait_ns);

  if (warp == 0) {
    // ---- TMA producer (one lane)
    if (lane == 0 && ok) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      uint32_t it = 0;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int m0 = (t / nN) * kBM, n0 = (t % nN) * BN;
        for (int k = 0; k < nk; ++k, ++it) {
          const int st = int(it % kStages);
          const uint32_t ph = (it / kStages) & 1u;
          if (!mbar_wait_bounded(&sm.empty[st], ph ^ 1u)) { ok = false; break; }
          mbar_expect_tx(&sm.full[st], kSliceA + kSliceB);
          tma_load_2d(sm.a[st], &tmA, k * kBK, m0, &sm.full[st]);
          tma_load_2d(sm.b[st], &tmB, k * kBK, n0, &sm.full[st]);
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer (one lane)
    if (lane == 0 && ok) {
      const uint32_t idesc = instr_desc(kBM, BN);
      uint32_t it = 0, ti = 0;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++ti) {
        const uint32_t buf = ti & 1u, aph = (ti >> 1) & 1u;
        if (!mbar_wait_bounded(&sm.acc_empty[buf], aph ^ 1u)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + buf * kAccCols;
        for (int k = 0; k < nk; ++k, ++it) {
          const int st = int(it % kStages);
          const uint32_t ph = (it / kStages) & 1u;
          if (!mbar_wait_bounded(&sm.full[st], ph)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = su32(sm.a[st]), b0 = su32(sm.b[st]);
#pragma unroll
          for (int j = 0; j < kBK / 16; ++j) {   // K = 16 per MMA: 32 bytes along the swizzled row
            const uint64_t ad = smem_desc_sw128(a0 + j * 32);
            const uint64_t bd = smem_desc_sw128(b0 + j * 32);
            const uint32_t accum = (k > 0 || j > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(&sm.empty[st]))
                       : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&sm.acc_full[buf]))
                     : "memory");
      }
      // before the tensor memory is freed, every committed MMA must be done:
      // the last commit of each stage covers the MMAs before it
      if (it > 0) {
        const uint32_t last = it - 1;
        for (uint32_t q = (last >= kStages ? last - kStages + 1 : 0); q <= last; ++q)
          if (!mbar_wait_bounded(&sm.empty[q % kStages], (q / kStages) & 1u)) ok = false;
      }
    }
  } else {
    // ---- epilogue (warps 2-5): tensor-memory lanes 32 (warp mod 4) ..
    const int lg = warp & 3;
    float *blk = sm.epi[warp - 2];
    uint32_t ti = 0;
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++ti) {
      const int m0 = (t / nN) * kBM, n0 = (t % nN) * BN;
      const uint32_t buf = ti & 1u, aph = (ti >> 1) & 1u;
      if (!mbar_wait_bounded(&sm.acc_full[buf], aph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + (uint32_t(lg * 32) << 16) + buf * kAccCols + uint32_t(c0);
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
#pragma unroll
        for (int i = 0; i < 32; ++i) blk[lane * 33 + i] = __uint_as_float(r[i]);
        __syncwarp();
        const int col = n0 + c0 + lane;
        const float bv = bias ? __ldg(bias + col) : 0.f;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
          const int64_t rr = m0 + lg * 32 + i;
          const float v = blk[i * 33 + lane] + bv;
          if (OUT_BF16) reinterpret_cast<__nv_bfloat16 *>(C)[rr * N + col] = __float2bfloat16_rn(v);
          else reinterpret_cast<float *>(C)[rr * N + col] = v;
        }
        __syncwarp();
      }
      // this warp is done with the accumulator
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
    }
  }
  if (!ok && lane == 0) atomicOr(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccCols) : "memory");
}

// cuTensorMapEncodeTiled from the driver, looked up through the runtime (the
// library does not link the driver library itself)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
std::mutex g_encode_mu;
EncodeTiledFn g_encode = nullptr;

wproj_status encode_fn(EncodeTiledFn *out) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (!g_encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(WPROJ_ERR_CUDA, "gemm: cuTensorMapEncodeTiled is not available");
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  *out = g_encode;
  return WPROJ_OK;
}

// tensor map of a rows x K bf16 row-major matrix, box box_rows x 64 (128 B), 128-byte swizzle
wproj_status tensor_map(CUtensorMap *map, const __nv_bfloat16 *p, int rows, int K, int box_rows) {
  EncodeTiledFn enc = nullptr;
  WPROJ_TRY(encode_fn(&enc));
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(K) * 2};
  const cuuint32_t box[2] = {cuuint32_t(kBK), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(WPROJ_ERR_CUDA, "gemm: cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
  return WPROJ_OK;
}

template <int BN>
wproj_status launch_gemm(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
                         void *C, bool out_bf16, int *err, cudaStream_t s) {
  CUtensorMap ta, tb;
  WPROJ_TRY(tensor_map(&ta, A, M, K, kBM));
  WPROJ_TRY(tensor_map(&tb, B, N, K, BN));
  int dev = 0, sms = 0;
  WPROJ_CUDA(cudaGetDevice(&dev));
  WPROJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int n_tiles = (M / kBM) * (N / BN);
  const int grid = std::max(1, std::min(n_tiles, sms));
  const size_t smem = sizeof(GemmSmem<BN>) + 1024;
  if (out_bf16) {
    WPROJ_CUDA(cudaFuncSetAttribute(k_gemm_ws<BN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gemm_ws<BN, true><<<grid, kThreads, smem, s>>>(ta, tb, M, N, K, bias, C, err);
  } else {
    WPROJ_CUDA(cudaFuncSetAttribute(k_gemm_ws<BN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gemm_ws<BN, false><<<grid, kThreads, smem, s>>>(ta, tb, M, N, K, bias, C, err);
  }
  WPROJ_CHECK_LAUNCH("gemm");
  return WPROJ_OK;
}

}  // namespace

// C = A B^T (+ bias); M, N multiples of 128, K a multiple of 64; A and B 16-byte
// aligned (TMA); err: device int.  Tiles of 128 x 256 when N is a multiple of
// 256, else 128 x 128.
wproj_status gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
                          void *C, bool out_bf16, int *err, cudaStream_t s) {
  if (M % kBM || N % 128 || K % kBK || M <= 0 || N <= 0 || K <= 0)
    return fail(WPROJ_ERR_INVALID_ARG, "gemm: M, N must be multiples of 128 and K of 64");
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
    return fail(WPROJ_ERR_INVALID_ARG, "gemm: A and B must be 16-byte aligned");
  if (N % 256 == 0) return launch_gemm<256>(M, N, K, A, B, bias, C, out_bf16, err, s);
  return launch_gemm<128>(M, N, K, A, B, bias, C, out_bf16, err, s);
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
