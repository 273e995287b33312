// y = Phi x for callers that cannot allocate device memory.
//
// wproj_phi needs scratch space between its kernels: the intermediate of the
// two FFT passes (N x G complex), the padded spectrum X (G x G complex) and the
// per-piece partial sums of the degridding (one complex per row piece).  The
// plan holds these buffers in memory it allocated itself.  This variant keeps
// them instead in one fixed-size array that lives in the library's own device
// image, so the call allocates nothing, and it does not touch the plan's work
// buffers.  It launches the same kernels as wproj_phi, so the results are the
// same.
#include <mutex>

#include "plan.h"

namespace {

// 16 MiB per GPU.  A plan fits when N*G + G*G complex values (FFT intermediate
// and padded spectrum) plus its degridding partial sums (one per row piece of
// the column format, four per (row, tile) segment of the tile stream), each
// part rounded up to 256 bytes, total at most this: N = 512 leaves room for
// 524,288 partial sums, N = 256 for 1.7 million; N >= 1024 never fits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_phi_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

// Device address of g_phi_scratch on the current device (looked up once per
// device and kept for the life of the process: a cudaDeviceReset, which also
// invalidates every plan, invalidates it too).
wproj_status scratch_address(void **out) {
  int dev = 0;
  WPROJ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return wproj::fail(WPROJ_ERR_UNSUPPORTED, "phi_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&ptr, g_phi_scratch);
    if (err != cudaSuccess) return wproj::cuda_fail(err, "phi_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return WPROJ_OK;
}

}  // namespace

extern "C" wproj_status wproj_phi_noalloc(wproj_plan *p, const float *x, void *y, void *stream) {
  using namespace wproj;
  if (!p) return fail(WPROJ_ERR_INVALID_ARG, "null plan");
  if (!p->built) return fail(WPROJ_ERR_NOT_BUILT, "G has not been built (call wproj_build_kernels)");
  if (!x || !y) return fail(WPROJ_ERR_INVALID_ARG, "null x or y");
  const size_t n_inter = round256(sizeof(float2) * size_t(p->g.N) * p->g.G);
  const size_t n_xt = round256(sizeof(float2) * size_t(p->g.G) * p->g.G);
  const size_t n_part = round256(sizeof(float2) * size_t(degrid_partials(p)));
  const size_t need = n_inter + n_xt + n_part;
  if (need > kNoAllocScratchBytes)
    return fail(WPROJ_ERR_INVALID_ARG,
                "phi_noalloc: this plan needs " + std::to_string(need) + " bytes of scratch (" +
                    std::to_string(degrid_partials(p)) + " degridding partial sums); the fixed limit is " +
                    std::to_string(kNoAllocScratchBytes) + " bytes: N*G + G*G + partials complex values");
  void *base = nullptr;
  WPROJ_TRY(scratch_address(&base));
  unsigned char *b = static_cast<unsigned char *>(base);
  float2 *inter = reinterpret_cast<float2 *>(b);
  float2 *Xt = reinterpret_cast<float2 *>(b + n_inter);
  float2 *partial = reinterpret_cast<float2 *>(b + n_inter + n_xt);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    // timed and counted like wproj_phi's two halves (FFT passes, then degridding)
    ScopedTimer t(p, TC_FFT, s);
    p->launches += p->g.upsampling ? 4 : 2;
    WPROJ_TRY(phi_forward_fft_into(p, x, inter, Xt, s));
  }
  p->launches += 2;
  return degrid_into(p, Xt, partial, static_cast<float2 *>(y), s);
}
