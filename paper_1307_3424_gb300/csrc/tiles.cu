// Degridding and gridding for G in the tile-stream format (TILE_MASK).
//
// The tile stream stores G tile-major: for every 32 x 32 grid tile (ascending)
// and every row of G with entries in that tile (rows ascending), one record of a
// multiple of 16 bytes:
//   header   int32 row, int32 count, int32 segment id (row-major), int32 0
//   mask     32 words, bit l of word r = cell (r, l) of the tile is stored
//   prefix   32 uint16, entries stored in the tile rows before row r
//   values   count values in row-major cell order, zero-padded to 16 bytes
// so the records of one tile are one contiguous byte range.  A chunk is a run of
// one tile's records holding about the same number of entries as the others;
// a block of 4 warps takes one chunk.  Warp w handles tile rows 8w..8w+7 of
// every record and lane l column l, so no two threads touch the same cell, the
// gridding accumulators (and the degridding's cells of X) stay in registers,
// and each warp has its rows' value loads in flight together.  A warp reads
// its 8 rows' mask words and prefixes with three 16-byte loads (the same
// address in every lane), so finding a lane's value takes no shuffles or scans.
// The next
// record's header and mask are loaded while the current one streams; its
// offset follows from the current count.  The gridding also asks the TMA engine
// to pull the chunk into L2 ahead of the warps (cp.async.bulk.prefetch.L2, 16 KB
// ahead); in the degridding that measured slower and is off.  Blocks take
// chunks in a strided order (chunk = block * stride mod chunks), which spreads
// the concurrently read chunks over more tiles (measured faster than in order).
//
//  degridding  out[4 s + w] = sum over warp w's cells of segment s of G[k, q] X[q];
//              y_k sums its row's segments and warps in a fixed order
//  gridding    the chunk's 32 x 32 partial of sum_k conj(G[k, q]) y_k, summed per
//              tile in chunk order afterwards
//
// No atomics: results are bit-reproducible.
#include "plan.h"

namespace wproj {

namespace {

constexpr int kWarps = kStreamWarps;   // warps per block
constexpr int kRows = 32 / kWarps;
constexpr int kThreads = kWarps * 32;
constexpr int kMinBlocks = 8;          // degridding: blocks per SM the register budget allows
constexpr int kMinBlocksGrid = 7;      // gridding: its 8 accumulators need 72 registers
constexpr int kPfAhead = 16384;        // gridding: bytes requested into L2 ahead of warp 0
constexpr int kPfStep = 8192;

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int VDT>
__device__ __forceinline__ float2 gval(const unsigned char *p) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    return __ldg(reinterpret_cast<const float2 *>(p));
  } else if constexpr (VDT == WPROJ_VAL_BF16) {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(p));
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw));
  } else {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(p));
    return __half22float2(*reinterpret_cast<const __half2 *>(&raw));
  }
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  return inc - v;
}

template <int VDT, bool DEGRID>
__global__ void __launch_bounds__(kThreads, DEGRID ? kMinBlocks : kMinBlocksGrid)
k_stream(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
         const int64_t *__restrict__ chunk_hi, const int64_t *__restrict__ rec_off, int stride,
         const unsigned char *__restrict__ stream, const float *__restrict__ row_scale,
         const float2 *__restrict__ y, const float2 *__restrict__ Xt, int logG, int nT,
         float2 *__restrict__ out) {
  constexpr int VB = (VDT == WPROJ_VAL_F32) ? 8 : 4;
  constexpr bool kPrefetch = !DEGRID;
  const int c = int((unsigned long long)blockIdx.x * unsigned(stride) % gridDim.x);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lbit = 1u << lane, lt = lbit - 1u;
  const int64_t j0 = chunk_lo[c], j1 = chunk_hi[c];
  const int64_t b0 = rec_off[j0], b1 = rec_off[j1];
  int64_t pf = b0;
  const bool pf_thread = kPrefetch && threadIdx.x == 0;
  auto prefetch_to = [&](int64_t upto) {   // request [pf, upto) of the chunk into L2
    if (upto > b1) upto = b1;
    while (pf < upto) {
      const int64_t n = b1 - pf < kPfStep ? b1 - pf : kPfStep;
      prefetch_l2(stream + pf, (uint32_t)n);
      pf += n;
    }
  };
  if (pf_thread) prefetch_to(b0 + kPfAhead);
  float2 xr[kRows];   // degridding: this thread's cells of the chunk's tile of X
  if constexpr (DEGRID) {
    const int tile = chunk_tile[c];
    const int tu = tile / nT, tv = tile % nT;
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr)
      xr[rr] = __ldg(Xt + ((int64_t(tu * 32 + kRows * w + rr)) << logG) + tv * 32 + lane);
  }
  float2 acc[kRows];
#pragma unroll
  for (int rr = 0; rr < kRows; ++rr) acc[rr] = make_float2(0.f, 0.f);
  static_assert(kRows == 8, "a warp reads 8 mask words and 8 prefixes");
  // this warp's rows' mask words (two uint4) and prefixes (one uint4 of 8 uint16)
  auto load_masks = [&](int64_t o, uint4 &a, uint4 &b, uint4 &p) {
    const uint4 *mk = reinterpret_cast<const uint4 *>(stream + o + kRecHeader) + 2 * w;
    a = __ldg(mk);
    b = __ldg(mk + 1);
    p = __ldg(reinterpret_cast<const uint4 *>(stream + o + kRecPrefix) + w);
  };
  int64_t off = b0;
  int4 hdr = make_int4(0, 0, 0, 0);
  uint4 wa = make_uint4(0, 0, 0, 0), wb = wa, pp = wa;
  float2 yk = make_float2(0.f, 0.f);
  if (j0 < j1) {
    hdr = __ldg(reinterpret_cast<const int4 *>(stream + off));
    load_masks(off, wa, wb, pp);
    if (!DEGRID) {
      yk = __ldg(y + hdr.x);
      if (row_scale) yk = cscale(yk, __ldg(row_scale + hdr.x));
    }
  }
  for (int64_t j = j0; j < j1; ++j) {
    const int64_t offn = off + kRecValues + ((hdr.y * VB + 15) & ~15);
    const bool more = j + 1 < j1;
    int4 hdrn = make_int4(0, 0, 0, 0);
    uint4 wan = make_uint4(0, 0, 0, 0), wbn = wan, ppn = wan;
    if (more) {
      hdrn = __ldg(reinterpret_cast<const int4 *>(stream + offn));
      load_masks(offn, wan, wbn, ppn);
    }
    if (pf_thread) prefetch_to(off + kPfAhead);
    const unsigned char *vb = stream + off + kRecValues;
    float2 v[kRows];
    const unsigned wrs[kRows] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    const unsigned pps[kRows / 2] = {pp.x, pp.y, pp.z, pp.w};
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) {
      const unsigned wr = wrs[rr];
      const int pr = int((pps[rr >> 1] >> (16 * (rr & 1))) & 0xffffu);
      v[rr] = (wr & lbit) ? gval<VDT>(vb + unsigned(pr + __popc(wr & lt)) * unsigned(VB)) : make_float2(0.f, 0.f);
    }
    if constexpr (DEGRID) {
      float ax = 0.f, ay = 0.f;
#pragma unroll
      for (int rr = 0; rr < kRows; ++rr) {
        const float2 x = xr[rr];
        ax = fmaf(v[rr].x, x.x, ax); ax = fmaf(-v[rr].y, x.y, ax);
        ay = fmaf(v[rr].x, x.y, ay); ay = fmaf(v[rr].y, x.x, ay);
      }
      // warp sum of (ax, ay) in 5 shuffles: after one exchange even lanes carry
      // pair sums of ax and odd lanes of ay, then both halve together
      const bool odd = lane & 1;
      float part = (odd ? ay : ax) + __shfl_xor_sync(0xffffffffu, odd ? ax : ay, 1);
#pragma unroll
      for (int o = 2; o < 32; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane < 2) reinterpret_cast<float *>(out + int64_t(hdr.z) * kWarps + w)[lane] = part;
    } else {
#pragma unroll
      for (int rr = 0; rr < kRows; ++rr) {
        // conj(v) * y
        acc[rr].x = fmaf(v[rr].x, yk.x, acc[rr].x); acc[rr].x = fmaf(v[rr].y, yk.y, acc[rr].x);
        acc[rr].y = fmaf(v[rr].x, yk.y, acc[rr].y); acc[rr].y = fmaf(-v[rr].y, yk.x, acc[rr].y);
      }
      if (more) {
        yk = __ldg(y + hdrn.x);
        if (row_scale) yk = cscale(yk, __ldg(row_scale + hdrn.x));
      }
    }
    off = offn;
    hdr = hdrn;
    wa = wan;
    wb = wbn;
    pp = ppn;
  }
  if constexpr (!DEGRID) {
    float2 *o = out + int64_t(c) * 1024;
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) o[(kRows * w + rr) * 32 + lane] = acc[rr];
  }
}

// smallest of a few small primes that is coprime with n: the block -> chunk
// stride (a bijection of [0, n))
int chunk_stride(int64_t n) {
  for (int s : {7, 11, 13, 17, 19, 23, 29, 31})
    if (n % s != 0) return s;
  return 1;
}

// y_k = sum over row k's segments s and warps w of partial[4 s + w], in that
// order, times the row scale
__global__ void k_stream_reduce(int64_t m, const int64_t *__restrict__ seg_base, const float2 *__restrict__ partial,
                                const float *__restrict__ row_scale, float2 *__restrict__ y) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= m) return;
  float2 acc = make_float2(0.f, 0.f);
  for (int64_t i = seg_base[k] * kWarps; i < seg_base[k + 1] * kWarps; ++i) acc = cadd(acc, partial[i]);
  if (row_scale) acc = cscale(acc, row_scale[k]);
  y[k] = acc;
}

template <int VDT, bool DEGRID>
wproj_status launch_stream(wproj_plan *p, const float2 *y, const float2 *Xt, float2 *out, cudaStream_t s) {
  k_stream<VDT, DEGRID><<<(unsigned)p->n_chunks, kThreads, 0, s>>>(
      p->chunk_tile.as<int32_t>(), p->chunk_lo.as<int64_t>(), p->chunk_hi.as<int64_t>(), p->rec_off.as<int64_t>(),
      chunk_stride(p->n_chunks), p->stream.as<unsigned char>(),
      p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(), y, Xt, ilog2(p->g.G), p->g.nT, out);
  WPROJ_CHECK_LAUNCH(DEGRID ? "degrid (tile stream)" : "grid (tile stream)");
  return WPROJ_OK;
}

// Entries of segments [s0, s1) (row-major order) written in CSR order at
// col_out / val_out + (seg_off[s] - first), warp per segment.
__global__ void k_stream_export(int64_t s0, int64_t s1, int64_t first, const int64_t *__restrict__ seg_rec,
                                const int64_t *__restrict__ seg_off, const int32_t *__restrict__ seg_tile,
                                const unsigned char *__restrict__ stream, int vb, int G, int nT,
                                int32_t *__restrict__ col_out, unsigned char *__restrict__ val_out) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t sg = s0 + warp; sg < s1; sg += nwarps) {
    const unsigned char *rec = stream + seg_rec[sg];
    const unsigned word = reinterpret_cast<const unsigned *>(rec + kRecHeader)[lane];
    const int pre = warp_excl_scan(__popc(word), lane);
    const int tile = seg_tile[sg];
    const int tu = tile / nT, tv = tile % nT;
    const int64_t o = seg_off[sg] - first;
    for (int r = 0; r < 32; ++r) {
      const unsigned wr = __shfl_sync(0xffffffffu, word, r);
      const int pr = __shfl_sync(0xffffffffu, pre, r);
      if (!((wr >> lane) & 1u)) continue;
      const int i = pr + __popc(wr & lt);
      if (col_out) col_out[o + i] = (tu * 32 + r) * G + tv * 32 + lane;
      if (val_out) {
        const unsigned char *src = rec + kRecValues + int64_t(i) * vb;
        if (vb == 8) reinterpret_cast<float2 *>(val_out)[o + i] = *reinterpret_cast<const float2 *>(src);
        else reinterpret_cast<unsigned *>(val_out)[o + i] = *reinterpret_cast<const unsigned *>(src);
      }
    }
  }
}

}  // namespace

int64_t degrid_stream_partials(const wproj_plan *p) { return p->n_seg * kWarps; }

// Tile-stream degridding: partials into `partial` (degrid_stream_partials float2).
wproj_status degrid_stream(wproj_plan *p, const float2 *Xt, float2 *partial, cudaStream_t s) {
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: return launch_stream<WPROJ_VAL_F32, true>(p, nullptr, Xt, partial, s);
    case WPROJ_VAL_BF16: return launch_stream<WPROJ_VAL_BF16, true>(p, nullptr, Xt, partial, s);
    default: return launch_stream<WPROJ_VAL_F16, true>(p, nullptr, Xt, partial, s);
  }
}

wproj_status degrid_stream_reduce(wproj_plan *p, const float2 *partial, float2 *y, cudaStream_t s) {
  k_stream_reduce<<<ceil_div(p->m, 256), 256, 0, s>>>(
      p->m, p->seg_base.as<int64_t>(), partial,
      p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(), y);
  WPROJ_CHECK_LAUNCH("degrid (tile stream) reduce");
  return WPROJ_OK;
}

// Tile-stream gridding: chunk partial tiles into p->grid_partial.
wproj_status grid_stream(wproj_plan *p, const float2 *y, cudaStream_t s) {
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: return launch_stream<WPROJ_VAL_F32, false>(p, y, nullptr, p->grid_partial.as<float2>(), s);
    case WPROJ_VAL_BF16: return launch_stream<WPROJ_VAL_BF16, false>(p, y, nullptr, p->grid_partial.as<float2>(), s);
    default: return launch_stream<WPROJ_VAL_F16, false>(p, y, nullptr, p->grid_partial.as<float2>(), s);
  }
}

wproj_status stream_export(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                           cudaStream_t s) {
  int64_t sb[2] = {0, 0}, first = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&sb[0], p->seg_base.as<int64_t>() + k0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&sb[1], p->seg_base.as<int64_t>() + k1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&first, p->row_ptr.as<int64_t>() + k0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (sb[1] <= sb[0]) return WPROJ_OK;
  const int blocks = (int)std::min<int64_t>(ceil_div((sb[1] - sb[0]) * 32, 256), 152 * 32);
  k_stream_export<<<blocks, 256, 0, s>>>(sb[0], sb[1], first, p->seg_rec.as<int64_t>(), p->seg_off.as<int64_t>(),
                                         p->seg_tile.as<int32_t>(), p->stream.as<unsigned char>(),
                                         p->g.value_dtype == WPROJ_VAL_F32 ? 8 : 4, p->g.G, p->g.nT, col_out,
                                         static_cast<unsigned char *>(val_out));
  WPROJ_CHECK_LAUNCH("export (tile stream)");
  return WPROJ_OK;
}

}  // namespace wproj
