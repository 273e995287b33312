// Degridding and gridding for G in the tile-mask format.
//
// A segment is a (row of G, 32 x 32 grid tile) pair: 32 mask words (bit l of
// word r = cell (r, l) stored) and its values, one contiguous run in row-major
// cell order, so row r's values sit at off + prefix(r) + popc(word_r & lanes
// below l).  Blocks of 4 warps take chunks of one tile's segments (the
// tile-sorted list); warp w handles tile rows 8w..8w+7 of every segment and lane
// l column l, so no two threads touch the same cell, accumulators stay in
// registers, and each warp has its rows' value loads in flight together.  The
// next segment's descriptor and mask are loaded while the current one streams.
//
//  degridding  out[4 s + w] = sum over warp w's cells of segment s of G[k, q] X[q]
//              (the tile of X staged in shared memory once per block); y_k sums
//              its row's segments and warps in a fixed order
//  gridding    the chunk's 32 x 32 partial of sum_k conj(G[k, q]) y_k, summed per
//              tile in chunk order afterwards
//
// No atomics anywhere: results are bit-reproducible.
#include "plan.h"

namespace wproj {

namespace {

constexpr int kWarps = 4;
constexpr int kRows = 32 / kWarps;

template <int VDT>
__device__ __forceinline__ float2 ldval(const void *__restrict__ val, int64_t i) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    return __ldg(reinterpret_cast<const float2 *>(val) + i);
  } else if constexpr (VDT == WPROJ_VAL_BF16) {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(val) + i);
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw));
  } else {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(val) + i);
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
__global__ void __launch_bounds__(kWarps * 32)
k_tiles(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
        const int64_t *__restrict__ chunk_hi, const SegMeta *__restrict__ meta,
        const uint32_t *__restrict__ mask, const void *__restrict__ val, const float *__restrict__ row_scale,
        const float2 *__restrict__ y, const float2 *__restrict__ Xt, int logG, int nT,
        float2 *__restrict__ out) {
  __shared__ float2 xs[DEGRID ? 32 * 33 : 1];     // the chunk's tile of X (degridding), padded rows
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t lo = chunk_lo[c], hi = chunk_hi[c];
  if constexpr (DEGRID) {
    const int tile = chunk_tile[c];
    const int tu = tile / nT, tv = tile % nT;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
      const int r = i >> 5, l = i & 31;
      xs[r * 33 + l] = __ldg(Xt + ((int64_t(tu * 32 + r)) << logG) + tv * 32 + l);
    }
    __syncthreads();
  }
  float2 acc[kRows];
#pragma unroll
  for (int rr = 0; rr < kRows; ++rr) acc[rr] = make_float2(0.f, 0.f);
  SegMeta m = {};
  unsigned word = 0;
  if (lo < hi) { m = meta[lo]; word = __ldg(mask + int64_t(m.seg) * 32 + lane); }
  for (int64_t j = lo; j < hi; ++j) {
    SegMeta mn = {};
    unsigned nword = 0;
    const bool more = j + 1 < hi;
    if (more) { mn = meta[j + 1]; nword = __ldg(mask + int64_t(mn.seg) * 32 + lane); }
    const int64_t off = meta_off(m);
    float2 yk = make_float2(0.f, 0.f);
    if (!DEGRID) {
      yk = __ldg(y + m.row);
      if (row_scale) yk = cscale(yk, __ldg(row_scale + m.row));
    }
    const int pre = warp_excl_scan(__popc(word), lane);
    float2 v[kRows];
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) {
      const int r = kRows * w + rr;
      const unsigned wr = __shfl_sync(0xffffffffu, word, r);
      const int pr = __shfl_sync(0xffffffffu, pre, r);
      v[rr] = ((wr >> lane) & 1u) ? ldval<VDT>(val, off + pr + __popc(wr & lt)) : make_float2(0.f, 0.f);
    }
    if constexpr (DEGRID) {
      float ax = 0.f, ay = 0.f;
#pragma unroll
      for (int rr = 0; rr < kRows; ++rr) {
        const float2 x = xs[(kRows * w + rr) * 33 + lane];
        ax = fmaf(v[rr].x, x.x, ax); ax = fmaf(-v[rr].y, x.y, ax);
        ay = fmaf(v[rr].x, x.y, ay); ay = fmaf(v[rr].y, x.x, ay);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
      }
      if (lane == 0) out[int64_t(m.seg) * kWarps + w] = make_float2(ax, ay);
    } else {
#pragma unroll
      for (int rr = 0; rr < kRows; ++rr) {
        // conj(v) * y
        acc[rr].x = fmaf(v[rr].x, yk.x, acc[rr].x); acc[rr].x = fmaf(v[rr].y, yk.y, acc[rr].x);
        acc[rr].y = fmaf(v[rr].x, yk.y, acc[rr].y); acc[rr].y = fmaf(-v[rr].y, yk.x, acc[rr].y);
      }
    }
    if (more) { m = mn; word = nword; }
  }
  if constexpr (!DEGRID) {
    float2 *o = out + int64_t(c) * 1024;
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) o[(kRows * w + rr) * 32 + lane] = acc[rr];
  }
}

// y_k = sum over row k's segments s and warps w of partial[4 s + w], in that
// order, times the row scale
__global__ void k_tiles_reduce(int64_t m, const int64_t *__restrict__ seg_base, const float2 *__restrict__ partial,
                               const float *__restrict__ row_scale, float2 *__restrict__ y) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= m) return;
  float2 acc = make_float2(0.f, 0.f);
  for (int64_t i = seg_base[k] * kWarps; i < seg_base[k + 1] * kWarps; ++i) acc = cadd(acc, partial[i]);
  if (row_scale) acc = cscale(acc, row_scale[k]);
  y[k] = acc;
}

template <int VDT, bool DEGRID>
wproj_status launch_tiles(wproj_plan *p, const float2 *y, const float2 *Xt, float2 *out, cudaStream_t s) {
  k_tiles<VDT, DEGRID><<<(unsigned)p->n_chunks, kWarps * 32, 0, s>>>(
      p->chunk_tile.as<int32_t>(), p->chunk_lo.as<int64_t>(), p->chunk_hi.as<int64_t>(), p->seg_meta.as<SegMeta>(),
      p->seg_mask.as<uint32_t>(), p->val.ptr, p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(),
      y, Xt, ilog2(p->g.G), p->g.nT, out);
  WPROJ_CHECK_LAUNCH(DEGRID ? "degrid (tile mask)" : "grid (tile mask)");
  return WPROJ_OK;
}

}  // namespace

int64_t degrid_mask_partials(const wproj_plan *p) { return p->n_seg * kWarps; }

// Tile-mask degridding: partials into `partial` (degrid_mask_partials float2).
wproj_status degrid_mask(wproj_plan *p, const float2 *Xt, float2 *partial, cudaStream_t s) {
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: return launch_tiles<WPROJ_VAL_F32, true>(p, nullptr, Xt, partial, s);
    case WPROJ_VAL_BF16: return launch_tiles<WPROJ_VAL_BF16, true>(p, nullptr, Xt, partial, s);
    default: return launch_tiles<WPROJ_VAL_F16, true>(p, nullptr, Xt, partial, s);
  }
}

wproj_status degrid_mask_reduce(wproj_plan *p, const float2 *partial, float2 *y, cudaStream_t s) {
  k_tiles_reduce<<<ceil_div(p->m, 256), 256, 0, s>>>(
      p->m, p->seg_base.as<int64_t>(), partial,
      p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(), y);
  WPROJ_CHECK_LAUNCH("degrid (tile mask) reduce");
  return WPROJ_OK;
}

// Tile-mask gridding: chunk partial tiles into p->grid_partial.
wproj_status grid_mask(wproj_plan *p, const float2 *y, cudaStream_t s) {
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: return launch_tiles<WPROJ_VAL_F32, false>(p, y, nullptr, p->grid_partial.as<float2>(), s);
    case WPROJ_VAL_BF16: return launch_tiles<WPROJ_VAL_BF16, false>(p, y, nullptr, p->grid_partial.as<float2>(), s);
    default: return launch_tiles<WPROJ_VAL_F16, false>(p, y, nullptr, p->grid_partial.as<float2>(), s);
  }
}

}  // namespace wproj
