// Part II: the measurement operator Phi = G F Z A (Eq. 8) and its adjoint.
//
//  degridding  y_k = sum_q G[k, q] X[q]          warp per row piece (<= 16384
//              entries), partial sums reduced per row in a fixed order
//  gridding    X'[q] = sum_k conj(G[k, q]) y_k    block per chunk of a grid
//              tile's segment list; every warp accumulates its segments into
//              a private shared-memory copy of the 32 x 32 tile, the copies are
//              summed in warp order, chunk partials are summed per tile in chunk
//              order.  No global atomics; results are bit-reproducible.
#include "plan.h"

namespace wproj {

namespace {

template <int VDT>
__device__ __forceinline__ float2 load_val(const void *__restrict__ val, int64_t i) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    return __ldg(reinterpret_cast<const float2 *>(val) + i);
  } else if constexpr (VDT == WPROJ_VAL_BF16) {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(val) + i);
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&raw);
    return __bfloat1622float2(h);
  } else {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(val) + i);
    __half2 h = *reinterpret_cast<const __half2 *>(&raw);
    return __half22float2(h);
  }
}

template <int VDT>
__global__ void __launch_bounds__(256)
k_degrid(int64_t n_pieces, const int32_t *__restrict__ piece_lo_row, const int64_t *__restrict__ piece_lo,
         const int32_t *__restrict__ piece_len, const int32_t *__restrict__ col,
         const void *__restrict__ val, const float2 *__restrict__ Xt, float2 *__restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t pc = warp; pc < n_pieces; pc += nwarps) {
    const int64_t lo = piece_lo[pc];
    const int len = piece_len[pc];
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    int i = lane;
    for (; i + 96 < len; i += 128) {
      const int c0 = __ldg(col + lo + i), c1 = __ldg(col + lo + i + 32);
      const int c2 = __ldg(col + lo + i + 64), c3 = __ldg(col + lo + i + 96);
      const float2 v0 = load_val<VDT>(val, lo + i), v1 = load_val<VDT>(val, lo + i + 32);
      const float2 v2 = load_val<VDT>(val, lo + i + 64), v3 = load_val<VDT>(val, lo + i + 96);
      const float2 x0 = __ldg(Xt + c0), x1 = __ldg(Xt + c1), x2 = __ldg(Xt + c2), x3 = __ldg(Xt + c3);
      ax = fmaf(v0.x, x0.x, ax); ax = fmaf(-v0.y, x0.y, ax); ay = fmaf(v0.x, x0.y, ay); ay = fmaf(v0.y, x0.x, ay);
      bx = fmaf(v1.x, x1.x, bx); bx = fmaf(-v1.y, x1.y, bx); by = fmaf(v1.x, x1.y, by); by = fmaf(v1.y, x1.x, by);
      ax = fmaf(v2.x, x2.x, ax); ax = fmaf(-v2.y, x2.y, ax); ay = fmaf(v2.x, x2.y, ay); ay = fmaf(v2.y, x2.x, ay);
      bx = fmaf(v3.x, x3.x, bx); bx = fmaf(-v3.y, x3.y, bx); by = fmaf(v3.x, x3.y, by); by = fmaf(v3.y, x3.x, by);
    }
    for (; i < len; i += 32) {
      const int c0 = __ldg(col + lo + i);
      const float2 v0 = load_val<VDT>(val, lo + i);
      const float2 x0 = __ldg(Xt + c0);
      ax = fmaf(v0.x, x0.x, ax); ax = fmaf(-v0.y, x0.y, ax); ay = fmaf(v0.x, x0.y, ay); ay = fmaf(v0.y, x0.x, ay);
    }
    ax += bx;
    ay += by;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) partial[pc] = make_float2(ax, ay);
  }
  (void)piece_lo_row;
}

__global__ void k_degrid_reduce(int64_t m, const int32_t *__restrict__ row_piece_ptr,
                                const float2 *__restrict__ partial, const float *__restrict__ row_scale,
                                float2 *__restrict__ y) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= m) return;
  float2 acc = make_float2(0.f, 0.f);
  for (int j = row_piece_ptr[k]; j < row_piece_ptr[k + 1]; ++j) acc = cadd(acc, partial[j]);
  if (row_scale) acc = cscale(acc, row_scale[k]);
  y[k] = acc;
}

// accumulate conj(v) * yk into this warp's copy of the tile (entries of one
// segment have distinct cells, so the lanes never collide)
__device__ __forceinline__ void grid_acc(float2 *my, int q, float2 v, float2 yk, int logG, int Gm, int ou,
                                         int ov, int TS) {
  const int lu = (q >> logG) - ou, lv = (q & Gm) - ov;
  if ((unsigned)lu >= (unsigned)TS || (unsigned)lv >= (unsigned)TS) return;   // not in this tile
  float2 *cell = my + lu * TS + lv;
  float2 a = *cell;
  a.x = fmaf(v.x, yk.x, a.x); a.x = fmaf(v.y, yk.y, a.x);
  a.y = fmaf(v.x, yk.y, a.y); a.y = fmaf(-v.y, yk.x, a.y);
  *cell = a;
}

template <int VDT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_grid(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
       const int64_t *__restrict__ chunk_hi, const SegMeta *__restrict__ meta,
       const int32_t *__restrict__ col, const void *__restrict__ val, const float *__restrict__ row_scale,
       const float2 *__restrict__ y, int logG, int TS, int nT, float2 *__restrict__ partial) {
  extern __shared__ float2 acc[];   // [WARPS][TS*TS]
  const int c = blockIdx.x;
  const int tile = chunk_tile[c];
  const int tu = tile / nT, tv = tile % nT;
  const int cells = TS * TS;
  for (int i = threadIdx.x; i < WARPS * cells; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2 *my = acc + w * cells;
  const int64_t lo = chunk_lo[c], hi = chunk_hi[c];
  const int Gm = (1 << logG) - 1;
  const int ou = tu * TS, ov = tv * TS;
  int64_t j = lo + w;
  SegMeta cur;
  if (j < hi) cur = meta[j];
  for (; j < hi; j += WARPS) {
    // prefetch the next segment's descriptor while this one streams
    SegMeta nxt;
    const bool more = j + WARPS < hi;
    if (more) nxt = meta[j + WARPS];
    float2 yk = __ldg(y + cur.row);
    if (row_scale) yk = cscale(yk, __ldg(row_scale + cur.row));
    const int64_t off = cur.off;
    const int n = cur.aux;
    int i = lane;
    for (; i + 96 < n; i += 128) {
      const int q0 = __ldg(col + off + i), q1 = __ldg(col + off + i + 32);
      const int q2 = __ldg(col + off + i + 64), q3 = __ldg(col + off + i + 96);
      const float2 v0 = load_val<VDT>(val, off + i), v1 = load_val<VDT>(val, off + i + 32);
      const float2 v2 = load_val<VDT>(val, off + i + 64), v3 = load_val<VDT>(val, off + i + 96);
      grid_acc(my, q0, v0, yk, logG, Gm, ou, ov, TS);
      grid_acc(my, q1, v1, yk, logG, Gm, ou, ov, TS);
      grid_acc(my, q2, v2, yk, logG, Gm, ou, ov, TS);
      grid_acc(my, q3, v3, yk, logG, Gm, ou, ov, TS);
    }
    for (; i < n; i += 32) grid_acc(my, __ldg(col + off + i), load_val<VDT>(val, off + i), yk, logG, Gm, ou, ov, TS);
    if (more) cur = nxt;
  }
  __syncthreads();
  float2 *out = partial + int64_t(c) * cells;
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    float2 s = acc[i];
#pragma unroll
    for (int ww = 1; ww < WARPS; ++ww) s = cadd(s, acc[ww * cells + i]);
    out[i] = s;
  }
}

__global__ void k_grid_reduce(const int32_t *__restrict__ tile_chunk_ptr, const float2 *__restrict__ partial,
                              int G, int TS, int nT, float2 *__restrict__ Xt2) {
  const int tile = blockIdx.x;
  const int tu = tile / nT, tv = tile % nT;
  const int cells = TS * TS;
  const int c0 = tile_chunk_ptr[tile], c1 = tile_chunk_ptr[tile + 1];
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int c = c0; c < c1; ++c) s = cadd(s, partial[int64_t(c) * cells + i]);
    const int lu = i / TS, lv = i % TS;
    Xt2[int64_t(tu * TS + lu) * G + tv * TS + lv] = s;
  }
}

constexpr int kGridWarps = 8;

// ---- tile-mask format -----------------------------------------------------------------
// A segment is a (row, 32x32 tile) pair: 32 mask words (bit l of word r = cell
// (r, l) stored) and its values contiguous in row-major cell order.  With
// lane = tile column, row r's values sit at off + prefix(r) + popc(word_r & lanes
// below), one contiguous run per tile row.

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  return inc - v;
}

// y partials: block (4 warps) per piece, a run of one row's segments.  Warp w
// handles tile rows 8w..8w+7 of every segment, lane l column l: it gathers the
// X values of its cells (coalesced 256-byte rows of X) and the stored values of
// its rows with predicated loads, all 16 in flight before the first multiply.
// The four warp sums are added in warp order at the end of the piece.
constexpr int kDegridMaskWarps = 4;

template <int VDT>
__global__ void __launch_bounds__(kDegridMaskWarps * 32)
k_degrid_mask(int64_t n_pieces, const int64_t *__restrict__ piece_seg, const int32_t *__restrict__ piece_nseg,
              const int32_t *__restrict__ seg_tile, const int64_t *__restrict__ seg_off,
              const uint32_t *__restrict__ mask, const void *__restrict__ val, const float2 *__restrict__ Xt,
              int logG, int lognT, float2 *__restrict__ partial) {
  constexpr int R = 32 / kDegridMaskWarps;
  __shared__ float2 red[kDegridMaskWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int nTm = (1 << lognT) - 1;
  for (int64_t pc = blockIdx.x; pc < n_pieces; pc += gridDim.x) {
    const int64_t s0 = piece_seg[pc];
    const int ns = piece_nseg[pc];
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    unsigned word = 0;
    int tile = 0;
    int64_t off = 0;
    if (ns > 0) { word = __ldg(mask + s0 * 32 + lane); tile = __ldg(seg_tile + s0); off = __ldg(seg_off + s0); }
    for (int64_t s = s0; s < s0 + ns; ++s) {
      // next segment's descriptor in flight while this one streams
      unsigned nword = 0;
      int ntile_ = 0;
      int64_t noff = 0;
      const bool more = s + 1 < s0 + ns;
      if (more) { nword = __ldg(mask + (s + 1) * 32 + lane); ntile_ = __ldg(seg_tile + s + 1); noff = __ldg(seg_off + s + 1); }
      const int pre = warp_excl_scan(__popc(word), lane);
      const float2 *xr = Xt + ((int64_t(tile >> lognT) << 5) << logG) + ((tile & nTm) << 5) + lane;
      float2 v[R], x[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = R * w + i;
        const unsigned wr = __shfl_sync(0xffffffffu, word, r);
        const int pr = __shfl_sync(0xffffffffu, pre, r);
        const bool bit = (wr >> lane) & 1u;
        v[i] = bit ? load_val<VDT>(val, off + pr + __popc(wr & lt)) : make_float2(0.f, 0.f);
        x[i] = __ldg(xr + (int64_t(r) << logG));
      }
#pragma unroll
      for (int i = 0; i < R; i += 2) {
        ax = fmaf(v[i].x, x[i].x, ax); ax = fmaf(-v[i].y, x[i].y, ax);
        ay = fmaf(v[i].x, x[i].y, ay); ay = fmaf(v[i].y, x[i].x, ay);
        bx = fmaf(v[i + 1].x, x[i + 1].x, bx); bx = fmaf(-v[i + 1].y, x[i + 1].y, bx);
        by = fmaf(v[i + 1].x, x[i + 1].y, by); by = fmaf(v[i + 1].y, x[i + 1].x, by);
      }
      if (more) { word = nword; tile = ntile_; off = noff; }
    }
    ax += bx;
    ay += by;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) red[w] = make_float2(ax, ay);
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 t = red[0];
#pragma unroll
      for (int i = 1; i < kDegridMaskWarps; ++i) t = cadd(t, red[i]);
      partial[pc] = t;
    }
    __syncthreads();
  }
}

// Gridding: block (4 warps) per chunk of one tile's segments; warp w owns tile
// rows 8w..8w+7 and lane l column l, so every accumulator lives in registers and
// no two threads ever touch the same cell.  Each warp walks all segments of the
// chunk (the mask words come through L1) and reads only its rows' values.
constexpr int kGridMaskWarps = 4;
constexpr int kGridMaskRows = 32 / kGridMaskWarps;

template <int VDT>
__global__ void __launch_bounds__(kGridMaskWarps * 32)
k_grid_mask(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
            const int64_t *__restrict__ chunk_hi, const SegMeta *__restrict__ meta,
            const uint32_t *__restrict__ mask, const void *__restrict__ val,
            const float *__restrict__ row_scale, const float2 *__restrict__ y, float2 *__restrict__ partial) {
  constexpr int R = kGridMaskRows;
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t lo = chunk_lo[c], hi = chunk_hi[c];
  float2 acc[R];
#pragma unroll
  for (int rr = 0; rr < R; ++rr) acc[rr] = make_float2(0.f, 0.f);
  SegMeta m = {};
  unsigned word = 0;
  if (lo < hi) { m = meta[lo]; word = __ldg(mask + int64_t(m.aux) * 32 + lane); }
  for (int64_t j = lo; j < hi; ++j) {
    SegMeta mn = {};
    unsigned nword = 0;
    const bool more = j + 1 < hi;
    if (more) { mn = meta[j + 1]; nword = __ldg(mask + int64_t(mn.aux) * 32 + lane); }
    float2 yk = __ldg(y + m.row);
    if (row_scale) yk = cscale(yk, __ldg(row_scale + m.row));
    const int pre = warp_excl_scan(__popc(word), lane);
    float2 v[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int r = R * w + rr;
      const unsigned wr = __shfl_sync(0xffffffffu, word, r);
      const int pr = __shfl_sync(0xffffffffu, pre, r);
      const bool bit = (wr >> lane) & 1u;
      v[rr] = bit ? load_val<VDT>(val, m.off + pr + __popc(wr & lt)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      // conj(v) * y
      acc[rr].x = fmaf(v[rr].x, yk.x, acc[rr].x); acc[rr].x = fmaf(v[rr].y, yk.y, acc[rr].x);
      acc[rr].y = fmaf(v[rr].x, yk.y, acc[rr].y); acc[rr].y = fmaf(-v[rr].y, yk.x, acc[rr].y);
    }
    if (more) { m = mn; word = nword; }
  }
  float2 *out = partial + int64_t(c) * 1024;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) out[(R * w + rr) * 32 + lane] = acc[rr];
  (void)chunk_tile;
}

// Column index of every stored entry (tile-mask format), warp per segment.
__global__ void k_expand_cols(int64_t n_seg, const int32_t *__restrict__ seg_tile,
                              const int64_t *__restrict__ seg_off, const uint32_t *__restrict__ mask,
                              int G, int nT, int32_t *__restrict__ col) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = warp; s < n_seg; s += nwarps) {
    const unsigned word = mask[s * 32 + lane];
    const int pre = warp_excl_scan(__popc(word), lane);
    const int tile = seg_tile[s];
    const int tu = tile / nT, tv = tile % nT;
    const int64_t off = seg_off[s];
    for (int r = 0; r < 32; ++r) {
      const unsigned wr = __shfl_sync(0xffffffffu, word, r);
      const int pr = __shfl_sync(0xffffffffu, pre, r);
      if ((wr >> lane) & 1u) col[off + pr + __popc(wr & lt)] = (tu * 32 + r) * G + tv * 32 + lane;
    }
  }
}

// Degridding kernels for the plan's index format and value type; partial sums
// per row piece go to `partial` (n_pieces float2).
wproj_status launch_degrid(wproj_plan *p, const float2 *Xt, float2 *partial, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(ceil_div(p->n_pieces * 32, 256), 152 * 16);
  const int logG = ilog2(p->g.G), lognT = ilog2(p->g.nT);
  const int mblocks = (int)std::max<int64_t>(1, std::min<int64_t>(p->n_pieces, 152 * 32));
#define DEGRID_COLS(VDT)                                                                                     \
  k_degrid<VDT><<<blocks, 256, 0, s>>>(p->n_pieces, p->piece_row.as<int32_t>(), p->piece_lo.as<int64_t>(),  \
                                       p->piece_len.as<int32_t>(), p->col.as<int32_t>(), p->val.ptr, Xt, partial)
#define DEGRID_MASK(VDT)                                                                                     \
  k_degrid_mask<VDT><<<mblocks, kDegridMaskWarps * 32, 0, s>>>(p->n_pieces, p->piece_lo.as<int64_t>(), p->piece_len.as<int32_t>(), \
                                            p->seg_tile.as<int32_t>(), p->seg_off.as<int64_t>(),              \
                                            p->seg_mask.as<uint32_t>(), p->val.ptr, Xt, logG, lognT, partial)
  const bool mask = p->fmt == WPROJ_INDEX_TILE_MASK;
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: if (mask) DEGRID_MASK(WPROJ_VAL_F32); else DEGRID_COLS(WPROJ_VAL_F32); break;
    case WPROJ_VAL_BF16: if (mask) DEGRID_MASK(WPROJ_VAL_BF16); else DEGRID_COLS(WPROJ_VAL_BF16); break;
    default: if (mask) DEGRID_MASK(WPROJ_VAL_F16); else DEGRID_COLS(WPROJ_VAL_F16);
  }
#undef DEGRID_COLS
#undef DEGRID_MASK
  WPROJ_CHECK_LAUNCH("degrid");
  return WPROJ_OK;
}

}  // namespace

wproj_status degrid(wproj_plan *p, const float2 *Xt, float2 *y, cudaStream_t s) {
  p->launches += 2;
  {
    ScopedTimer t(p, TC_DEGRID, s);
    WPROJ_TRY(launch_degrid(p, Xt, p->piece_partial.as<float2>(), s));
  }
  ScopedTimer t(p, TC_REDUCE, s);
  k_degrid_reduce<<<ceil_div(p->m, 256), 256, 0, s>>>(p->m, p->row_piece_ptr.as<int32_t>(), p->piece_partial.as<float2>(),
                                                      p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(), y);
  WPROJ_CHECK_LAUNCH("degrid reduce");
  return WPROJ_OK;
}

// Degridding with a caller-provided buffer for the per-piece partial sums
// (n_pieces float2); the kernels and their launch shape are those of degrid().
wproj_status degrid_into(wproj_plan *p, const float2 *Xt, float2 *partial, float2 *y, cudaStream_t s) {
  WPROJ_TRY(launch_degrid(p, Xt, partial, s));
  k_degrid_reduce<<<ceil_div(p->m, 256), 256, 0, s>>>(p->m, p->row_piece_ptr.as<int32_t>(), partial,
                                                      p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(), y);
  WPROJ_CHECK_LAUNCH("degrid reduce");
  return WPROJ_OK;
}

wproj_status grid(wproj_plan *p, const float2 *y, float2 *Xt2, cudaStream_t s) {
  p->launches += 2;
  const GridGeom &g = p->g;
  const size_t smem = sizeof(float2) * kGridWarps * g.tile * g.tile;
  const int logG = ilog2(g.G);
  const float *rs = g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>();
  {
    ScopedTimer t(p, TC_GRID, s);
#define LAUNCH_GRID(VDT)                                                                                    \
  do {                                                                                                      \
    if (p->fmt == WPROJ_INDEX_TILE_MASK) {                                                                  \
      k_grid_mask<VDT><<<(unsigned)p->n_chunks, kGridMaskWarps * 32, 0, s>>>(                               \
          p->chunk_tile.as<int32_t>(), p->chunk_lo.as<int64_t>(), p->chunk_hi.as<int64_t>(),                \
          p->seg_meta.as<SegMeta>(), p->seg_mask.as<uint32_t>(), p->val.ptr, rs, y,                         \
          p->grid_partial.as<float2>());                                                                    \
    } else {                                                                                                \
      WPROJ_CUDA(cudaFuncSetAttribute(k_grid<VDT, kGridWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
      k_grid<VDT, kGridWarps><<<(unsigned)p->n_chunks, kGridWarps * 32, smem, s>>>(                         \
          p->chunk_tile.as<int32_t>(), p->chunk_lo.as<int64_t>(), p->chunk_hi.as<int64_t>(),                \
          p->seg_meta.as<SegMeta>(), p->col.as<int32_t>(), p->val.ptr, rs, y, logG, g.tile, g.nT,           \
          p->grid_partial.as<float2>());                                                                    \
    }                                                                                                       \
  } while (0)
    switch (g.value_dtype) {
      case WPROJ_VAL_F32: LAUNCH_GRID(WPROJ_VAL_F32); break;
      case WPROJ_VAL_BF16: LAUNCH_GRID(WPROJ_VAL_BF16); break;
      default: LAUNCH_GRID(WPROJ_VAL_F16);
    }
#undef LAUNCH_GRID
    WPROJ_CHECK_LAUNCH("grid");
  }
  ScopedTimer t(p, TC_REDUCE, s);
  k_grid_reduce<<<g.nT * g.nT, 256, 0, s>>>(p->tile_chunk_ptr.as<int32_t>(), p->grid_partial.as<float2>(), g.G, g.tile,
                                             g.nT, Xt2);
  WPROJ_CHECK_LAUNCH("grid reduce");
  return WPROJ_OK;
}

wproj_status csr_columns(const wproj_plan *p, int32_t *col_out, cudaStream_t s) {
  if (p->fmt == WPROJ_INDEX_COLUMNS) {
    WPROJ_CUDA(cudaMemcpyAsync(col_out, p->col.ptr, sizeof(int32_t) * p->nnz, cudaMemcpyDeviceToDevice, s));
    return WPROJ_OK;
  }
  const int blocks = (int)std::min<int64_t>(ceil_div(p->n_seg * 32, 256), 152 * 32);
  k_expand_cols<<<std::max(blocks, 1), 256, 0, s>>>(p->n_seg, p->seg_tile.as<int32_t>(), p->seg_off.as<int64_t>(),
                                                    p->seg_mask.as<uint32_t>(), p->g.G, p->g.nT, col_out);
  WPROJ_CHECK_LAUNCH("expand columns");
  return WPROJ_OK;
}

wproj_status apply_phi(wproj_plan *p, const float *x, const float2 *xc, float2 *y, cudaStream_t s) {
  WPROJ_TRY(phi_forward_fft(p, x, xc, p->Xt.as<float2>(), s));
  return degrid(p, p->Xt.as<float2>(), y, s);
}

wproj_status apply_phi_adj(wproj_plan *p, const float2 *y, float *x_re, float2 *x_cplx, const float *z,
                           int mode, cudaStream_t s) {
  WPROJ_TRY(grid(p, y, p->Xt2.as<float2>(), s));
  return phi_adjoint_fft(p, p->Xt2.as<float2>(), x_re, x_cplx, z, mode, s);
}

}  // namespace wproj
