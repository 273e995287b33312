// Part II: the measurement operator Phi = G F Z A (Eq. 8) and its adjoint.
// Kernels for G in the COLUMNS format (TILE_MASK: tiles.cu) and the dispatch:
//
//  degridding  y_k = sum_q G[k, q] X[q]          32, 16, 8 or 4 lanes per row
//              piece (<= 16384 entries, or a batch's tuned size), partial sums
//              reduced per row in a fixed order
//  gridding    X'[q] = sum_k conj(G[k, q]) y_k    from the cell-major copy
//              (cells.cu) when it exists; otherwise (m > 2^22) block per chunk
//              of a grid tile's segment list, every warp accumulating its
//              segments into a private shared-memory copy of the 32 x 32 tile,
//              the copies summed in warp order, chunk partials summed per tile
//              in chunk order.  No global atomics; results are bit-reproducible.
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

// A stored value as loaded (float2, or one 32-bit word of two 16-bit halves)
// and its conversion, so that prefetched values stay unconverted until used.
template <int VDT> struct RawVal { using type = unsigned; };
template <> struct RawVal<WPROJ_VAL_F32> { using type = float2; };

template <int VDT>
__device__ __forceinline__ typename RawVal<VDT>::type load_raw(const void *__restrict__ val, int64_t i) {
  if constexpr (VDT == WPROJ_VAL_F32) return __ldg(reinterpret_cast<const float2 *>(val) + i);
  else return __ldg(reinterpret_cast<const unsigned *>(val) + i);
}

template <int VDT>
__device__ __forceinline__ float2 raw_to_float2(typename RawVal<VDT>::type r) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    return r;
  } else if constexpr (VDT == WPROJ_VAL_BF16) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r));
  } else {
    return __half22float2(*reinterpret_cast<const __half2 *>(&r));
  }
}

constexpr int kDegridBlocksPerSm = 4;   // 56 registers a thread: four resident 256-thread blocks

// LPP lanes per row piece (32, 16, 8 or 4): 32 / LPP pieces per warp step, so
// that short pieces still put several independent loads in flight per lane.
// Each lane takes up to four entries per step (predicated, all issued before
// the first use); the next step's columns and values are loaded while this
// step's grid values are gathered, and the next piece's header one piece
// ahead, so the column -> grid-value chain is the only dependent pair of loads
// and it overlaps the next step's loads.
template <int VDT, int LPP>
__global__ void __launch_bounds__(256, kDegridBlocksPerSm)
k_degrid(int64_t n_pieces, const int64_t *__restrict__ piece_lo, const int32_t *__restrict__ piece_len,
         const int32_t *__restrict__ col, const void *__restrict__ val, const float2 *__restrict__ Xt,
         float2 *__restrict__ partial) {
  constexpr int kPer = 32 / LPP;   // pieces per warp step
  const int lane = threadIdx.x & 31, sl = lane % LPP;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t stride = ((int64_t(gridDim.x) * blockDim.x) >> 5) * kPer;
  int64_t pc = warp * kPer + lane / LPP;
  int64_t lo = pc < n_pieces ? piece_lo[pc] : 0;
  int len = pc < n_pieces ? piece_len[pc] : 0;
  for (int64_t base = warp * kPer; base < n_pieces; base += stride, pc += stride) {
    const int64_t npc = pc + stride;
    const int64_t nlo = npc < n_pieces ? piece_lo[npc] : 0;
    const int nlen = npc < n_pieces ? piece_len[npc] : 0;
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    using Raw = typename RawVal<VDT>::type;
    int c[4];
    Raw v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = sl + k * LPP < len;
      c[k] = ok ? __ldg(col + lo + sl + k * LPP) : 0;
      v[k] = ok ? load_raw<VDT>(val, lo + sl + k * LPP) : Raw{};
    }
    for (int i = sl; i < len; i += 4 * LPP) {
      float2 x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = i + k * LPP < len ? __ldg(Xt + c[k]) : make_float2(0.f, 0.f);
      // the next step's columns and values, in flight with this step's gathers
      int cn[4];
      Raw vn[4];
      const int in = i + 4 * LPP;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = in + k * LPP < len;
        cn[k] = ok ? __ldg(col + lo + in + k * LPP) : 0;
        vn[k] = ok ? load_raw<VDT>(val, lo + in + k * LPP) : Raw{};
      }
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        const float2 v0 = raw_to_float2<VDT>(v[k]), v1 = raw_to_float2<VDT>(v[k + 1]);
        ax = fmaf(v0.x, x[k].x, ax); ax = fmaf(-v0.y, x[k].y, ax);
        ay = fmaf(v0.x, x[k].y, ay); ay = fmaf(v0.y, x[k].x, ay);
        bx = fmaf(v1.x, x[k + 1].x, bx); bx = fmaf(-v1.y, x[k + 1].y, bx);
        by = fmaf(v1.x, x[k + 1].y, by); by = fmaf(v1.y, x[k + 1].x, by);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c[k] = cn[k];
        v[k] = vn[k];
      }
    }
    ax += bx;
    ay += by;
#pragma unroll
    for (int o = LPP / 2; o; o >>= 1) {   // within the piece's lanes
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (pc < n_pieces && sl == 0) partial[pc] = make_float2(ax, ay);
    lo = nlo;
    len = nlen;
  }
}

template <int VDT>
wproj_status launch_degrid_pieces(int64_t n_pieces, const int64_t *piece_lo, const int32_t *piece_len,
                                  const int32_t *col, const void *val, const float2 *Xt, float2 *partial, int lpp,
                                  cudaStream_t s) {
  const int64_t warps = ceil_div(n_pieces, int64_t(32 / lpp));
  // one resident wave: every block strides over the same share of pieces
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps * 32, 256), 152 * kDegridBlocksPerSm));
  switch (lpp) {
    case 4: k_degrid<VDT, 4><<<blocks, 256, 0, s>>>(n_pieces, piece_lo, piece_len, col, val, Xt, partial); break;
    case 8: k_degrid<VDT, 8><<<blocks, 256, 0, s>>>(n_pieces, piece_lo, piece_len, col, val, Xt, partial); break;
    case 16: k_degrid<VDT, 16><<<blocks, 256, 0, s>>>(n_pieces, piece_lo, piece_len, col, val, Xt, partial); break;
    default: k_degrid<VDT, 32><<<blocks, 256, 0, s>>>(n_pieces, piece_lo, piece_len, col, val, Xt, partial);
  }
  WPROJ_CHECK_LAUNCH("degrid");
  return WPROJ_OK;
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

// chunk_prob / tab (batches): the chunk's problem supplies logG, nT and the
// offset of its grid, which the stored columns include
template <int VDT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_grid(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
       const int64_t *__restrict__ chunk_hi, const SegMeta *__restrict__ meta,
       const int32_t *__restrict__ col, const void *__restrict__ val, const float *__restrict__ row_scale,
       const float2 *__restrict__ y, int logG, int TS, int nT, const int32_t *__restrict__ chunk_prob,
       const BProb *__restrict__ tab, float2 *__restrict__ partial) {
  extern __shared__ float2 acc[];   // [WARPS][TS*TS]
  const int c = blockIdx.x;
  int cbase = 0;
  if (chunk_prob) {
    const BProb &P = tab[chunk_prob[c]];
    logG = P.logG;
    nT = P.nT;
    cbase = int(P.grid_off);
  }
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
    const int64_t off = meta_off(cur);
    const int n = meta_cnt(cur);
    int i = lane;
    for (; i + 96 < n; i += 128) {
      const int q0 = __ldg(col + off + i) - cbase, q1 = __ldg(col + off + i + 32) - cbase;
      const int q2 = __ldg(col + off + i + 64) - cbase, q3 = __ldg(col + off + i + 96) - cbase;
      const float2 v0 = load_val<VDT>(val, off + i), v1 = load_val<VDT>(val, off + i + 32);
      const float2 v2 = load_val<VDT>(val, off + i + 64), v3 = load_val<VDT>(val, off + i + 96);
      grid_acc(my, q0, v0, yk, logG, Gm, ou, ov, TS);
      grid_acc(my, q1, v1, yk, logG, Gm, ou, ov, TS);
      grid_acc(my, q2, v2, yk, logG, Gm, ou, ov, TS);
      grid_acc(my, q3, v3, yk, logG, Gm, ou, ov, TS);
    }
    for (; i < n; i += 32)
      grid_acc(my, __ldg(col + off + i) - cbase, load_val<VDT>(val, off + i), yk, logG, Gm, ou, ov, TS);
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

// tile_prob / tab (batches): blockIdx.x is a tile of the whole batch
__global__ void k_grid_reduce(const int32_t *__restrict__ tile_chunk_ptr, const float2 *__restrict__ partial,
                              int G, int TS, int nT, const int32_t *__restrict__ tile_prob,
                              const BProb *__restrict__ tab, float2 *__restrict__ Xt2) {
  int tile = blockIdx.x;
  const int c0 = tile_chunk_ptr[tile], c1 = tile_chunk_ptr[tile + 1];
  if (tile_prob) {
    const BProb &P = tab[tile_prob[tile]];
    G = P.G;
    nT = P.nT;
    tile -= int(P.tile_off);
    Xt2 += P.grid_off;
  }
  const int tu = tile / nT, tv = tile % nT;
  const int cells = TS * TS;
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int c = c0; c < c1; ++c) s = cadd(s, partial[int64_t(c) * cells + i]);
    const int lu = i / TS, lv = i % TS;
    Xt2[int64_t(tu * TS + lu) * G + tv * TS + lv] = s;
  }
}

constexpr int kGridWarps = 8;

// Column-format degridding kernels; partial sums per row piece into `partial`.
// A piece takes the fewest lanes whose two four-entry steps cover its average
// length (the second step's loads overlap the first's gathers).
wproj_status launch_degrid_cols(wproj_plan *p, const float2 *Xt, float2 *partial, cudaStream_t s) {
  int lpp = 4;
  while (lpp < 32 && 8 * lpp * p->n_pieces < p->nnz) lpp *= 2;
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32:
      return launch_degrid_pieces<WPROJ_VAL_F32>(p->n_pieces, p->piece_lo.as<int64_t>(), p->piece_len.as<int32_t>(),
                                                 p->col.as<int32_t>(), p->val.ptr, Xt, partial, lpp, s);
    case WPROJ_VAL_BF16:
      return launch_degrid_pieces<WPROJ_VAL_BF16>(p->n_pieces, p->piece_lo.as<int64_t>(), p->piece_len.as<int32_t>(),
                                                  p->col.as<int32_t>(), p->val.ptr, Xt, partial, lpp, s);
    default:
      return launch_degrid_pieces<WPROJ_VAL_F16>(p->n_pieces, p->piece_lo.as<int64_t>(), p->piece_len.as<int32_t>(),
                                                 p->col.as<int32_t>(), p->val.ptr, Xt, partial, lpp, s);
  }
}

}  // namespace

wproj_status degrid(wproj_plan *p, const float2 *Xt, float2 *y, cudaStream_t s) {
  p->launches += p->fmt == WPROJ_INDEX_TILE_RUNS ? 1 : 2;
  return degrid_into(p, Xt, p->piece_partial.as<float2>(), y, s);
}

// Degridding with a caller-provided buffer for the partial sums
// (degrid_partials(p) float2); the kernels and their launch shape are those of
// degrid().
wproj_status degrid_into(wproj_plan *p, const float2 *Xt, float2 *partial, float2 *y, cudaStream_t s) {
  if (p->fmt == WPROJ_INDEX_TILE_RUNS) {   // warp per row, no partial sums
    ScopedTimer t(p, TC_DEGRID, s);
    return degrid_runs(p, Xt, y, s);
  }
  {
    ScopedTimer t(p, TC_DEGRID, s);
    if (p->fmt == WPROJ_INDEX_TILE_MASK) WPROJ_TRY(degrid_stream(p, Xt, partial, s));
    else WPROJ_TRY(launch_degrid_cols(p, Xt, partial, s));
  }
  ScopedTimer t(p, TC_REDUCE, s);
  if (p->fmt == WPROJ_INDEX_TILE_MASK) return degrid_stream_reduce(p, partial, y, s);
  k_degrid_reduce<<<ceil_div(p->m, 256), 256, 0, s>>>(p->m, p->row_piece_ptr.as<int32_t>(), partial,
                                                      p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>(), y);
  WPROJ_CHECK_LAUNCH("degrid reduce");
  return WPROJ_OK;
}

int64_t degrid_partials(const wproj_plan *p) {
  if (p->fmt == WPROJ_INDEX_TILE_RUNS) return 0;
  return p->fmt == WPROJ_INDEX_TILE_MASK ? degrid_stream_partials(p) : p->n_pieces;
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
    WPROJ_CUDA(cudaFuncSetAttribute(k_grid<VDT, kGridWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_grid<VDT, kGridWarps><<<(unsigned)p->n_chunks, kGridWarps * 32, smem, s>>>(                           \
        p->chunk_tile.as<int32_t>(), p->chunk_lo.as<int64_t>(), p->chunk_hi.as<int64_t>(),                  \
        p->seg_meta.as<SegMeta>(), p->col.as<int32_t>(), p->val.ptr, rs, y, logG, g.tile, g.nT, nullptr,    \
        nullptr, p->grid_partial.as<float2>());                                                             \
  } while (0)
    if (p->fmt == WPROJ_INDEX_TILE_RUNS) {
      int nl = 0;
      WPROJ_TRY(grid_runs(p, y, Xt2, &nl, s));
      p->launches += nl - 2;
      return WPROJ_OK;
    } else if (p->fmt == WPROJ_INDEX_TILE_MASK) {
      WPROJ_TRY(grid_stream(p, y, s));
    } else if (p->has_cells) {
      p->launches -= 1;   // one kernel, no chunk reduction
      return grid_cells(p, y, Xt2, s);
    } else {
      switch (g.value_dtype) {
        case WPROJ_VAL_F32: LAUNCH_GRID(WPROJ_VAL_F32); break;
        case WPROJ_VAL_BF16: LAUNCH_GRID(WPROJ_VAL_BF16); break;
        default: LAUNCH_GRID(WPROJ_VAL_F16);
      }
    }
#undef LAUNCH_GRID
    WPROJ_CHECK_LAUNCH("grid");
  }
  ScopedTimer t(p, TC_REDUCE, s);
  k_grid_reduce<<<g.nT * g.nT, 256, 0, s>>>(p->tile_chunk_ptr.as<int32_t>(), p->grid_partial.as<float2>(), g.G, g.tile,
                                             g.nT, nullptr, nullptr, Xt2);
  WPROJ_CHECK_LAUNCH("grid reduce");
  return WPROJ_OK;
}

wproj_status csr_rows(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                      cudaStream_t s) {
  if (p->fmt == WPROJ_INDEX_TILE_MASK) return stream_export(p, k0, k1, col_out, val_out, s);
  if (p->fmt == WPROJ_INDEX_TILE_RUNS) return runs_export(p, k0, k1, col_out, val_out, s);
  int64_t r[2] = {0, 0};
  WPROJ_CUDA(cudaMemcpyAsync(&r[0], p->row_ptr.as<int64_t>() + k0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&r[1], p->row_ptr.as<int64_t>() + k1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  const int64_t n = r[1] - r[0];
  if (n <= 0) return WPROJ_OK;
  const size_t vb = p->g.value_dtype == WPROJ_VAL_F32 ? 8 : 4;
  if (col_out)
    WPROJ_CUDA(cudaMemcpyAsync(col_out, p->col.as<int32_t>() + r[0], sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  if (val_out)
    WPROJ_CUDA(cudaMemcpyAsync(val_out, static_cast<const unsigned char *>(p->val.ptr) + vb * r[0], vb * n,
                               cudaMemcpyDeviceToDevice, s));
  return WPROJ_OK;
}

// ---- batches: the column-format kernels over a batch's concatenated arrays ------

wproj_status batch_degrid(const BatchOps &b, const float2 *Xt, float2 *partial, float2 *y, cudaStream_t s) {
  WPROJ_TRY(launch_degrid_pieces<WPROJ_VAL_F32>(b.n_pieces, b.piece_lo, b.piece_len, b.col, b.val, Xt, partial,
                                                b.lpp, s));
  k_degrid_reduce<<<ceil_div(b.m, 256), 256, 0, s>>>(b.m, b.row_piece_ptr, partial, nullptr, y);
  WPROJ_CHECK_LAUNCH("batch degrid reduce");
  return WPROJ_OK;
}

wproj_status batch_grid(const BatchOps &b, const float2 *y, float2 *partial, float2 *Xt2, cudaStream_t s) {
  if (b.cell_ent) return batch_grid_cells(b, y, Xt2, s);
  const size_t smem = sizeof(float2) * kGridWarps * kTile * kTile;
  WPROJ_CUDA(cudaFuncSetAttribute(k_grid<WPROJ_VAL_F32, kGridWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  k_grid<WPROJ_VAL_F32, kGridWarps><<<(unsigned)b.n_chunks, kGridWarps * 32, smem, s>>>(
      b.chunk_tile, b.chunk_lo, b.chunk_hi, b.meta, b.col, b.val, nullptr, y, 0, kTile, 0, b.chunk_prob, b.tab,
      partial);
  WPROJ_CHECK_LAUNCH("batch grid");
  k_grid_reduce<<<(unsigned)b.n_tiles, 256, 0, s>>>(b.tile_chunk_ptr, partial, 0, kTile, 0, b.tile_prob, b.tab, Xt2);
  WPROJ_CHECK_LAUNCH("batch grid reduce");
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
