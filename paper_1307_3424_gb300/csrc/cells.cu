// Gridding X'[q] = sum_k conj(G[k, q]) y_k for G with column indices, from a
// cell-major copy of G (Eq. 8's adjoint, Section 3.1).
//
// The copy holds, for every 32 x 32 grid tile (ascending), the tile's entries
// sorted by cell and, within a cell, by row: one packed word per entry
// (row << 10 | cell within the tile; rows < 2^22) and its value.  The gridding
// then needs no accumulators: a block owns a tile, its warps take equal slices
// of the tile's entries in windows of 128, a lane four consecutive entries.
// Cells are sorted, so a cell's entries are adjacent: a lane sums its entries
// run by run (a run that begins and ends inside the lane is written at once),
// and the runs open at the lanes' ends are summed across lanes by a segmented
// shuffle scan.  A run of one cell that crosses a window boundary is carried
// to the next window; a run that crosses a warp boundary is merged by thread 0
// in warp order.  Every cell therefore gets a fixed summation order
// (bit-reproducible), each cell is written once, and the tile's empty cells are
// zeroed by the same block.  Grids with few tiles split every tile's entries
// into `parts` contiguous slices, one block each; a block then writes its
// slice's sums into a private 32 x 32 partial tile and the partials are added
// per cell in slice order.
//
// The copy is built from the tile-ordered segment list by a block per tile:
// count entries per cell, scan, then place the segments' entries in segment
// (row) order, one segment at a time.
#include "plan.h"

namespace wproj {

namespace {

constexpr int kCellWarps = 8;
constexpr unsigned kCellMask = 1023u;
constexpr int kCellJ = 4;   // consecutive entries per lane in the gridding

// exclusive scan of v over a block of 1024 threads; returns the thread's prefix
__device__ __forceinline__ int block_excl_scan_1024(int v, int *wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int t = wsum[lane];
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += n;
    }
    wsum[lane] = ti - t;
  }
  __syncthreads();
  return wsum[w] + inc - v;
}

template <int VB>
__global__ void __launch_bounds__(1024)
k_cellsort(const int64_t *__restrict__ tptr, const SegMeta *__restrict__ meta, const int32_t *__restrict__ col,
           const unsigned char *__restrict__ val, const int64_t *__restrict__ tile_ent, int logG, int nT,
           uint32_t *__restrict__ cell_ent, unsigned char *__restrict__ cell_val) {
  __shared__ int cnt[1024];
  __shared__ int base[1024];
  __shared__ int wsum[32];
  const int t = blockIdx.x;
  const int tu = t / nT, tv = t % nT;
  const int Gm = (1 << logG) - 1;
  const int64_t s0 = tptr[t], s1 = tptr[t + 1];
  const int64_t e0 = tile_ent[t];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  auto cell_of = [&](int q) { return (((q >> logG) - tu * 32) << 5) | ((q & Gm) - tv * 32); };
  for (int64_t s = s0; s < s1; ++s) {
    const SegMeta m = meta[s];
    if ((int)threadIdx.x < meta_cnt(m)) atomicAdd(&cnt[cell_of(col[meta_off(m) + threadIdx.x])], 1);
  }
  __syncthreads();
  base[threadIdx.x] = block_excl_scan_1024(cnt[threadIdx.x], wsum);
  cnt[threadIdx.x] = 0;
  __syncthreads();
  // place entries segment by segment (rows ascending); the cells of one segment
  // are distinct, so each cell's counter has one writer per step
  for (int64_t s = s0; s < s1; ++s) {
    const SegMeta m = meta[s];
    if ((int)threadIdx.x < meta_cnt(m)) {
      const int64_t src = meta_off(m) + threadIdx.x;
      const int c = cell_of(col[src]);
      const int64_t dst = e0 + base[c] + cnt[c];
      cnt[c] += 1;
      cell_ent[dst] = (uint32_t(m.row) << 10) | uint32_t(c);
      if constexpr (VB == 8) {
        reinterpret_cast<float2 *>(cell_val)[dst] = reinterpret_cast<const float2 *>(val)[src];
      } else {
        reinterpret_cast<unsigned *>(cell_val)[dst] = reinterpret_cast<const unsigned *>(val)[src];
      }
    }
    __syncthreads();
  }
}

template <int VDT>
__device__ __forceinline__ float2 cell_value(const void *__restrict__ v, int64_t i) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    return __ldg(reinterpret_cast<const float2 *>(v) + i);
  } else if constexpr (VDT == WPROJ_VAL_BF16) {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(v) + i);
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw));
  } else {
    const unsigned raw = __ldg(reinterpret_cast<const unsigned *>(v) + i);
    return __half22float2(*reinterpret_cast<const __half2 *>(&raw));
  }
}

// y_k times the row scale of the 16-bit value forms
__global__ void k_scale_y(int64_t m, const float2 *__restrict__ y, const float *__restrict__ rs,
                          float2 *__restrict__ ys) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < m) ys[k] = cscale(y[k], rs[k]);
}

// y: visibilities, already multiplied by the row scales for 16-bit values.
// tile_prob / tab (batches): blockIdx.x is a tile of the whole batch
template <int VDT>
__global__ void __launch_bounds__(kCellWarps * 32, 4)   // four blocks an SM: 64 registers
k_grid_cells(const int64_t *__restrict__ tile_ent, const uint32_t *__restrict__ cell_ent,
             const void *__restrict__ cell_val, const float2 *__restrict__ y,
             int logG, int nT, const int32_t *__restrict__ tile_prob, const BProb *__restrict__ tab,
             float2 *__restrict__ Xt2, int parts, float2 *__restrict__ partial) {
  __shared__ int h_cell[kCellWarps], t_cell[kCellWarps], h_closed[kCellWarps];
  __shared__ float2 h_val[kCellWarps], t_val[kCellWarps];
  int tile = blockIdx.x, part = 0;
  if (parts > 1) {
    tile = blockIdx.x / parts;
    part = blockIdx.x - tile * parts;
  }
  const int64_t te0 = tile_ent[tile], tn = tile_ent[tile + 1] - te0;
  int64_t e0 = te0, e1 = te0 + tn;
  if (parts > 1) {
    e0 = te0 + tn * part / parts;
    e1 = te0 + tn * (part + 1) / parts;
  }
  if (tile_prob) {
    const BProb &P = tab[tile_prob[tile]];
    logG = P.logG;
    nT = P.nT;
    tile -= int(P.tile_off);
    Xt2 += P.grid_off;
    y += P.vis_off;
  }
  int G = 1 << logG;
  const int tu = tile >> (logG - 5), tv = tile & (nT - 1);   // nT = G / 32
  float2 *out = Xt2 + int64_t(tu * 32) * G + tv * 32;   // cell c at out[(c >> 5) G + (c & 31)]
  if (parts > 1) {                                      // this slice's partial tile (row stride 32)
    out = partial + int64_t(blockIdx.x) * 1024;
    G = 32;
  }
  for (int c = threadIdx.x; c < 1024; c += blockDim.x) out[int64_t(c >> 5) * G + (c & 31)] = make_float2(0.f, 0.f);
  __syncthreads();

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = e1 - e0;
  const int64_t a = e0 + (n * w >> 3), b = e0 + (n * (w + 1) >> 3);
  static_assert(kCellWarps == 8 && kCellJ == 4, "eight warps; a lane takes one 16-byte word of entries");
  constexpr int J = kCellJ, WIN = 32 * J;
  int carry_cell = -1;          // run left open by the previous window
  float2 carry = make_float2(0.f, 0.f);
  bool head_done = false;       // the warp's first run has been closed
  auto cell_of = [](uint32_t e) { return int(e & kCellMask); };
  auto term = [](float2 v, float2 yv) {   // conj(v) y
    return make_float2(v.x * yv.x + v.y * yv.y, v.x * yv.y - v.y * yv.x);
  };
  // Windows start at a multiple of 4 entries at or below a, so that lane l's
  // entries wb + o + 4 l + j (j < 4) are one aligned 16-byte word of entries
  // and one (16-bit values) or two (f32) aligned 16-byte words of values; the
  // arrays carry 4 entries of padding for the last word.  Entries outside
  // [a, b) are loaded but not used.  Offsets within a warp's slice fit 32 bits
  // (a tile holds <= 2^32 entries, rows < 2^22 with <= 1024 cells each, and a
  // warp takes an eighth of a tile at most).
  const int64_t wb = a & ~int64_t(3);
  const int span = int(b - wb);
  const int lo = int(a - wb);
  const uint32_t *__restrict__ ent_w = cell_ent + wb;
  // software pipeline: entries two windows ahead, values and y one window ahead
  auto load_e = [&](int o, uint32_t(&e)[J]) {
    const int li = o + J * lane;
    if (li < span) {
      const uint4 q = __ldg(reinterpret_cast<const uint4 *>(ent_w + li));
      e[0] = q.x; e[1] = q.y; e[2] = q.z; e[3] = q.w;
    } else {
      e[0] = e[1] = e[2] = e[3] = 0u;
    }
  };
  auto load_v = [&](int o, float2(&v)[J]) {
    const int li = o + J * lane;
    if (li < span) {
      if constexpr (VDT == WPROJ_VAL_F32) {
        const float4 *p4 = reinterpret_cast<const float4 *>(static_cast<const float2 *>(cell_val) + wb + li);
        const float4 q0 = __ldg(p4), q1 = __ldg(p4 + 1);
        v[0] = make_float2(q0.x, q0.y); v[1] = make_float2(q0.z, q0.w);
        v[2] = make_float2(q1.x, q1.y); v[3] = make_float2(q1.z, q1.w);
      } else {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(static_cast<const unsigned *>(cell_val) + wb + li));
        const unsigned r[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < J; ++j) {
          if constexpr (VDT == WPROJ_VAL_BF16) v[j] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r[j]));
          else v[j] = __half22float2(*reinterpret_cast<const __half2 *>(&r[j]));
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) v[j] = make_float2(0.f, 0.f);
    }
  };
  auto load_y = [&](int o, const uint32_t(&e)[J], float2(&yv)[J]) {
    const int li = o + J * lane;
#pragma unroll
    for (int j = 0; j < J; ++j)
      yv[j] = (li + j >= lo && li + j < span) ? __ldg(y + (e[j] >> 10)) : make_float2(0.f, 0.f);
  };
  uint32_t ec[J], en[J], ef[J];
  float2 vc[J], vn[J], yc[J], yn[J];
  load_e(0, ec);
  load_e(WIN, en);
  load_v(0, vc);
  load_y(0, ec, yc);
  for (int o = 0; o < span; o += WIN) {
    load_e(o + 2 * WIN, ef);
    load_v(o + WIN, vn);
    load_y(o + WIN, en, yn);
    const int li = o + J * lane;
    const int last_valid = (span - 1 - o) / J < 31 ? (span - 1 - o) / J : 31;
    // Branch-free form over the lane's 4 entries: an entry outside [a, b)
    // takes the cell of its valid neighbour in the lane and the value 0, so it
    // joins that run without changing its sum; a lane without entries takes a
    // cell of its own.
    bool val[J];
    int c[J];
    float2 t[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      val[j] = li + j >= lo && li + j < span;
      c[j] = val[j] ? cell_of(ec[j]) : -1;
      t[j] = val[j] ? term(vc[j], yc[j]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 1; j < J; ++j) c[j] = val[j] ? c[j] : c[j - 1];       // trailing
#pragma unroll
    for (int j = J - 2; j >= 0; --j) c[j] = c[j] >= 0 ? c[j] : c[j + 1];   // leading
    const bool any = c[0] >= 0;
#pragma unroll
    for (int j = 0; j < J; ++j) c[j] = any ? c[j] : 4096 + lane;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      ec[j] = en[j];
      en[j] = ef[j];
      vc[j] = vn[j];
      yc[j] = yn[j];
    }
    // in-lane segmented inclusive sums
    bool bnd[J];
    float2 sj[J];
    bnd[0] = false;
    sj[0] = t[0];
#pragma unroll
    for (int j = 1; j < J; ++j) {
      bnd[j] = c[j] != c[j - 1];
      sj[j] = bnd[j] ? t[j] : cadd(sj[j - 1], t[j]);
    }
    const bool multi = bnd[1] || bnd[2] || bnd[3];
    // does the run open at the previous lane's end (the carry for lane 0) continue here?
    int prev_c = __shfl_up_sync(0xffffffffu, c[J - 1], 1);
    if (lane == 0) prev_c = carry_cell;
    const bool chain_in = any && prev_c == c[0];
    // segmented inclusive scan of the runs open at the lanes' ends; a segment
    // starts at lane 0, at a lane holding a run boundary and at a lane whose
    // first cell is new
    float2 cs = sj[J - 1];
    if (lane == 0 && chain_in && !multi) cs = cadd(carry, cs);
    const bool head = lane == 0 || multi || !chain_in;
    const unsigned hm = __ballot_sync(0xffffffffu, head);
    const int seg = 31 - __clz(hm & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u)));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float ux = __shfl_up_sync(0xffffffffu, cs.x, d);
      const float uy = __shfl_up_sync(0xffffffffu, cs.y, d);
      if (lane - d >= seg) cs = make_float2(ux + cs.x, uy + cs.y);
    }
    // the open run before the lane (the carry for lane 0), added to the lane's first run
    float2 cin = make_float2(__shfl_up_sync(0xffffffffu, cs.x, 1), __shfl_up_sync(0xffffffffu, cs.y, 1));
    if (lane == 0) cin = carry;
    if (!chain_in) cin = make_float2(0.f, 0.f);
    float2 full[J];
    bool first = true;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      first = first && !bnd[j];
      full[j] = first ? cadd(cin, sj[j]) : sj[j];
    }
    // entry j closes its run when the next entry is valid and holds another cell
    const int next_c0 = __shfl_down_sync(0xffffffffu, c[0], 1);
    const bool next_any = __shfl_down_sync(0xffffffffu, any, 1) && lane < 31;
    bool cls[J];
#pragma unroll
    for (int j = 0; j + 1 < J; ++j) cls[j] = val[j] && val[j + 1] && bnd[j + 1];
    cls[J - 1] = val[J - 1] && next_any && next_c0 != c[J - 1];
    if (carry_cell >= 0 && !__shfl_sync(0xffffffffu, chain_in, 0)) {
      // the carried run ended exactly at the window boundary
      if (!head_done) {
        if (lane == 0) {
          h_cell[w] = carry_cell;
          h_val[w] = carry;
          h_closed[w] = 1;
        }
        head_done = true;
      } else if (lane == 0) {
        out[int64_t(carry_cell >> 5) * G + (carry_cell & 31)] = carry;
      }
    }
    // the warp's first closed run may have begun in the previous warp: its
    // first closing entry is recorded instead of written
    int hj = -1;
    const unsigned cm = __ballot_sync(0xffffffffu, cls[0] || cls[1] || cls[2] || cls[3]);
    if (!head_done && cm) {
      if (lane == __ffs(cm) - 1) {
        hj = cls[0] ? 0 : (cls[1] ? 1 : (cls[2] ? 2 : 3));
#pragma unroll
        for (int j = 0; j < J; ++j) {   // static indices: the arrays stay in registers
          if (j == hj) {
            h_cell[w] = c[j];
            h_val[w] = full[j];
          }
        }
        h_closed[w] = 1;
      }
      head_done = true;
    }
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (cls[j] && j != hj) out[int64_t(c[j] >> 5) * G + (c[j] & 31)] = full[j];
    carry_cell = __shfl_sync(0xffffffffu, c[J - 1], last_valid);
    carry.x = __shfl_sync(0xffffffffu, full[J - 1].x, last_valid);
    carry.y = __shfl_sync(0xffffffffu, full[J - 1].y, last_valid);
  }
  if (lane == 0) {
    if (!head_done) h_closed[w] = 0;
    t_cell[w] = (a < b) ? carry_cell : -1;
    t_val[w] = carry;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // merge the runs that cross warp boundaries, in warp order
    int oc = -1;
    float2 ov = make_float2(0.f, 0.f);
    for (int k = 0; k < kCellWarps; ++k) {
      if (t_cell[k] < 0) continue;   // no entries
      if (h_closed[k]) {
        if (oc == h_cell[k]) {
          out[int64_t(oc >> 5) * G + (oc & 31)] = cadd(ov, h_val[k]);
        } else {
          if (oc >= 0) out[int64_t(oc >> 5) * G + (oc & 31)] = ov;
          out[int64_t(h_cell[k] >> 5) * G + (h_cell[k] & 31)] = h_val[k];
        }
        oc = t_cell[k];
        ov = t_val[k];
      } else if (oc == t_cell[k]) {   // one run spans the whole slice
        ov = cadd(ov, t_val[k]);
      } else {
        if (oc >= 0) out[int64_t(oc >> 5) * G + (oc & 31)] = ov;
        oc = t_cell[k];
        ov = t_val[k];
      }
    }
    if (oc >= 0) out[int64_t(oc >> 5) * G + (oc & 31)] = ov;
  }
}

// Xt2 cell = sum of the tile's partial tiles in slice order
__global__ void k_cells_reduce(int n_tiles, int parts, int logG, int nT, const float2 *__restrict__ partial,
                               float2 *__restrict__ Xt2) {
  const int tile = blockIdx.x;
  const int tu = tile / nT, tv = tile % nT;
  for (int c = threadIdx.x; c < 1024; c += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < parts; ++q) acc = cadd(acc, partial[(int64_t(tile) * parts + q) * 1024 + c]);
    Xt2[(int64_t(tu * 32 + (c >> 5)) << logG) + tv * 32 + (c & 31)] = acc;
  }
}

__global__ void k_tile_ent(int n_tiles, const int64_t *__restrict__ tptr, const int64_t *__restrict__ cum,
                           int64_t n_seg, int64_t nnz, int64_t *__restrict__ tile_ent) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  const int64_t s = tptr[t];
  tile_ent[t] = s < n_seg ? cum[s] : nnz;
}

}  // namespace

// Cell-major copy of a plan's column-format G (needs p->m <= 2^22, the tile
// segment list in p->seg_meta and its tile ranges tptr with entry prefix cum).
wproj_status build_cells(wproj_plan *p, const int64_t *tptr, const int64_t *cum, int64_t n_seg, cudaStream_t s) {
  const int n_tiles = p->g.nT * p->g.nT;
  const int vb = p->g.value_dtype == WPROJ_VAL_F32 ? 8 : 4;
  WPROJ_TRY(p->tile_ent.alloc(sizeof(int64_t) * (n_tiles + 1)));
  // 4 entries of padding: the gridding reads whole 16-byte words of 4 entries
  WPROJ_TRY(p->cell_ent.alloc(sizeof(uint32_t) * (p->nnz + kCellPad)));
  WPROJ_TRY(p->cell_val.alloc(int64_t(vb) * (p->nnz + kCellPad)));
  k_tile_ent<<<ceil_div(n_tiles + 1, 256), 256, 0, s>>>(n_tiles, tptr, cum, n_seg, p->nnz,
                                                       p->tile_ent.as<int64_t>());
  WPROJ_CHECK_LAUNCH("tile entries");
  const int logG = ilog2(p->g.G);
  if (vb == 8) {
    k_cellsort<8><<<n_tiles, 1024, 0, s>>>(tptr, p->seg_meta.as<SegMeta>(), p->col.as<int32_t>(),
                                          p->val.as<unsigned char>(), p->tile_ent.as<int64_t>(), logG, p->g.nT,
                                          p->cell_ent.as<uint32_t>(), p->cell_val.as<unsigned char>());
  } else {
    k_cellsort<4><<<n_tiles, 1024, 0, s>>>(tptr, p->seg_meta.as<SegMeta>(), p->col.as<int32_t>(),
                                          p->val.as<unsigned char>(), p->tile_ent.as<int64_t>(), logG, p->g.nT,
                                          p->cell_ent.as<uint32_t>(), p->cell_val.as<unsigned char>());
  }
  WPROJ_CHECK_LAUNCH("cell sort");
  // small grids: split every tile over several blocks so that the SMs fill
  // (about six blocks per SM, each slice at least 4096 entries)
  const int64_t want = (152 * 6 + n_tiles - 1) / n_tiles;
  const int64_t cap = std::max<int64_t>(1, p->nnz / (int64_t(n_tiles) * 4096));
  p->cell_parts = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, cap), 64));
  if (p->cell_parts > 1) {
    WPROJ_TRY(p->cell_partial.alloc(sizeof(float2) * size_t(n_tiles) * p->cell_parts * 1024));
  } else {
    p->cell_partial.release();
  }
  return WPROJ_OK;
}

namespace {
// first segment of every tile from the plan's chunk list
__global__ void k_tptr_from_chunks(int n_tiles, const int64_t *__restrict__ chunk_lo,
                                   const int32_t *__restrict__ tile_chunk_ptr, int64_t n_seg,
                                   int64_t *__restrict__ tptr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_tiles) tptr[t] = chunk_lo[tile_chunk_ptr[t]];
  if (t == n_tiles) tptr[t] = n_seg;
}
}  // namespace

// Refresh the cell-major copy after the row-major values changed (same support).
wproj_status rebuild_cells(wproj_plan *p, cudaStream_t s) {
  if (!p->has_cells) return WPROJ_OK;
  const int n_tiles = p->g.nT * p->g.nT;
  DevBuf tptr;
  WPROJ_TRY(tptr.alloc(sizeof(int64_t) * (n_tiles + 1)));
  k_tptr_from_chunks<<<ceil_div(n_tiles + 1, 256), 256, 0, s>>>(n_tiles, p->chunk_lo.as<int64_t>(),
                                                               p->tile_chunk_ptr.as<int32_t>(), p->n_seg,
                                                               tptr.as<int64_t>());
  WPROJ_CHECK_LAUNCH("tile ranges");
  const int logG = ilog2(p->g.G);
  if (p->g.value_dtype == WPROJ_VAL_F32) {
    k_cellsort<8><<<n_tiles, 1024, 0, s>>>(tptr.as<int64_t>(), p->seg_meta.as<SegMeta>(), p->col.as<int32_t>(),
                                          p->val.as<unsigned char>(), p->tile_ent.as<int64_t>(), logG, p->g.nT,
                                          p->cell_ent.as<uint32_t>(), p->cell_val.as<unsigned char>());
  } else {
    k_cellsort<4><<<n_tiles, 1024, 0, s>>>(tptr.as<int64_t>(), p->seg_meta.as<SegMeta>(), p->col.as<int32_t>(),
                                          p->val.as<unsigned char>(), p->tile_ent.as<int64_t>(), logG, p->g.nT,
                                          p->cell_ent.as<uint32_t>(), p->cell_val.as<unsigned char>());
  }
  WPROJ_CHECK_LAUNCH("cell sort");
  WPROJ_CUDA(cudaStreamSynchronize(s));
  return WPROJ_OK;
}

wproj_status grid_cells(wproj_plan *p, const float2 *y, float2 *Xt2, cudaStream_t s) {
  const int n_tiles = p->g.nT * p->g.nT;
  const int logG = ilog2(p->g.G);
  if (p->g.value_dtype != WPROJ_VAL_F32) {
    k_scale_y<<<ceil_div(p->m, 256), 256, 0, s>>>(p->m, y, p->row_scale.as<float>(), p->ytmp.as<float2>());
    WPROJ_CHECK_LAUNCH("scaled visibilities");
    y = p->ytmp.as<float2>();
    p->launches += 1;
  }
  const int parts = p->cell_parts;
  float2 *partial = parts > 1 ? p->cell_partial.as<float2>() : nullptr;
#define GC(VDT)                                                                                                  \
  k_grid_cells<VDT><<<n_tiles * parts, kCellWarps * 32, 0, s>>>(p->tile_ent.as<int64_t>(),                      \
                                                                p->cell_ent.as<uint32_t>(), p->cell_val.ptr, y, \
                                                                logG, p->g.nT, nullptr, nullptr, Xt2, parts, partial)
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: GC(WPROJ_VAL_F32); break;
    case WPROJ_VAL_BF16: GC(WPROJ_VAL_BF16); break;
    default: GC(WPROJ_VAL_F16);
  }
#undef GC
  WPROJ_CHECK_LAUNCH("grid (cells)");
  if (parts > 1) {
    k_cells_reduce<<<n_tiles, 256, 0, s>>>(n_tiles, parts, logG, p->g.nT, partial, Xt2);
    WPROJ_CHECK_LAUNCH("grid (cells) partial tiles");
    p->launches += 1;
  }
  return WPROJ_OK;
}

wproj_status batch_grid_cells(const BatchOps &b, const float2 *y, float2 *Xt2, cudaStream_t s) {
  k_grid_cells<WPROJ_VAL_F32><<<(unsigned)b.n_tiles, kCellWarps * 32, 0, s>>>(
      b.tile_ent, b.cell_ent, b.cell_val, y, 0, 0, b.tile_prob, b.tab, Xt2, 1, nullptr);
  WPROJ_CHECK_LAUNCH("batch grid (cells)");
  return WPROJ_OK;
}

}  // namespace wproj
