// Degridding and gridding for G in the run-length format (TILE_RUNS), for plans
// whose kernel boxes are at most 64 x 64 cells (the box rule's small kernels).
//
// A small w-kernel holds its kept entries in one contiguous run of cells per
// grid row of its box (on the precision-form workload: 283 entries per row in
// 16.6 runs over 16.6 grid rows).  A run costs a 2- or 4-byte descriptor where
// column indices cost 4 bytes per entry, as much as a bf16 complex value, so
// run descriptors shrink the index to a few per cent of the value bytes.
//
// Every run is stored padded to an even length by one zero value, so that a
// lane always takes two consecutive entries of one run (one 8-byte load of
// two bf16/f16 pairs or one 16-byte load of two f32 pairs).  For a chunk of 64
// padded entries of a window of <= 32 runs held one per lane, lane l takes the
// entries i0 + 2l and i0 + 2l + 1; its run is the number of runs of the window
// that end at or before i0 + 2l, i.e. a popcount of the OR-reduced bit mask of
// the run ends that fall inside the chunk.
//
// Two copies of the values:
//   row-major (degridding)   per row k: window origin a = (j0 - S/2) mod G per
//       axis (rm_org), runs in window order (rm_run: window row dr, window column
//       dc of the first entry, true length - 1), values run after run (rm_val,
//       first value of row k at rm_vptr[k], first run at rm_rptr[k]).  A warp
//       takes a row, gathers X from L2 and writes y_k: no partial sums.
//   tile-major records (gridding and row export)  for every 32 x 32 grid tile
//       (ascending) and every row with entries in it (rows ascending) one
//       16-byte-aligned record: int32 row, uint16 stored count, uint16 runs;
//       the runs as uint16 (tile column of the first entry | (length - 1) << 5 |
//       tile row << 10), zero-padded to 16 bytes; the values, zero-padded to 16
//       bytes.  A record's values are its segment's entries in CSR order (row-
//       major inside the tile) with the run pads.  A block of 4 warps takes a
//       chunk of one tile's records; each warp accumulates its records into a
//       private 32 x 33 shared-memory tile (column 32 takes the pads' zeros),
//       and the four tiles are summed in warp order.  Tiles split over several
//       chunks are summed in chunk order afterwards.
//
// No atomics in the operators: results are bit-reproducible.
#include "plan.h"

namespace wproj {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRecHdr = 8;          // int32 row, uint16 stored count, uint16 runs
constexpr int kGridWarps = 4;       // warps per gridding block
constexpr int kTileStride = 34;     // shared-memory tile row (pairs stay 16-byte aligned, rows shift banks)
constexpr int kMaxRuns = 64;        // runs of one row or record (two per lane)

__host__ __device__ __forceinline__ int64_t runs_rec_bytes(int nruns, int pcount, int vb) {
  return int64_t((kRecHdr + 4 * nruns + 15) & ~15) + ((int64_t(pcount) * vb + 15) & ~15);
}
__host__ __device__ __forceinline__ int rec_values_at(int nruns) { return (kRecHdr + 4 * nruns + 15) & ~15; }

__device__ __forceinline__ int warp_incl_scan_i(int v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += n;
  }
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---- run lookup for a chunk of 128 stored entries -------------------------------------
//
// The runs of one row (or record), at most 64, are held two per lane: lane j
// holds runs j (lo) and j + 32 (hi) as words with their first stored position P
// in the high bits, and their end E (first stored position after the run).
// Every run is stored with an even length, so a chunk of 128 stored entries is
// 64 pairs; lane l takes pairs l and l + 32, so that each load or store
// instruction covers 32 consecutive pairs.  A pair's run is the number of runs
// ending at or before it: `base` (runs ending at or before the chunk) plus the
// popcount of the chunk's run-end mask (bit e: a run ends at pair e) up to it.

struct RunPair {
  uint32_t wlo, whi;   // run words (0 past the last run)
  int Elo, Ehi;        // run ends (stored positions)
  bool vlo, vhi;
};

__device__ __forceinline__ void pair_runs(const RunPair &R, int i0, int lane, uint32_t &qA, uint32_t &qB) {
  const int dl = R.Elo - i0, dh = R.Ehi - i0;
  unsigned long long b = 0ull;
  if (R.vlo && dl > 0 && dl < 128) b |= 1ull << (dl >> 1);
  if (R.vhi && dh > 0 && dh < 128) b |= 1ull << (dh >> 1);
  const unsigned lo = __reduce_or_sync(kFull, unsigned(b)), hi = __reduce_or_sync(kFull, unsigned(b >> 32));
  const int base = __popc(__ballot_sync(kFull, R.vlo && dl <= 0)) + __popc(__ballot_sync(kFull, R.vhi && dh <= 0));
  const int rA = base + __popc(lo & ((2u << lane) - 1u));
  const int rB = base + __popc(lo) + __popc(hi & ((2u << lane) - 1u));
  const uint32_t a0 = __shfl_sync(kFull, R.wlo, rA & 31), a1 = __shfl_sync(kFull, R.whi, rA & 31);
  const uint32_t b0 = __shfl_sync(kFull, R.wlo, rB & 31), b1 = __shfl_sync(kFull, R.whi, rB & 31);
  qA = rA < 32 ? a0 : a1;
  qB = rB < 32 ? b0 : b1;
}

// two consecutive stored values (8-byte aligned for 16-bit pairs, 16 for f32)
template <int VDT>
__device__ __forceinline__ void load_pair(const unsigned char *p, float2 &a, float2 &b) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    const float4 u = __ldg(reinterpret_cast<const float4 *>(p));
    a = make_float2(u.x, u.y);
    b = make_float2(u.z, u.w);
  } else {
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    if constexpr (VDT == WPROJ_VAL_BF16) {
      a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
      b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    } else {
      a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
      b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    }
  }
}

__device__ __forceinline__ void cfma(float2 &acc, float2 g, float2 x) {
  acc.x += g.x * x.x - g.y * x.y;
  acc.y += g.x * x.y + g.y * x.x;
}

// ---- degridding: warp per row of the row-major copy ---------------------------------

// NC chunks of one row: lane l's pairs l and l + 32 of each chunk
template <int VDT, int NC>
__device__ __forceinline__ void degrid_step(const RunPair &R, int i0, int lane, int pc, int au, int av, int Gm,
                                            int logG, const unsigned char *vb, const float4 *__restrict__ X4,
                                            float2 &acc) {
  constexpr int VB = VDT == WPROJ_VAL_F32 ? 8 : 4;
  uint32_t q[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) pair_runs(R, i0 + 128 * c, lane, q[2 * c], q[2 * c + 1]);
  float2 g[2 * NC][2];
  float4 x[2 * NC];
#pragma unroll
  for (int u = 0; u < 2 * NC; ++u) {
    const int pu = i0 + 2 * lane + 64 * u;
    const bool ok = pu < pc;
    const int dc = int((q[u] >> 6) & 63u);
    const int col = ok ? av + dc - ((av + dc) & 1) + pu - int(q[u] >> 18) : 0;
    load_pair<VDT>(vb + int64_t(ok ? pu : 0) * VB, g[u][0], g[u][1]);
    x[u] = X4[(((au + int(q[u] & 63u)) & Gm) << (logG - 1)) + ((col & Gm) >> 1)];
    if (!ok) x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < 2 * NC; ++u) {
    cfma(acc, g[u][0], make_float2(x[u].x, x[u].y));
    cfma(acc, g[u][1], make_float2(x[u].z, x[u].w));
  }
}
//
// A warp takes tasks of 32 consecutive rows (lane t loads row t's offsets and
// origin) and walks the rows one by one in chunks of 128 stored entries, a
// quad per lane: one 16-byte (bf16/f16) or two 16-byte (f32) value loads and
// four gathers of X, which sit on one or two grid rows per pair, so neighbouring
// lanes read neighbouring cells.

template <int VDT>
__global__ void __launch_bounds__(256, 4)
k_runs_degrid(int64_t m, const int64_t *__restrict__ vptr, const int64_t *__restrict__ rptr,
              const uint32_t *__restrict__ org, const uint32_t *__restrict__ runs,
              const unsigned char *__restrict__ val, const float *__restrict__ row_scale,
              const float2 *__restrict__ X, int logG, float2 *__restrict__ y) {
  constexpr int VB = VDT == WPROJ_VAL_F32 ? 8 : 4;
  const int lane = threadIdx.x & 31;
  const int Gm = (1 << logG) - 1;
  const float4 *__restrict__ X4 = reinterpret_cast<const float4 *>(X);
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ntask = (m + 31) >> 5;
  for (int64_t task = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nw) {
    const int64_t kb = task << 5;
    const int nrows = int(min(int64_t(32), m - kb));
    const int64_t kl = kb + min(lane, nrows - 1);
    const long long v0_l = vptr[kl];
    const int pc_l = int(vptr[kl + 1] - v0_l);
    const long long r0_l = rptr[kl];
    const int nr_l = int(rptr[kl + 1] - r0_l);
    const uint32_t org_l = __ldg(org + kl);
    // the runs of row t + 1 are loaded while row t is reduced
    uint32_t nlo = 0u, nhi = 0u;
    {
      const long long r0 = __shfl_sync(kFull, r0_l, 0);
      const int nr = __shfl_sync(kFull, nr_l, 0);
      if (lane < nr) nlo = __ldg(runs + r0 + lane);
      if (lane + 32 < nr) nhi = __ldg(runs + r0 + 32 + lane);
    }
    float2 yout = make_float2(0.f, 0.f);
    for (int t = 0; t < nrows; ++t) {
      const long long v0 = __shfl_sync(kFull, v0_l, t);
      const int nr = __shfl_sync(kFull, nr_l, t), pc = __shfl_sync(kFull, pc_l, t);
      const uint32_t o = __shfl_sync(kFull, org_l, t);
      const int au = int(o & 0xffffu), av = int(o >> 16);
      RunPair R;
      R.vlo = lane < nr;
      R.vhi = lane + 32 < nr;
      R.wlo = nlo;
      R.whi = nhi;
      if (t + 1 < nrows) {
        const long long r0n = __shfl_sync(kFull, r0_l, t + 1);
        const int nrn = __shfl_sync(kFull, nr_l, t + 1);
        nlo = lane < nrn ? __ldg(runs + r0n + lane) : 0u;
        nhi = lane + 32 < nrn ? __ldg(runs + r0n + 32 + lane) : 0u;
      }
      // end = start + stored length: the run's length plus its left pad (when its
      // first column is odd), rounded up to even
      R.Elo = R.vlo ? int(R.wlo >> 18) + ((int((R.wlo >> 12) & 63u) + 2 + int((av + (R.wlo >> 6)) & 1u)) & ~1) : 0;
      R.Ehi = R.vhi ? int(R.whi >> 18) + ((int((R.whi >> 12) & 63u) + 2 + int((av + (R.whi >> 6)) & 1u)) & ~1) : 0;
      const unsigned char *vb = val + v0 * VB;
      float2 acc = make_float2(0.f, 0.f);
      // steps of two chunks (four pairs per lane) while the row has more than
      // one chunk left, then one; every load of a step is issued before its
      // first product (indices past the row are clamped to its first pair and
      // their products dropped)
      int i0 = 0;
      for (; i0 + 128 < pc; i0 += 256) degrid_step<VDT, 2>(R, i0, lane, pc, au, av, Gm, logG, vb, X4, acc);
      if (i0 < pc) degrid_step<VDT, 1>(R, i0, lane, pc, au, av, Gm, logG, vb, X4, acc);
      for (int sft = 16; sft; sft >>= 1) {
        acc.x += __shfl_xor_sync(kFull, acc.x, sft);
        acc.y += __shfl_xor_sync(kFull, acc.y, sft);
      }
      if (lane == t) yout = acc;
    }
    if (lane < nrows) y[kb + lane] = row_scale ? cscale(yout, __ldg(row_scale + kb + lane)) : yout;
  }
}

// ---- gridding: a chunk of one tile's records per block -----------------------------
//
// Warp w takes the w-th quarter of the chunk's records, in groups of 32 (lane t
// loads record t's offset, header and y value), and accumulates each record
// into its private shared-memory tile, a quad of stored entries per lane.

template <int VDT>
__global__ void __launch_bounds__(kGridWarps * 32)
k_runs_grid(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
            const int64_t *__restrict__ chunk_hi, const int32_t *__restrict__ tile_chunk_ptr,
            const int64_t *__restrict__ rec_off, const unsigned char *__restrict__ stream,
            const float *__restrict__ row_scale, const float2 *__restrict__ y, int logG, int nT,
            float2 *__restrict__ partial, float2 *__restrict__ Xt2) {
  constexpr int VB = VDT == WPROJ_VAL_F32 ? 8 : 4;
  __shared__ __align__(16) float2 acc[kGridWarps][32 * kTileStride];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2 *a = acc[w];
  float4 *a4 = reinterpret_cast<float4 *>(a);
  for (int i = lane; i < 32 * kTileStride; i += 32) a[i] = make_float2(0.f, 0.f);
  __syncwarp();
  const int c = blockIdx.x;
  const int64_t clo = chunk_lo[c], chi = chunk_hi[c], cn = chi - clo;
  const int64_t lo = clo + cn * w / kGridWarps, hi = clo + cn * (w + 1) / kGridWarps;
  for (int64_t gb = lo; gb < hi; gb += 32) {
    const int nrec = int(min(int64_t(32), hi - gb));
    const int64_t il = gb + min(lane, nrec - 1);
    const long long off_l = rec_off[il];
    const int2 hdr_l = __ldg(reinterpret_cast<const int2 *>(stream + off_l));
    float2 y_l = __ldg(y + hdr_l.x);
    if (row_scale) y_l = cscale(y_l, __ldg(row_scale + hdr_l.x));
    // record t + 1's runs and first chunk of values are loaded while record t
    // is accumulated
    uint32_t nwl = 0u, nwh = 0u;
    float2 nv[4];
    auto fetch = [&](int tt) {
      const long long o2 = __shfl_sync(kFull, off_l, tt);
      const int h2 = __shfl_sync(kFull, hdr_l.y, tt);
      const int nr2 = int(unsigned(h2) >> 16), pc2 = h2 & 0xffff;
      const unsigned char *r2 = stream + o2;
      const uint32_t *w2 = reinterpret_cast<const uint32_t *>(r2 + kRecHdr);
      nwl = lane < nr2 ? __ldg(w2 + lane) : 0u;
      nwh = lane + 32 < nr2 ? __ldg(w2 + 32 + lane) : 0u;
      const unsigned char *v2 = r2 + rec_values_at(nr2);
      load_pair<VDT>(v2 + int64_t(2 * lane < pc2 ? 2 * lane : 0) * VB, nv[0], nv[1]);
      load_pair<VDT>(v2 + int64_t(2 * lane + 64 < pc2 ? 2 * lane + 64 : 0) * VB, nv[2], nv[3]);
    };
    fetch(0);
    for (int t = 0; t < nrec; ++t) {
      const long long off = __shfl_sync(kFull, off_l, t);
      const int hy = __shfl_sync(kFull, hdr_l.y, t);
      const int nr = int(unsigned(hy) >> 16), pc = hy & 0xffff;
      const float2 yk = make_float2(__shfl_sync(kFull, y_l.x, t), __shfl_sync(kFull, y_l.y, t));
      const unsigned char *vals = stream + off + rec_values_at(nr);
      // record run word: tile column | (length - 1) << 5 | tile row << 10 | P << 16
      RunPair R;
      R.vlo = lane < nr;
      R.vhi = lane + 32 < nr;
      R.wlo = nwl;
      R.whi = nwh;
      const float2 f0 = nv[0], f1 = nv[1], f2 = nv[2], f3 = nv[3];
      if (t + 1 < nrec) fetch(t + 1);
      R.Elo = R.vlo ? int(R.wlo >> 16) + ((int((R.wlo >> 5) & 31u) + 2 + int(R.wlo & 1u)) & ~1) : 0;
      R.Ehi = R.vhi ? int(R.whi >> 16) + ((int((R.whi >> 5) & 31u) + 2 + int(R.whi & 1u)) & ~1) : 0;
      for (int i0 = 0; i0 < pc; i0 += 128) {
        uint32_t qA, qB;
        pair_runs(R, i0, lane, qA, qB);
        // a stored pair starts on an even tile column: one 16-byte read-modify-write;
        // both pairs' loads are issued first (indices past the record clamped)
        const int pA = i0 + 2 * lane, pB = pA + 64;
        const bool okA = pA < pc, okB = pB < pc;
        float2 ga0, ga1, gb0, gb1;
        if (i0 == 0) {   // prefetched with the record
          ga0 = f0; ga1 = f1; gb0 = f2; gb1 = f3;
        } else {
          load_pair<VDT>(vals + int64_t(okA ? pA : 0) * VB, ga0, ga1);
          load_pair<VDT>(vals + int64_t(okB ? pB : 0) * VB, gb0, gb1);
        }
        if (okA) {
          const int cell = int((qA >> 10) & 31u) * kTileStride + int(qA & 30u) + (pA - int(qA >> 16));
          float4 s4 = a4[cell >> 1];
          s4.x += ga0.x * yk.x + ga0.y * yk.y;
          s4.y += ga0.x * yk.y - ga0.y * yk.x;
          s4.z += ga1.x * yk.x + ga1.y * yk.y;
          s4.w += ga1.x * yk.y - ga1.y * yk.x;
          a4[cell >> 1] = s4;
        }
        if (okB) {
          const int cell = int((qB >> 10) & 31u) * kTileStride + int(qB & 30u) + (pB - int(qB >> 16));
          float4 s4 = a4[cell >> 1];
          s4.x += gb0.x * yk.x + gb0.y * yk.y;
          s4.y += gb0.x * yk.y - gb0.y * yk.x;
          s4.z += gb1.x * yk.x + gb1.y * yk.y;
          s4.w += gb1.x * yk.y - gb1.y * yk.x;
          a4[cell >> 1] = s4;
        }
      }
    }
  }
  __syncthreads();
  const int t = chunk_tile[c];
  const bool single = tile_chunk_ptr[t + 1] - tile_chunk_ptr[t] == 1;
  const int tu = t / nT, tv = t % nT;
  for (int e = threadIdx.x; e < 1024; e += kGridWarps * 32) {
    const int r = e >> 5, cc = e & 31, at = r * kTileStride + cc;
    float2 s = acc[0][at];
#pragma unroll
    for (int q = 1; q < kGridWarps; ++q) s = cadd(s, acc[q][at]);
    if (single) Xt2[(int64_t(tu * 32 + r) << logG) + tv * 32 + cc] = s;
    else partial[int64_t(c) * 1024 + e] = s;
  }
}

// tiles split over several chunks: their partial tiles summed in chunk order
__global__ void __launch_bounds__(256)
k_runs_grid_reduce(const int32_t *__restrict__ tile_chunk_ptr, const float2 *__restrict__ partial, int logG, int nT,
                   float2 *__restrict__ Xt2) {
  const int t = blockIdx.x;
  const int c0 = tile_chunk_ptr[t], c1 = tile_chunk_ptr[t + 1];
  if (c1 - c0 <= 1) return;
  const int tu = t / nT, tv = t % nT;
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int c = c0; c < c1; ++c) s = cadd(s, partial[int64_t(c) * 1024 + e]);
    Xt2[(int64_t(tu * 32 + (e >> 5)) << logG) + tv * 32 + (e & 31)] = s;
  }
}

// ---- rows of G in CSR order from the records ------------------------------------------

__global__ void k_runs_export(int64_t s0, int64_t s1, int64_t first, const int64_t *__restrict__ seg_rec,
                              const int64_t *__restrict__ seg_off, const int32_t *__restrict__ seg_tile,
                              const unsigned char *__restrict__ stream, int vb, int logG, int nT,
                              int32_t *__restrict__ col_out, unsigned char *__restrict__ val_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t sg = s0 + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); sg < s1; sg += nw) {
    if (seg_rec[sg] < 0) continue;   // an empty segment has no record
    const unsigned char *rp = stream + seg_rec[sg];
    const int nr = int(unsigned(reinterpret_cast<const int2 *>(rp)->y) >> 16);
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(rp + kRecHdr);
    const unsigned char *vals = rp + rec_values_at(nr);
    const int tile = seg_tile[sg];
    const int tu = tile / nT, tv = tile % nT;
    const int64_t o = seg_off[sg] - first;
    int tw = 0, pw = 0;   // true and padded entries before the window
    for (int j0 = 0; j0 < nr; j0 += 32) {
      const bool valid = j0 + lane < nr;
      const uint32_t wd = valid ? uint32_t(rw[j0 + lane]) : 0u;
      const int len = valid ? int((wd >> 5) & 31u) + 1 : 0;
      const int lp = valid ? int(wd & 1u) : 0;   // a pad before runs that start on an odd column
      const int plen = (len + lp + 1) & ~1;
      const int T = warp_incl_scan_i(len, lane), E = warp_incl_scan_i(plen, lane);
      if (valid) {
        const int c0 = int(wd & 31u), tr = int((wd >> 10) & 31u);
        const int ti = tw + T - len, pi = pw + E - plen + lp;
        for (int i = 0; i < len; ++i) {
          if (col_out) col_out[o + ti + i] = ((tu * 32 + tr) << logG) + tv * 32 + c0 + i;
          if (val_out) {
            const unsigned char *src = vals + int64_t(pi + i) * vb;
            if (vb == 8) reinterpret_cast<float2 *>(val_out)[o + ti + i] = *reinterpret_cast<const float2 *>(src);
            else reinterpret_cast<unsigned *>(val_out)[o + ti + i] = *reinterpret_cast<const unsigned *>(src);
          }
        }
      }
      tw += __shfl_sync(kFull, T, 31);
      pw += __shfl_sync(kFull, E, 31);
    }
  }
}

// ---- transcoding from the column form ----------------------------------------------------

// Runs of one window row (bit b = column b; par = parity of the absolute grid
// column of bit 0): the number of runs, the stored entries (every run padded
// with zeros to start on an even absolute column and to an even length), and
// the masks of the first entries that get a pad before them (lpad) and of the
// last entries that get one after them (rpad).  An entry at bit c is stored at
// popc(w & lt) + popc(lpad & le) + popc(rpad & lt) of its row, lt / le the bits
// below / up to c.
__device__ __forceinline__ void row_runs64(unsigned long long w, int par, int &nr, int &pc, unsigned long long &lpad,
                                           unsigned long long &rpad) {
  unsigned long long st = w & ~(w << 1), en = w & ~(w >> 1);
  nr = __popcll(st);
  pc = __popcll(w);
  lpad = rpad = 0;
  while (st) {
    const int b0 = __ffsll((long long)st) - 1, b1 = __ffsll((long long)en) - 1;
    const int lp = (b0 + par) & 1;
    if (lp) { lpad |= 1ull << b0; ++pc; }
    if ((b1 - b0 + 1 + lp) & 1) { rpad |= 1ull << b1; ++pc; }
    st &= st - 1;
    en &= en - 1;
  }
}
__device__ __forceinline__ void row_runs32(unsigned w, int &nr, int &pc, unsigned &lpad, unsigned &rpad) {
  unsigned st = w & ~(w << 1), en = w & ~(w >> 1);
  nr = __popc(st);
  pc = __popc(w);
  lpad = rpad = 0;
  while (st) {
    const int b0 = __ffs(int(st)) - 1, b1 = __ffs(int(en)) - 1;
    const int lp = b0 & 1;   // tiles start on even columns
    if (lp) { lpad |= 1u << b0; ++pc; }
    if ((b1 - b0 + 1 + lp) & 1) { rpad |= 1u << b1; ++pc; }
    st &= st - 1;
    en &= en - 1;
  }
}

// Row-major copy, block of 64 threads per row (thread t = window row t).
// Pass 1 (out_pc != null): stored entries (runs padded to even lengths, the row
// to a multiple of 4) and runs per row; err |= 1 for a row of more than
// kMaxRuns runs.  Pass 2: run words (with each run's first stored position),
// origin and values (rm_val zeroed beforehand: the pads stay zero).
__global__ void __launch_bounds__(64)
k_rm_build(int64_t m, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
           const unsigned char *__restrict__ val, int vb, const int2 *__restrict__ j0, const int32_t *__restrict__ Sk,
           int logG, int32_t *__restrict__ out_pc, int32_t *__restrict__ out_nr, int *__restrict__ err,
           const int64_t *__restrict__ vptr,
           const int64_t *__restrict__ rptr, uint32_t *__restrict__ org, uint32_t *__restrict__ runs,
           unsigned char *__restrict__ rm_val) {
  __shared__ unsigned long long bm[64], lpad_s[64], rpad_s[64];
  __shared__ int pbase[64];
  __shared__ int red[4];
  const int t = threadIdx.x, lane = t & 31;
  const int G = 1 << logG, Gm = G - 1;
  for (int64_t k = blockIdx.x; k < m; k += gridDim.x) {
    const int S = Sk[k];
    const int au = (j0[k].x - S / 2) & Gm, av = (j0[k].y - S / 2) & Gm;
    bm[t] = 0;
    __syncthreads();
    const int64_t e0 = row_ptr[k], e1 = row_ptr[k + 1];
    for (int64_t e = e0 + t; e < e1; e += 64) {
      const int q = col[e];
      const int du = ((q >> logG) - au) & Gm, dv = ((q & Gm) - av) & Gm;
      atomicOr(&bm[du], 1ull << dv);
    }
    __syncthreads();
    const unsigned long long wv = bm[t];
    int nr, pc;
    unsigned long long lpm, rpm;
    row_runs64(wv, av & 1, nr, pc, lpm, rpm);
    if (out_pc) {
      const int a = warp_sum_i(pc), b = warp_sum_i(nr);
      if (lane == 0) { red[2 * (t >> 5)] = a; red[2 * (t >> 5) + 1] = b; }
      __syncthreads();
      if (t == 0) {
        out_pc[k] = red[0] + red[2];
        out_nr[k] = red[1] + red[3];
        if (red[1] + red[3] > kMaxRuns) atomicOr(err, 1);
      }
      __syncthreads();
      continue;
    }
    // exclusive prefixes over the 64 window rows
    const int ip = warp_incl_scan_i(pc, lane), ir = warp_incl_scan_i(nr, lane);
    if (lane == 31) { red[2 * (t >> 5)] = ip; red[2 * (t >> 5) + 1] = ir; }
    __syncthreads();
    const int pb = ip - pc + (t >= 32 ? red[0] : 0);
    int rb = ir - nr + (t >= 32 ? red[1] : 0);
    pbase[t] = pb;
    lpad_s[t] = lpm;
    rpad_s[t] = rpm;
    {
      uint32_t *rr = runs + rptr[k];
      unsigned long long st = wv & ~(wv << 1), en = wv & ~(wv >> 1);
      int pp = pb;   // stored position of the run's first (padded) entry
      while (st) {
        const int b0 = __ffsll((long long)st) - 1, b1 = __ffsll((long long)en) - 1;
        const int len = b1 - b0 + 1, lp = (av + b0) & 1;
        rr[rb++] = uint32_t(t) | (uint32_t(b0) << 6) | (uint32_t(len - 1) << 12) | (uint32_t(pp) << 18);
        pp += (len + lp + 1) & ~1;
        st &= st - 1;
        en &= en - 1;
      }
    }
    if (t == 0) org[k] = uint32_t(au) | (uint32_t(av) << 16);
    __syncthreads();
    unsigned char *dst = rm_val + vptr[k] * vb;
    for (int64_t e = e0 + t; e < e1; e += 64) {
      const int q = col[e];
      const int du = ((q >> logG) - au) & Gm, dv = ((q & Gm) - av) & Gm;
      const unsigned long long lt = (1ull << dv) - 1ull;
      const int pos = pbase[du] + __popcll(bm[du] & lt) + __popcll(lpad_s[du] & (lt | (lt + 1))) +
                      __popcll(rpad_s[du] & lt);
      if (vb == 8) reinterpret_cast<float2 *>(dst)[pos] = reinterpret_cast<const float2 *>(val)[e];
      else reinterpret_cast<unsigned *>(dst)[pos] = reinterpret_cast<const unsigned *>(val)[e];
    }
    __syncthreads();
  }
}

// Tile-major records, warp per segment.  Pass 1 (out_bytes != null): record
// bytes per segment (stored count padded to a multiple of 4); err |= 1 for a
// segment of more than kMaxRuns runs.  Pass 2: header, runs and values (stream
// zeroed beforehand).
__global__ void __launch_bounds__(256)
k_tr_build(int64_t n_seg, const int64_t *__restrict__ seg_off, const int32_t *__restrict__ seg_cnt,
           const int32_t *__restrict__ seg_row, const int32_t *__restrict__ seg_tile, const int32_t *__restrict__ col,
           const unsigned char *__restrict__ val, int vb, int logG, int nT, int32_t *__restrict__ out_bytes,
           const int64_t *__restrict__ seg_rec, unsigned char *__restrict__ stream, int *__restrict__ err) {
  __shared__ unsigned bm[8][32], lpad_s[8][32], rpad_s[8][32];
  __shared__ int pbase[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int Gm = (1 << logG) - 1;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t sg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; sg < n_seg; sg += nw) {
    bm[w][lane] = 0;
    __syncwarp();
    const int tile = seg_tile[sg];
    const int tu = tile / nT, tv = tile % nT;
    const int64_t off = seg_off[sg];
    const int cnt = seg_cnt[sg];
    for (int e = lane; e < cnt; e += 32) {
      const int q = col[off + e];
      atomicOr(&bm[w][(q >> logG) - tu * 32], 1u << ((q & Gm) - tv * 32));
    }
    __syncwarp();
    const unsigned wv = bm[w][lane];
    int nr, pc;
    unsigned lpm, rpm;
    row_runs32(wv, nr, pc, lpm, rpm);
    const int tnr = warp_sum_i(nr), tpc = warp_sum_i(pc);
    const int spc = tpc;
    if (out_bytes) {
      if (lane == 0) {
        out_bytes[sg] = int32_t(runs_rec_bytes(tnr, spc, vb));
        if (tnr > kMaxRuns) atomicOr(err, 1);
      }
      continue;
    }
    if (cnt == 0) continue;   // empty segments have no record
    unsigned char *rp = stream + seg_rec[sg];
    if (lane == 0) {
      *reinterpret_cast<int2 *>(rp) = make_int2(seg_row[sg], int(uint32_t(spc) | (uint32_t(tnr) << 16)));
    }
    int rb = warp_incl_scan_i(nr, lane) - nr;
    const int pb = warp_incl_scan_i(pc, lane) - pc;
    {
      uint32_t *rw = reinterpret_cast<uint32_t *>(rp + kRecHdr);
      unsigned st = wv & ~(wv << 1), en = wv & ~(wv >> 1);
      int pp = pb;   // stored position of the run's first (padded) entry
      while (st) {
        const int b0 = __ffs(int(st)) - 1, b1 = __ffs(int(en)) - 1;
        const int len = b1 - b0 + 1, lp = b0 & 1;
        rw[rb++] = uint32_t(b0) | (uint32_t(len - 1) << 5) | (uint32_t(lane) << 10) | (uint32_t(pp) << 16);
        pp += (len + lp + 1) & ~1;
        st &= st - 1;
        en &= en - 1;
      }
    }
    pbase[w][lane] = pb;
    lpad_s[w][lane] = lpm;
    rpad_s[w][lane] = rpm;
    __syncwarp();
    unsigned char *vals = rp + rec_values_at(tnr);
    for (int e = lane; e < cnt; e += 32) {
      const int q = col[off + e];
      const int r = (q >> logG) - tu * 32, c = (q & Gm) - tv * 32;
      const unsigned lt = (1u << c) - 1u;
      const int pos = pbase[w][r] + __popc(bm[w][r] & lt) + __popc(lpad_s[w][r] & (lt | (lt + 1))) +
                      __popc(rpad_s[w][r] & lt);
      if (vb == 8) reinterpret_cast<float2 *>(vals)[pos] = reinterpret_cast<const float2 *>(val)[off + e];
      else reinterpret_cast<unsigned *>(vals)[pos] = reinterpret_cast<const unsigned *>(val)[off + e];
    }
    __syncwarp();
  }
}

// 1 for the tile-order positions whose segment holds entries
__global__ void k_nonempty(int64_t n, const int32_t *__restrict__ tile_seg, const int32_t *__restrict__ seg_cnt,
                           int32_t *__restrict__ flag) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = seg_cnt[tile_seg[i]] > 0 ? 1 : 0;
}
__global__ void k_compact_i32(int64_t n, const int32_t *__restrict__ flag, const int64_t *__restrict__ pos,
                              const int32_t *__restrict__ src, int32_t *__restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) dst[pos[i]] = src[i];
}
// tile pointers into the compacted list: tptr[t] -> pos[tptr[t]] (pos[n] = total)
__global__ void k_remap_ptr(int n_tiles, int64_t *__restrict__ tptr, const int64_t *__restrict__ pos) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= n_tiles) tptr[t] = pos[tptr[t]];
}

__global__ void k_gather_i32(int64_t n, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                             int32_t *__restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_scatter_i64(int64_t n, const int32_t *__restrict__ idx, const int64_t *__restrict__ src,
                              int64_t *__restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = src[i];
}

// last element of an exclusive scan plus the last count: the total
wproj_status scan_total(const int32_t *cnt, int64_t *out, int64_t n, int64_t *total, cudaStream_t s) {
  WPROJ_TRY(exclusive_scan_i32_to_i64(cnt, out, n, s));
  int64_t lb = 0;
  int32_t lc = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&lb, out + (n - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&lc, cnt + (n - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  *total = lb + lc;
  WPROJ_CUDA(cudaMemcpyAsync(out + n, total, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  return WPROJ_OK;
}

int grid_blocks(int64_t units, int per_block) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(units, per_block), 152 * 64));
}

}  // namespace

// Both copies from the column form held in p->col / p->val (CSR order), then the
// column form is released.  tile_seg / tptr: segments in tile order and the
// first of each tile; on success they are compacted in place to the segments
// that hold entries (the records; *n_rec of them).  A row or segment of more
// than kMaxRuns runs returns WPROJ_ERR_UNSUPPORTED before anything is
// allocated, and the column form stays as it was.
wproj_status build_runs(wproj_plan *p, const int2 *j0, const int32_t *Sk, int32_t *tile_seg, int64_t *tptr,
                        int64_t *n_rec, cudaStream_t s) {
  const GridGeom &g = p->g;
  const int64_t m = p->m, n_seg = p->n_seg;
  const int vb = g.value_dtype == WPROJ_VAL_F32 ? 8 : 4;
  const int logG = ilog2(g.G);
  const int nb_rows = grid_blocks(m, 1), nb_seg = grid_blocks(std::max<int64_t>(1, n_seg), 8);
  // ---- counting passes
  DevBuf pc, nr, bytes, err;
  WPROJ_TRY(pc.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(nr.alloc(sizeof(int32_t) * m));
  WPROJ_TRY(bytes.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
  WPROJ_TRY(err.alloc(sizeof(int)));
  WPROJ_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
  k_rm_build<<<nb_rows, 64, 0, s>>>(m, p->row_ptr.as<int64_t>(), p->col.as<int32_t>(), p->val.as<unsigned char>(),
                                    vb, j0, Sk, logG, pc.as<int32_t>(), nr.as<int32_t>(), err.as<int>(), nullptr,
                                    nullptr, nullptr, nullptr, nullptr);
  WPROJ_CHECK_LAUNCH("runs: row counts");
  if (n_seg > 0) {
    k_tr_build<<<nb_seg, 256, 0, s>>>(n_seg, p->seg_off.as<int64_t>(), p->seg_cnt.as<int32_t>(),
                                      p->seg_row.as<int32_t>(), p->seg_tile.as<int32_t>(), p->col.as<int32_t>(),
                                      p->val.as<unsigned char>(), vb, logG, g.nT, bytes.as<int32_t>(), nullptr,
                                      nullptr, err.as<int>());
    WPROJ_CHECK_LAUNCH("runs: record sizes");
  }
  int herr = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels: a row or segment holds more than 64 runs");
  // ---- row-major copy
  {
    WPROJ_TRY(p->rm_vptr.alloc(sizeof(int64_t) * (m + 1)));
    WPROJ_TRY(p->rm_rptr.alloc(sizeof(int64_t) * (m + 1)));
    WPROJ_TRY(p->rm_org.alloc(sizeof(uint32_t) * m));
    int64_t n_vals = 0, n_runs = 0;
    WPROJ_TRY(scan_total(pc.as<int32_t>(), p->rm_vptr.as<int64_t>(), m, &n_vals, s));
    WPROJ_TRY(scan_total(nr.as<int32_t>(), p->rm_rptr.as<int64_t>(), m, &n_runs, s));
    WPROJ_TRY(p->rm_run.alloc(sizeof(uint32_t) * std::max<int64_t>(1, n_runs)));
    WPROJ_TRY(p->rm_val.alloc(int64_t(vb) * std::max<int64_t>(4, n_vals)));
    WPROJ_CUDA(cudaMemsetAsync(p->rm_val.ptr, 0, int64_t(vb) * std::max<int64_t>(4, n_vals), s));
    k_rm_build<<<nb_rows, 64, 0, s>>>(m, p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
                                      p->val.as<unsigned char>(), vb, j0, Sk, logG, nullptr, nullptr, nullptr,
                                      p->rm_vptr.as<int64_t>(), p->rm_rptr.as<int64_t>(), p->rm_org.as<uint32_t>(),
                                      p->rm_run.as<uint32_t>(), p->rm_val.as<unsigned char>());
    WPROJ_CHECK_LAUNCH("runs: row-major copy");
    p->rm_runs = n_runs;
    p->rm_vals = n_vals;
  }
  // ---- tile-major records, one per segment that holds entries (the box of a
  // small kernel touches more tiles than its support)
  {
    const int n_tiles = g.nT * g.nT;
    int64_t nr_ = 0;
    {
      DevBuf flag, pos, tmp;
      WPROJ_TRY(flag.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
      WPROJ_TRY(pos.alloc(sizeof(int64_t) * (n_seg + 1)));
      WPROJ_TRY(tmp.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
      if (n_seg > 0) {
        k_nonempty<<<ceil_div(n_seg, 256), 256, 0, s>>>(n_seg, tile_seg, p->seg_cnt.as<int32_t>(), flag.as<int32_t>());
        WPROJ_CHECK_LAUNCH("runs: non-empty segments");
        WPROJ_TRY(scan_total(flag.as<int32_t>(), pos.as<int64_t>(), n_seg, &nr_, s));
        k_compact_i32<<<ceil_div(n_seg, 256), 256, 0, s>>>(n_seg, flag.as<int32_t>(), pos.as<int64_t>(), tile_seg,
                                                           tmp.as<int32_t>());
        WPROJ_CHECK_LAUNCH("runs: compact segments");
        WPROJ_CUDA(cudaMemcpyAsync(tile_seg, tmp.ptr, sizeof(int32_t) * nr_, cudaMemcpyDeviceToDevice, s));
      } else {
        WPROJ_CUDA(cudaMemsetAsync(pos.ptr, 0, sizeof(int64_t), s));
      }
      k_remap_ptr<<<ceil_div(n_tiles + 1, 256), 256, 0, s>>>(n_tiles, tptr, pos.as<int64_t>());
      WPROJ_CHECK_LAUNCH("runs: tile pointers");
      WPROJ_CUDA(cudaStreamSynchronize(s));
    }
    *n_rec = nr_;
    DevBuf bytes_t;
    WPROJ_TRY(bytes_t.alloc(sizeof(int32_t) * std::max<int64_t>(1, nr_)));
    WPROJ_TRY(p->rec_off.alloc(sizeof(int64_t) * (nr_ + 1)));
    WPROJ_TRY(p->seg_rec.alloc(sizeof(int64_t) * std::max<int64_t>(1, n_seg)));
    WPROJ_CUDA(cudaMemsetAsync(p->seg_rec.ptr, 0xff, sizeof(int64_t) * std::max<int64_t>(1, n_seg), s));   // -1
    int64_t total = 0;
    if (nr_ > 0) {
      k_gather_i32<<<ceil_div(nr_, 256), 256, 0, s>>>(nr_, tile_seg, bytes.as<int32_t>(), bytes_t.as<int32_t>());
      WPROJ_CHECK_LAUNCH("runs: record sizes in tile order");
      WPROJ_TRY(scan_total(bytes_t.as<int32_t>(), p->rec_off.as<int64_t>(), nr_, &total, s));
      k_scatter_i64<<<ceil_div(nr_, 256), 256, 0, s>>>(nr_, tile_seg, p->rec_off.as<int64_t>(),
                                                       p->seg_rec.as<int64_t>());
      WPROJ_CHECK_LAUNCH("runs: record offsets");
    } else {
      WPROJ_CUDA(cudaMemsetAsync(p->rec_off.ptr, 0, sizeof(int64_t), s));
    }
    WPROJ_TRY(p->stream.alloc(std::max<int64_t>(16, total)));
    WPROJ_CUDA(cudaMemsetAsync(p->stream.ptr, 0, std::max<int64_t>(16, total), s));
    p->stream_bytes = total;
    if (n_seg > 0) {
      k_tr_build<<<nb_seg, 256, 0, s>>>(n_seg, p->seg_off.as<int64_t>(), p->seg_cnt.as<int32_t>(),
                                        p->seg_row.as<int32_t>(), p->seg_tile.as<int32_t>(), p->col.as<int32_t>(),
                                        p->val.as<unsigned char>(), vb, logG, g.nT, nullptr,
                                        p->seg_rec.as<int64_t>(), p->stream.as<unsigned char>(), err.as<int>());
      WPROJ_CHECK_LAUNCH("runs: records");
    }
    WPROJ_CUDA(cudaStreamSynchronize(s));
  }
  p->col.release();
  p->val.release();
  return WPROJ_OK;
}

wproj_status degrid_runs(wproj_plan *p, const float2 *Xt, float2 *y, cudaStream_t s) {
  const int nb = grid_blocks(p->m, 8);
  const float *rs = p->g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>();
  const int logG = ilog2(p->g.G);
#define LAUNCH(VDT)                                                                                             \
  k_runs_degrid<VDT><<<nb, 256, 0, s>>>(p->m, p->rm_vptr.as<int64_t>(), p->rm_rptr.as<int64_t>(),               \
                                        p->rm_org.as<uint32_t>(), p->rm_run.as<uint32_t>(),                     \
                                        p->rm_val.as<unsigned char>(), rs, Xt, logG, y)
  switch (p->g.value_dtype) {
    case WPROJ_VAL_F32: LAUNCH(WPROJ_VAL_F32); break;
    case WPROJ_VAL_BF16: LAUNCH(WPROJ_VAL_BF16); break;
    default: LAUNCH(WPROJ_VAL_F16);
  }
#undef LAUNCH
  WPROJ_CHECK_LAUNCH("degrid (runs)");
  return WPROJ_OK;
}

// Gridding into Xt2; returns the number of kernels launched in *launches.
wproj_status grid_runs(wproj_plan *p, const float2 *y, float2 *Xt2, int *launches, cudaStream_t s) {
  const GridGeom &g = p->g;
  const float *rs = g.value_dtype == WPROJ_VAL_F32 ? nullptr : p->row_scale.as<float>();
  const int logG = ilog2(g.G);
#define LAUNCH(VDT)                                                                                             \
  k_runs_grid<VDT><<<(unsigned)p->n_chunks, kGridWarps * 32, 0, s>>>(                                          \
      p->chunk_tile.as<int32_t>(), p->chunk_lo.as<int64_t>(), p->chunk_hi.as<int64_t>(),                        \
      p->tile_chunk_ptr.as<int32_t>(), p->rec_off.as<int64_t>(), p->stream.as<unsigned char>(), rs, y, logG,    \
      g.nT, p->grid_partial.as<float2>(), Xt2)
  switch (g.value_dtype) {
    case WPROJ_VAL_F32: LAUNCH(WPROJ_VAL_F32); break;
    case WPROJ_VAL_BF16: LAUNCH(WPROJ_VAL_BF16); break;
    default: LAUNCH(WPROJ_VAL_F16);
  }
#undef LAUNCH
  WPROJ_CHECK_LAUNCH("grid (runs)");
  *launches = 1;
  if (p->n_chunks > int64_t(g.nT) * g.nT) {
    k_runs_grid_reduce<<<g.nT * g.nT, 256, 0, s>>>(p->tile_chunk_ptr.as<int32_t>(), p->grid_partial.as<float2>(),
                                                    logG, g.nT, Xt2);
    WPROJ_CHECK_LAUNCH("grid (runs) reduce");
    *launches = 2;
  }
  return WPROJ_OK;
}

wproj_status runs_export(const wproj_plan *p, int64_t k0, int64_t k1, int32_t *col_out, void *val_out,
                         cudaStream_t s) {
  int64_t sb[2] = {0, 0}, first = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&sb[0], p->seg_base.as<int64_t>() + k0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&sb[1], p->seg_base.as<int64_t>() + k1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaMemcpyAsync(&first, p->row_ptr.as<int64_t>() + k0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (sb[1] <= sb[0]) return WPROJ_OK;
  k_runs_export<<<grid_blocks(sb[1] - sb[0], 8), 256, 0, s>>>(
      sb[0], sb[1], first, p->seg_rec.as<int64_t>(), p->seg_off.as<int64_t>(), p->seg_tile.as<int32_t>(),
      p->stream.as<unsigned char>(), p->g.value_dtype == WPROJ_VAL_F32 ? 8 : 4, ilog2(p->g.G), p->g.nT, col_out,
      static_cast<unsigned char *>(val_out));
  WPROJ_CHECK_LAUNCH("export (runs)");
  return WPROJ_OK;
}

}  // namespace wproj
