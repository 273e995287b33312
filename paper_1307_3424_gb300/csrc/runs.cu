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
constexpr int kTileStride = 33;     // shared-memory tile row: 32 cells + the pad column
constexpr int kDegU = 4;            // degridding: chunks of 64 stored entries in flight per row
constexpr int kGridU = 2;           // gridding: chunks in flight per record

__host__ __device__ __forceinline__ int64_t runs_rec_bytes(int nruns, int pcount, int vb) {
  return int64_t((kRecHdr + 2 * nruns + 15) & ~15) + ((int64_t(pcount) * vb + 15) & ~15);
}
__host__ __device__ __forceinline__ int rec_values_at(int nruns) { return (kRecHdr + 2 * nruns + 15) & ~15; }

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

// ---- value pairs -------------------------------------------------------------------

template <int VDT> struct PairT { using T = uint2; };
template <> struct PairT<WPROJ_VAL_F32> { using T = float4; };

template <int VDT>
__device__ __forceinline__ typename PairT<VDT>::T ld_pair(const unsigned char *p) {
  return __ldg(reinterpret_cast<const typename PairT<VDT>::T *>(p));
}
template <int VDT>
__device__ __forceinline__ void unpack_pair(const typename PairT<VDT>::T &v, float2 &a, float2 &b) {
  if constexpr (VDT == WPROJ_VAL_F32) {
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  } else if constexpr (VDT == WPROJ_VAL_BF16) {
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
  } else {
    a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
  }
}
template <int VDT>
__device__ __forceinline__ typename PairT<VDT>::T zero_pair() {
  typename PairT<VDT>::T z;
  memset(&z, 0, sizeof(z));
  return z;
}

// ---- degridding: warp per row of the row-major copy ---------------------------------
//
// A warp takes groups of 32 consecutive rows; lane t loads row t's offsets and
// origin, and while row t is reduced the warp already loads row t + 1's first
// 32 runs and first 64 stored values, so a row costs one wait for X (in L2).

template <int VDT>
__global__ void __launch_bounds__(256, 3)
k_runs_degrid(int64_t m, const int64_t *__restrict__ vptr, const int64_t *__restrict__ rptr,
              const uint32_t *__restrict__ org, const uint32_t *__restrict__ runs,
              const unsigned char *__restrict__ val, const float *__restrict__ row_scale,
              const float2 *__restrict__ X, int logG, float2 *__restrict__ y) {
  constexpr int VB = VDT == WPROJ_VAL_F32 ? 8 : 4;
  using VT = typename PairT<VDT>::T;
  const int lane = threadIdx.x & 31;
  const int Gm = (1 << logG) - 1;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ngroups = (m + 31) >> 5;
  for (int64_t gi = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; gi < ngroups; gi += nw) {
    const int64_t kb = gi << 5;
    const int nrows = int(min(int64_t(32), m - kb));
    const int64_t kl = kb + min(lane, nrows - 1);
    const long long v0_l = vptr[kl];
    const int pc_l = int(vptr[kl + 1] - v0_l);
    const long long r0_l = rptr[kl];
    const int nr_l = int(rptr[kl + 1] - r0_l);
    const uint32_t org_l = __ldg(org + kl);
    // row 0 of the group: first runs and values
    uint32_t w_nx = 0u;
    VT v_nx = zero_pair<VDT>();
    {
      const long long r0 = __shfl_sync(kFull, r0_l, 0), v0 = __shfl_sync(kFull, v0_l, 0);
      const int nr = __shfl_sync(kFull, nr_l, 0), pc = __shfl_sync(kFull, pc_l, 0);
      if (lane < nr) w_nx = __ldg(runs + r0 + lane);
      if (2 * lane < pc) v_nx = ld_pair<VDT>(val + (v0 + 2 * lane) * VB);
    }
    float2 yout = make_float2(0.f, 0.f);
    for (int t = 0; t < nrows; ++t) {
      const long long r0 = __shfl_sync(kFull, r0_l, t), v0 = __shfl_sync(kFull, v0_l, t);
      const int nr = __shfl_sync(kFull, nr_l, t);
      const uint32_t o = __shfl_sync(kFull, org_l, t);
      const int au = int(o & 0xffffu), av = int(o >> 16);
      uint32_t w = w_nx;
      const VT vfirst = v_nx;
      if (t + 1 < nrows) {   // prefetch the next row
        const long long r0n = __shfl_sync(kFull, r0_l, t + 1), v0n = __shfl_sync(kFull, v0_l, t + 1);
        const int nrn = __shfl_sync(kFull, nr_l, t + 1), pcn = __shfl_sync(kFull, pc_l, t + 1);
        w_nx = lane < nrn ? __ldg(runs + r0n + lane) : 0u;
        v_nx = 2 * lane < pcn ? ld_pair<VDT>(val + (v0n + 2 * lane) * VB) : zero_pair<VDT>();
      }
      const unsigned char *vb = val + v0 * VB;
      float2 acc = make_float2(0.f, 0.f);
      int pw = 0;
      for (int j0 = 0; j0 < nr; j0 += 32) {
        const bool valid = j0 + lane < nr;
        if (j0 > 0) w = valid ? __ldg(runs + r0 + j0 + lane) : 0u;
        const int len = valid ? int((w >> 12) & 63u) + 1 : 0;
        const int plen = len + (len & 1);
        const int E = pw + warp_incl_scan_i(plen, lane);
        w |= uint32_t(E - plen) << 18;
        const int p1 = __shfl_sync(kFull, E, 31);
        // chunks of 64 stored entries, kDegU at a time: every load of the group
        // is issued before the first product
        for (int i0 = pw; i0 < p1; i0 += 64 * kDegU) {
          VT v[kDegU];
          float2 x0[kDegU], x1[kDegU];
#pragma unroll
          for (int u = 0; u < kDegU; ++u) {
            const int ib = i0 + 64 * u;
            const int d = E - ib;
            const unsigned bit = (valid && d > 0 && d <= 62) ? (1u << (d >> 1)) : 0u;
            const unsigned ends = __reduce_or_sync(kFull, bit);
            const int base = __popc(__ballot_sync(kFull, valid && d <= 0));
            const int r = base + __popc(ends & ((2u << lane) - 1u));
            const uint32_t q = __shfl_sync(kFull, w, r & 31);
            const int p = ib + 2 * lane;
            v[u] = zero_pair<VDT>();
            x0[u] = x1[u] = make_float2(0.f, 0.f);
            if (p < p1) {
              v[u] = (ib == 0) ? vfirst : ld_pair<VDT>(vb + int64_t(p) * VB);
              const int dr = int(q & 63u), dc = int((q >> 6) & 63u), P = int(q >> 18);
              const int qu = (au + dr) & Gm, qv = (av + dc + p - P) & Gm;
              const float2 *xr = X + (int64_t(qu) << logG);
              x0[u] = __ldg(xr + qv);
              x1[u] = __ldg(xr + ((qv + 1) & Gm));
            }
          }
#pragma unroll
          for (int u = 0; u < kDegU; ++u) {
            float2 g0, g1;
            unpack_pair<VDT>(v[u], g0, g1);
            acc.x += g0.x * x0[u].x - g0.y * x0[u].y + g1.x * x1[u].x - g1.y * x1[u].y;
            acc.y += g0.x * x0[u].y + g0.y * x0[u].x + g1.x * x1[u].y + g1.y * x1[u].x;
          }
        }
        pw = p1;
      }
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
// Warp w takes the w-th quarter of the chunk's records, in groups of 32: lane
// t loads record t's offset, header and y value; while record t is
// accumulated the warp already loads record t + 1's first 32 runs and first
// 64 stored values.

template <int VDT>
__global__ void __launch_bounds__(kGridWarps * 32)
k_runs_grid(const int32_t *__restrict__ chunk_tile, const int64_t *__restrict__ chunk_lo,
            const int64_t *__restrict__ chunk_hi, const int32_t *__restrict__ tile_chunk_ptr,
            const int64_t *__restrict__ rec_off, const unsigned char *__restrict__ stream,
            const float *__restrict__ row_scale, const float2 *__restrict__ y, int logG, int nT,
            float2 *__restrict__ partial, float2 *__restrict__ Xt2) {
  constexpr int VB = VDT == WPROJ_VAL_F32 ? 8 : 4;
  using VT = typename PairT<VDT>::T;
  __shared__ float2 acc[kGridWarps][32 * kTileStride];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2 *a = acc[w];
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
    const int nr_l = int(unsigned(hdr_l.y) >> 16), pc_l = hdr_l.y & 0xffff;
    uint32_t w_nx = 0u;
    VT v_nx = zero_pair<VDT>();
    {
      const long long off = __shfl_sync(kFull, off_l, 0);
      const int nr = __shfl_sync(kFull, nr_l, 0), pc = __shfl_sync(kFull, pc_l, 0);
      const unsigned char *rp = stream + off;
      if (lane < nr) w_nx = reinterpret_cast<const uint16_t *>(rp + kRecHdr)[lane];
      if (2 * lane < pc) v_nx = ld_pair<VDT>(rp + rec_values_at(nr) + 2 * lane * VB);
    }
    for (int t = 0; t < nrec; ++t) {
      const long long off = __shfl_sync(kFull, off_l, t);
      const int nr = __shfl_sync(kFull, nr_l, t);
      const float2 yk = make_float2(__shfl_sync(kFull, y_l.x, t), __shfl_sync(kFull, y_l.y, t));
      uint32_t wd = w_nx;
      const VT vfirst = v_nx;
      if (t + 1 < nrec) {   // prefetch the next record
        const long long offn = __shfl_sync(kFull, off_l, t + 1);
        const int nrn = __shfl_sync(kFull, nr_l, t + 1), pcn = __shfl_sync(kFull, pc_l, t + 1);
        const unsigned char *rpn = stream + offn;
        w_nx = lane < nrn ? uint32_t(reinterpret_cast<const uint16_t *>(rpn + kRecHdr)[lane]) : 0u;
        v_nx = 2 * lane < pcn ? ld_pair<VDT>(rpn + rec_values_at(nrn) + 2 * lane * VB) : zero_pair<VDT>();
      }
      const unsigned char *rp = stream + off;
      const uint16_t *rw = reinterpret_cast<const uint16_t *>(rp + kRecHdr);
      const unsigned char *vals = rp + rec_values_at(nr);
      int pw = 0;
      for (int j0 = 0; j0 < nr; j0 += 32) {
        const bool valid = j0 + lane < nr;
        if (j0 > 0) wd = valid ? uint32_t(rw[j0 + lane]) : 0u;
        const int len = valid ? int((wd >> 5) & 31u) + 1 : 0;
        const int plen = len + (len & 1);
        const int E = pw + warp_incl_scan_i(plen, lane);
        wd |= uint32_t(E - plen) << 16;
        const int p1 = __shfl_sync(kFull, E, 31);
        for (int i0 = pw; i0 < p1; i0 += 64 * kGridU) {
          VT v[kGridU];
          int cell[kGridU];
#pragma unroll
          for (int u = 0; u < kGridU; ++u) {
            const int ib = i0 + 64 * u;
            const int d = E - ib;
            const unsigned bit = (valid && d > 0 && d <= 62) ? (1u << (d >> 1)) : 0u;
            const unsigned ends = __reduce_or_sync(kFull, bit);
            const int base = __popc(__ballot_sync(kFull, valid && d <= 0));
            const int r = base + __popc(ends & ((2u << lane) - 1u));
            const uint32_t q = __shfl_sync(kFull, wd, r & 31);
            const int p = ib + 2 * lane;
            cell[u] = -1;
            v[u] = zero_pair<VDT>();
            if (p < p1) {
              v[u] = (ib == 0) ? vfirst : ld_pair<VDT>(vals + int64_t(p) * VB);
              const int c0 = int(q & 31u), tr = int((q >> 10) & 31u), P = int(q >> 16);
              cell[u] = tr * kTileStride + c0 + (p - P);
            }
          }
#pragma unroll
          for (int u = 0; u < kGridU; ++u) {
            if (cell[u] < 0) continue;
            float2 g0, g1;
            unpack_pair<VDT>(v[u], g0, g1);
            float2 s0 = a[cell[u]], s1 = a[cell[u] + 1];
            s0.x += g0.x * yk.x + g0.y * yk.y;
            s0.y += g0.x * yk.y - g0.y * yk.x;
            s1.x += g1.x * yk.x + g1.y * yk.y;
            s1.y += g1.x * yk.y - g1.y * yk.x;
            a[cell[u]] = s0;
            a[cell[u] + 1] = s1;
          }
        }
        pw = p1;
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
    const unsigned char *rp = stream + seg_rec[sg];
    const int nr = int(unsigned(reinterpret_cast<const int2 *>(rp)->y) >> 16);
    const uint16_t *rw = reinterpret_cast<const uint16_t *>(rp + kRecHdr);
    const unsigned char *vals = rp + rec_values_at(nr);
    const int tile = seg_tile[sg];
    const int tu = tile / nT, tv = tile % nT;
    const int64_t o = seg_off[sg] - first;
    int tw = 0, pw = 0;   // true and padded entries before the window
    for (int j0 = 0; j0 < nr; j0 += 32) {
      const bool valid = j0 + lane < nr;
      const uint32_t wd = valid ? uint32_t(rw[j0 + lane]) : 0u;
      const int len = valid ? int((wd >> 5) & 31u) + 1 : 0;
      const int plen = len + (len & 1);
      const int T = warp_incl_scan_i(len, lane), E = warp_incl_scan_i(plen, lane);
      if (valid) {
        const int c0 = int(wd & 31u), tr = int((wd >> 10) & 31u);
        const int ti = tw + T - len, pi = pw + E - plen;
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

// Runs of one 64-bit window row: count, stored (padded) entries and the mask of
// the last entries of odd-length runs (a pad follows each of them).
__device__ __forceinline__ void row_runs64(unsigned long long w, int &nr, int &pc, unsigned long long &padm) {
  unsigned long long st = w & ~(w << 1), en = w & ~(w >> 1);
  nr = __popcll(st);
  pc = __popcll(w);
  padm = 0;
  while (st) {
    const int b0 = __ffsll((long long)st) - 1, b1 = __ffsll((long long)en) - 1;
    if ((b1 - b0 + 1) & 1) { padm |= 1ull << b1; ++pc; }
    st &= st - 1;
    en &= en - 1;
  }
}
__device__ __forceinline__ void row_runs32(unsigned w, int &nr, int &pc, unsigned &padm) {
  unsigned st = w & ~(w << 1), en = w & ~(w >> 1);
  nr = __popc(st);
  pc = __popc(w);
  padm = 0;
  while (st) {
    const int b0 = __ffs(st) - 1, b1 = __ffs(en) - 1;
    if ((b1 - b0 + 1) & 1) { padm |= 1u << b1; ++pc; }
    st &= st - 1;
    en &= en - 1;
  }
}

// Row-major copy, block of 64 threads per row (thread t = window row t).
// Pass 1 (out_pc != null): stored entries and runs per row.  Pass 2: runs,
// origin and values (rm_val zeroed beforehand: the pads stay zero).
__global__ void __launch_bounds__(64)
k_rm_build(int64_t m, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
           const unsigned char *__restrict__ val, int vb, const int2 *__restrict__ j0, const int32_t *__restrict__ Sk,
           int logG, int32_t *__restrict__ out_pc, int32_t *__restrict__ out_nr, const int64_t *__restrict__ vptr,
           const int64_t *__restrict__ rptr, uint32_t *__restrict__ org, uint32_t *__restrict__ runs,
           unsigned char *__restrict__ rm_val) {
  __shared__ unsigned long long bm[64], padm_s[64];
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
    unsigned long long pm;
    row_runs64(wv, nr, pc, pm);
    if (out_pc) {
      const int a = warp_sum_i(pc), b = warp_sum_i(nr);
      if (lane == 0) { red[2 * (t >> 5)] = a; red[2 * (t >> 5) + 1] = b; }
      __syncthreads();
      if (t == 0) { out_pc[k] = red[0] + red[2]; out_nr[k] = red[1] + red[3]; }
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
    padm_s[t] = pm;
    {
      uint32_t *rr = runs + rptr[k];
      unsigned long long st = wv & ~(wv << 1), en = wv & ~(wv >> 1);
      while (st) {
        const int b0 = __ffsll((long long)st) - 1, b1 = __ffsll((long long)en) - 1;
        rr[rb++] = uint32_t(t) | (uint32_t(b0) << 6) | (uint32_t(b1 - b0) << 12);
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
      const int pos = pbase[du] + __popcll(bm[du] & lt) + __popcll(padm_s[du] & lt);
      if (vb == 8) reinterpret_cast<float2 *>(dst)[pos] = reinterpret_cast<const float2 *>(val)[e];
      else reinterpret_cast<unsigned *>(dst)[pos] = reinterpret_cast<const unsigned *>(val)[e];
    }
    __syncthreads();
  }
}

// Tile-major records, warp per segment.  Pass 1 (out_bytes != null): record
// bytes per segment.  Pass 2: header, runs and values (stream zeroed beforehand).
__global__ void __launch_bounds__(256)
k_tr_build(int64_t n_seg, const int64_t *__restrict__ seg_off, const int32_t *__restrict__ seg_cnt,
           const int32_t *__restrict__ seg_row, const int32_t *__restrict__ seg_tile, const int32_t *__restrict__ col,
           const unsigned char *__restrict__ val, int vb, int logG, int nT, int32_t *__restrict__ out_bytes,
           const int64_t *__restrict__ seg_rec, unsigned char *__restrict__ stream, int *__restrict__ err) {
  __shared__ unsigned bm[8][32], padm_s[8][32];
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
    unsigned pm;
    row_runs32(wv, nr, pc, pm);
    const int tnr = warp_sum_i(nr), tpc = warp_sum_i(pc);
    if (out_bytes) {
      if (lane == 0) out_bytes[sg] = int32_t(runs_rec_bytes(tnr, tpc, vb));
      continue;
    }
    unsigned char *rp = stream + seg_rec[sg];
    if (lane == 0) {
      *reinterpret_cast<int2 *>(rp) = make_int2(seg_row[sg], int(uint32_t(tpc) | (uint32_t(tnr) << 16)));
      if (tpc > 0xffff || tnr > 0xffff) atomicOr(err, 1);
    }
    int rb = warp_incl_scan_i(nr, lane) - nr;
    {
      uint16_t *rw = reinterpret_cast<uint16_t *>(rp + kRecHdr);
      unsigned st = wv & ~(wv << 1), en = wv & ~(wv >> 1);
      while (st) {
        const int b0 = __ffs(st) - 1, b1 = __ffs(en) - 1;
        rw[rb++] = uint16_t(b0 | ((b1 - b0) << 5) | (lane << 10));
        st &= st - 1;
        en &= en - 1;
      }
    }
    pbase[w][lane] = warp_incl_scan_i(pc, lane) - pc;
    padm_s[w][lane] = pm;
    __syncwarp();
    unsigned char *vals = rp + rec_values_at(tnr);
    for (int e = lane; e < cnt; e += 32) {
      const int q = col[off + e];
      const int r = (q >> logG) - tu * 32, c = (q & Gm) - tv * 32;
      const unsigned lt = (1u << c) - 1u;
      const int pos = pbase[w][r] + __popc(bm[w][r] & lt) + __popc(padm_s[w][r] & lt);
      if (vb == 8) reinterpret_cast<float2 *>(vals)[pos] = reinterpret_cast<const float2 *>(val)[off + e];
      else reinterpret_cast<unsigned *>(vals)[pos] = reinterpret_cast<const unsigned *>(val)[off + e];
    }
    __syncwarp();
  }
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
// column form is released.  tile_seg: segments in tile order.
wproj_status build_runs(wproj_plan *p, const int2 *j0, const int32_t *Sk, const int32_t *tile_seg, cudaStream_t s) {
  const GridGeom &g = p->g;
  const int64_t m = p->m, n_seg = p->n_seg;
  const int vb = g.value_dtype == WPROJ_VAL_F32 ? 8 : 4;
  const int logG = ilog2(g.G);
  // ---- row-major copy
  {
    DevBuf pc, nr;
    WPROJ_TRY(pc.alloc(sizeof(int32_t) * m));
    WPROJ_TRY(nr.alloc(sizeof(int32_t) * m));
    WPROJ_TRY(p->rm_vptr.alloc(sizeof(int64_t) * (m + 1)));
    WPROJ_TRY(p->rm_rptr.alloc(sizeof(int64_t) * (m + 1)));
    WPROJ_TRY(p->rm_org.alloc(sizeof(uint32_t) * m));
    const int nb = grid_blocks(m, 1);
    k_rm_build<<<nb, 64, 0, s>>>(m, p->row_ptr.as<int64_t>(), p->col.as<int32_t>(), p->val.as<unsigned char>(), vb,
                                 j0, Sk, logG, pc.as<int32_t>(), nr.as<int32_t>(), nullptr, nullptr, nullptr,
                                 nullptr, nullptr);
    WPROJ_CHECK_LAUNCH("runs: row counts");
    int64_t n_vals = 0, n_runs = 0;
    WPROJ_TRY(scan_total(pc.as<int32_t>(), p->rm_vptr.as<int64_t>(), m, &n_vals, s));
    WPROJ_TRY(scan_total(nr.as<int32_t>(), p->rm_rptr.as<int64_t>(), m, &n_runs, s));
    WPROJ_TRY(p->rm_run.alloc(sizeof(uint32_t) * std::max<int64_t>(1, n_runs)));
    WPROJ_TRY(p->rm_val.alloc(int64_t(vb) * std::max<int64_t>(2, n_vals)));
    WPROJ_CUDA(cudaMemsetAsync(p->rm_val.ptr, 0, int64_t(vb) * std::max<int64_t>(2, n_vals), s));
    k_rm_build<<<nb, 64, 0, s>>>(m, p->row_ptr.as<int64_t>(), p->col.as<int32_t>(), p->val.as<unsigned char>(), vb,
                                 j0, Sk, logG, nullptr, nullptr, p->rm_vptr.as<int64_t>(), p->rm_rptr.as<int64_t>(),
                                 p->rm_org.as<uint32_t>(), p->rm_run.as<uint32_t>(), p->rm_val.as<unsigned char>());
    WPROJ_CHECK_LAUNCH("runs: row-major copy");
    p->rm_runs = n_runs;
    p->rm_vals = n_vals;
  }
  // ---- tile-major records
  {
    DevBuf bytes, bytes_t, err;
    WPROJ_TRY(bytes.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
    WPROJ_TRY(bytes_t.alloc(sizeof(int32_t) * std::max<int64_t>(1, n_seg)));
    WPROJ_TRY(err.alloc(sizeof(int)));
    WPROJ_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    WPROJ_TRY(p->rec_off.alloc(sizeof(int64_t) * (n_seg + 1)));
    WPROJ_TRY(p->seg_rec.alloc(sizeof(int64_t) * std::max<int64_t>(1, n_seg)));
    int64_t total = 0;
    if (n_seg > 0) {
      const int nb = grid_blocks(n_seg, 8);
      k_tr_build<<<nb, 256, 0, s>>>(n_seg, p->seg_off.as<int64_t>(), p->seg_cnt.as<int32_t>(),
                                    p->seg_row.as<int32_t>(), p->seg_tile.as<int32_t>(), p->col.as<int32_t>(),
                                    p->val.as<unsigned char>(), vb, logG, g.nT, bytes.as<int32_t>(), nullptr,
                                    nullptr, err.as<int>());
      WPROJ_CHECK_LAUNCH("runs: record sizes");
      k_gather_i32<<<ceil_div(n_seg, 256), 256, 0, s>>>(n_seg, tile_seg, bytes.as<int32_t>(), bytes_t.as<int32_t>());
      WPROJ_CHECK_LAUNCH("runs: record sizes in tile order");
      WPROJ_TRY(scan_total(bytes_t.as<int32_t>(), p->rec_off.as<int64_t>(), n_seg, &total, s));
      k_scatter_i64<<<ceil_div(n_seg, 256), 256, 0, s>>>(n_seg, tile_seg, p->rec_off.as<int64_t>(),
                                                         p->seg_rec.as<int64_t>());
      WPROJ_CHECK_LAUNCH("runs: record offsets");
    } else {
      WPROJ_CUDA(cudaMemsetAsync(p->rec_off.ptr, 0, sizeof(int64_t), s));
    }
    WPROJ_TRY(p->stream.alloc(std::max<int64_t>(16, total)));
    WPROJ_CUDA(cudaMemsetAsync(p->stream.ptr, 0, std::max<int64_t>(16, total), s));
    p->stream_bytes = total;
    if (n_seg > 0) {
      k_tr_build<<<grid_blocks(n_seg, 8), 256, 0, s>>>(
          n_seg, p->seg_off.as<int64_t>(), p->seg_cnt.as<int32_t>(), p->seg_row.as<int32_t>(),
          p->seg_tile.as<int32_t>(), p->col.as<int32_t>(), p->val.as<unsigned char>(), vb, logG, g.nT, nullptr,
          p->seg_rec.as<int64_t>(), p->stream.as<unsigned char>(), err.as<int>());
      WPROJ_CHECK_LAUNCH("runs: records");
    }
    int herr = 0;
    WPROJ_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WPROJ_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(WPROJ_ERR_UNSUPPORTED, "build_kernels: a run record exceeds 65535 entries or runs");
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
