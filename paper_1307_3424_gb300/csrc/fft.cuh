// Shared-memory Stockham FFT building blocks (radix 4, one radix-2 stage when
// log2 n is odd).  A block holds C transforms of length N = 2^LOGN in shared
// memory, rows of `ld` elements; T threads cooperate on every stage.  Each
// stage reads all its butterflies into registers, synchronises, and writes the
// outputs in Stockham (self-sorting) order, so no bit reversal is needed.
//
// Twiddles come from tables tw_n[k] = exp(-2 pi i k / n), k < n, for every power
// of two n (stored at offset n), computed once in double precision and rounded
// to float.
#pragma once

#include "common.cuh"

namespace wproj {

// Twiddle tables for N = 2 .. 4096, table of size N stored at offset N.
constexpr int kMaxLogN = 12;
constexpr int kTwiddleLen = 2 << kMaxLogN;

template <int R, int DIR>
__device__ __forceinline__ void small_dft(float2 (&a)[R]) {
  if constexpr (R == 2) {
    float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  } else {
    static_assert(R == 4, "radix");
    float2 t0 = cadd(a[0], a[2]);
    float2 t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]);
    float2 t3 = csub(a[1], a[3]);
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    // forward: X1 = t1 - i t3, X3 = t1 + i t3; inverse swaps them
    float2 m = make_float2(t1.x + t3.y, t1.y - t3.x);   // t1 - i t3
    float2 p = make_float2(t1.x - t3.y, t1.y + t3.x);   // t1 + i t3
    if (DIR < 0) { a[1] = m; a[3] = p; } else { a[1] = p; a[3] = m; }
  }
}

// Stage of span Ns: butterfly k < Ns multiplies input r by exp(-+2 pi i k r /
// (Ns R)), read from the table of length Ns R (lanes with consecutive k read
// words r apart, not N / (Ns R) r apart as in the length-N table).
template <int R, int LOGN, int C, int T, int DIR>
__device__ __forceinline__ void fft_stage(float2 *s, int ld, int Ns, const float2 *__restrict__ twtab) {
  constexpr int N = 1 << LOGN;
  constexpr int NB = N / R;
  constexpr int TOT = NB * C;
  constexpr int PER = (TOT + T - 1) / T;
  float2 v[PER][R];
  const int tid = threadIdx.x;
  const float2 *tw = twtab + Ns * R;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = tid + i * T;
    if ((TOT % T == 0) || b < TOT) {
      const int c = b / NB, j = b % NB;
      const float2 *src = s + c * ld;
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 x = src[j + r * NB];
        if (r > 0) {
          float2 w = __ldg(&tw[k * r]);
          if (DIR > 0) w.y = -w.y;
          x = cmul(x, w);
        }
        v[i][r] = x;
      }
      small_dft<R, DIR>(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = tid + i * T;
    if ((TOT % T == 0) || b < TOT) {
      const int c = b / NB, j = b % NB;
      const int k = j & (Ns - 1);
      float2 *dst = s + c * ld + (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * Ns] = v[i][r];
    }
  }
  __syncthreads();
}

// Full transform of the C rows held in shared memory.  DIR = -1 forward
// (exp(-2 pi i ...)), +1 inverse (unnormalised).  Caller synchronises before.
template <int LOGN, int C, int T, int DIR>
__device__ __forceinline__ void fft_block(float2 *s, int ld, const float2 *__restrict__ twtab) {
  int Ns = 1;
  if constexpr (LOGN & 1) {
    fft_stage<2, LOGN, C, T, DIR>(s, ld, Ns, twtab);
    Ns = 2;
  }
#pragma unroll
  for (int st = 0; st < LOGN / 2; ++st) {
    fft_stage<4, LOGN, C, T, DIR>(s, ld, Ns, twtab);
    Ns *= 4;
  }
}

// Launch shapes.  Row passes hold C = 4096/N rows (at least 1); column passes
// hold max(4, 8192/N) columns so that every global row segment is >= 32 bytes.
template <int LOGN> struct RowCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int C = (N >= 4096) ? 1 : 4096 / N;
  static constexpr int T = 256;
  static constexpr int LD = N + 1;
  static constexpr size_t SMEM = size_t(C) * LD * sizeof(float2);
};
template <int LOGN> struct ColCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int C = (8192 / N >= 4) ? ((8192 / N > 64) ? 64 : 8192 / N) : 4;
  static constexpr int T = (C * N >= 16384) ? 1024 : 512;
  static constexpr int LD = N + 1;
  static constexpr size_t SMEM = size_t(C) * LD * sizeof(float2);
};

}  // namespace wproj
