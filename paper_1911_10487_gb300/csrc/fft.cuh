// Batched 1D FFTs of length N = 2^a 3^b on lines held in shared memory.
//
// The horizontal transform F_r of Sec. 2 (and its inverse, Algorithm 2 step 2)
// is a 2D DFT on the periodic N x N grid, done as two passes of 1D transforms:
// along x (contiguous rows) and along y (strided columns).  Each pass stages a
// tile of lines in shared memory and runs a Stockham autosort FFT on it: every
// stage reads all butterfly inputs into registers, synchronises, and writes the
// outputs back in place, so one buffer per tile suffices.
//
// Radices: 3 (once per factor 3), then the cap MAXR (16, 8 or 4) for as many powers of
// two as it covers, then one stage of 8, 4 or 2 for the rest: few stages, so few
// passes of the tile through shared memory.  The cap is set per kernel (measured):
// a large radix leaves threads idle when a tile has few butterflies.  For stage s with radix
// R and Ns = product of the earlier radices, butterfly j of a line reads elements
// j + r N/R, multiplies by w^(r (j mod Ns) N/(Ns R)) (w = exp(-2 pi i/N), conjugated
// for the inverse), applies the R-point DFT and writes element
// (j / Ns) Ns R + (j mod Ns) + r Ns.  Forward = unnormalised exp(-i...) DFT;
// inverse = unnormalised exp(+i...) DFT (the caller applies 1/N^2).
#pragma once

#include "common.cuh"

namespace fl {

__host__ __device__ constexpr int count_factor(int n, int f) { return (n % f == 0) ? 1 + count_factor(n / f, f) : 0; }
__host__ __device__ constexpr int strip(int n, int f) { return (n % f == 0) ? strip(n / f, f) : n; }

__host__ __device__ constexpr int log2i(int n) { return n > 1 ? 1 + log2i(n / 2) : 0; }

// MAXR (4, 8 or 16) caps the power-of-two radix
template <int N, int MAXR> struct FftPlan {
  static_assert(MAXR == 4 || MAXR == 8 || MAXR == 16, "radix cap 4, 8 or 16");
  static constexpr int n3 = count_factor(N, 3);
  static constexpr int p2 = count_factor(N, 2);
  static constexpr int q = log2i(MAXR);
  static constexpr int nbig = p2 / q;
  static constexpr int rest = 1 << (p2 % q);  // 1 (no further stage), 2, 4 or 8
  static constexpr int stages = n3 + nbig + (rest > 1 ? 1 : 0);
  static_assert(strip(strip(N, 2), 3) == 1, "N must be 2^a 3^b");
  __host__ __device__ static constexpr int radix(int s) { return s < n3 ? 3 : (s < n3 + nbig ? MAXR : rest); }
};

// cos and sin of 2 pi e / 16
__host__ __device__ constexpr double cos16(int e) {
  return (e & 15) == 0 ? 1.0 : (e & 15) == 1 ? 0.92387953251128674 : (e & 15) == 2 ? 0.70710678118654752
       : (e & 15) == 3 ? 0.38268343236508977 : (e & 15) == 4 ? 0.0 : (e & 15) == 5 ? -0.38268343236508977
       : (e & 15) == 6 ? -0.70710678118654752 : (e & 15) == 7 ? -0.92387953251128674 : (e & 15) == 8 ? -1.0
       : (e & 15) == 9 ? -0.92387953251128674 : (e & 15) == 10 ? -0.70710678118654752
       : (e & 15) == 11 ? -0.38268343236508977 : (e & 15) == 12 ? 0.0 : (e & 15) == 13 ? 0.38268343236508977
       : (e & 15) == 14 ? 0.70710678118654752 : 0.92387953251128674;
}
__host__ __device__ constexpr double sin16(int e) { return cos16(e + 12); }  // sin x = cos(x - pi/2)

// Line layouts inside a shared-memory tile.
//  ROW:  element i of line b at b*(N + N/S) + i + i/S    (rows of a plane), S = SKEW:
//        one padding element after every S keeps the stride-S writes of a radix-S
//        stage on distinct shared-memory banks (S = 0: b*N + i, no padding)
//  COL:  element i of line b sits at i*LINES + b         (columns of a plane tile)
enum class Lay { ROW, COL };

template <Lay L, int N, int LINES, int SKEW> struct LayIdx {
  static constexpr int STRIDE = (L == Lay::ROW && SKEW > 0) ? N + N / SKEW : N;
  static constexpr int ELEMS = LINES * STRIDE;  // elements of the tile, padding included
  __host__ __device__ __forceinline__ static int at(int b, int i) {
    return (L == Lay::ROW) ? b * STRIDE + i + (SKEW > 0 ? i / SKEW : 0) : i * LINES + b;
  }
  // thread-item -> (line, butterfly) so that neighbouring threads touch
  // neighbouring shared-memory words
  __device__ __forceinline__ static void map(int t, int nb, int& b, int& j) {
    if (L == Lay::ROW) { j = t % nb; b = t / nb; } else { b = t % LINES; j = t / LINES; }
  }
};

template <typename R, bool INV> struct Dft {
  using C = cx<R>;
  __device__ __forceinline__ static void d2(C* v) {
    C a = v[0], b = v[1];
    v[0] = a + b; v[1] = a - b;
  }
  __device__ __forceinline__ static void d4(C* v) {
    C s02 = v[0] + v[2], d02 = v[0] - v[2];
    C s13 = v[1] + v[3], d13 = rot90<INV>(v[1] - v[3]);
    v[0] = s02 + s13; v[2] = s02 - s13;
    v[1] = d02 + d13; v[3] = d02 - d13;
  }
  // x w16^e, w16 = exp(-2 pi i/16) (conjugated for the inverse); e is a constant
  __device__ __forceinline__ static C tw16(C x, int e) {
    const R c = R(cos16(e)), sn = INV ? R(sin16(e)) : -R(sin16(e));
    return mk<R>(x.x * c - x.y * sn, x.x * sn + x.y * c);
  }
  // 8 points: 4-point DFTs of the even and odd inputs, X[k] = E[k] + w8^k O[k],
  // X[k + 4] = E[k] - w8^k O[k]
  __device__ __forceinline__ static void d8(C* v) {
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    d4(e);
    d4(o);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const C t = tw16(o[k], 2 * k);
      v[k] = e[k] + t;
      v[k + 4] = e[k] - t;
    }
  }
  // 16 points as 4 x 4: with n = 4 n1 + n2 and k = k1 + 4 k2, 4-point DFTs over n1,
  // twiddles w16^(n2 k1), then 4-point DFTs over n2
  __device__ __forceinline__ static void d16(C* v) {
    C y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2];
      y[n2][1] = v[n2 + 4];
      y[n2][2] = v[n2 + 8];
      y[n2][3] = v[n2 + 12];
      d4(y[n2]);
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) y[n2][k1] = tw16(y[n2][k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      d4(z);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
    }
  }
  __device__ __forceinline__ static void d3(C* v) {
    // y1,2 = a0 - (a1+a2)/2 -/+ i (sqrt(3)/2)(a1 - a2)  (forward; signs swap for the inverse)
    const R h = R(0.86602540378443864676);
    C s = v[1] + v[2];
    C t = v[0] - R(0.5) * s;
    C d = h * rot90<INV>(v[1] - v[2]);
    v[0] = v[0] + s; v[1] = t + d; v[2] = t - d;
  }
};

template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int SKEW, int RAD, int NS>
__device__ __forceinline__ void fft_stage(cx<R>* buf, const cx<R>* tw) {
  using C = cx<R>;
  using IX = LayIdx<L, N, LINES, SKEW>;
  constexpr int NB = N / RAD;                 // butterflies per line
  constexpr int TOTAL = LINES * NB;
  constexpr int PER = (TOTAL + THREADS - 1) / THREADS;
  constexpr int STRIDE_TW = N / (NS * RAD);
  C v[PER][RAD];
  int out_b[PER], out_i[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int t = threadIdx.x + p * THREADS;
    if (TOTAL % THREADS == 0 || t < TOTAL) {
      int b, j;
      IX::map(t, NB, b, j);
      const int k = j % NS;
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        C x = buf[IX::at(b, j + r * NB)];
        if (r > 0 && NS > 1) {
          C w = tw[r * k * STRIDE_TW];
          if (INV) w.y = -w.y;
          x = x * w;
        }
        v[p][r] = x;
      }
      if constexpr (RAD == 2) Dft<R, INV>::d2(v[p]);
      else if constexpr (RAD == 4) Dft<R, INV>::d4(v[p]);
      else if constexpr (RAD == 8) Dft<R, INV>::d8(v[p]);
      else if constexpr (RAD == 16) Dft<R, INV>::d16(v[p]);
      else Dft<R, INV>::d3(v[p]);
      out_b[p] = b;
      out_i[p] = (j / NS) * NS * RAD + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int t = threadIdx.x + p * THREADS;
    if (TOTAL % THREADS == 0 || t < TOTAL) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[IX::at(out_b[p], out_i[p] + r * NS)] = v[p][r];
    }
  }
  __syncthreads();
}

// stage S of the plan, with NS = product of the earlier radices (compile-time)
template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int SKEW, int MAXR, int S, int NS>
struct FftStages {
  __device__ __forceinline__ static void run(cx<R>* buf, const cx<R>* tw) {
    if constexpr (S < FftPlan<N, MAXR>::stages) {
      constexpr int RAD = FftPlan<N, MAXR>::radix(S);
      fft_stage<R, N, INV, LINES, THREADS, L, SKEW, RAD, NS>(buf, tw);
      FftStages<R, N, INV, LINES, THREADS, L, SKEW, MAXR, S + 1, NS * RAD>::run(buf, tw);
    }
  }
};

// Transform all LINES lines of the tile in place.  `tw` holds w^j, j < N
// (w = exp(-2 pi i/N)), in shared or global memory.  Must be called by all
// THREADS threads of the block; contains __syncthreads().
template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int MAXR, int SKEW = 0>
__device__ __forceinline__ void fft_lines(cx<R>* buf, const cx<R>* tw) {
  FftStages<R, N, INV, LINES, THREADS, L, SKEW, MAXR, 0, 1>::run(buf, tw);
}

// Out-of-place form of a stage: reads `src`, writes `dst`, one butterfly of a thread
// at a time (few values live, for tiles with many butterflies per thread, where the
// in-place form would hold them all in registers); one barrier per stage.
template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int SKEW, int RAD, int NS>
__device__ __forceinline__ void fft_stage_pp(const cx<R>* src, cx<R>* dst, const cx<R>* tw) {
  using C = cx<R>;
  using IX = LayIdx<L, N, LINES, SKEW>;
  constexpr int NB = N / RAD;
  constexpr int TOTAL = LINES * NB;
  constexpr int STRIDE_TW = N / (NS * RAD);
#pragma unroll 1
  for (int t = threadIdx.x; t < TOTAL; t += THREADS) {
    int b, j;
    IX::map(t, NB, b, j);
    const int k = j % NS;
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      C x = src[IX::at(b, j + r * NB)];
      if (r > 0 && NS > 1) {
        C w = tw[r * k * STRIDE_TW];
        if (INV) w.y = -w.y;
        x = x * w;
      }
      v[r] = x;
    }
    if constexpr (RAD == 2) Dft<R, INV>::d2(v);
    else if constexpr (RAD == 4) Dft<R, INV>::d4(v);
    else if constexpr (RAD == 8) Dft<R, INV>::d8(v);
    else if constexpr (RAD == 16) Dft<R, INV>::d16(v);
    else Dft<R, INV>::d3(v);
    const int oi = (j / NS) * NS * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[IX::at(b, oi + r * NS)] = v[r];
  }
  __syncthreads();
}

template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int SKEW, int MAXR, int S, int NS>
struct FftStagesPP {
  __device__ __forceinline__ static cx<R>* run(cx<R>* a, cx<R>* b, const cx<R>* tw) {
    if constexpr (S < FftPlan<N, MAXR>::stages) {
      constexpr int RAD = FftPlan<N, MAXR>::radix(S);
      fft_stage_pp<R, N, INV, LINES, THREADS, L, SKEW, RAD, NS>(a, b, tw);
      return FftStagesPP<R, N, INV, LINES, THREADS, L, SKEW, MAXR, S + 1, NS * RAD>::run(b, a, tw);
    } else {
      return a;
    }
  }
};

// Transform the LINES lines of tile `a` through `b` (same layout); returns the one
// that holds the result (a after an even number of stages, b after an odd one).  The
// input tile must be complete before the call (a barrier), as for fft_lines.
template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int MAXR, int SKEW = 0>
__device__ __forceinline__ cx<R>* fft_lines_pp(cx<R>* a, cx<R>* b, const cx<R>* tw) {
  return FftStagesPP<R, N, INV, LINES, THREADS, L, SKEW, MAXR, 0, 1>::run(a, b, tw);
}

}  // namespace fl
