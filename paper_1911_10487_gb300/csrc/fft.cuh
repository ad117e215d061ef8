// Batched 1D FFTs of length N = 2^a 3^b on lines held in shared memory.
//
// The horizontal transform F_r of Sec. 2 (and its inverse, Algorithm 2 step 2)
// is a 2D DFT on the periodic N x N grid, done as two passes of 1D transforms:
// along x (contiguous rows) and along y (strided columns).  Each pass stages a
// tile of lines in shared memory and runs a Stockham autosort FFT on it: every
// stage reads all butterfly inputs into registers, synchronises, and writes the
// outputs back in place, so one buffer per tile suffices.
//
// Radices: 3 (once per factor 3), then 4, then a final 2.  For stage s with radix
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

template <int N> struct FftPlan {
  static constexpr int n3 = count_factor(N, 3);
  static constexpr int p2 = count_factor(N, 2);
  static constexpr int n4 = p2 / 2;
  static constexpr int n2 = p2 % 2;
  static constexpr int stages = n3 + n4 + n2;
  static_assert(strip(strip(N, 2), 3) == 1, "N must be 2^a 3^b");
  __host__ __device__ static constexpr int radix(int s) { return s < n3 ? 3 : (s < n3 + n4 ? 4 : 2); }
};

// Line layouts inside a shared-memory tile.
//  ROW:  line b occupies [b*(N+PAD), b*(N+PAD)+N)      (rows of a plane)
//  COL:  element i of line b sits at i*LINES + b         (columns of a plane tile)
enum class Lay { ROW, COL };

template <Lay L, int N, int LINES, int PAD> struct LayIdx {
  __device__ __forceinline__ static int at(int b, int i) {
    return (L == Lay::ROW) ? b * (N + PAD) + i : i * LINES + b;
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
  __device__ __forceinline__ static void d3(C* v) {
    // y1,2 = a0 - (a1+a2)/2 -/+ i (sqrt(3)/2)(a1 - a2)  (forward; signs swap for the inverse)
    const R h = R(0.86602540378443864676);
    C s = v[1] + v[2];
    C t = v[0] - R(0.5) * s;
    C d = h * rot90<INV>(v[1] - v[2]);
    v[0] = v[0] + s; v[1] = t + d; v[2] = t - d;
  }
};

template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int PAD, int RAD, int NS>
__device__ __forceinline__ void fft_stage(cx<R>* buf, const cx<R>* tw) {
  using C = cx<R>;
  using IX = LayIdx<L, N, LINES, PAD>;
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
      if (RAD == 2) Dft<R, INV>::d2(v[p]);
      else if (RAD == 4) Dft<R, INV>::d4(v[p]);
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
template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int PAD, int S, int NS>
struct FftStages {
  __device__ __forceinline__ static void run(cx<R>* buf, const cx<R>* tw) {
    if constexpr (S < FftPlan<N>::stages) {
      constexpr int RAD = FftPlan<N>::radix(S);
      fft_stage<R, N, INV, LINES, THREADS, L, PAD, RAD, NS>(buf, tw);
      FftStages<R, N, INV, LINES, THREADS, L, PAD, S + 1, NS * RAD>::run(buf, tw);
    }
  }
};

// Transform all LINES lines of the tile in place.  `tw` holds w^j, j < N
// (w = exp(-2 pi i/N)), in shared or global memory.  Must be called by all
// THREADS threads of the block; contains __syncthreads().
template <typename R, int N, bool INV, int LINES, int THREADS, Lay L, int PAD = 0>
__device__ __forceinline__ void fft_lines(cx<R>* buf, const cx<R>* tw) {
  FftStages<R, N, INV, LINES, THREADS, L, PAD, 0, 1>::run(buf, tw);
}

}  // namespace fl
