// Shared-memory FFT passes of the 2D transforms (fft.cuh holds the line transforms):
// the dense pass along x (rows), the dense pass along y (columns, in place) and the
// per-mode norms, with their tile shapes.  Included by the forward and the inverse
// translation units (fft_forward.cu, fft_inverse.cu).
#pragma once

#include <math.h>

#include <type_traits>

#include "fft.cuh"
#include "modes.cuh"
#include "pipeline.cuh"

namespace fl {

namespace {

// Tile shapes of the transform passes (fs_options.fft_tile, chosen by the batch tuner):
//   0  shared-memory tiles of 2048 elements, 16 (FP32) or 8 (FP64) columns per column
//      tile, radix cap 16 (8 in the recovery pass) -- measured best on one 128^2 problem;
//   1  tiles of 1024 elements, 8 or 4 columns, radix cap 8: twice the blocks with half
//      the shared memory each, for many concurrent problems.
// Row tiles are padded after every SKEW elements (LayIdx): the first (radix-SKEW) stage
// of a row pass writes with that stride.
template <int T> struct Tile;
template <> struct Tile<0> {
  static constexpr int ELEMS = 2048, TC32 = 16, TC64 = 8;
  static constexpr int RADIX_ROWS = 16, RADIX_COLS = 16, RADIX_GATHER = 16, RADIX_RECOVER = 8;
  static constexpr int SKEW_ROWS = 16, SKEW_RECOVER = 8;
};
template <> struct Tile<1> {
  static constexpr int ELEMS = 1024, TC32 = 8, TC64 = 4;
  static constexpr int RADIX_ROWS = 8, RADIX_COLS = 8, RADIX_GATHER = 8, RADIX_RECOVER = 8;
  static constexpr int SKEW_ROWS = 8, SKEW_RECOVER = 8;
};
template <typename R, int T> __host__ __device__ constexpr int tile_cols() {
  return sizeof(R) == 4 ? Tile<T>::TC32 : Tile<T>::TC64;
}

constexpr int THREADS = 256;

// rows of one tile of the dense row pass: the tile's elements over N; FP32 at N = 256
// with the default tile: 4096 elements (16 rows), fewer CTAs with less fixed cost
// (measured: the row pass of 256^2 x 64 with 19 planes and 8 frequencies 61.5 -> 55.5 us;
// at 192, 21 rows a tile, slower: 53.6 -> 57.8 us)
template <typename R, int N, int T> __host__ __device__ constexpr int row_lines() {
  constexpr int E = (sizeof(R) == 4 && T == 0 && N >= 256) ? 4096 : Tile<T>::ELEMS;
  return E / N > 0 ? E / N : 1;
}

// CTAs per plane of the single-pass (cluster) transforms: the smallest power of two,
// at most 8 (the portable cluster size), that leaves each CTA at most 16 rows (24 for
// N = 192, 32 for N = 256)
template <int N, int MAXRB = 16> __host__ __device__ constexpr int plane_cluster() {
  int c = 1;
  while (c < 8 && N / c > MAXRB && N % (2 * c) == 0) c *= 2;
  return c;
}
// the one-pass forward transform's cluster: up to 32 rows per CTA (4 CTAs at N = 128;
// measured 2 us faster on the 128^2 step than 8 CTAs of 16 rows, and 16 CTAs of 8 rows
// slower still: fewer, larger tiles have less fixed cost)
template <int N> __host__ __device__ constexpr int fwd_cluster() { return plane_cluster<N, 32>(); }

template <typename R, int N>
__device__ __forceinline__ void load_twiddles(cx<R>* tw_s, const cx<R>* __restrict__ tw) {
  for (int j = threadIdx.x; j < N; j += THREADS) tw_s[j] = tw[j];
}

// ---- dense pass along x (rows): forward, or inverse with 1/N^2 scaling --------
// TI: element type of `in` (cx<R>, or float2 read into an FP64 transform)
template <typename R, int N, bool INV, typename TI = cx<R>, int T = 0>
__global__ void __launch_bounds__(THREADS)
k_fft_rows(const TI* __restrict__ in, cx<R>* __restrict__ out, long long nrows,
           const cx<R>* __restrict__ tw, R scale) {
  constexpr int LINES = row_lines<R, N, T>();
  using IX = LayIdx<Lay::ROW, N, LINES, Tile<T>::SKEW_ROWS>;
  __shared__ cx<R> buf[IX::ELEMS];
  __shared__ cx<R> tw_s[N];
  load_twiddles<R, N>(tw_s, tw);  // a constant table: read while the predecessor drains
  pdl_wait();
  pdl_trigger();
  const long long row0 = (long long)blockIdx.x * LINES;
  const long long base = row0 * N;
  const long long limit = nrows * N;
  for (int e = threadIdx.x; e < LINES * N; e += THREADS) {
    cx<R> v = czero<R>();
    if (base + e < limit) {
      if constexpr (std::is_same<TI, cx<R>>::value) v = in[base + e];
      else v = from_d<R>(to_d(in[base + e]));
    }
    buf[IX::at(e / N, e % N)] = v;
  }
  __syncthreads();
  fft_lines<R, N, INV, LINES, THREADS, Lay::ROW, Tile<T>::RADIX_ROWS, Tile<T>::SKEW_ROWS>(buf, tw_s);
  for (int e = threadIdx.x; e < LINES * N; e += THREADS)
    if (base + e < limit) {
      const cx<R> v = buf[IX::at(e / N, e % N)];
      out[base + e] = INV ? scale * v : v;
    }
}

// ---- dense pass along y (columns), in place; grid (ceil(N/TC), planes) ---------
// clear (may be null): nclear counters zeroed by block (0, 0) -- the barrier counters
// of the classification kernel that follows
template <typename R, int N, bool INV, int T = 0>
__global__ void __launch_bounds__(THREADS)
k_fft_cols(cx<R>* __restrict__ data, const cx<R>* __restrict__ tw, unsigned* __restrict__ clear, int nclear) {
  constexpr int TC = tile_cols<R, T>();
  constexpr int E = N * TC;
  __shared__ cx<R> buf[E];
  __shared__ cx<R> tw_s[N];
  load_twiddles<R, N>(tw_s, tw);  // a constant table: read while the predecessor drains
  pdl_wait();
  pdl_trigger();
  if (clear && blockIdx.x == 0 && blockIdx.y == 0)
    for (int i = threadIdx.x; i < nclear; i += THREADS) clear[i] = 0u;
  const int c0 = blockIdx.x * TC;
  cx<R>* pl = data + (long long)blockIdx.y * N * N;
  for (int e = threadIdx.x; e < E; e += THREADS) {
    const int i = e / TC, b = e % TC;
    buf[e] = (c0 + b < N) ? pl[(long long)i * N + c0 + b] : czero<R>();
  }
  __syncthreads();
  fft_lines<R, N, INV, TC, THREADS, Lay::COL, Tile<T>::RADIX_COLS>(buf, tw_s);
  for (int e = threadIdx.x; e < E; e += THREADS) {
    const int i = e / TC, b = e % TC;
    if (c0 + b < N) pl[(long long)i * N + c0 + b] = buf[e];
  }
}

// ---- per-mode norms ||W~_nu||^2 = sum_k |W~_k(nu)|^2 ----------------------------
// grid (n_partial, n_omega), NORM_MB modes per block and NORM_Q threads per mode: warp
// w sums the planes of quarter q = w / 2 (a contiguous quarter of the planes, its loads
// in flight together) for 32 consecutive modes, and the quarters are added in a fixed
// order; each block also writes the sum of its modes' norms (fixed-order tree) for ||W||.
constexpr int NORM_T = 256, NORM_Q = 4, NORM_MB = NORM_T / NORM_Q;

template <typename R>
__global__ void __launch_bounds__(NORM_T)
k_mode_norms(const cx<R>* __restrict__ wt, double* __restrict__ norms, double* __restrict__ partial, int m1,
             int N2, unsigned long long* __restrict__ ctr) {
  pdl_wait();
  pdl_trigger();
  __shared__ R part[NORM_Q][NORM_MB];
  __shared__ double red[NORM_MB];
  const int om = blockIdx.y;
  const int q = threadIdx.x / NORM_MB, j = threadIdx.x % NORM_MB;
  const int nu = blockIdx.x * NORM_MB + j;
  // summed in the working precision R (FP32 in the mixed path: FP64 arithmetic
  // here would run on the slow FP64 pipe for every mode)
  R acc = R(0);
  const int k0 = q * m1 / NORM_Q, k1 = (q + 1) * m1 / NORM_Q;
  if (nu < N2) {
    const cx<R>* p = wt + (long long)om * m1 * N2 + nu;
    int k = k0;
    for (; k + 8 <= k1; k += 8) {  // eight independent loads in flight, summed in plane order
      cx<R> v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = p[(long long)(k + t) * N2];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc += v[t].x * v[t].x + v[t].y * v[t].y;
    }
    for (; k < k1; ++k) {
      const cx<R> v = p[(long long)k * N2];
      acc += v.x * v.x + v.y * v.y;
    }
  }
  part[q][j] = acc;
  __syncthreads();
  R nrm = R(0);
  if (q == 0) {
    nrm = (part[0][j] + part[1][j]) + (part[2][j] + part[3][j]);
    if (nu < N2) norms[(long long)om * N2 + nu] = (double)nrm;
    red[j] = (double)nrm;
  }
  // modes whose norm is not finite (a NaN or Inf in W), counted at the barrier
  // the reduction needs anyway
  const int n_bad = __syncthreads_count(q == 0 && nu < N2 && !isfinite(nrm));
  if (n_bad && threadIdx.x == 0) atomicAdd(ctr + C_NONFINITE, (unsigned long long)n_bad);
  for (int h = NORM_MB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long long)om * gridDim.x + blockIdx.x] = red[0];
}

}  // namespace

#define FL_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256)

}  // namespace fl
