// Inverse 2D FFT passes of Algorithm 2 (step 2) with the pointwise recovery of step
// 3 fused into the last, for N = 2^a 3^b <= 256, in FP64 (double2) or FP32 (float2).
//
//   fft2_forward  : W -> W~ on every data plane (Sec. 4, Algorithm 2 step 1 needs
//                   W~ = F_r[W]), then ||W~_nu||^2 summed over the planes of a
//                   frequency, which the discrepancy test needs.
//   recover       : V~, U~ -> V = F^-1[V~], u = F^-1[U~] (Algorithm 2 step 2) and
//                   xi = Re(sum conj(u) V)/sum |u|^2, c = (c0^-2 - xi)^-1/2
//                   (step 3, Sec. 5.2; Sec. 1 for c).  The inverse column pass
//                   gathers the solved profiles of the active modes only and
//                   transforms only the columns nu1 that hold a nonzero mode; the
//                   row pass scatters those columns and transforms full rows.
#include "fft_pass.cuh"

namespace fl {

namespace {

// ---- inverse pass 1: gather active profiles, columns (along y) ----------------
// grid (ceil(N/TC), M, 2 n_omega).  Column chunk `blockIdx.x` of the compact column
// list of frequency om; field f = 0 (V~) or 1 (U~).  Inactive modes are zero in
// V~ and equal the incident field U~0 in U~; the plane wave exp(-i k0 z) has
// U~0 = N^2 exp(-i k0 z'_l) at nu = 0 and zero elsewhere.
template <typename R, int N, int T>
__global__ void __launch_bounds__(THREADS)
k_ifft_cols_gather(Problem P, const cx<R>* __restrict__ prof, const int* __restrict__ slot,
                   const int* __restrict__ cols, const int* __restrict__ ncol,
                   cx<R>* __restrict__ t2, const cx<R>* __restrict__ tw) {
  pdl_wait();
  pdl_trigger();
  constexpr int TC = tile_cols<R, T>();
  constexpr int E = N * TC;
  constexpr int PER = (E + THREADS - 1) / THREADS;
  const int om = blockIdx.z >> 1, f = blockIdx.z & 1;
  const int l = blockIdx.y;
  const int nc = ncol[om];
  const int cb = blockIdx.x * TC;
  if (cb >= nc) return;
  __shared__ cx<R> buf[E];
  __shared__ cx<R> tw_s[N];
  load_twiddles<R, N>(tw_s, tw);
  const long long N2 = (long long)N * N;
  const int M = P.m;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (e < E) {
      const int i = e / TC, b = e % TC;
      const int c = cb + b;
      cx<R> v = czero<R>();
      if (c < nc) {
        const int nu1 = cols[om * N + c];
        const int s = slot[om * N2 + (long long)i * N + nu1];
        if (s >= 0) {
          v = prof[(((long long)om * N2 + s) * 2 + f) * M + l];
        } else if (f == 1 && i == 0 && nu1 == 0 && !P.incident) {  // one thread: FP64 is slow on this GPU
          double sn, cs;
          sincos(-(P.omega[om] / P.c0) * (P.z1 + (l + 0.5) * P.hz), &sn, &cs);
          v = from_d<R>(make_double2((double)N2 * cs, (double)N2 * sn));
        }
      }
      buf[e] = v;
    }
  }
  __syncthreads();
  fft_lines<R, N, true, TC, THREADS, Lay::COL, Tile<T>::RADIX_GATHER>(buf, tw_s);
  const long long ob = (((long long)om * 2 + f) * M + l) * N2;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (e < E) {
      const int i = e / TC, b = e % TC;
      if (cb + b < nc) t2[ob + (long long)i * N + cb + b] = buf[e];
    }
  }
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned v, unsigned* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
  return s;
}

// ---- inverse pass 2: rows (along x) + step 3 ----------------------------------
// grid ceil(M N / LINES); a block owns LINES rows (l, y) of the X grid, loops over
// the frequencies, transforms V and u rows and accumulates the least-squares sums
// in the accumulator type A.  Returns (block-uniform) whether any sum overflowed.
// a / b and 1/sqrt(x) of the pointwise recovery: IEEE in FP32; in FP64 by
// Newton-Raphson from FP32 seeds (rcp64, rsqrt64), a few dependent FP64 operations
// instead of the FP64 division and square root, which dominate this kernel on a
// GPU whose FP64 pipe runs at 1/64 of the FP32 rate.
template <typename R> __device__ __forceinline__ R quot(R a, R b);
template <> __device__ __forceinline__ float quot<float>(float a, float b) { return a / b; }
template <> __device__ __forceinline__ double quot<double>(double a, double b) { return a * rcp64(b); }
template <typename R> __device__ __forceinline__ R inv_sqrt(R x);
template <> __device__ __forceinline__ float inv_sqrt<float>(float x) { return 1.0f / sqrtf(x); }
template <> __device__ __forceinline__ double inv_sqrt<double>(double x) { return rsqrt64(x); }

template <typename R, int N, typename A, bool INC, int T>
__device__ __forceinline__ bool recover_pass(const Problem& P, const cx<R>* __restrict__ t2,
                                             const int* __restrict__ cols, const int* __restrict__ ncol,
                                             const cx<R>* __restrict__ u0, cx<R>* buf, const cx<R>* tw_s, A* num,
                                             A* den) {
  constexpr int LINES = row_lines<N, T>() / 2 > 0 ? row_lines<N, T>() / 2 : 1;
  constexpr int E = LINES * N;
  using IX = LayIdx<Lay::ROW, N, 2 * LINES, Tile<T>::SKEW_RECOVER>;  // V~ lines, then U~ lines
  constexpr int PER = (E + THREADS - 1) / THREADS;
  const int M = P.m;
  const long long N2 = (long long)N * N;
  const long long nrows = (long long)M * N;
  const long long row0 = (long long)blockIdx.x * LINES;
  const R scale = R(1.0 / (double)N2);
#pragma unroll
  for (int p = 0; p < PER; ++p) { num[p] = A(0); den[p] = A(0); }
  for (int om = 0; om < P.n_omega; ++om) {
    for (int e = threadIdx.x; e < IX::ELEMS; e += THREADS) buf[e] = czero<R>();
    __syncthreads();
    const int nc = ncol[om];
    const int* cl = cols + om * N;
    const int tot = 2 * LINES * nc;
    for (int q = threadIdx.x; q < tot; q += THREADS) {
      const int line = q / nc, c = q - line * nc;
      const int f = line / LINES, b = line - f * LINES;
      const long long r = row0 + b;
      if (r < nrows) {
        const long long l = r / N, i = r - l * N;
        buf[IX::at(line, cl[c])] = t2[(((long long)om * 2 + f) * M + l) * N2 + i * N + c];
      }
    }
    __syncthreads();
    fft_lines<R, N, true, 2 * LINES, THREADS, Lay::ROW, Tile<T>::RADIX_RECOVER, Tile<T>::SKEW_RECOVER>(buf, tw_s);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * THREADS;
      if (e < E) {
        const cx<R> v = scale * buf[IX::at(e / N, e % N)];
        cx<R> u = scale * buf[IX::at(LINES + e / N, e % N)];
        if (INC) {  // the given incident field (the transform holds U~ - U~0)
          const long long r = row0 + e / N;
          if (r < nrows) u = u + u0[((long long)om * M + r / N) * N2 + (r % N) * N + (e % N)];
        }
        num[p] += (A)u.x * (A)v.x + (A)u.y * (A)v.y;  // Re(conj(u) V)
        den[p] += (A)u.x * (A)u.x + (A)u.y * (A)u.y;  // |u|^2
      }
    }
    __syncthreads();
  }
  bool bad = false;
#pragma unroll
  for (int p = 0; p < PER; ++p) bad |= !(isfinite(num[p]) && isfinite(den[p]));
  return __syncthreads_or(bad) != 0;
}

// INC: u0 (the incident field on X) is given and added to u; otherwise the transform
// already holds the plane wave
template <typename R, int N, bool INC, int T>
__global__ void __launch_bounds__(THREADS)
k_ifft_rows_recover(Problem P, const cx<R>* __restrict__ t2, const int* __restrict__ cols,
                    const int* __restrict__ ncol, const cx<R>* __restrict__ u0, R* __restrict__ xi,
                    R* __restrict__ cout, unsigned long long* __restrict__ ctr, const cx<R>* __restrict__ tw) {
  pdl_wait();
  pdl_trigger();
  constexpr int LINES = row_lines<N, T>() / 2 > 0 ? row_lines<N, T>() / 2 : 1;
  constexpr int E = LINES * N;            // elements of one field
  constexpr int PER = (E + THREADS - 1) / THREADS;
  __shared__ cx<R> buf[LayIdx<Lay::ROW, N, 2 * LINES, Tile<T>::SKEW_RECOVER>::ELEMS];
  __shared__ cx<R> tw_s[N];
  __shared__ unsigned red[THREADS / 32];
  load_twiddles<R, N>(tw_s, tw);
  const long long nrows = (long long)P.m * N;
  const long long row0 = (long long)blockIdx.x * LINES;
  R num[PER], den[PER];
  if (recover_pass<R, N, R, INC, T>(P, t2, cols, ncol, u0, buf, tw_s, num, den)) {
    // the sums left the range of R (|u| |V| beyond FP32 for huge evanescent
    // profiles): redo this block with FP64 sums; xi itself is in range
    double nd[PER], dd[PER];
    recover_pass<R, N, double, INC, T>(P, t2, cols, ncol, u0, buf, tw_s, nd, dd);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const bool g = !(dd[p] >= (double)P.n_omega * P.eps_u * P.eps_u);
      num[p] = g ? R(0) : R(nd[p] / dd[p]);
      den[p] = g ? R(0) : R(1);
    }
  }
  const R guard = R(P.u_guard);  // host-derived: no FP64 division on the device
  const R inv_c02 = R(P.inv_c02);
  unsigned n_guard = 0, n_nan = 0, n_bad = 0;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (e < E) {
      const long long r = row0 + e / N;
      if (r < nrows) {
        const bool g = !(den[p] >= guard);
        const R x = g ? R(0) : quot<R>(num[p], den[p]);
        n_guard += g;
        n_bad += !isfinite(x);
        const long long o = r * N + (e % N);
        xi[o] = x;
        if (cout) {
          const bool ok = x < inv_c02;
          n_nan += !ok;
          cout[o] = ok ? inv_sqrt<R>(inv_c02 - x) : R(NAN);
        }
      }
    }
  }
  // the counters of guarded, NaN-c and non-finite voxels: almost always zero, so one
  // barrier decides
  if (__syncthreads_or((n_guard | n_nan | n_bad) != 0u)) {
    const unsigned long long sg = block_sum_u64(n_guard, red);
    __syncthreads();
    const unsigned long long sn = block_sum_u64(n_nan, red);
    __syncthreads();
    const unsigned long long sb = block_sum_u64(n_bad, red);
    if (threadIdx.x == 0) {
      if (sg) atomicAdd(ctr + C_U_GUARD, sg);
      if (sn) atomicAdd(ctr + C_NAN_C, sn);
      if (sb) atomicAdd(ctr + C_NONFINITE, sb);
    }
  }
}

template <typename R, int N, int T>
cudaError_t rec_tiled(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  constexpr int TC = tile_cols<R, T>();
  dim3 g1((N + TC - 1) / TC, P.m, 2 * P.n_omega);
  cudaError_t e = launch_pdl(k_ifft_cols_gather<R, N, T>, g1, dim3(THREADS), 0, s, P, (const cx<R>*)w.prof,
                             (const int*)w.slot, (const int*)w.cols, (const int*)w.ncol, w.t2, (const cx<R>*)w.tw);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  constexpr int LINES = row_lines<N, T>() / 2 > 0 ? row_lines<N, T>() / 2 : 1;
  const long long nrows = (long long)P.m * N;
  const dim3 gr((unsigned)((nrows + LINES - 1) / LINES));
  if (w.u0)
    e = launch_pdl(k_ifft_rows_recover<R, N, true, T>, gr, dim3(THREADS), 0, s, P, (const cx<R>*)w.t2,
                   (const int*)w.cols, (const int*)w.ncol, w.u0, xi, c, w.ctr, (const cx<R>*)w.tw);
  else
    e = launch_pdl(k_ifft_rows_recover<R, N, false, T>, gr, dim3(THREADS), 0, s, P, (const cx<R>*)w.t2,
                   (const int*)w.cols, (const int*)w.ncol, w.u0, xi, c, w.ctr, (const cx<R>*)w.tw);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, int N>
cudaError_t rec_impl(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  return P.fft_tile == 1 ? rec_tiled<R, N, 1>(P, w, xi, c, s, mid) : rec_tiled<R, N, 0>(P, w, xi, c, s, mid);
}

}  // namespace

template <typename R>
cudaError_t launch_recover(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  switch (P.n) {
#define FL_CASE(K) case K: return rec_impl<R, K>(P, w, xi, c, s, mid);
    FL_SIZES(FL_CASE)
#undef FL_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_recover<double>(const Problem&, const Work<double>&, double*, double*, cudaStream_t,
                                            cudaEvent_t);
template cudaError_t launch_recover<float>(const Problem&, const Work<float>&, float*, float*, cudaStream_t,
                                           cudaEvent_t);

}  // namespace fl
