// 2D FFT passes of Algorithm 2 (steps 1 and 2) with their fused prologues and
// epilogues, for N = 2^a 3^b <= 256, in FP64 (double2) or FP32 (float2).
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
#include <math.h>

#include <type_traits>

#include "fft.cuh"
#include "modes.cuh"
#include "pipeline.cuh"

namespace fl {

namespace {

template <typename R> struct Cfg;
template <> struct Cfg<double> { static constexpr int TC = 8; };
template <> struct Cfg<float> { static constexpr int TC = 16; };

constexpr int THREADS = 256;
// radix caps of the passes (FftPlan), measured on the 128^2 workload
constexpr int RADIX_ROWS = 16, RADIX_COLS = 16, RADIX_GATHER = 16, RADIX_RECOVER = 8;
// row tiles padded after every SKEW elements (LayIdx): the first, radix-16 or radix-8,
// stage of a row pass writes with that stride
constexpr int SKEW_ROWS = 16, SKEW_RECOVER = 8;
constexpr int TILE_ELEMS = 2048;  // elements of one shared-memory tile

template <int N> __host__ __device__ constexpr int row_lines() { return TILE_ELEMS / N > 0 ? TILE_ELEMS / N : 1; }

template <typename R, int N>
__device__ __forceinline__ void load_twiddles(cx<R>* tw_s, const cx<R>* __restrict__ tw) {
  for (int j = threadIdx.x; j < N; j += THREADS) tw_s[j] = tw[j];
}

// ---- dense pass along x (rows): forward, or inverse with 1/N^2 scaling --------
// TI: element type of `in` (cx<R>, or float2 read into an FP64 transform)
template <typename R, int N, bool INV, typename TI = cx<R>>
__global__ void __launch_bounds__(THREADS)
k_fft_rows(const TI* __restrict__ in, cx<R>* __restrict__ out, long long nrows,
           const cx<R>* __restrict__ tw, R scale) {
  pdl_wait();
  pdl_trigger();
  constexpr int LINES = row_lines<N>();
  using IX = LayIdx<Lay::ROW, N, LINES, SKEW_ROWS>;
  __shared__ cx<R> buf[IX::ELEMS];
  __shared__ cx<R> tw_s[N];
  load_twiddles<R, N>(tw_s, tw);
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
  fft_lines<R, N, INV, LINES, THREADS, Lay::ROW, RADIX_ROWS, SKEW_ROWS>(buf, tw_s);
  for (int e = threadIdx.x; e < LINES * N; e += THREADS)
    if (base + e < limit) {
      const cx<R> v = buf[IX::at(e / N, e % N)];
      out[base + e] = INV ? scale * v : v;
    }
}

// ---- dense pass along y (columns), in place; grid (ceil(N/TC), planes) ---------
// clear (may be null): nclear counters zeroed by block (0, 0) -- the barrier counters
// of the classification kernel that follows
template <typename R, int N, bool INV>
__global__ void __launch_bounds__(THREADS)
k_fft_cols(cx<R>* __restrict__ data, const cx<R>* __restrict__ tw, unsigned* __restrict__ clear, int nclear) {
  pdl_wait();
  pdl_trigger();
  if (clear && blockIdx.x == 0 && blockIdx.y == 0)
    for (int i = threadIdx.x; i < nclear; i += THREADS) clear[i] = 0u;
  constexpr int TC = Cfg<R>::TC;
  constexpr int E = N * TC;
  __shared__ cx<R> buf[E];
  __shared__ cx<R> tw_s[N];
  load_twiddles<R, N>(tw_s, tw);
  const int c0 = blockIdx.x * TC;
  cx<R>* pl = data + (long long)blockIdx.y * N * N;
  for (int e = threadIdx.x; e < E; e += THREADS) {
    const int i = e / TC, b = e % TC;
    buf[e] = (c0 + b < N) ? pl[(long long)i * N + c0 + b] : czero<R>();
  }
  __syncthreads();
  fft_lines<R, N, INV, TC, THREADS, Lay::COL, RADIX_COLS>(buf, tw_s);
  for (int e = threadIdx.x; e < E; e += THREADS) {
    const int i = e / TC, b = e % TC;
    if (c0 + b < N) pl[(long long)i * N + c0 + b] = buf[e];
  }
}

// ---- per-mode norms ||W~_nu||^2 = sum_k |W~_k(nu)|^2, summed in plane order ------
// grid (n_partial, n_omega), one mode per thread; each block also writes the sum
// of its modes' norms (fixed-order tree) for ||W||.
constexpr int NORM_T = 256;

template <typename R>
__global__ void __launch_bounds__(NORM_T)
k_mode_norms(const cx<R>* __restrict__ wt, double* __restrict__ norms, double* __restrict__ partial, int m1,
             int N2, unsigned long long* __restrict__ ctr) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[NORM_T];
  const int om = blockIdx.y;
  const int nu = blockIdx.x * NORM_T + threadIdx.x;
  // summed in the working precision R (FP32 in the mixed path: FP64 arithmetic
  // here would run on the slow FP64 pipe for every mode)
  R acc = R(0);
  if (nu < N2) {
    const cx<R>* p = wt + (long long)om * m1 * N2 + nu;
    int k = 0;
    for (; k + 8 <= m1; k += 8) {  // eight independent loads in flight, summed in plane order
      cx<R> v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = p[(long long)(k + q) * N2];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc += v[q].x * v[q].x + v[q].y * v[q].y;
    }
    for (; k < m1; ++k) {
      const cx<R> v = p[(long long)k * N2];
      acc += v.x * v.x + v.y * v.y;
    }
    norms[(long long)om * N2 + nu] = (double)acc;
  }
  red[threadIdx.x] = (double)acc;
  // modes whose norm is not finite (a NaN or Inf in W), counted at the barrier
  // the reduction needs anyway
  const int n_bad = __syncthreads_count(nu < N2 && !isfinite(acc));
  if (n_bad && threadIdx.x == 0) atomicAdd(ctr + C_NONFINITE, (unsigned long long)n_bad);
  for (int h = NORM_T / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long long)om * gridDim.x + blockIdx.x] = red[0];
}

// ---- inverse pass 1: gather active profiles, columns (along y) ----------------
// grid (ceil(N/TC), M, 2 n_omega).  Column chunk `blockIdx.x` of the compact column
// list of frequency om; field f = 0 (V~) or 1 (U~).  Inactive modes are zero in
// V~ and equal the incident field U~0 in U~; the plane wave exp(-i k0 z) has
// U~0 = N^2 exp(-i k0 z'_l) at nu = 0 and zero elsewhere.
template <typename R, int N>
__global__ void __launch_bounds__(THREADS)
k_ifft_cols_gather(Problem P, const cx<R>* __restrict__ prof, const int* __restrict__ slot,
                   const int* __restrict__ cols, const int* __restrict__ ncol,
                   cx<R>* __restrict__ t2, const cx<R>* __restrict__ tw) {
  pdl_wait();
  pdl_trigger();
  constexpr int TC = Cfg<R>::TC;
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
  fft_lines<R, N, true, TC, THREADS, Lay::COL, RADIX_GATHER>(buf, tw_s);
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

template <typename R, int N, typename A, bool INC>
__device__ __forceinline__ bool recover_pass(const Problem& P, const cx<R>* __restrict__ t2,
                                             const int* __restrict__ cols, const int* __restrict__ ncol,
                                             const cx<R>* __restrict__ u0, cx<R>* buf, const cx<R>* tw_s, A* num,
                                             A* den) {
  constexpr int LINES = row_lines<N>() / 2 > 0 ? row_lines<N>() / 2 : 1;
  constexpr int E = LINES * N;
  using IX = LayIdx<Lay::ROW, N, 2 * LINES, SKEW_RECOVER>;  // V~ lines, then U~ lines
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
    fft_lines<R, N, true, 2 * LINES, THREADS, Lay::ROW, RADIX_RECOVER, SKEW_RECOVER>(buf, tw_s);
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
template <typename R, int N, bool INC>
__global__ void __launch_bounds__(THREADS)
k_ifft_rows_recover(Problem P, const cx<R>* __restrict__ t2, const int* __restrict__ cols,
                    const int* __restrict__ ncol, const cx<R>* __restrict__ u0, R* __restrict__ xi,
                    R* __restrict__ cout, unsigned long long* __restrict__ ctr, const cx<R>* __restrict__ tw) {
  pdl_wait();
  pdl_trigger();
  constexpr int LINES = row_lines<N>() / 2 > 0 ? row_lines<N>() / 2 : 1;
  constexpr int E = LINES * N;            // elements of one field
  constexpr int PER = (E + THREADS - 1) / THREADS;
  __shared__ cx<R> buf[LayIdx<Lay::ROW, N, 2 * LINES, SKEW_RECOVER>::ELEMS];
  __shared__ cx<R> tw_s[N];
  __shared__ unsigned red[THREADS / 32];
  load_twiddles<R, N>(tw_s, tw);
  const long long nrows = (long long)P.m * N;
  const long long row0 = (long long)blockIdx.x * LINES;
  R num[PER], den[PER];
  if (recover_pass<R, N, R, INC>(P, t2, cols, ncol, u0, buf, tw_s, num, den)) {
    // the sums left the range of R (|u| |V| beyond FP32 for huge evanescent
    // profiles): redo this block with FP64 sums; xi itself is in range
    double nd[PER], dd[PER];
    recover_pass<R, N, double, INC>(P, t2, cols, ncol, u0, buf, tw_s, nd, dd);
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

template <typename R>
__global__ void k_twiddles(cx<R>* tw, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)n, &s, &c);
    tw[j] = from_d<R>(make_double2(c, s));
  }
}

// W (complex64) -> W~ (complex128 in w.wt64) and the norms: the forward transform
// of the mixed truncated-SVD route, in FP64
template <int N>
cudaError_t fwd_wide_impl(const float2* W, const Problem& P, const Work<float>& w, cudaStream_t s, cudaEvent_t mid) {
  constexpr int LINES = row_lines<N>();
  const long long nrows = (long long)P.n_omega * P.m1 * N;
  const long long nblk = (nrows + LINES - 1) / LINES;
  cudaError_t e = launch_pdl(k_fft_rows<double, N, false, float2>, dim3((unsigned)nblk), dim3(THREADS), 0, s, W,
                             w.wt64, nrows, w.tw64, 1.0);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  const dim3 g2((N + Cfg<double>::TC - 1) / Cfg<double>::TC, (unsigned)(P.n_omega * P.m1));
  e = launch_pdl(k_fft_cols<double, N, false>, g2, dim3(THREADS), 0, s, w.wt64, w.tw64, (unsigned*)nullptr, 0);
  if (e != cudaSuccess) return e;
  const dim3 gn((unsigned)w.n_partial, (unsigned)P.n_omega);
  e = launch_pdl(k_mode_norms<double>, gn, dim3(NORM_T), 0, s, (const double2*)w.wt64, w.norms, w.partial, P.m1,
                 N * N, w.ctr);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, int N>
cudaError_t fwd_impl(const cx<R>* W, const Problem& P, const Work<R>& w, cudaStream_t s, cudaEvent_t mid,
                     bool norms) {
  if constexpr (std::is_same<R, float>::value) {
    if (w.wt64) return fwd_wide_impl<N>(W, P, w, s, mid);
  }
  constexpr int LINES = row_lines<N>();
  const long long nrows = (long long)P.n_omega * P.m1 * N;
  const long long nblk = (nrows + LINES - 1) / LINES;
  cudaError_t e = launch_pdl(k_fft_rows<R, N, false>, dim3((unsigned)nblk), dim3(THREADS), 0, s, W, w.wt, nrows,
                             (const cx<R>*)w.tw, R(1));
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  const dim3 g2((N + Cfg<R>::TC - 1) / Cfg<R>::TC, (unsigned)(P.n_omega * P.m1));
  e = launch_pdl(k_fft_cols<R, N, false>, g2, dim3(THREADS), 0, s, w.wt, (const cx<R>*)w.tw,
                 norms ? (unsigned*)nullptr : w.bar, P.n_omega);
  if (e != cudaSuccess) return e;
  if (!norms) return cudaGetLastError();
  return launch_mode_norms<R>(P, w, s);
}

template <typename R, int N>
cudaError_t rec_impl(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  dim3 g1((N + Cfg<R>::TC - 1) / Cfg<R>::TC, P.m, 2 * P.n_omega);
  cudaError_t e = launch_pdl(k_ifft_cols_gather<R, N>, g1, dim3(THREADS), 0, s, P, (const cx<R>*)w.prof,
                             (const int*)w.slot, (const int*)w.cols, (const int*)w.ncol, w.t2, (const cx<R>*)w.tw);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  constexpr int LINES = row_lines<N>() / 2 > 0 ? row_lines<N>() / 2 : 1;
  const long long nrows = (long long)P.m * N;
  const dim3 gr((unsigned)((nrows + LINES - 1) / LINES));
  if (w.u0)
    e = launch_pdl(k_ifft_rows_recover<R, N, true>, gr, dim3(THREADS), 0, s, P, (const cx<R>*)w.t2,
                   (const int*)w.cols, (const int*)w.ncol, w.u0, xi, c, w.ctr, (const cx<R>*)w.tw);
  else
    e = launch_pdl(k_ifft_rows_recover<R, N, false>, gr, dim3(THREADS), 0, s, P, (const cx<R>*)w.t2,
                   (const int*)w.cols, (const int*)w.ncol, w.u0, xi, c, w.ctr, (const cx<R>*)w.tw);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, int N>
cudaError_t dense_impl(cx<R>* in, cx<R>* out, long long planes, bool inverse, const cx<R>* tw, cudaStream_t s) {
  constexpr int LINES = row_lines<N>();
  constexpr long long MAX_Y = 32768;  // planes per column launch (grid y <= 65535)
  const long long nrows = planes * N;
  const unsigned nblk = (unsigned)((nrows + LINES - 1) / LINES);
  auto cols = [&](cx<R>* buf, bool inv) {
    for (long long p0 = 0; p0 < planes; p0 += MAX_Y) {
      const long long np = planes - p0 < MAX_Y ? planes - p0 : MAX_Y;
      const dim3 gc((N + Cfg<R>::TC - 1) / Cfg<R>::TC, (unsigned)np);
      if (inv) k_fft_cols<R, N, true><<<gc, THREADS, 0, s>>>(buf + p0 * N * N, tw, nullptr, 0);
      else k_fft_cols<R, N, false><<<gc, THREADS, 0, s>>>(buf + p0 * N * N, tw, nullptr, 0);
    }
  };
  if (!inverse) {
    k_fft_rows<R, N, false><<<nblk, THREADS, 0, s>>>(in, out, nrows, tw, R(1));
    cols(out, false);
  } else {
    cols(in, true);
    k_fft_rows<R, N, true><<<nblk, THREADS, 0, s>>>(in, out, nrows, tw, R(1.0 / ((double)N * N)));
  }
  return cudaGetLastError();
}

#define FL_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256)

}  // namespace

bool fft_size_supported(int n) {
#define FL_CASE(K) if (n == K) return true;
  FL_SIZES(FL_CASE)
#undef FL_CASE
  return false;
}

template <typename R>
cudaError_t launch_mode_norms(const Problem& P, const Work<R>& w, cudaStream_t s) {
  const dim3 gn((unsigned)w.n_partial, (unsigned)P.n_omega);
  cudaError_t e = launch_pdl(k_mode_norms<R>, gn, dim3(NORM_T), 0, s, (const cx<R>*)w.wt, w.norms, w.partial, P.m1,
                             P.n * P.n, w.ctr);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template cudaError_t launch_mode_norms<double>(const Problem&, const Work<double>&, cudaStream_t);
template cudaError_t launch_mode_norms<float>(const Problem&, const Work<float>&, cudaStream_t);

template <typename R>
cudaError_t launch_fft2_forward(const cx<R>* W, const Problem& P, const Work<R>& w, cudaStream_t s,
                                cudaEvent_t mid, bool norms) {
  switch (P.n) {
#define FL_CASE(K) case K: return fwd_impl<R, K>(W, P, w, s, mid, norms);
    FL_SIZES(FL_CASE)
#undef FL_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_recover(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  switch (P.n) {
#define FL_CASE(K) case K: return rec_impl<R, K>(P, w, xi, c, s, mid);
    FL_SIZES(FL_CASE)
#undef FL_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_fft2_dense(cx<R>* in, cx<R>* out, int n, long long planes, bool inverse, const cx<R>* tw,
                              cudaStream_t s) {
  switch (n) {
#define FL_CASE(K) case K: return dense_impl<R, K>(in, out, planes, inverse, tw, s);
    FL_SIZES(FL_CASE)
#undef FL_CASE
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_fft2_dense<double>(double2*, double2*, int, long long, bool, const double2*, cudaStream_t);
template cudaError_t launch_fft2_dense<float>(float2*, float2*, int, long long, bool, const float2*, cudaStream_t);

template <typename R>
cudaError_t launch_twiddles(cx<R>* tw, int n, cudaStream_t s) {
  k_twiddles<R><<<(n + 255) / 256, 256, 0, s>>>(tw, n);
  return cudaGetLastError();
}

template cudaError_t launch_fft2_forward<double>(const double2*, const Problem&, const Work<double>&, cudaStream_t,
                                                 cudaEvent_t, bool);
template cudaError_t launch_fft2_forward<float>(const float2*, const Problem&, const Work<float>&, cudaStream_t,
                                                cudaEvent_t, bool);
template cudaError_t launch_recover<double>(const Problem&, const Work<double>&, double*, double*, cudaStream_t,
                                            cudaEvent_t);
template cudaError_t launch_recover<float>(const Problem&, const Work<float>&, float*, float*, cudaStream_t,
                                           cudaEvent_t);
template cudaError_t launch_twiddles<double>(double2*, int, cudaStream_t);
template cudaError_t launch_twiddles<float>(float2*, int, cudaStream_t);

}  // namespace fl
