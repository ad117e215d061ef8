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
constexpr int GATHER_COLS = 32;  // active columns the gather's grid covers in one pass (see rec_tiled)

// Column chunks blockIdx.z, blockIdx.z + gridDim.z, ... of the compact column list of
// frequency om (grid below); field f = 0 (V~) or 1 (U~).  Inactive modes are zero in
// V~ and equal the incident field U~0 in U~; the plane wave exp(-i k0 z) has
// U~0 = N^2 exp(-i k0 z'_l) at nu = 0 and zero elsewhere.
template <typename R, int N, int T>
__global__ void __launch_bounds__(THREADS)
k_ifft_cols_gather(Problem P, const cx<R>* __restrict__ prof, const int* __restrict__ slot,
                   const int* __restrict__ cols, const int* __restrict__ ncol,
                   cx<R>* __restrict__ t2, const cx<R>* __restrict__ tw) {
  constexpr int TC = tile_cols<R, T>();
  constexpr int E = N * TC;
  constexpr int PER = (E + THREADS - 1) / THREADS;
  __shared__ cx<R> buf[E];
  __shared__ cx<R> tw_s[N];
  load_twiddles<R, N>(tw_s, tw);  // a constant table: read while the predecessor drains
  pdl_wait();
  pdl_trigger();
  // grid (M, 2 n_omega, gather_chunks): the column chunk is the slowest index, so that
  // the chunks that hold active columns (the first ceil(ncol / TC)) are dispatched first
  // and the rest, which return at once, last; a block loops when ncol needs more chunks
  const int om = blockIdx.y >> 1, f = blockIdx.y & 1;
  const int l = blockIdx.x;
  const int nc = ncol[om];
  const long long N2 = (long long)N * N;
  const int M = P.m;
  for (int cb = blockIdx.z * TC; cb < nc; cb += gridDim.z * TC) {
    if (cb != (int)blockIdx.z * TC) __syncthreads();  // the previous chunk's stores have read buf
    // element e = t + p THREADS is row i = e / TC of line b = t mod TC (THREADS is a
    // multiple of TC): one column per thread, its PER slot loads and then its profile
    // loads issued together
    static_assert(THREADS % TC == 0, "one column per thread");
    const int b = threadIdx.x % TC;
    const int nu1 = cb + b < nc ? cols[om * N + cb + b] : -1;
    int sl[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * THREADS, i = e / TC;
      sl[p] = (nu1 >= 0 && e < E) ? slot[om * N2 + (long long)i * N + nu1] : -1;
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * THREADS;
      if (e < E) {
        const int i = e / TC;
        cx<R> v = czero<R>();
        if (sl[p] >= 0) {
          v = prof[(((long long)om * N2 + sl[p]) * 2 + f) * M + l];
        } else if (f == 1 && i == 0 && nu1 == 0 && !P.incident) {  // one thread: FP64 is slow on this GPU
          double sn, cs;
          sincos(-(P.omega[om] / P.c0) * (P.z1 + (l + 0.5) * P.hz), &sn, &cs);
          v = from_d<R>(make_double2((double)N2 * cs, (double)N2 * sn));
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
      if (e < E && nu1 >= 0) t2[ob + (long long)(e / TC) * N + cb + b] = buf[e];
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
template <> __device__ __forceinline__ float inv_sqrt<float>(float x) { return rsqrtf(x); }  // <= 2 ulp
template <> __device__ __forceinline__ double inv_sqrt<double>(double x) { return rsqrt64(x); }

// The recovery pass's tile.  FP32, default tile (fs_options.fft_tile = 0): from N = 96
// up, 4096 elements (the V and u rows of 4096 / (2N) rows of X) with radix-16 stages
// (a 128-point row in two stages, 16 and 8, every thread busy in both), transformed out
// of place (PP: two tiles in shared memory, one butterfly per thread at a time, one
// barrier per stage; in place, the radix-3 stages of N = 96 and 192 would hold five
// butterflies a thread in registers and spill); below 96 at N = 2^k, 1024 elements in
// place (small problems need the CTAs: 64^2 x 16 recovers in 18 us instead of 33 with
// 4096); otherwise the tile of fs_options.fft_tile.  MINB: CTAs per SM the register
// allocation is held to -- three at N = 2^k (at most 80 registers a thread; 1 us faster
// at 128^2 than two CTAs of 102), two with PP at radix-3 sizes (128 registers, no
// spill), one elsewhere.
template <typename R, int N, int T> struct RecTile {
  static constexpr bool F32 = sizeof(R) == 4 && T == 0;
  static constexpr bool PP = F32 && N >= 96;
  static constexpr bool BIG = F32 && (PP || N % 3 != 0);
  static constexpr int ELEMS = BIG ? (N >= 96 ? 4096 : 1024) : Tile<T>::ELEMS;
  static constexpr int RADIX = BIG ? 16 : Tile<T>::RADIX_RECOVER;
  static constexpr int SKEW = BIG ? 16 : Tile<T>::SKEW_RECOVER;
  static constexpr int MINB = T == 0 && N % 3 != 0 ? 3 : (PP ? 2 : 1);
};
template <typename R, int N, int T> __host__ __device__ constexpr int rec_lines() {
  return RecTile<R, N, T>::ELEMS / N / 2 > 0 ? RecTile<R, N, T>::ELEMS / N / 2 : 1;
}
// the recovery pass's dynamic shared memory: its tile (two with PP)
template <typename R, int N, int T> __host__ __device__ constexpr size_t rec_smem() {
  return sizeof(cx<R>) * (RecTile<R, N, T>::PP ? 2 : 1) *
         (size_t)LayIdx<Lay::ROW, N, 2 * rec_lines<R, N, T>(), RecTile<R, N, T>::SKEW>::ELEMS;
}

// filled: the tile is already zero for the first frequency.  In FP64 without a given
// incident field the sums are taken of the unscaled transforms (N^2 V, N^2 u): xi is
// their quotient either way, and the guard on sum |u|^2 is scaled instead
// (Problem::u_guard_raw), which saves four FP64 products per voxel and frequency.
template <typename R, bool INC> __host__ __device__ constexpr bool raw_sums() { return sizeof(R) == 8 && !INC; }

template <typename R, int N, typename A, bool INC, int T>
__device__ __forceinline__ bool recover_pass(const Problem& P, const cx<R>* __restrict__ t2,
                                             const int* __restrict__ cols, const int* __restrict__ ncol,
                                             const cx<R>* __restrict__ u0, cx<R>* buf, const cx<R>* tw_s, A* num,
                                             A* den, bool filled) {
  constexpr int LINES = rec_lines<R, N, T>();
  constexpr int E = LINES * N;
  using IX = LayIdx<Lay::ROW, N, 2 * LINES, RecTile<R, N, T>::SKEW>;  // V~ lines, then U~ lines
  constexpr int PER = (E + THREADS - 1) / THREADS;
  const int M = P.m;
  const long long N2 = (long long)N * N;
  const long long nrows = (long long)M * N;
  const long long row0 = (long long)blockIdx.x * LINES;
  const R scale = raw_sums<R, INC>() ? R(1) : R(1.0 / (double)N2);
#pragma unroll
  for (int p = 0; p < PER; ++p) { num[p] = A(0); den[p] = A(0); }
  for (int om = 0; om < P.n_omega; ++om) {
    if (om > 0 || !filled)
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
    const cx<R>* res = buf;
    if constexpr (RecTile<R, N, T>::PP)
      res = fft_lines_pp<R, N, true, 2 * LINES, THREADS, Lay::ROW, RecTile<R, N, T>::RADIX, RecTile<R, N, T>::SKEW>(
          buf, buf + IX::ELEMS, tw_s);
    else
      fft_lines<R, N, true, 2 * LINES, THREADS, Lay::ROW, RecTile<R, N, T>::RADIX, RecTile<R, N, T>::SKEW>(buf, tw_s);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * THREADS;
      if (e < E) {
        cx<R> v = res[IX::at(e / N, e % N)];
        cx<R> u = res[IX::at(LINES + e / N, e % N)];
        if constexpr (!raw_sums<R, INC>()) {
          v = scale * v;
          u = scale * u;
        }
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

// xi and c of the elements e = threadIdx.x + p THREADS < E of rows row0 + e / N (below
// nrows) from the least-squares sums, and the counters of guarded, NaN-c and non-finite
// voxels (almost always zero, so one barrier decides).  guard: the least den of a kept
// voxel (host-derived: no FP64 division on the device)
template <typename R, int PER, int N>
__device__ __forceinline__ void recover_epilogue(const Problem& P, const R* num, const R* den, R guard,
                                                 long long row0, long long nrows, int E, R* __restrict__ xi,
                                                 R* __restrict__ cout, unsigned long long* __restrict__ ctr,
                                                 unsigned* red) {
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

// INC: u0 (the incident field on X) is given and added to u; otherwise the transform
// already holds the plane wave
template <typename R, int N, bool INC, int T>
__global__ void __launch_bounds__(THREADS, (RecTile<R, N, T>::MINB))
k_ifft_rows_recover(Problem P, const cx<R>* __restrict__ t2, const int* __restrict__ cols,
                    const int* __restrict__ ncol, const cx<R>* __restrict__ u0, R* __restrict__ xi,
                    R* __restrict__ cout, unsigned long long* __restrict__ ctr, const cx<R>* __restrict__ tw) {
  constexpr int LINES = rec_lines<R, N, T>();
  constexpr int E = LINES * N;            // elements of one field
  constexpr int PER = (E + THREADS - 1) / THREADS;
  using IX = LayIdx<Lay::ROW, N, 2 * LINES, RecTile<R, N, T>::SKEW>;
  extern __shared__ __align__(16) unsigned char rec_smem_raw[];  // rec_smem<R, N, T>() bytes
  cx<R>* buf = reinterpret_cast<cx<R>*>(rec_smem_raw);
  __shared__ cx<R> tw_s[N];
  __shared__ unsigned red[THREADS / 32];
  // the constant twiddle table and the cleared tile of the first frequency, while the
  // predecessor drains
  load_twiddles<R, N>(tw_s, tw);
  for (int e = threadIdx.x; e < IX::ELEMS; e += THREADS) buf[e] = czero<R>();
  pdl_wait();
  pdl_trigger();
  const long long nrows = (long long)P.m * N;
  const long long row0 = (long long)blockIdx.x * LINES;
  R num[PER], den[PER];
  const double gd = raw_sums<R, INC>() ? P.u_guard_raw : P.u_guard;
  R guard = R(gd);
  if (P.sums64 || recover_pass<R, N, R, INC, T>(P, t2, cols, ncol, u0, buf, tw_s, num, den, true)) {
    // the sums left the range of R (|u| |V| beyond FP32 for huge evanescent
    // profiles): redo this block with FP64 sums; xi itself is in range
    double nd[PER], dd[PER];
    recover_pass<R, N, double, INC, T>(P, t2, cols, ncol, u0, buf, tw_s, nd, dd, P.sums64 != 0);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const bool g = !(dd[p] >= gd);
      num[p] = g ? R(0) : R(nd[p] / dd[p]);
      den[p] = g ? R(0) : R(1);
    }
    guard = R(0.5);  // den is now 1 (kept) or 0 (guarded)
  }
  recover_epilogue<R, PER, N>(P, num, den, guard, row0, nrows, E, xi, cout, ctr, red);
}

// ---- single-pass inverse transform and recovery: one X plane per cluster ---------
// grid (C, M), clusters of C = plane_cluster<N>() CTAs along x; CTA r of the cluster
// of plane l owns rows r RB .. r RB + RB - 1 (RB = N / C) of both fields (V and u) in
// its shared memory.  For every frequency the cluster splits the 2 nc active columns
// (V~ and U~ columns nu1 of cols) among its CTAs; each gathers its columns' profiles
// (as k_ifft_cols_gather), transforms them along y and stores every value in the row
// tile of the CTA that owns its row (distributed shared memory).  After a cluster
// barrier each CTA transforms its rows along x and accumulates the least-squares sums
// (as recover_pass).  No intermediate array goes through global memory, and one launch
// replaces two.
constexpr int REC_CL = 8;  // column lines per chunk (a divisor of THREADS)

template <typename R, int N> __host__ __device__ constexpr size_t plane_rec_smem() {
  constexpr int RB = N / plane_cluster<N>();
  return sizeof(cx<R>) * ((size_t)LayIdx<Lay::ROW, N, 2 * RB, 8>::ELEMS + (size_t)REC_CL * N + N);
}

// The sums of the elements p0 .. p0 + G - 1 (of threadIdx.x + p THREADS < RB N) over
// the frequencies, in the accumulator type A.  Called by every thread of every CTA of
// the cluster (it holds cluster barriers).
template <typename R, int N, bool INC, typename A, int G>
__device__ __forceinline__ void plane_rec_pass(const Problem& P, const cx<R>* __restrict__ prof,
                                               const int* __restrict__ slot, const int* __restrict__ cols,
                                               const int* __restrict__ ncol, const cx<R>* __restrict__ u0, int l,
                                               unsigned r, cx<R>* rt, cx<R>* ct, const cx<R>* tw_s, int p0, A* num,
                                               A* den) {
  constexpr int C = plane_cluster<N>(), RB = N / C;
  using IX = LayIdx<Lay::ROW, N, 2 * RB, 8>;  // V rows, then u rows
  constexpr int E = RB * N;
  const int M = P.m;
  const long long N2 = (long long)N * N;
  const R scale = R(1.0 / (double)N2);
#pragma unroll
  for (int k = 0; k < G; ++k) { num[k] = A(0); den[k] = A(0); }
  for (int om = 0; om < P.n_omega; ++om) {
    for (int e = threadIdx.x; e < IX::ELEMS; e += THREADS) rt[e] = czero<R>();
    cluster_sync();  // every row tile is cleared (and was read) before any CTA stores into it
    const int nc = ncol[om];
    const int* cl = cols + om * N;
    const int nl = 2 * nc, lpc = (nl + C - 1) / C;  // line q: field q / nc, column cl[q % nc]
    const int q0 = min(nl, (int)r * lpc), q1 = min(nl, q0 + lpc);
    // thread t handles line b = t % REC_CL of each chunk, rows i = t / REC_CL + p THREADS / REC_CL:
    // one column per thread, its CPER values' loads issued together
    constexpr int CPER = (REC_CL * N + THREADS - 1) / THREADS;
    const int b = threadIdx.x % REC_CL;
    for (int c0 = q0; c0 < q1; c0 += REC_CL) {
      const int q = c0 + b;
      const int f = q >= nc ? 1 : 0;
      const int nu1 = q < q1 ? cl[q - f * nc] : -1;
      int sl[CPER];
#pragma unroll
      for (int p = 0; p < CPER; ++p) {
        const int i = threadIdx.x / REC_CL + p * (THREADS / REC_CL);
        sl[p] = (nu1 >= 0 && i < N) ? slot[om * N2 + (long long)i * N + nu1] : -1;
      }
#pragma unroll
      for (int p = 0; p < CPER; ++p) {
        const int i = threadIdx.x / REC_CL + p * (THREADS / REC_CL);
        if (i < N) {
          cx<R> v = czero<R>();
          if (sl[p] >= 0) {
            v = prof[(((long long)om * N2 + sl[p]) * 2 + f) * M + l];
          } else if (!INC && f == 1 && i == 0 && nu1 == 0) {
            // the plane wave's U~0 = N^2 exp(-i k0 z'_l) at nu = 0: the phase reduced to
            // [-pi, pi] in FP64, its sine and cosine in FP32 (the precision of R)
            const double ph = -(P.omega[om] / P.c0) * (P.z1 + (l + 0.5) * P.hz);
            const double red = fma(-6.283185307179586, rint(ph * 0.15915494309189535), ph);
            float sn, cs;
            sincosf((float)red, &sn, &cs);
            v = mk<R>(R(N2) * R(cs), R(N2) * R(sn));
          }
          ct[i * REC_CL + b] = v;  // element i of line b
        }
      }
      __syncthreads();
      fft_lines<R, N, true, REC_CL, THREADS, Lay::COL, 8>(ct, tw_s);
      if (nu1 >= 0) {  // value i of the line -> row i % RB of CTA i / RB
#pragma unroll
        for (int p = 0; p < CPER; ++p) {
          const int i = threadIdx.x / REC_CL + p * (THREADS / REC_CL);
          if (i < N) dsmem_st(dsmem_addr(rt + IX::at(f * RB + i % RB, nu1), (unsigned)(i / RB)), ct[i * REC_CL + b]);
        }
      }
      __syncthreads();
    }
    cluster_sync();  // every active column has reached its rows
    fft_lines<R, N, true, 2 * RB, THREADS, Lay::ROW, 8, 8>(rt, tw_s);
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int e = threadIdx.x + (p0 + k) * THREADS;
      if (e < E) {
        const cx<R> v = scale * rt[IX::at(e / N, e % N)];
        cx<R> u = scale * rt[IX::at(RB + e / N, e % N)];
        if (INC) u = u + u0[((long long)om * M + l) * N2 + (long long)((int)r * RB + e / N) * N + (e % N)];
        num[k] += (A)u.x * (A)v.x + (A)u.y * (A)v.y;  // Re(conj(u) V)
        den[k] += (A)u.x * (A)u.x + (A)u.y * (A)u.y;  // |u|^2
      }
    }
    __syncthreads();
  }
}

template <typename R, int N, bool INC>
__global__ void __launch_bounds__(THREADS, 2)
k_ifft2_plane_recover(Problem P, const cx<R>* __restrict__ prof, const int* __restrict__ slot,
                      const int* __restrict__ cols, const int* __restrict__ ncol, const cx<R>* __restrict__ u0,
                      R* __restrict__ xi, R* __restrict__ cout, unsigned long long* __restrict__ ctr,
                      const cx<R>* __restrict__ tw) {
  constexpr int C = plane_cluster<N>(), RB = N / C;
  constexpr int E = RB * N;
  constexpr int PER = (E + THREADS - 1) / THREADS;
  static_assert(PER <= 32, "one bit per element in the redo mask");
  constexpr int G = 2;  // elements per thread of one redo pass
  extern __shared__ __align__(16) unsigned char plane_smem[];
  cx<R>* rt = reinterpret_cast<cx<R>*>(plane_smem);
  cx<R>* ct = rt + LayIdx<Lay::ROW, N, 2 * RB, 8>::ELEMS;
  cx<R>* tw_s = ct + REC_CL * N;
  __shared__ unsigned red[THREADS / 32];
  __shared__ unsigned vote[8];
  load_twiddles<R, N>(tw_s, tw);  // a constant table: read while the predecessor drains
  pdl_wait();
  pdl_trigger();
  const unsigned r = cluster_rank();
  const int l = blockIdx.y;
  const long long row0 = (long long)l * N + (long long)r * RB;
  R num[PER], den[PER];
  unsigned any = 1;
  if (!P.sums64) {
    plane_rec_pass<R, N, INC, R, PER>(P, prof, slot, cols, ncol, u0, l, r, rt, ct, tw_s, 0, num, den);
    bool bad = false;
#pragma unroll
    for (int p = 0; p < PER; ++p) bad |= !(isfinite(num[p]) && isfinite(den[p]));
    const unsigned mine = __syncthreads_or(bad) ? 1u : 0u;
    // every CTA of the cluster learns whether any of them overflowed
    if (threadIdx.x < C) dsmem_st(dsmem_addr(&vote[r], threadIdx.x), mine);
    cluster_sync();
    any = 0;
#pragma unroll
    for (int q = 0; q < C; ++q) any |= vote[q];
  }
  if (any) {
    // the sums left the range of R (|u| |V| beyond FP32 for huge evanescent profiles):
    // the cluster redoes the plane with FP64 sums, G elements per thread at a time;
    // the quotient goes through xi (written and read back by the same thread)
    unsigned gated = 0;
    for (int p0 = 0; p0 < PER; p0 += G) {
      double nd[G], dd[G];
      plane_rec_pass<R, N, INC, double, G>(P, prof, slot, cols, ncol, u0, l, r, rt, ct, tw_s, p0, nd, dd);
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const int e = threadIdx.x + (p0 + k) * THREADS;
        if (p0 + k < PER && e < E) {
          const bool g = !(dd[k] >= (double)P.n_omega * P.eps_u * P.eps_u);
          gated |= (g ? 1u : 0u) << (p0 + k);
          xi[(row0 + e / N) * N + (e % N)] = g ? R(0) : R(nd[k] / dd[k]);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * THREADS;
      const bool g = (gated >> p) & 1u;
      num[p] = (g || e >= E) ? R(0) : xi[(row0 + e / N) * N + (e % N)];
      den[p] = g ? R(0) : R(1);
    }
  }
  // after a redo den is 1 (kept) or 0 (guarded)
  recover_epilogue<R, PER, N>(P, num, den, any ? R(0.5) : R(P.u_guard), row0, (long long)P.m * N, E, xi, cout, ctr,
                              red);
}

template <typename R, int N, bool INC>
cudaError_t rec_plane(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s) {
  constexpr size_t smem = plane_rec_smem<R, N>();
  static SmemOptIn attr;
  cudaError_t e = opt_in_smem(attr, (const void*)k_ifft2_plane_recover<R, N, INC>, smem, true);
  if (e != cudaSuccess) return e;
  constexpr int C = plane_cluster<N>();
  e = launch_pdl_cluster(k_ifft2_plane_recover<R, N, INC>, dim3(C, (unsigned)P.m), dim3(THREADS), C, smem, s, P,
                         (const cx<R>*)w.prof, (const int*)w.slot, (const int*)w.cols, (const int*)w.ncol, w.u0, xi,
                         c, w.ctr, (const cx<R>*)w.tw);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, int N, int T>
cudaError_t rec_tiled(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  constexpr int TC = tile_cols<R, T>();
  // column chunks for the first GATHER_COLS active columns in the grid (the blocks loop
  // over more): the active columns are few in the usual case, and a grid of blocks that
  // return at once only delays the successor's launch (measured, 64-problem batch: 6.17
  // ms with every chunk in the grid, 6.07 with 32 columns; FP64 128^2 step +0.5 us)
  constexpr int NCH = (N + TC - 1) / TC, GZ = (GATHER_COLS + TC - 1) / TC;
  dim3 g1(P.m, 2 * P.n_omega, NCH < GZ ? NCH : GZ);
  cudaError_t e = launch_pdl(k_ifft_cols_gather<R, N, T>, g1, dim3(THREADS), 0, s, P, (const cx<R>*)w.prof,
                             (const int*)w.slot, (const int*)w.cols, (const int*)w.ncol, w.t2, (const cx<R>*)w.tw);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  constexpr int LINES = rec_lines<R, N, T>();
  constexpr size_t smem = rec_smem<R, N, T>();
  const long long nrows = (long long)P.m * N;
  const dim3 gr((unsigned)((nrows + LINES - 1) / LINES));
  static SmemOptIn attr[2];
  if (w.u0) {
    if ((e = opt_in_smem(attr[1], (const void*)k_ifft_rows_recover<R, N, true, T>, smem)) != cudaSuccess) return e;
    e = launch_pdl(k_ifft_rows_recover<R, N, true, T>, gr, dim3(THREADS), smem, s, P, (const cx<R>*)w.t2,
                   (const int*)w.cols, (const int*)w.ncol, w.u0, xi, c, w.ctr, (const cx<R>*)w.tw);
  } else {
    if ((e = opt_in_smem(attr[0], (const void*)k_ifft_rows_recover<R, N, false, T>, smem)) != cudaSuccess) return e;
    e = launch_pdl(k_ifft_rows_recover<R, N, false, T>, gr, dim3(THREADS), smem, s, P, (const cx<R>*)w.t2,
                   (const int*)w.cols, (const int*)w.ncol, w.u0, xi, c, w.ctr, (const cx<R>*)w.tw);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, int N>
cudaError_t rec_impl(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s, cudaEvent_t mid) {
  // the mixed path: one pass unless asked otherwise (N = 96, 192 and 256 hold too many
  // values per thread for the cluster pass: two passes)
  if constexpr (sizeof(R) == 4 && N <= 128 && N != 96) {
    if (P.inverse_single) {
      if (mid) cudaEventRecord(mid, s);
      return w.u0 ? rec_plane<R, N, true>(P, w, xi, c, s) : rec_plane<R, N, false>(P, w, xi, c, s);
    }
  }
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
