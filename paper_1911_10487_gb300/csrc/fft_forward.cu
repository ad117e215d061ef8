// Forward 2D FFT passes of Algorithm 2 (step 1) and the dense 2D transforms of the
// forward solvers and derivatives, for N = 2^a 3^b <= 256, in FP64 (double2) or FP32
// (float2).
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

template <typename R>
__global__ void k_twiddles(cx<R>* tw, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)n, &s, &c);
    tw[j] = from_d<R>(make_double2(c, s));
  }
}

// ---- single-pass forward 2D transform: one data plane per cluster ------------------
// grid (C, planes), clusters of C = fwd_cluster<N>() CTAs along x.  CTA r of the
// cluster of plane p loads rows r RB .. r RB + RB - 1 (RB = N / C) of the plane into
// its shared memory and transforms them along x; after a cluster barrier it reads
// columns r RB .. r RB + RB - 1 of all N rows from the CTAs that hold them
// (distributed shared memory), transforms them along y and writes them to W~.  The
// plane crosses global memory once each way, in one launch.
// clear (may be null): nclear counters zeroed by CTA (0, 0), as in k_fft_cols.
template <typename R, int N> __host__ __device__ constexpr size_t plane_fwd_smem() {
  constexpr int RB = N / fwd_cluster<N>();
  return sizeof(cx<R>) * ((size_t)LayIdx<Lay::ROW, N, RB, 16>::ELEMS + (size_t)RB * N + N);
}

template <typename R, int N>
__global__ void __launch_bounds__(THREADS)
k_fft2_plane(const cx<R>* __restrict__ in, cx<R>* __restrict__ out, const cx<R>* __restrict__ tw,
             unsigned* __restrict__ clear, int nclear) {
  constexpr int C = fwd_cluster<N>(), RB = N / C;
  using IA = LayIdx<Lay::ROW, N, RB, 16>;  // this CTA's rows
  constexpr int E = RB * N;                // elements of the row tile and of the column tile
  constexpr int PER = (E + THREADS - 1) / THREADS;
  extern __shared__ __align__(16) unsigned char plane_smem[];
  cx<R>* rows = reinterpret_cast<cx<R>*>(plane_smem);
  cx<R>* colt = rows + IA::ELEMS;  // column tile: element i of column b at i RB + b
  cx<R>* tw_s = colt + E;
  const unsigned r = cluster_rank();
  load_twiddles<R, N>(tw_s, tw);  // a constant table: read while the predecessor drains
  pdl_wait();
  pdl_trigger();
  if (clear && blockIdx.x == 0 && blockIdx.y == 0)
    for (int i = threadIdx.x; i < nclear; i += THREADS) clear[i] = 0u;
  const long long pb = (long long)blockIdx.y * N * N;
  const cx<R>* src = in + pb + (long long)r * E;
  cx<R> v[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (E % THREADS == 0 || e < E) v[p] = src[e];
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (E % THREADS == 0 || e < E) rows[IA::at(e / N, e % N)] = v[p];
  }
  __syncthreads();
  fft_lines<R, N, false, RB, THREADS, Lay::ROW, 16, 16>(rows, tw_s);
  cluster_sync();  // every CTA's rows are transformed
  // row i of column r RB + b sits in row i % RB of CTA i / RB: all loads first, then
  // the stores, so that the remote loads overlap
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (E % THREADS == 0 || e < E) {
      const int i = e / RB, b = e - (e / RB) * RB;
      v[p] = dsmem_ld(dsmem_addr(rows + IA::at(i % RB, (int)r * RB + b), (unsigned)(i / RB)), v[p]);
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (E % THREADS == 0 || e < E) colt[e] = v[p];
  }
  cluster_arrive();  // this CTA has read the others' rows
  __syncthreads();
  fft_lines<R, N, false, RB, THREADS, Lay::COL, 16>(colt, tw_s);
  cx<R>* dst = out + pb + (long long)r * RB;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * THREADS;
    if (E % THREADS == 0 || e < E) dst[(long long)(e / RB) * N + e % RB] = colt[e];
  }
  cluster_wait();  // no CTA leaves while another may still read its rows
}

template <typename R, int N>
cudaError_t fwd_plane(const cx<R>* W, const Problem& P, const Work<R>& w, cudaStream_t s, cudaEvent_t mid,
                      bool norms) {
  constexpr size_t smem = plane_fwd_smem<R, N>();
  static SmemOptIn attr;
  cudaError_t e = opt_in_smem(attr, (const void*)k_fft2_plane<R, N>, smem, true);
  if (e != cudaSuccess) return e;
  constexpr int C = fwd_cluster<N>();
  e = launch_pdl_cluster(k_fft2_plane<R, N>, dim3(C, (unsigned)(P.n_omega * P.m1)), dim3(THREADS), C, smem, s, W,
                         w.wt, (const cx<R>*)w.tw, norms ? (unsigned*)nullptr : w.bar, P.n_omega);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  if (!norms) return cudaGetLastError();
  return launch_mode_norms<R>(P, w, s);
}

// W (complex64) -> W~ (complex128 in w.wt64) and the norms: the forward transform
// of the mixed truncated-SVD route, in FP64
template <int N>
cudaError_t fwd_wide_impl(const float2* W, const Problem& P, const Work<float>& w, cudaStream_t s, cudaEvent_t mid) {
  constexpr int LINES = row_lines<double, N, 0>();
  const long long nrows = (long long)P.n_omega * P.m1 * N;
  const long long nblk = (nrows + LINES - 1) / LINES;
  cudaError_t e = launch_pdl(k_fft_rows<double, N, false, float2>, dim3((unsigned)nblk), dim3(THREADS), 0, s, W,
                             w.wt64, nrows, w.tw64, 1.0);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  const dim3 g2((N + tile_cols<double, 0>() - 1) / tile_cols<double, 0>(), (unsigned)(P.n_omega * P.m1));
  e = launch_pdl(k_fft_cols<double, N, false>, g2, dim3(THREADS), 0, s, w.wt64, w.tw64, (unsigned*)nullptr, 0);
  if (e != cudaSuccess) return e;
  const dim3 gn((unsigned)w.n_partial, (unsigned)P.n_omega);
  e = launch_pdl(k_mode_norms<double>, gn, dim3(NORM_T), 0, s, (const double2*)w.wt64, w.norms, w.partial, P.m1,
                 N * N, w.ctr);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, int N, int T>
cudaError_t fwd_tiled(const cx<R>* W, const Problem& P, const Work<R>& w, cudaStream_t s, cudaEvent_t mid,
                      bool norms) {
  constexpr int LINES = row_lines<R, N, T>();
  const long long nrows = (long long)P.n_omega * P.m1 * N;
  const long long nblk = (nrows + LINES - 1) / LINES;
  cudaError_t e = launch_pdl(k_fft_rows<R, N, false, cx<R>, T>, dim3((unsigned)nblk), dim3(THREADS), 0, s, W, w.wt,
                             nrows, (const cx<R>*)w.tw, R(1));
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  constexpr int TC = tile_cols<R, T>();
  const dim3 g2((N + TC - 1) / TC, (unsigned)(P.n_omega * P.m1));
  e = launch_pdl(k_fft_cols<R, N, false, T>, g2, dim3(THREADS), 0, s, w.wt, (const cx<R>*)w.tw,
                 norms ? (unsigned*)nullptr : w.bar, P.n_omega);
  if (e != cudaSuccess) return e;
  if (!norms) return cudaGetLastError();
  return launch_mode_norms<R>(P, w, s);
}

template <typename R, int N>
cudaError_t fwd_impl(const cx<R>* W, const Problem& P, const Work<R>& w, cudaStream_t s, cudaEvent_t mid,
                     bool norms) {
  if constexpr (std::is_same<R, float>::value) {
    if (w.wt64) return fwd_wide_impl<N>(W, P, w, s, mid);
    // N = 192 and 256: the cluster's row tiles (77 / 134 KB per CTA) leave one or two
    // CTAs per SM, and the two passes are faster (measured at 256^2 x 64, 29 planes, 6
    // frequencies: 0.139 ms vs 0.122 ms)
    if constexpr (N <= 128) {
      if (P.forward_single) return fwd_plane<R, N>(W, P, w, s, mid, norms);
    }
  }
  return P.fft_tile == 1 ? fwd_tiled<R, N, 1>(W, P, w, s, mid, norms) : fwd_tiled<R, N, 0>(W, P, w, s, mid, norms);
}

template <typename R, int N>
cudaError_t dense_impl(cx<R>* in, cx<R>* out, long long planes, bool inverse, const cx<R>* tw, cudaStream_t s) {
  constexpr int LINES = row_lines<R, N, 0>();
  constexpr long long MAX_Y = 32768;  // planes per column launch (grid y <= 65535)
  const long long nrows = planes * N;
  const unsigned nblk = (unsigned)((nrows + LINES - 1) / LINES);
  auto cols = [&](cx<R>* buf, bool inv) {
    for (long long p0 = 0; p0 < planes; p0 += MAX_Y) {
      const long long np = planes - p0 < MAX_Y ? planes - p0 : MAX_Y;
      const dim3 gc((N + tile_cols<R, 0>() - 1) / tile_cols<R, 0>(), (unsigned)np);
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
template cudaError_t launch_twiddles<double>(double2*, int, cudaStream_t);
template cudaError_t launch_twiddles<float>(float2*, int, cudaStream_t);

}  // namespace fl
