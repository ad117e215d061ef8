// Per-mode part of Algorithm 2: classification of the modes (discrepancy test)
// and, for every active mode nu, the regularised solution of the SLAE of eq. (8)
// followed by eq. (9) (Sec. 4 steps 1-2, Sec. 5.2).
//
// For every active mode one thread block:
//   1. builds A_nu[k, l] = omega^2 h_z K_nu(z_k - z'_l) (FP64) with the Weyl closed
//      form K_nu(dz) = -i exp(i k_z |dz|)/(2 k_z) (horizontal Fourier transform of
//      G = -exp(i k0 rho)/(4 pi rho)); every data plane lies above X, so
//      exp(i k_z (z_k - z'_l)) is evaluated as exp(i k_z (z_k - z'_top)) *
//      exp(i k_z (z'_top - z'_l)) with both factors of modulus <= 1;
//   2. applies the dual normal matrix G = A A^H (M1 x M1, Hermitian) only as
//      A (A^H q), never forming it;
//   3. reduces G to a real symmetric tridiagonal T = Q^H G Q by the Lanczos process
//      started from q_1 = b / ||b|| (full reorthogonalisation), stopped when the
//      Krylov space is invariant to working precision -- after two steps for these
//      kernels, whose matrices are rank one up to rounding;
//   4. picks alpha by the discrepancy principle: since q_1 = b / ||b|| and the
//      residual of the Tikhonov solution is b - A A^H y = alpha y,
//      phi(alpha) = ||A V~ - b|| = ||b|| alpha ||(T + alpha I)^-1 e_1||; the root of
//      phi = delta_nu lies in the bracket [alpha_floor, tr(G) delta_nu/(||b|| - delta_nu)],
//      alpha_floor = alpha_rel tr(G); phi(alpha_floor) >= delta_nu selects alpha_floor;
//   5. y = (G + alpha I)^-1 b, V~ = A^H y (the Tikhonov solution
//      (A^H A + alpha I)^-1 A^H b in its dual form);
//   6. U~ = U~0 + omega^2 T_nu V~ with T_nu[l, l'] = h_z K_nu(z'_l - z'_l'): since the
//      X planes are uniform, T_nu is h_z(-i/2k_z) q^|l-l'| with q = exp(i k_z h_z),
//      applied as one forward and one backward first-order recurrence (the z part
//      of the zero-padded convolution u = u0 + G * w, done exactly).
//
// Cost model on this GPU: a dependent FP64 operation costs ~64 cycles and an FP64
// division ~640, while FP32 runs at 64x the FP64 rate.  So every sequential chain
// (the Lanczos scalars, tridiagonal solves, the root-find) is kept short and runs
// in FP32 wherever the precision allows.
//  FS_FP64 : steps 2-3 in FP64; the root is seeded by an FP32 search on T and
//            finished by FP64 Newton steps in log(alpha) (reciprocals by
//            Newton-Raphson from an FP32 seed instead of FP64 division);
//            y = (||b||/tr) Q (T/tr + a I)^-1 e_1.
//  FS_MIXED: steps 2-4 in FP32 on the scaled problem; y is then refined against
//            the residual b - A (A^H y) - alpha y evaluated in two-float arithmetic
//            (about 48 bits), each correction solved from the Lanczos model
//            (exactly on its Krylov space, 1/alpha on the complement).  Modes whose
//            corrections do not contract or whose alpha/tr(G) falls below
//            fp64_switch, floor cases and FP32 breakdowns take the FS_FP64 route.
#include <math.h>

#include <atomic>

#include "modes.cuh"
#include "pipeline.cuh"
#include "twofloat.cuh"

// FL_PHASE_TIMING (development builds only) records clock64() at phase
// boundaries of the first mode of block 0; it is compiled out otherwise.
#ifdef FL_PHASE_TIMING
__device__ long long g_phase[24];
__device__ long long g_mode_cycles[4096];
__device__ int g_mode_sweeps[4096];
extern "C" int fs_debug_phases(long long* out) {
  return (int)cudaMemcpyFromSymbol(out, g_phase, sizeof(long long) * 24);
}
extern "C" int fs_debug_modes(long long* cycles, int* sweeps) {
  int e = (int)cudaMemcpyFromSymbol(cycles, g_mode_cycles, sizeof(long long) * 4096);
  if (e) return e;
  return (int)cudaMemcpyFromSymbol(sweeps, g_mode_sweeps, sizeof(int) * 4096);
}
#define FL_MARK(i) \
  if (blockIdx.x == 0 && (threadIdx.x & 31) == 0 && item == 0) g_phase[i] = clock64()
#define FL_MARK_S(i) \
  if (S.tflag && (threadIdx.x & 31) == 0) g_phase[i] = clock64()
#else
#define FL_MARK(i)
#define FL_MARK_S(i)
#endif

namespace fl {

namespace {

// Threads per solve block: 4 warps.  The per-mode critical path is warp 0's
// sequential part (Lanczos scalars, root, model solves); with 4 warps on the 4
// schedulers of an SM that warp does not share its issue slots with another warp
// of the same block (8 warps measured slower).  The per-mode code runs once per
// mode and is latency-bound, so its loops are not unrolled ("#pragma unroll 1"):
// unrolling only multiplies the code (measured 2-5 us slower per mode).
constexpr int ST = 128;
// Lanczos stops when the next off-diagonal of T is at most this fraction of
// tr(G): a few units of round-off of the normal matrix in each precision
constexpr float LANCZOS_TOL32 = 1e-6f;
constexpr double LANCZOS_TOL64 = 1e-14;
static_assert(ST == 2 * DENSE_M && ST == 4 * DENSE_M1, "thread maps of the solve assume 2 threads per plane l and 4 per data plane k");

// ------------------------------------------------------------------------------
// classification (integer arithmetic only), in two passes over blocks of CMB
// consecutive modes of one frequency:
//  k_classify_flags   delta_nu (every block sums the same norm partials in the
//                     same order), the active-mode bitmask, and per block the
//                     count of active and of grazing modes and a column mask;
//  k_classify_scatter slot and the ascending active list from the per-block
//                     prefix; block 0 of a frequency compacts the column list and
//                     adds the counters.
// Everything a later kernel reads is a fixed-order function of the inputs.
// ------------------------------------------------------------------------------
constexpr int CT = 256;            // threads per classify block
constexpr int CMB = 4 * CT;        // modes per classify block
constexpr int CWB = CMB / 32;      // bitmask words per block
constexpr int NWC = (MAX_N + 31) / 32;
static_assert((MAX_N * MAX_N + CMB - 1) / CMB <= 64, "the scatter prefix covers at most 64 blocks");

__global__ void __launch_bounds__(CT)
k_classify_flags(Problem P, const double* __restrict__ norms, const double* __restrict__ partial, int n_partial,
                 unsigned* __restrict__ flagbits, int* __restrict__ blkcnt, int* __restrict__ blkgz,
                 unsigned* __restrict__ colblk, double* __restrict__ dnu_out) {
  pdl_wait();
  pdl_trigger();
  const int om = blockIdx.y, b = blockIdx.x, CB = gridDim.x;
  const int N = P.n, N2 = N * N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ long long thr_bits;
  __shared__ unsigned cm[NWC];
  __shared__ int wc[CT / 32], wg[CT / 32];
  __shared__ double psum[CT / 32];
  if (threadIdx.x < NWC) cm[threadIdx.x] = 0u;
  {
    // ||W||^2 = sum_nu ||W~_nu||^2 / N^2 (Parseval): the block partial sums of the
    // norms kernel, thread-strided (up to eight loads of a thread in flight together),
    // then a tree over the lanes and the warps (the same order in every block)
    double s = 0.0;
    for (int i0 = threadIdx.x; i0 < n_partial; i0 += 8 * CT) {
      double v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = i0 + t * CT;
        v[t] = i < n_partial ? partial[(long long)om * n_partial + i] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) s += v[t];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) psum[wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = lane < CT / 32 ? psum[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      // ||W|| = sqrt(s / N^2) by the Newton reciprocal square root (no FP64 division or
      // square root on this block's critical path); every block computes it alike
      const double sn = s * P.inv_n2;
      const double wnorm = (sn > 0.0 && isfinite(sn)) ? sn * rsqrt64(sn) : sqrt(sn);
      const double dnu = P.dscale * wnorm;
      if (b == 0) dnu_out[om] = dnu;
      // a non-finite ||W|| (W holds a NaN or Inf, counted by the norms kernel) leaves
      // delta_nu undefined: no mode passes the test
      thr_bits = isfinite(dnu) ? __double_as_longlong(dnu * dnu) : 0x7fffffffffffffffLL;
    }
  }
  __syncthreads();
  // non-negative doubles order like their bit patterns: nrm > dnu^2 is an
  // integer comparison
  const long long tb = thr_bits;
  const int glo = P.graz_lo[om], ghi = P.graz_hi[om];
  const long long* nb = reinterpret_cast<const long long*>(norms + (long long)om * N2);
  int cnt = 0, ngz = 0;
#pragma unroll
  for (int k = 0; k < CMB / CT; ++k) {
    const int v = b * CMB + k * CT + threadIdx.x;
    bool on = false;
    if (v < N2) {
      const int i2 = v / N, i1 = v - i2 * N;
      const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
      const int msq = m1 * m1 + m2 * m2;
      const bool graz = msq >= glo && msq <= ghi;
      ngz += graz;
      on = !graz && (P.alpha_mode == 1 || nb[v] > tb);
      if (on) atomicOr(&cm[i1 >> 5], 1u << (i1 & 31));
    }
    const unsigned word = __ballot_sync(0xffffffffu, on);  // modes v0 .. v0 + 31, v0 = v - lane
    if (lane == 0) {
      flagbits[((long long)om * CB + b) * CWB + k * (CT / 32) + wid] = word;
      cnt += __popc(word);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ngz += __shfl_xor_sync(0xffffffffu, ngz, o);
  if (lane == 0) {
    wc[wid] = cnt;
    wg[wid] = ngz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0, g = 0;
    for (int w = 0; w < CT / 32; ++w) {
      c += wc[w];
      g += wg[w];
    }
    blkcnt[om * CB + b] = c;
    blkgz[om * CB + b] = g;
  }
  if (threadIdx.x < NWC) colblk[((long long)om * CB + b) * NWC + threadIdx.x] = cm[threadIdx.x];
}

__global__ void __launch_bounds__(CT)
k_classify_scatter(Problem P, const unsigned* __restrict__ flagbits, const int* __restrict__ blkcnt,
                   const int* __restrict__ blkgz, const unsigned* __restrict__ colblk, int* __restrict__ slot,
                   int* __restrict__ act, int* __restrict__ cols, int* __restrict__ ncol, int* __restrict__ count,
                   unsigned long long* __restrict__ ctr) {
  pdl_wait();
  pdl_trigger();
  const int om = blockIdx.y, b = blockIdx.x, CB = gridDim.x;
  const int N = P.n, N2 = N * N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ int base_s, total_s;
  __shared__ unsigned words[CWB];
  __shared__ int wpre[CWB];
  if (wid == 0) {
    // active modes of the blocks before this one (fixed order), and the total
    const int c0 = lane < CB ? blkcnt[om * CB + lane] : 0;
    const int c1 = lane + 32 < CB ? blkcnt[om * CB + lane + 32] : 0;
    int before = (lane < b ? c0 : 0) + (lane + 32 < b ? c1 : 0), all = c0 + c1;
    for (int o = 16; o > 0; o >>= 1) {
      before += __shfl_xor_sync(0xffffffffu, before, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    // exclusive prefix of the popcounts of this block's words (ascending modes)
    const unsigned w = flagbits[((long long)om * CB + b) * CWB + lane];
    const int c = __popc(w);
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    words[lane] = w;
    wpre[lane] = incl - c;
    if (lane == 0) {
      base_s = before;
      total_s = all;
    }
  }
  __syncthreads();
  static_assert(CWB == 32, "one warp holds the words of a block");
#pragma unroll
  for (int k = 0; k < CMB / CT; ++k) {
    const int v = b * CMB + k * CT + threadIdx.x;
    if (v < N2) {
      const int j = k * (CT / 32) + wid;
      const unsigned w = words[j];
      if (w >> lane & 1u) {
        const int pos = base_s + wpre[j] + __popc(w & ((1u << lane) - 1u));
        slot[(long long)om * N2 + v] = pos;
        act[(long long)om * N2 + pos] = v;
      } else {
        slot[(long long)om * N2 + v] = -1;
      }
    }
  }
  if (b == 0 && wid == 0) {  // columns holding an active mode, in order, and the counters
    int gz = 0;
    for (int i = lane; i < CB; i += 32) gz += blkgz[om * CB + i];
    for (int o = 16; o > 0; o >>= 1) gz += __shfl_xor_sync(0xffffffffu, gz, o);
    // OR of the blocks' column masks: lanes i and i + 32 load every word of blocks i and
    // i + 32 (all these loads in flight together), then one warp reduction per word
    static_assert(NWC <= 8 && 64 >= (MAX_N * MAX_N + CMB - 1) / CMB, "column words and blocks of one warp");
    const int nw = (N + 31) >> 5;
    unsigned cw[NWC];
#pragma unroll
    for (int w = 0; w < NWC; ++w) {
      unsigned a = 0u;
      if (w < nw) {
        if (lane < CB) a |= colblk[((long long)om * CB + lane) * NWC + w];
        if (lane + 32 < CB) a |= colblk[((long long)om * CB + lane + 32) * NWC + w];
      }
      cw[w] = a;
    }
    int base = 0;
#pragma unroll
    for (int w = 0; w < NWC; ++w) {
      if (w < nw) {
        unsigned cmw = __reduce_or_sync(0xffffffffu, cw[w]);
        if (w == 0) cmw |= 1u;  // the incident plane wave lives at nu = 0
        const int j = 32 * w + lane;
        const bool f = j < N && (cmw >> lane & 1u);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (f) cols[om * N + base + __popc(bal & ((1u << lane) - 1u))] = j;
        base += __popc(bal);
      }
    }
    if (lane == 0) {
      const int total = total_s;
      ncol[om] = base;
      count[om] = total;
      atomicAdd(ctr + C_MODES, (unsigned long long)N2);
      atomicAdd(ctr + C_COLUMNS, (unsigned long long)base);
      atomicAdd(ctr + C_ACTIVE, (unsigned long long)total);
      atomicAdd(ctr + C_GRAZING, (unsigned long long)gz);
      atomicAdd(ctr + C_ZEROED, (unsigned long long)(N2 - total - gz));
    }
  }
}

// ------------------------------------------------------------------------------
// single-pass classification: one cooperative launch, grid (CB, n_omega), blocks of
// CMB modes as above, in three phases separated by barriers over the blocks of a
// frequency:
//   1. the norms ||W~_nu||^2 of the block's modes (summed over the data planes in
//      plane order, in the working precision, kept in registers) and their block sum;
//   2. delta_nu from the CB block sums (every block adds them in the same order), the
//      active-mode bitmask (shared memory), the block's active and grazing counts and
//      column mask;
//   3. slots and the ascending active list from the prefix of the block counts;
//      block 0 compacts the columns and adds the counters.
// It replaces k_mode_norms, k_classify_flags and k_classify_scatter (three launches and
// their tails).  The barrier counters (Work::bar) are zeroed by the forward column
// pass.  Each wait polls at most BAR_POLLS times (about a quarter of a second); a wait
// that runs out adds to C_TIMEOUT and its block stops (fs_sync_status: FS_ETIMEOUT).
// ------------------------------------------------------------------------------
constexpr unsigned BAR_POLLS = 1u << 22;

// arrive at the barrier `bar` and wait until `target` blocks have arrived; false when
// the wait ran out (uniform over the block)
__device__ __forceinline__ bool grid_wait(unsigned* bar, unsigned target, unsigned polls_max,
                                          unsigned long long* ctr, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's writes before its arrival
    atomicAdd(bar, 1u);
    unsigned polls = 0;
    int ok = 1;
    while (*(volatile unsigned*)bar < target) {
      if (++polls > polls_max) {
        ok = 0;
        atomicAdd(ctr + C_TIMEOUT, 1ull);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();  // the other blocks' writes after the wait
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

constexpr int FT = CMB / 2;  // threads per block of the single-pass classification: two modes each

template <typename R>
__global__ void __launch_bounds__(FT)
k_classify_fused(Problem P, const cx<R>* __restrict__ wt, double* __restrict__ partial, unsigned* __restrict__ bar,
                 int* __restrict__ blkcnt, int* __restrict__ blkgz, unsigned* __restrict__ colblk,
                 int* __restrict__ slot, int* __restrict__ act, int* __restrict__ cols, int* __restrict__ ncol,
                 int* __restrict__ count, double* __restrict__ dnu_out, unsigned long long* __restrict__ ctr) {
  pdl_wait();
  pdl_trigger();
  const int om = blockIdx.y, b = blockIdx.x, CB = gridDim.x;
  const int N = P.n, N2 = N * N, M1 = P.m1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int K = CMB / FT;  // modes per thread
  constexpr int BATCH = sizeof(R) == 4 ? 16 : 8;  // plane loads in flight per thread
  __shared__ double red[FT / 32];
  __shared__ double thr_s;
  __shared__ unsigned cm[NWC];
  __shared__ int wc[FT / 32], wg[FT / 32];
  __shared__ unsigned words[CWB];
  __shared__ int wpre[CWB];
  __shared__ int base_s, total_s, ok_s;
  if (threadIdx.x < NWC) cm[threadIdx.x] = 0u;
  // phase 1: norms, BATCH planes' loads in flight, summed in plane order
  R nrm[K];
  double mine = 0.0;
  int bad = 0;
  const cx<R>* base = wt + (long long)om * M1 * N2;
#pragma unroll
  for (int k = 0; k < K; ++k) nrm[k] = R(0);
  for (int p = 0; p < M1; p += BATCH) {  // the K modes' loads of BATCH planes all in flight
    cx<R> q[K][BATCH];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int v = b * CMB + k * FT + threadIdx.x;
#pragma unroll
      for (int j = 0; j < BATCH; ++j)
        q[k][j] = (v < N2 && p + j < M1) ? base[(long long)(p + j) * N2 + v] : czero<R>();
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < BATCH; ++j) nrm[k] += q[k][j].x * q[k][j].x + q[k][j].y * q[k][j].y;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int v = b * CMB + k * FT + threadIdx.x;
    if (v < N2) bad += !isfinite(nrm[k]);
    mine += (double)nrm[k];
  }
  mine = warp_sum(mine);
  if (lane == 0) red[wid] = mine;
  const int n_bad = __syncthreads_count(bad);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < FT / 32; ++w) t += red[w];
    partial[om * CB + b] = t;
    if (n_bad) atomicAdd(ctr + C_NONFINITE, (unsigned long long)n_bad);
  }
  if (!grid_wait(bar + om, (unsigned)CB, BAR_POLLS, ctr, &ok_s)) return;
  // phase 2: delta_nu from the block sums (||W||^2 = sum_nu ||W~_nu||^2 / N^2, Parseval),
  // the same order in every block, then the bitmask
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = lane; i < CB; i += 32) t += __ldcg(partial + om * CB + i);
    t = warp_sum(t);
    if (lane == 0) {
      const double sn = t * P.inv_n2;  // as k_classify_flags
      const double dnu = P.dscale * ((sn > 0.0 && isfinite(sn)) ? sn * rsqrt64(sn) : sqrt(sn));
      if (b == 0) dnu_out[om] = dnu;
      // a non-finite ||W|| (W holds a NaN or Inf) leaves delta_nu undefined: no mode passes
      thr_s = isfinite(dnu) ? dnu * dnu : INFINITY;
    }
  }
  __syncthreads();
  const double thr = thr_s;
  const int glo = P.graz_lo[om], ghi = P.graz_hi[om];
  int cnt = 0, ngz = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int v = b * CMB + k * FT + threadIdx.x;
    bool on = false;
    if (v < N2) {
      const int i2 = v / N, i1 = v - i2 * N;
      const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
      const int msq = m1 * m1 + m2 * m2;
      const bool graz = msq >= glo && msq <= ghi;
      ngz += graz;
      on = !graz && (P.alpha_mode == 1 || (double)nrm[k] > thr);
      if (on) atomicOr(&cm[i1 >> 5], 1u << (i1 & 31));
    }
    const unsigned word = __ballot_sync(0xffffffffu, on);
    if (lane == 0) {
      words[k * (FT / 32) + wid] = word;
      cnt += __popc(word);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ngz += __shfl_xor_sync(0xffffffffu, ngz, o);
  if (lane == 0) {
    wc[wid] = cnt;
    wg[wid] = ngz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0, g = 0;
    for (int w = 0; w < FT / 32; ++w) {
      c += wc[w];
      g += wg[w];
    }
    blkcnt[om * CB + b] = c;
    blkgz[om * CB + b] = g;
  }
  if (threadIdx.x < NWC) colblk[((long long)om * CB + b) * NWC + threadIdx.x] = cm[threadIdx.x];
  if (!grid_wait(bar + om, 2u * (unsigned)CB, BAR_POLLS, ctr, &ok_s)) return;
  // phase 3: slots and the active list (as k_classify_scatter, the words from shared memory)
  if (wid == 0) {
    const int c0 = lane < CB ? __ldcg(blkcnt + om * CB + lane) : 0;
    const int c1 = lane + 32 < CB ? __ldcg(blkcnt + om * CB + lane + 32) : 0;
    int before = (lane < b ? c0 : 0) + (lane + 32 < b ? c1 : 0), all = c0 + c1;
    for (int o = 16; o > 0; o >>= 1) {
      before += __shfl_xor_sync(0xffffffffu, before, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    const unsigned w = words[lane];
    const int c = __popc(w);
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    wpre[lane] = incl - c;
    if (lane == 0) {
      base_s = before;
      total_s = all;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int v = b * CMB + k * FT + threadIdx.x;
    if (v < N2) {
      const int j = k * (FT / 32) + wid;
      const unsigned w = words[j];
      if (w >> lane & 1u) {
        const int pos = base_s + wpre[j] + __popc(w & ((1u << lane) - 1u));
        slot[(long long)om * N2 + v] = pos;
        act[(long long)om * N2 + pos] = v;
      } else {
        slot[(long long)om * N2 + v] = -1;
      }
    }
  }
  if (b == 0 && wid == 0) {  // columns holding an active mode, in order, and the counters
    int gz = 0;
    for (int i = lane; i < CB; i += 32) gz += __ldcg(blkgz + om * CB + i);
    for (int o = 16; o > 0; o >>= 1) gz += __shfl_xor_sync(0xffffffffu, gz, o);
    int cbase = 0;
    for (int j0 = 0; j0 < N; j0 += 32) {
      unsigned cmw = 0u;
      for (int i = lane; i < CB; i += 32) cmw |= __ldcg(colblk + ((long long)om * CB + i) * NWC + (j0 >> 5));
      cmw = __reduce_or_sync(0xffffffffu, cmw);
      if (j0 == 0) cmw |= 1u;  // the incident plane wave lives at nu = 0
      const int j = j0 + lane;
      const bool f = j < N && (cmw >> lane & 1u);
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (f) cols[om * N + cbase + __popc(bal & ((1u << lane) - 1u))] = j;
      cbase += __popc(bal);
    }
    if (lane == 0) {
      const int total = total_s;
      ncol[om] = cbase;
      count[om] = total;
      atomicAdd(ctr + C_MODES, (unsigned long long)N2);
      atomicAdd(ctr + C_COLUMNS, (unsigned long long)cbase);
      atomicAdd(ctr + C_ACTIVE, (unsigned long long)total);
      atomicAdd(ctr + C_GRAZING, (unsigned long long)gz);
      atomicAdd(ctr + C_ZEROED, (unsigned long long)(N2 - total - gz));
    }
  }
}

// ------------------------------------------------------------------------------
// scalar helpers
// ------------------------------------------------------------------------------

// ------------------------------------------------------------------------------
// shared state of one block
// ------------------------------------------------------------------------------
// The union below holds what one phase of a mode needs and is dead in the next:
// the FP64 route's Lanczos basis, the mixed route's FP32 model (whose copy of A is
// dead after the Lanczos process, so the root search reuses it), and the arrays of
// eq. (9), written once the solve is done.
template <typename B> struct Bulk {
  cx<B> V[DENSE_M1][DENSE_M1 + 1];  // Lanczos basis, column j = q_j (FP64 route)
  cx<B> t[DENSE_M];               // A^H q_j of the Lanczos step
  cx<B> w[DENSE_M1];              // G q_j of the Lanczos step
};
struct BulkF {
  float2 Q[DENSE_M1][DENSE_M1 + 1];  // Lanczos basis, column j = q_j
  float2 t[DENSE_M];               // A^H q_j of the Lanczos step
  float2 w[DENSE_M1];              // G q_j of the Lanczos step
  float2 p[DENSE_M1];              // model solve (T + a I)^-1 Q^H r
  union {
    float2 A[DENSE_M1][DENSE_M + 1];  // A_nu / sqrt(tr G) in FP32, for the Lanczos products
    struct {
      float2 ts[DENSE_M1][32];  // per-lane tridiagonal solves of the root search: scaled values
      float tmu[DENSE_M1][32];  //                                                 and multipliers
    } rs;
  } m;
};
struct Eq9 {
  double2 Vt[DENSE_M], t[DENSE_M], F[DENSE_M], Bk[DENSE_M], z64[DENSE_M];
};

struct Shared {
  double2 A[DENSE_M1][DENSE_M + 1];  // A_nu in FP64 (FP64 route), Ah in two-float (mixed route)
  union { Bulk<double> d; BulkF f; Eq9 q; } u;
  double2 E[DENSE_M1], Pz[DENSE_M], b[DENSE_M1], c[DENSE_M1], y[DENSE_M1], z[DENSE_M1];
  double2 Tk[DENSE_M];  // sampled kernel: row omega^2 h_z K~(j h_z) of the Toeplitz T_nu of eq. (9)
  double d[DENSE_M1], e[DENSE_M1];     // tridiagonal T (FP64 route: of G; scaled by 1/tr after the factor)
  float d32[DENSE_M1], e32[DENSE_M1];  // T / tr in FP32
  float2 c32[DENSE_M1], r32[DENSE_M1];
  ffc yh[DENSE_M1], bh[DENSE_M1], th[DENSE_M], Ef[DENSE_M1], Pf[DENSE_M];  // two-float (mixed route)
  double tr, sb, inv_sb, dnu, lo, hi, a_s, red[8];  // a_s = alpha / tr
  double2 qz;  // exp(i k_z h_z)
  int fp64, tflag, kd, go;  // kd: dimension of the Lanczos model; go: Lanczos continues
};
static_assert(sizeof(Shared) <= 75 * 1024, "three solve blocks per SM");


// Lanczos tridiagonalisation of the Hermitian G = A A^H (n x n; A is n x m in
// shared memory) from the unit vector in column 0 of Q, with full
// reorthogonalisation (classical Gram-Schmidt, twice): Q^H G Q = T, real symmetric
// tridiagonal with diagonal d and off-diagonal e >= 0.  G is never formed: each
// step applies it as A (A^H q_j), 2 n m complex products instead of the n^2 m of
// the normal matrix, spread over the whole block (two threads per column of A for
// t = A^H q_j, four per row for A t); warp 0 then orthogonalises (lane r owning
// row r).  Stops when the next off-diagonal is not above tol (the Krylov space of
// q_0 is then invariant to that level) or at n columns, and returns the number k
// of columns (the same in every thread).  Called by all ST threads; t (m entries),
// w (n entries) and *go are scratch.
// The (1,1) entries of (T + a I)^-1 and (T + a I)^-2, from which the discrepancy
// is computed, depend on e only through the squares e_j^2, so stopping at
// e_k <= tol changes phi^2 by O(tol^2 / a^2) relative.
template <typename T>
__device__ int lanczos_block(const cx<T> (*A)[DENSE_M + 1], int n, int m, cx<T>* t, cx<T>* wv,
                             cx<T> (*Q)[DENSE_M1 + 1], T* d, T* e, T tol, int* go) {
  const int lane = threadIdx.x & 31;
  int k = n;
#pragma unroll 1
  for (int j = 0; j < n; ++j) {
    {  // t = A^H q_j: two threads per column l
      const int l = threadIdx.x >> 1, h = threadIdx.x & 1;
      cx<T> acc = czero<T>();
      if (l < m)
#pragma unroll 1
        for (int r = h; r < n; r += 2) acc = acc + cmul_conj_a(A[r][l], Q[r][j]);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      if (l < m && h == 0) t[l] = acc;
    }
    __syncthreads();
    {  // w = A t = G q_j: four threads per row r
      const int r = threadIdx.x >> 2, h = threadIdx.x & 3;
      cx<T> acc = czero<T>();
      if (r < n)
#pragma unroll 1
        for (int l = h; l < m; l += 4) acc = acc + A[r][l] * t[l];
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (r < n && h == 0) wv[r] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      cx<T> w = lane < n ? wv[lane] : czero<T>();
      const cx<T> qj = lane < n ? Q[lane][j] : czero<T>();
      const T aj = warp_sum(qj.x * w.x + qj.y * w.y);  // q_j^H G q_j (real)
      w = w - aj * qj;
      if (j > 0 && lane < n) w = w - e[j - 1] * Q[lane][j - 1];
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {  // w -= Q (Q^H w) over q_0 .. q_j
        cx<T> corr = czero<T>();
#pragma unroll 1
        for (int i = 0; i <= j; ++i) {
          const cx<T> qi = lane < n ? Q[lane][i] : czero<T>();
          const cx<T> hh = warp_sum(cmul_conj_a(qi, w));  // q_i^H w
          corr = corr + qi * hh;
        }
        w = w - corr;
      }
      const T beta = sqrt(warp_sum(abs2(w)));
      const bool stop = j + 1 == n || !(beta > tol);
      if (lane == 0) {
        d[j] = aj;
        if (!stop) e[j] = beta;
        *go = stop ? 0 : 1;
      }
      if (!stop && lane < n) Q[lane][j + 1] = rcp<T>(beta) * w;
    }
    __syncthreads();
    if (!*go) {
      k = j + 1;
      break;
    }
  }
  return k;
}

// (T + a I) z = rhs, T real symmetric tridiagonal (d, e); single thread.
// Returns false if a pivot is not positive (T + a I not numerically SPD).
template <typename T>
__device__ bool tri_solve(const T* d, const T* e, int n, T a, const cx<T>* rhs, cx<T>* z) {
  T mu[DENSE_M1], il[DENSE_M1];
  T lp = d[0] + a;
  if (!(lp > T(0))) return false;
  il[0] = rcp<T>(lp);
  mu[0] = T(0);
  z[0] = rhs[0];
#pragma unroll 1
  for (int i = 1; i < n; ++i) {
    mu[i] = e[i - 1] * il[i - 1];
    lp = d[i] + a - mu[i] * e[i - 1];
    if (!(lp > T(0))) return false;
    il[i] = rcp<T>(lp);
    z[i] = rhs[i] - mu[i] * z[i - 1];
  }
#pragma unroll 1
  for (int i = 0; i < n; ++i) z[i] = il[i] * z[i];
#pragma unroll 1
  for (int i = n - 2; i >= 0; --i) z[i] = z[i] - mu[i + 1] * z[i + 1];
  return true;
}

__device__ __forceinline__ float exp_t(float t) { return expf(t); }
__device__ __forceinline__ double exp_t(double t) { return exp(t); }
__device__ __forceinline__ float log_t(float t) { return logf(t); }
__device__ __forceinline__ double log_t(double t) { return log(t); }

// Safeguarded Newton in t = log(a) on g(t) = log(a^2 ||(T + a I)^-1 c||^2) - log(target),
// on the scaled problem (T = G / tr, c = D^H Q^H b / ||b||, a = alpha / tr), single
// thread.  [lo, hi] brackets the root (g(lo) < 0 < g(hi)); t0 is the start.
// Returns t; gp = dg/dt at the last point; ok = false on a breakdown.
template <typename T>
__device__ double newton_log_alpha(const T* d, const T* e, const cx<T>* c, int n, double lo, double hi,
                                   double target, double t0, double tol, int max_iter, double& gp_out,
                                   bool& ok, int& iters) {
  cx<T> z[DENSE_M1], s[DENSE_M1];
  T tl = log_t((T)lo), th = log_t((T)hi), t = (T)t0;
  const T lt = log_t((T)target);
  const T eps_t = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
  gp_out = 0.0;
  ok = true;
  int it = 0;
#pragma unroll 1
  for (; it < max_iter; ++it) {
    const T a = exp_t(t);
    if (!tri_solve<T>(d, e, n, a, c, z)) { ok = false; break; }
    T zz = T(0);
#pragma unroll 1
    for (int i = 0; i < n; ++i) zz += abs2(z[i]);
    const T g = log_t(a * a * zz) - lt;
    if (g > T(0)) th = t; else tl = t;
    if (!tri_solve<T>(d, e, n, a, z, s)) { ok = false; break; }
    T zs = T(0);
#pragma unroll 1
    for (int i = 0; i < n; ++i) zs += z[i].x * s[i].x + z[i].y * s[i].y;
    const T gp = T(2) - T(2) * a * zs * rcp<T>(zz);  // d log(a^2 ||z||^2) / d log a
    gp_out = (double)gp;
    if (fabs(g) < (T)tol || th - tl < eps_t * fmax(T(1), fabs(t))) break;
    T tn = (gp > T(0)) ? t - g * rcp<T>(gp) : T(0.5) * (tl + th);
    if (!(tn > tl && tn < th)) tn = T(0.5) * (tl + th);
    t = tn;
  }
  iters = it;
  return (double)t;
}

// a^2 ||(T + a I)^-1 c||^2 in precision T; single thread.
template <typename T>
__device__ double phi2(const T* d, const T* e, const cx<T>* c, int n, double a, bool& ok) {
  cx<T> z[DENSE_M1];
  ok = tri_solve<T>(d, e, n, (T)a, c, z);
  T zz = T(0);
#pragma unroll 1
  for (int i = 0; i < n; ++i) zz += abs2(z[i]);
  return a * a * (double)zz;
}

// block-wide sums of one double per thread (all threads get them)

// FP64 route: FP64 Lanczos model of the normal matrix, FP32-seeded root on the
// scaled tridiagonal, FP64 Newton to full accuracy, y = (||b||/tr) Q (T/tr + a I)^-1 e_1.
__device__ void solve_fp64(Shared& S, int n, int m, const Problem& P, int om, unsigned long long* ctr) {
  FL_MARK_S(13);
  Bulk<double>& K = S.u.d;
  const double inv_sb = rcp64(S.sb), inv_tr = rcp64(S.tr);
  if (threadIdx.x < n) K.V[threadIdx.x][0] = inv_sb * S.b[threadIdx.x];
  __syncthreads();
  const int kd = lanczos_block<double>(S.A, n, m, K.t, K.w, K.V, S.d, S.e, LANCZOS_TOL64 * S.tr, &S.go);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane < kd) {  // scaled model T / tr, c = e_1, and FP32 copies for the seed
      S.d[lane] *= inv_tr;
      S.d32[lane] = (float)S.d[lane];
      if (lane + 1 < kd) {
        S.e[lane] *= inv_tr;
        S.e32[lane] = (float)S.e[lane];
      }
      S.c[lane] = make_double2(lane == 0 ? 1.0 : 0.0, 0.0);
      S.c32[lane] = make_float2(lane == 0 ? 1.f : 0.f, 0.f);
    }
    if (lane == 0) S.kd = kd;
  }
  __syncthreads();
  FL_MARK_S(14);
  if (threadIdx.x == 0) {
    const double target = (S.dnu * inv_sb) * (S.dnu * inv_sb);
    const double lo = P.alpha_rel, hi = S.hi * inv_tr;
    bool ok = true;
    double a;
    if (P.alpha_mode == 1) {
      a = P.alpha_given[om] * inv_tr;
    } else if (phi2<double>(S.d, S.e, S.c, kd, lo, ok) >= target) {
      a = lo;
      atomicAdd(ctr + C_ALPHA_FLOOR, 1ull);
    } else {
      double gp;
      bool ok32;
      int it32, it64;
      const double t_mid = 0.5 * (log(lo) + log(hi));
      double t = newton_log_alpha<float>(S.d32, S.e32, S.c32, kd, lo, hi, target, t_mid, 1e-5, P.max_iter, gp,
                                         ok32, it32);
      if (!ok32 || !(t > log(lo) && t < log(hi))) t = t_mid;
      t = newton_log_alpha<double>(S.d, S.e, S.c, kd, lo, hi, target, t, 1e-14, P.max_iter, gp, ok, it64);
      if (it64 >= P.max_iter) atomicAdd(ctr + C_ROOT_CAPPED, 1ull);
      a = exp(t);
    }
    S.a_s = a;
    tri_solve<double>(S.d, S.e, kd, a, S.c, S.z);
  }
  __syncthreads();
  FL_MARK_S(15);
  if (threadIdx.x < n) {  // y = (||b|| / tr) Q z
    double2 acc = make_double2(0, 0);
#pragma unroll 1
    for (int j = 0; j < kd; ++j) acc = acc + K.V[threadIdx.x][j] * S.z[j];
    S.y[threadIdx.x] = (S.sb * inv_tr) * acc;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------
// mixed precision route: warp-synchronous FP32 factorisation held in registers
// ------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ cx<T> pick(const cx<T>* v, int j) {  // v[j] for a runtime j, register-resident v
  cx<T> r = czero<T>();
#pragma unroll
  for (int c = 0; c < DENSE_M1; ++c)
    if (c == j) r = v[c];
  return r;
}

// Approximate (G + a I)^-1 r from the Lanczos model of the FP32 normal matrix,
// exact on the Krylov space spanned by the model and r/a on its orthogonal
// complement:  Q (T + a I)^-1 Q^H r + (r - Q Q^H r)/a.  The complement holds the
// eigenvalues the Lanczos process did not reach, round-off for these kernels
// (rank one in exact arithmetic); the refinement around it checks that its
// corrections contract and sends the mode to the FP64 route otherwise.  Warp 0,
// lane k holding r_k (zero for lanes >= n).
__device__ float2 lanczos_apply32(Shared& S, int n, int kd, float a, float2 r) {
  BulkF& K = S.u.f;
  const int lane = threadIdx.x & 31;
  float2 mine = make_float2(0.f, 0.f), proj = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int i = 0; i < kd; ++i) {
    const float2 qi = lane < n ? K.Q[lane][i] : make_float2(0.f, 0.f);
    const float2 ci = warp_sum(cmul_conj_a(qi, r));  // q_i^H r
    if (lane == i) mine = ci;
    proj = proj + qi * ci;
  }
  if (lane < kd) S.c32[lane] = mine;
  __syncwarp();
  if (lane == 0) tri_solve<float>(S.d32, S.e32, kd, a, S.c32, K.p);  // z = (T + a I)^-1 Q^H r
  __syncwarp();
  float2 y = make_float2(0.f, 0.f);
  if (lane < n) {
#pragma unroll 1
    for (int i = 0; i < kd; ++i) y = y + K.Q[lane][i] * K.p[i];
    y = y + rcp<float>(a) * (r - proj);
  }
  __syncwarp();
  return y;
}

// Ah^H yh (two-float, m columns): two threads per column l, lanes 8 apart (l = t mod 8 +
// 8 (t / 16)), each summing every other row in two compensated chains.  Eight
// consecutive threads read eight consecutive columns of one row: the 16-byte loads of a
// quarter warp fall on distinct banks.  Returns the column sum on both threads.
__device__ __forceinline__ ffc colsum_ff(const ffc (*Af)[DENSE_M + 1], const ffc* yh, int n, int l, int h) {
  dot2c a0 = dot2c_zero(), a1 = dot2c_zero();
#pragma unroll 1
  for (int k = h; k < n; k += 4) {
    dot2c_conj_mac(a0, Af[k][l], yh[k]);
    if (k + 2 < n) dot2c_conj_mac(a1, Af[k + 2][l], yh[k + 2]);
  }
  ffc acc = ffc_add(dot2c_ffc(a0), dot2c_ffc(a1));
  return ffc_add(acc, ffc_shfl_xor(acc, 8));
}

// two-float residual of the scaled dual system: th = Ah^H yh, rh = bh - Ah th - a yh
__device__ void residual_ff(Shared& S, int n, int m, ff a) {
  const ffc (*Af)[DENSE_M + 1] = reinterpret_cast<const ffc (*)[DENSE_M + 1]>(S.A);
  {  // 2 threads per column l
    const int t = threadIdx.x, l = (t & 7) + 8 * (t >> 4), h = (t >> 3) & 1;
    const bool on = l < m;
    const ffc acc = colsum_ff(Af, S.yh, on ? n : 0, l, h);
    if (on && h == 0) S.th[l] = acc;
  }
  __syncthreads();
  {  // 4 threads per row k (lanes 8 apart): eight consecutive rows at one column per
     // quarter warp, distinct banks (row stride 65 entries)
    const int t = threadIdx.x, k = (t & 7) + 8 * (t >> 5), h = (t >> 3) & 3;
    dot2c a0 = dot2c_zero(), a1 = dot2c_zero();
    if (k < n)
#pragma unroll 1
      for (int l = h; l < m; l += 8) {
        dot2c_mac(a0, Af[k][l], S.th[l]);
        if (l + 4 < m) dot2c_mac(a1, Af[k][l + 4], S.th[l + 4]);
      }
    ffc acc = ffc_add(dot2c_ffc(a0), dot2c_ffc(a1));
    acc = ffc_add(acc, ffc_shfl_xor(acc, 8));
    acc = ffc_add(acc, ffc_shfl_xor(acc, 16));
    if (k < n && h == 0) {
      const ffc ay = ffc{ff_mul(a, S.yh[k].re), ff_mul(a, S.yh[k].im)};
      const ffc r = ffc_sub(ffc_sub(S.bh[k], acc), ay);
      S.r32[k] = make_float2(r.re.hi, r.im.hi);
    }
  }
  __syncthreads();
}

// (T + a I) z = c with per-lane scratch in shared memory; returns a^2 ||z||^2 (FP32 T)
__device__ float lane_phi2(Shared& S, int n, float a, const float2* c, bool& ok) {
  BulkF& K = S.u.f;
  const int L = threadIdx.x & 31;
  float lp = S.d32[0] + a;
  ok = lp > 0.f;
  float il = __fdividef(1.f, lp);
  float2 w = c[0];
  K.m.rs.ts[0][L] = il * w;
#pragma unroll 1
  for (int i = 1; i < n; ++i) {
    const float mu = S.e32[i - 1] * il;
    lp = S.d32[i] + a - mu * S.e32[i - 1];
    ok = ok && lp > 0.f;
    il = __fdividef(1.f, lp);
    w = c[i] - mu * w;
    K.m.rs.tmu[i][L] = mu;
    K.m.rs.ts[i][L] = il * w;
  }
  float2 x = K.m.rs.ts[n - 1][L];
  float zz = abs2(x);
#pragma unroll 1
  for (int i = n - 2; i >= 0; --i) {
    x = K.m.rs.ts[i][L] - K.m.rs.tmu[i + 1][L] * x;
    zz += abs2(x);
  }
  return a * a * zz;
}

// Discrepancy root on the scaled FP32 model by three rounds of a 32-point search
// in log(a) (one point per lane) and a final secant step.  Warp 0.  Returns a;
// floor = g(lo) >= 0; ok = false on a breakdown.
__device__ float root32_warp(Shared& S, int n, float lo, float hi, float target, bool& floor_case, bool& ok) {
  const int lane = threadIdx.x;
  float tl = logf(lo), th = logf(hi);
  const float lt = logf(target);
  float gl = 0.f, gh = 0.f;
  floor_case = false;
  ok = true;
#pragma unroll 1
  for (int round = 0; round < 3; ++round) {
    const float t = tl + (th - tl) * (float)lane * (1.f / 31.f);
    bool okl;
    const float f = lane_phi2(S, n, expf(t), S.c32, okl);
    const float g = logf(f) - lt;
    if (!__all_sync(0xffffffffu, okl && isfinite(g))) { ok = false; return 0.f; }
    const unsigned above = __ballot_sync(0xffffffffu, g >= 0.f);
    if (round == 0 && (above & 1u)) { floor_case = true; return lo; }
    const int k = above ? __ffs(above) - 1 : 31;  // first grid point at or above the target
    const float gk = __shfl_sync(0xffffffffu, g, k), gk1 = __shfl_sync(0xffffffffu, g, k > 0 ? k - 1 : 0);
    const float tk = __shfl_sync(0xffffffffu, t, k), tk1 = __shfl_sync(0xffffffffu, t, k > 0 ? k - 1 : 0);
    if (!above) return expf(th);  // phi stays below target up to hi: cannot happen for an active mode
    tl = tk1; th = tk; gl = gk1; gh = gk;
  }
  const float t = gh > gl ? tl + (th - tl) * (-gl / (gh - gl)) : 0.5f * (tl + th);
  return expf(t);
}

// The block's shared state through the dynamic shared-memory symbol, so that an
// out-of-line device function addresses it with shared-memory instructions.
extern __shared__ __align__(16) unsigned char smem_dyn[];
__device__ __forceinline__ Shared& shm() { return *reinterpret_cast<Shared*>(smem_dyn); }

// U~ - U~0 = gamma (F + B) of eq. (9): the forward recurrence F_l = q F_{l-1} + V~_l
// and the backward one B_l = q (B_{l+1} + V~_{l+1}), each an inclusive scan over
// the planes (warp 0: F, warp 1: B in reversed order).  Kept out of line: compiled
// on its own, this FP64 code runs about three times faster than inlined into the
// solve kernel (measured).
__device__ __noinline__ void eq9_scans(int m) {
  Shared& S = shm();
  if (threadIdx.x < 64) {
    const double2 qz = S.qz;
    if (threadIdx.x < 32) {
      affine_scan64(S.u.q.Vt, m, qz, S.u.q.F);
    } else {
      const int r = threadIdx.x - 32;  // reversed sequence s'_r = q V~_{m-r} (s'_0 = 0)
#pragma unroll 1
      for (int rr = r; rr < m; rr += 32) S.u.q.t[rr] = rr == 0 ? make_double2(0, 0) : qz * S.u.q.Vt[m - rr];
      __syncwarp();
      affine_scan64(S.u.q.t, m, qz, S.u.q.z64);
      __syncwarp();
#pragma unroll 1
      for (int rr = r; rr < m; rr += 32) S.u.q.Bk[m - 1 - rr] = S.u.q.z64[rr];
    }
  }
}

// SAMPLED: A_nu and the row of T_nu come from the tables of a kernel plan (the
// sampled-G kernel: ktab, ktr, layout in Work::ktab) instead of the Weyl closed form;
// eq. (9) is then the Toeplitz product itself rather than its recurrences.
template <typename B, bool MIXED, bool SAMPLED>
__global__ void __launch_bounds__(ST)
k_solve(Problem P, const cx<B>* __restrict__ wt, const int* __restrict__ act,
        const int* __restrict__ count, const double* __restrict__ dnu_arr,
        cx<B>* __restrict__ prof, double* __restrict__ alpha_out, unsigned long long* __restrict__ ctr,
        const void* __restrict__ ktab, const double* __restrict__ ktr) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared& S = *reinterpret_cast<Shared*>(smem_raw);
  const int N = P.n, n = P.m1, m = P.m;
  const long long N2 = (long long)N * N;
  long long total = 0;
#pragma unroll 1
  for (int w = 0; w < P.n_omega; ++w) total += count[w];
#pragma unroll 1
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    int om = 0;
    long long i = item;
    while (i >= count[om]) { i -= count[om]; ++om; }
    const int nu = act[om * N2 + i];
    FL_MARK(0);
#ifdef FL_PHASE_TIMING
    if (threadIdx.x == 0) S.tflag = blockIdx.x == 0 && item == 0;
    const long long t_mode0 = clock64();
#endif
    const int i2 = nu / N, i1 = nu - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const double k0 = P.k0[om], kn = P.kn;
    const double q = k0 * k0 - kn * kn * (double)(m1 * m1 + m2 * m2);
    // k_z = sqrt(|q|) (real, or i sqrt(|q|) for an evanescent mode; active modes are
    // never grazing, q != 0) and 1/k_z from one reciprocal square root
    const double rq = rsqrt64(fabs(q));
    const double2 kz = q >= 0.0 ? make_double2(fabs(q) * rq, 0.0) : make_double2(0.0, fabs(q) * rq);
    // gamma = omega^2 h_z (-i / (2 k_z))
    const double g0 = P.g0[om];
    const double2 gamma = q >= 0.0 ? make_double2(0.0, -g0 * rq) : make_double2(-g0 * rq, 0.0);
    const double ztop = P.z1 + (m - 0.5) * P.hz;
    const long long mb = ((long long)om * N2 + nu) * (long long)(n * m + m);  // the mode's table row
    // the exponentials, one per thread: threads 0..63 take P, threads 64..95 take E
    // (FP32 in the mixed route), thread 96 the plane-to-plane factor q of eq. (9)
    // in FP64 (the mixed route takes it later, while warp 0 finds the root).  The
    // sampled kernel reads the row of T_nu (threads 0..63) instead.
    if (SAMPLED) {
      if (threadIdx.x < m) {
        const long long at = mb + n * m + threadIdx.x;
        if (MIXED) {
          const float4 v = reinterpret_cast<const float4*>(ktab)[at];
          S.Tk[threadIdx.x] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
        } else {
          S.Tk[threadIdx.x] = reinterpret_cast<const double2*>(ktab)[at];
        }
      } else if (threadIdx.x >= DENSE_M && threadIdx.x < DENSE_M + n) {
        const int k = threadIdx.x - DENSE_M;
        S.b[k] = to_d(wt[((long long)om * n + k) * N2 + nu]);
      }
    } else if (threadIdx.x < m) {
      const int l = threadIdx.x;
      S.Pz[l] = MIXED ? exp_ikz32(kz, ztop - (P.z1 + (l + 0.5) * P.hz)) : exp_ikz(kz, ztop - (P.z1 + (l + 0.5) * P.hz));
      if (MIXED) S.Pf[l] = ffc_from(S.Pz[l]);
    } else if (threadIdx.x >= DENSE_M && threadIdx.x < DENSE_M + n) {
      const int k = threadIdx.x - DENSE_M;
      S.b[k] = to_d(wt[((long long)om * n + k) * N2 + nu]);
      S.E[k] = gamma * (MIXED ? exp_ikz32(kz, P.zy[k] - ztop) : exp_ikz(kz, P.zy[k] - ztop));
    } else if (!MIXED && threadIdx.x == DENSE_M + DENSE_M1) {
      S.qz = exp_ikz(kz, P.hz);
    }
    __syncthreads();
    FL_MARK(1);
    // ||A||_F^2 = tr(G) = (sum_k |E_k|^2)(sum_l |P_l|^2) since A_kl = E_k P_l, and ||b||^2, in
    // FP64 in both routes (|E|^2 and |P|^2 of strongly evanescent modes leave the FP32
    // range), one sum per warp: a warp issues its FP64 instructions one per 64 cycles,
    // so the FP64 work of a mode is spread over the warps
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      double v = 0.0;
      if (wid == 0) v = (lane < m ? abs2(S.Pz[lane]) : 0.0) + (lane + 32 < m ? abs2(S.Pz[lane + 32]) : 0.0);
      else if (wid == 1) v = lane < n ? abs2(S.b[lane]) : 0.0;
      else if (wid == 2) v = lane < n ? abs2(S.E[lane]) : 0.0;
      if (SAMPLED && wid != 1) {
        // tr(G) from the plan: S.red[0] S.red[2] = tr
        if (wid < 3 && lane == 0) S.red[wid] = wid == 0 ? ktr[(long long)om * N2 + nu] : 1.0;
      } else if (wid < 3) {
        v = warp_sum(v);
        if (lane == 0) S.red[wid] = v;
      }
    }
    __syncthreads();
    FL_MARK(3);
    {
      // the scalars of the mode, and in the mixed route the scaled factors of A and b in
      // two-float (warp 0: E, warp 1: b, warp 3: the root bracket)
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      const double tr = S.red[0] * S.red[2], bb = S.red[1];
      // 1/||b||: FP32 seed and one FP64 Newton step in the mixed route (||bh|| = 1 to
      // FP64), the full FP64 reciprocal square root otherwise
      const auto inv_norm_b = [&]() {
        if (!MIXED) return rsqrt64(bb);
        const double y = rsqrt32(bb);
        return fma(0.5 * y, fma(-bb * y, y, 1.0), y);
      };
      if (MIXED && !SAMPLED && wid == 0 && lane < n) {
        // the scale factor need only be used consistently: FP32-accurate 1/sqrt(tr)
        S.Ef[lane] = ffc_from(rsqrt32(tr) * S.E[lane]);
      } else if (wid == 1) {
        const double ib = inv_norm_b();
        if (MIXED && lane < n) S.bh[lane] = ffc_from(ib * S.b[lane]);
        if (lane == 0) {
          S.inv_sb = ib;
          S.sb = bb * ib;
          S.tr = tr;
          S.dnu = dnu_arr[om];
          S.fp64 = MIXED ? 0 : 1;
        }
      } else if (wid == 3 && lane == 0) {
        const double dnu = dnu_arr[om], sb = bb * inv_norm_b();
        S.lo = P.alpha_rel * tr;
        // the root's upper bracket: FP32 accuracy is enough in the mixed route
        S.hi = fmax(tr * dnu * (MIXED ? rcp32(sb - dnu) : rcp64(sb - dnu)), S.lo);
      }
    }
    __syncthreads();
    FL_MARK(16);
    const double tr = S.tr, bb = S.red[1];
    const double dnu0 = S.dnu;
    // A_nu underflowed to zero (the mode carries no information), or, under the
    // discrepancy rule, ||b|| recomputed here does not exceed delta_nu after all (a
    // rounding tie at the threshold of the classification): V~ = 0
    if (!(tr > 0.0) || (P.alpha_mode == 0 && !(bb > dnu0 * dnu0))) {
      if (threadIdx.x == 0) {
        atomicAdd(ctr + C_ACTIVE, ~0ull);  // -1: counted as zeroed instead
        atomicAdd(ctr + C_ZEROED, 1ull);
        if (alpha_out) alpha_out[om * N2 + nu] = INFINITY;
      }
      cx<B>* out0 = prof + ((long long)om * N2 + i) * 2 * m;
#pragma unroll 1
      for (int l = threadIdx.x; l < m; l += ST) {
        double2 u = make_double2(0, 0);
        if (nu == 0 && !P.incident) {
          double s0, c0;
          sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s0, &c0);
          u = make_double2((double)N2 * c0, (double)N2 * s0);
        }
        out0[l] = czero<B>();
        out0[m + l] = from_d<B>(u);
      }
      __syncthreads();
      continue;
    }
    if (MIXED) {
      // scaled problem Ah = A / sqrt(tr) (||Ah||_F ~ 1), bh = b / ||b||, a = alpha / tr:
      // Ah in two-float (for the residual and V~) and its FP32 part (for the model);
      // thread t builds column t mod 64, rows t / 64, t / 64 + 2, ...
      ffc (*Af)[DENSE_M + 1] = reinterpret_cast<ffc (*)[DENSE_M + 1]>(S.A);
      // the sampled tables hold A exactly scaled by 1/sqrt(tr) (FP64 in the plan)
      const double sa = SAMPLED ? rsqrt64(tr) : rsqrt32(tr);
      if (SAMPLED) {
        const float4* t4 = reinterpret_cast<const float4*>(ktab) + mb;
#pragma unroll 1
        for (int e = threadIdx.x; e < n * m; e += ST) {
          const int k = e / m, l = e - k * m;
          const float4 v = t4[e];
          Af[k][l] = ffc{ff{v.x, v.y}, ff{v.z, v.w}};
          S.u.f.m.A[k][l] = make_float2(v.x, v.z);
        }
      } else {
        const int l = threadIdx.x & (DENSE_M - 1);
        if (l < m) {
          const ffc pl = S.Pf[l];
#pragma unroll 1
          for (int k = threadIdx.x / DENSE_M; k < n; k += ST / DENSE_M) {
            const ffc a = ffc_mul(S.Ef[k], pl);
            Af[k][l] = a;
            S.u.f.m.A[k][l] = make_float2(a.re.hi, a.im.hi);
          }
        }
      }
      __syncthreads();
      FL_MARK(2);
      BulkF& K = S.u.f;
      if (threadIdx.x < 32) {
        // Lanczos model of the scaled G from q_0 = bh (renormalised in FP32)
        const int lane = threadIdx.x;
        const float2 q0 = lane < n ? make_float2(S.bh[lane].re.hi, S.bh[lane].im.hi) : make_float2(0.f, 0.f);
        const float inq = rsqrtf(warp_sum(abs2(q0)));
        if (lane < n) K.Q[lane][0] = inq * q0;
      }
      __syncthreads();
      const int kd = lanczos_block<float>(K.m.A, n, m, K.t, K.w, K.Q, S.d32, S.e32, LANCZOS_TOL32, &S.go);
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) S.kd = kd;
        FL_MARK(4);
        if (lane < kd) S.c32[lane] = make_float2(lane == 0 ? 1.f : 0.f, 0.f);  // c = e_1
        __syncwarp();
        FL_MARK(5);
        bool ok = true, fl = false;
        float a;
        if (P.alpha_mode == 1) {
          a = (float)P.alpha_given[om] / (float)S.tr;
        } else {
          const float target = (float)((S.dnu * S.inv_sb) * (S.dnu * S.inv_sb));
          a = root32_warp(S, kd, (float)P.alpha_rel, (float)S.hi / (float)S.tr, target, fl, ok);
        }
        FL_MARK(6);
        // floor cases, breakdowns and small alpha/tr are decided and solved in FP64
        const bool fp64 = !ok || fl || a < (float)P.fp64_switch;
        if (lane == 0) {
          S.a_s = (double)a;
          S.fp64 = fp64 ? 1 : 0;
          if (fp64) atomicAdd(ctr + C_FP64_FALLBACK, 1ull);
        }
      } else if (!SAMPLED && threadIdx.x == DENSE_M + DENSE_M1) {
        S.qz = exp_ikz(kz, P.hz);  // FP64, on an idle warp; first read by eq. (9)
      }
      __syncthreads();
      FL_MARK(7);
      if (!S.fp64) {
        // yh by refinement against the two-float residual, to ||dy|| <= 1e-9 ||y||
#pragma unroll 1
        for (int k = threadIdx.x; k < n; k += ST) {
          S.yh[k] = ffc_zero();
          S.r32[k] = make_float2(S.bh[k].re.hi, S.bh[k].im.hi);
        }
        __syncthreads();
        FL_MARK(17);
        const float a32 = (float)S.a_s;
        const ff a_ff = ff{a32, 0.f};  // the FP32 root is exact in two-float
        // stop once the next correction, predicted from the contraction of the last
        // two (||dy_k||^2 rho^2, rho = ||dy_k|| / ||dy_k-1||), is below 1e-18 ||y||^2;
        // a correction that does not shrink ends the refinement unconverged
        int sweeps = 0;
        float prev = 0.f, rel = 1.f;
        bool conv = false;
#pragma unroll 1
        for (; sweeps < P.refine_iters; ++sweeps) {
          if (sweeps == 1 && rel <= 1e-18f) { conv = true; break; }
          if (sweeps >= 2) {
            if (rel * rel <= 1e-18f * prev) { conv = true; break; }
            if (!(rel < prev)) break;
          }
          prev = rel;
          if (sweeps) residual_ff(S, n, m, a_ff);
          if (sweeps == 1) FL_MARK(19);
          if (threadIdx.x < 32) {
            const int j = threadIdx.x;
            const float2 dy = lanczos_apply32(S, n, kd, a32, j < n ? S.r32[j] : make_float2(0.f, 0.f));
            float dd = 0.f, yy = 0.f;
            if (j < n) {
              const ffc yn = ffc_add(S.yh[j], ffc{ff{dy.x, 0.f}, ff{dy.y, 0.f}});
              S.yh[j] = yn;
              dd = abs2(dy);
              yy = yn.re.hi * yn.re.hi + yn.im.hi * yn.im.hi;
            }
            dd = warp_sum(dd);
            yy = warp_sum(yy);
            if (j == 0) S.red[4] = yy > 0.f ? dd / yy : 0.f;
          }
          __syncthreads();
          rel = (float)S.red[4];
          if (sweeps == 0) FL_MARK(18);
          if (sweeps == 1) FL_MARK(20);
        }
        if (!conv) conv = rel <= 1e-18f || (sweeps >= 2 && rel * rel <= 1e-18f * prev);
        if (threadIdx.x == 0) {
#ifdef FL_PHASE_TIMING
          if (item < 4096) g_mode_sweeps[item] = sweeps;
#endif
          atomicAdd(ctr + C_REFINE_ITERS, (unsigned long long)sweeps);
          if (!conv) {
            S.fp64 = 1;
            atomicAdd(ctr + C_FP64_FALLBACK, 1ull);
          }
        }
        FL_MARK(8);
        if (conv) {
          // V~ = A^H y = (||b|| / sqrt(tr)) Ah^H yh, two-float, 2 threads per column
          const int t = threadIdx.x, l = (t & 7) + 8 * (t >> 4), h = (t >> 3) & 1;
          const bool on = l < m;
          const ffc acc = colsum_ff(Af, S.yh, on ? n : 0, l, h);
          if (on && h == 0) S.u.q.Vt[l] = (S.sb * sa) * ffc_to(acc);
        }
        __syncthreads();
      }
      if (S.fp64) {
        // FP64 route for this mode: A in FP64 over the two-float storage (each entry
        // read and rewritten by the same thread)
        const double sq = tr * sa;  // sqrt(tr), the sampled tables' scale
#pragma unroll 1
        for (int e = threadIdx.x; e < n * m; e += ST) {
          const int k = e / m, l = e - k * m;
          if (SAMPLED) {
            const ffc a = Af[k][l];
            S.A[k][l] = sq * ffc_to(a);
          } else {
            S.A[k][l] = S.E[k] * S.Pz[l];
          }
        }
        __syncthreads();
      }
    } else {
#pragma unroll 1
      for (int e = threadIdx.x; e < n * m; e += ST) {
        const int k = e / m, l = e - k * m;
        S.A[k][l] = SAMPLED ? reinterpret_cast<const double2*>(ktab)[mb + e] : S.E[k] * S.Pz[l];
      }
      __syncthreads();
    }
    FL_MARK(9);
    if (S.fp64) {
      solve_fp64(S, n, m, P, om, ctr);
      // V~ = A^H y (FP64), 2 threads per column
      const int l = threadIdx.x >> 1, h = threadIdx.x & 1;
      double2 acc = make_double2(0, 0);
      if (l < m)
#pragma unroll 1
        for (int k = h; k < n; k += 2) acc = acc + cmul_conj_a(S.A[k][l], S.y[k]);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      if (l < m && h == 0) S.u.q.Vt[l] = acc;
      __syncthreads();
    }
    FL_MARK(10);
    // U~ = U~0 + gamma (F + B), eq. (9); with the sampled kernel U~ - U~0 = T_nu V~ by
    // the Toeplitz product (F), two threads per plane
    if (SAMPLED) {
      const int l = threadIdx.x >> 1, h = threadIdx.x & 1;
      double2 acc = make_double2(0.0, 0.0);
      if (l < m)
#pragma unroll 1
        for (int j = h; j < m; j += 2) acc = acc + S.Tk[l > j ? l - j : j - l] * S.u.q.Vt[j];
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      if (l < m && h == 0) S.u.q.F[l] = acc;
    } else {
      eq9_scans(m);
    }
    __syncthreads();
    FL_MARK(11);
    cx<B>* out = prof + ((long long)om * N2 + i) * 2 * m;
    bool overflow = false;  // a profile beyond the range of B (FP32 in the mixed path)
    {  // V~ by threads l < 64, U~ by threads 64 + l (its FP64 arithmetic on warps 2 and 3)
      const int l = threadIdx.x & (DENSE_M - 1);
      if (l < m) {
        if (threadIdx.x < DENSE_M) {
          const cx<B> v = from_d<B>(S.u.q.Vt[l]);
          overflow = !(isfinite(v.x) && isfinite(v.y));
          out[l] = v;
        } else {
          double2 u;
          if (SAMPLED) {
            u = S.u.q.F[l];
          } else {
            const double2 f = S.u.q.F[l] + S.u.q.Bk[l];
            // gamma is imaginary (propagating mode) or real (evanescent)
            u = q >= 0.0 ? make_double2(-gamma.y * f.y, gamma.y * f.x) : make_double2(gamma.x * f.x, gamma.x * f.y);
          }
          if (nu == 0 && !P.incident) {  // the plane wave; a given incident field is added in the recovery
            double s, c;
            sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
            u = u + make_double2((double)N2 * c, (double)N2 * s);
          }
          const cx<B> uo = from_d<B>(u);
          overflow = !(isfinite(uo.x) && isfinite(uo.y));
          out[m + l] = uo;
        }
      }
    }
    if (threadIdx.x == 0 && alpha_out) alpha_out[om * N2 + nu] = S.a_s * S.tr;
    // counted as non-finite (fs_sync_status: FS_ENONFINITE): the working precision
    // cannot hold this mode's solution
    if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicAdd(ctr + C_NONFINITE, 1ull);
    FL_MARK(12);
#ifdef FL_PHASE_TIMING
    if (threadIdx.x == 0 && item < 4096) g_mode_cycles[item] = clock64() - t_mode0;
#endif
  }
}

int solve_grid(int bps) { return (bps < 1 ? 1 : (bps > 3 ? 3 : bps)) * sm_count(); }

template <typename B, bool MIXED, bool SAMPLED>
cudaError_t solve_variant(const Problem& P, const Work<B>& w, cudaStream_t s) {
  const size_t smem = sizeof(Shared);
  static SmemOptIn attr;
  cudaError_t e = opt_in_smem(attr, (const void*)k_solve<B, MIXED, SAMPLED>, smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_solve<B, MIXED, SAMPLED>, dim3(solve_grid(P.solve_bps)), dim3(ST), smem, s, P,
                    (const cx<B>*)w.wt, (const int*)w.act, (const int*)w.count, (const double*)w.dnu, w.prof,
                    w.alpha_out, w.ctr, w.ktab, w.ktr);
}

template <typename B, bool MIXED>
cudaError_t solve_impl(const Problem& P, const Work<B>& w, cudaStream_t s) {
  if (P.sampled) {
    if (!w.ktab || !w.ktr) return cudaErrorInvalidValue;
    return solve_variant<B, MIXED, true>(P, w, s);
  }
  return solve_variant<B, MIXED, false>(P, w, s);
}

}  // namespace

template <typename R>
cudaError_t launch_classify(const Problem& P, const Work<R>& w, cudaStream_t s) {
  const dim3 g(classify_blocks(P.n), P.n_omega);
  cudaError_t e = launch_pdl(k_classify_flags, g, dim3(CT), 0, s, P, (const double*)w.norms, (const double*)w.partial,
                             w.n_partial, w.flagbits, w.blkcnt, w.blkgz, w.colblk, w.dnu);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_classify_scatter, g, dim3(CT), 0, s, P, (const unsigned*)w.flagbits, (const int*)w.blkcnt,
                    (const int*)w.blkgz, (const unsigned*)w.colblk, w.slot, w.act, w.cols, w.ncol, w.count, w.ctr);
}
template cudaError_t launch_classify<double>(const Problem&, const Work<double>&, cudaStream_t);
template cudaError_t launch_classify<float>(const Problem&, const Work<float>&, cudaStream_t);

template <typename R>
cudaError_t launch_classify_fused(const Problem& P, const Work<R>& w, cudaStream_t s) {
  const int cb = classify_blocks(P.n);
  if (cb * CMB < P.n * P.n || cb > 64) return cudaErrorInvalidValue;
  // every block of the grid must be resident at once (they wait on one another): the
  // resident blocks per SM of this kernel, looked up once per device; a device on
  // which the launch failed once takes the two-kernel classification from then on
  static std::atomic<int> occ[MAX_DEVICES], refused[MAX_DEVICES];
  int dev = 0;
  cudaGetDevice(&dev);
  const bool known = dev >= 0 && dev < MAX_DEVICES;
  if (known && refused[dev].load(std::memory_order_relaxed)) return cudaErrorNotSupported;
  int per_sm = known ? occ[dev].load(std::memory_order_relaxed) : 0;
  if (per_sm <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_classify_fused<R>, FT, 0);
    if (e != cudaSuccess) return e;
    if (known) occ[dev].store(per_sm, std::memory_order_relaxed);
  }
  if ((long long)per_sm * sm_count() < (long long)cb * P.n_omega) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cb, P.n_omega);
  cfg.blockDim = dim3(FT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_classify_fused<R>, P, (const cx<R>*)w.wt, w.partial, w.bar,
                                           w.blkcnt, w.blkgz, w.colblk, w.slot, w.act, w.cols, w.ncol, w.count,
                                           w.dnu, w.ctr);
  if (e != cudaSuccess && known) refused[dev].store(1, std::memory_order_relaxed);
  return e;
}
template cudaError_t launch_classify_fused<double>(const Problem&, const Work<double>&, cudaStream_t);
template cudaError_t launch_classify_fused<float>(const Problem&, const Work<float>&, cudaStream_t);

namespace {
// every block arrives at a barrier whose target is one more than the grid: nothing
// ever completes it, so each wait runs out after `polls` polls
__global__ void k_wait_never(unsigned* bar, unsigned target, unsigned polls, unsigned long long* ctr) {
  __shared__ int ok_s;
  grid_wait(bar, target, polls, ctr, &ok_s);
}
}  // namespace

}  // namespace fl

extern "C" int fs_check_bounded_wait(int blocks, unsigned polls, long long* timeouts) {
  using namespace fl;
  if (blocks < 1 || blocks > 64 || polls < 1 || polls > (1u << 20) || !timeouts) return 1;
  // one buffer: the barrier counter (bytes 0-3), the counters [C_COUNT] from byte 16
  constexpr size_t CTR_OFF = 16, BYTES = CTR_OFF + sizeof(unsigned long long) * C_COUNT;
  unsigned char* mem = nullptr;
  if (cudaMalloc(&mem, BYTES) != cudaSuccess) return 2;
  unsigned* bar = reinterpret_cast<unsigned*>(mem);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(mem + CTR_OFF);
  cudaError_t e = cudaMemset(mem, 0, BYTES);
  if (e == cudaSuccess) {
    k_wait_never<<<blocks, 32>>>(bar, (unsigned)blocks + 1u, polls, ctr);
    e = cudaGetLastError();
  }
  unsigned long long h[C_COUNT] = {};
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, ctr, sizeof(unsigned long long) * C_COUNT, cudaMemcpyDeviceToHost);
  cudaFree(mem);
  if (e != cudaSuccess) return 3;
  *timeouts = (long long)h[C_TIMEOUT];
  return 0;
}

namespace fl {

cudaError_t launch_solve_fp64(const Problem& P, const Work<double>& w, cudaStream_t s) {
  return solve_impl<double, false>(P, w, s);
}
cudaError_t launch_solve_mixed(const Problem& P, const Work<float>& w, cudaStream_t s) {
  return solve_impl<float, true>(P, w, s);
}

}  // namespace fl
