// Internal interface of the fixed-alpha derivative kernels (diff.cu) used by the
// C-ABI layer; the public interface is include/flatlayer_diff.h.
#pragma once

#include "pipeline.cuh"

namespace fl {

constexpr int JVP_CHUNK = 16;  // directions per JVP launch

// blocks per frequency of the per-mode kernels (fixed for a device and shape, so
// that the per-block partial sums, and hence the results, are reproducible)
int diff_blocks_per_omega(int n, int n_omega);

// G^ = A^ A^^H per mode, packed lower triangle: [n_omega][N*N][M1(M1+1)/2]
cudaError_t launch_diff_gram(const Problem& P, double2* gram, cudaStream_t s);

template <typename R>
cudaError_t launch_diff_forward(const Problem& P, int gb, const double2* gram, const cx<R>* wt,
                                const double* log_alpha, double2* Ls, double2* ys, cx<R>* vt, cx<R>* ut,
                                double* partial, unsigned long long* ctr, cudaStream_t s);
template <typename R>
cudaError_t launch_diff_vjp(const Problem& P, int gb, const double2* Ls, const double2* ys, const cx<R>* vbt,
                            const cx<R>* ubt, const double* log_alpha, const double* grad_phi, cx<R>* wbt,
                            double* partial, cudaStream_t s);
template <typename R>
cudaError_t launch_diff_jvp(const Problem& P, int gb, int nd, const double2* Ls, const double2* ys,
                            const cx<R>* dwt, const double* log_alpha, const double* dlog_alpha, cx<R>* dvt,
                            cx<R>* dut, double* partial, cudaStream_t s);
template <typename R>
cudaError_t launch_diff_combine(const Problem& P, const cx<R>* Vx, const cx<R>* ux, R* xi, R* c, R* xis,
                                cudaStream_t s);
template <typename R>
cudaError_t launch_diff_vjp_point(const Problem& P, const R* gxi, const cx<R>* Vx, const cx<R>* ux, const R* xis,
                                  cx<R>* Vb, cx<R>* ub, cudaStream_t s);
template <typename R>
cudaError_t launch_diff_jvp_point(const Problem& P, int nd, const cx<R>* Vx, const cx<R>* ux, const R* xis,
                                  const cx<R>* dVx, const cx<R>* dux, R* dxi, cudaStream_t s);
cudaError_t launch_reduce_rows(const double* partial, int rows, int cols, double* out, cudaStream_t s);

}  // namespace fl
