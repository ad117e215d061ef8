// ALU microbenchmarks of the device the library runs on: FP64 and FP32 FMA
// throughput (many independent chains over a full grid) and the latency of a
// dependent FP64 FMA chain and of dependent FP64 divisions issued by one lane
// or by a full warp.  They give the denominators of the ALU rooflines of the
// per-mode solve and the per-instruction cost of sequential FP64 code.
#include <cuda_runtime.h>

#include "../../include/flatlayer_peaks.h"
#include "modes.cuh"

namespace {

constexpr int TP_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_tp(T* out, int iters, T a, T b) {
  T x[TP_CHAINS];
#pragma unroll
  for (int c = 0; c < TP_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < TP_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < TP_CHAINS; ++c) s += x[c];
  if (s == (T)12345.678) out[blockIdx.x] = s;  // keeps the chains alive
}

// one warp; `lanes` lanes run a dependent chain of `iters` FMAs (or divisions)
template <bool DIV>
__global__ void k_lat(long long* cycles, double* out, int iters, int lanes, double a, double b) {
  double x = 1.0 + threadIdx.x * 1e-3;
  long long t0 = 0, t1 = 0;
  __syncwarp();
  if ((int)threadIdx.x < lanes) {
    t0 = clock64();
    for (int i = 0; i < iters; ++i) x = DIV ? (b / x + a) : fma(x, a, b);
    t1 = clock64();
  }
  __syncwarp();
  if (threadIdx.x == 0) cycles[0] = t1 - t0;
  if (x == 12345.678) out[0] = x;
}

// the library's reciprocal helpers beside CUDA's own operations, one input per thread
__global__ void k_eval_reciprocals(const double* __restrict__ x, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  out[0 * (long long)n + i] = fl::rcp64(v);
  out[1 * (long long)n + i] = 1.0 / v;
  out[2 * (long long)n + i] = fl::rsqrt64(v);
  out[3 * (long long)n + i] = rsqrt(v);
  out[4 * (long long)n + i] = fl::rcp32(v);
  out[5 * (long long)n + i] = fl::rsqrt32(v);
}

}  // namespace

extern "C" int fs_eval_reciprocals(const double* x, int n, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return 1;
  if (n == 0) return 0;
  k_eval_reciprocals<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, n, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int fs_measure_alu_peaks(int device, fs_alu_peaks* r) {
  if (!r) return 1;
  if (cudaSetDevice(device) != cudaSuccess) return 3;
  int sms = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
  double* dout = nullptr;
  float* fout = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&dout, 4096 * sizeof(double)) != cudaSuccess) return 2;
  if (cudaMalloc(&fout, 4096 * sizeof(float)) != cudaSuccess) return 2;
  if (cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  float ms = 0.f;
  // FP64 throughput
  k_fma_tp<double><<<blocks, 256>>>(dout, 64, 0.999, 1e-3);
  const int it64 = 4096;
  cudaEventRecord(e0);
  k_fma_tp<double><<<blocks, 256>>>(dout, it64, 0.999, 1e-3);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  r->fp64_tflops = 2.0 * blocks * 256.0 * it64 * TP_CHAINS / (ms * 1e-3) / 1e12;
  // FP32 throughput
  k_fma_tp<float><<<blocks, 256>>>(fout, 64, 0.999f, 1e-3f);
  const int it32 = 65536;
  cudaEventRecord(e0);
  k_fma_tp<float><<<blocks, 256>>>(fout, it32, 0.999f, 1e-3f);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  r->fp32_tflops = 2.0 * blocks * 256.0 * it32 * TP_CHAINS / (ms * 1e-3) / 1e12;
  // latencies (cycles per dependent operation)
  const int li = 2048;
  long long c = 0;
  k_lat<false><<<1, 32>>>(cyc, dout, li, 1, 0.999, 1e-3);
  cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
  r->fp64_fma_cycles_1lane = (double)c / li;
  k_lat<false><<<1, 32>>>(cyc, dout, li, 32, 0.999, 1e-3);
  cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
  r->fp64_fma_cycles_warp = (double)c / li;
  k_lat<true><<<1, 32>>>(cyc, dout, li / 4, 1, 0.5, 1.5);
  cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
  r->fp64_div_cycles_1lane = (double)c / (li / 4);
  r->sms = sms;
  r->clock_mhz = clk_khz / 1000.0;
  cudaError_t err = cudaDeviceSynchronize();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dout);
  cudaFree(fout);
  cudaFree(cyc);
  return err == cudaSuccess ? 0 : 3;
}
