/*
 * flatlayer_peaks.h -- ALU microbenchmarks used as roofline denominators for the
 * per-mode solve of the flat-layer reconstruction (the paper has no counterpart:
 * it reports CPU wall times only, Sec. 6).
 */
#ifndef FLATLAYER_PEAKS_H
#define FLATLAYER_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double fp64_tflops;            /* FP64 FMA throughput over a full grid (2 flops per FMA) */
  double fp32_tflops;            /* FP32 FMA throughput over a full grid                    */
  double fp64_fma_cycles_1lane;  /* cycles per dependent FP64 FMA, one active lane          */
  double fp64_fma_cycles_warp;   /* cycles per dependent FP64 FMA, 32 active lanes          */
  double fp64_div_cycles_1lane;  /* cycles per dependent FP64 division (+ add), one lane    */
  int sms;                       /* streaming multiprocessors                               */
  double clock_mhz;              /* nominal SM clock reported by the driver                 */
} fs_alu_peaks;

/* Run the microbenchmarks on `device` (synchronous, ~0.1 s; allocates and frees a
   few KB).  Returns 0 on success, 1 for a NULL argument, 2 if allocation fails,
   3 on a CUDA error. */
int fs_measure_alu_peaks(int device, fs_alu_peaks* out);

/* The scalar reciprocals the per-mode kernels use in place of FP64 division and
   square root (Newton-Raphson iterations from FP32 seeds: rcp64 and rsqrt64 to FP64
   accuracy, rcp32 and rsqrt32 to FP32 accuracy at any exponent), evaluated beside
   CUDA's own 1.0/x and rsqrt(x), so that a test can compare them over the whole
   exponent range.  The paper has no counterpart.
     x    device, n doubles.
     out  device, [6][n] doubles: rcp64(x), 1.0/x, rsqrt64(x), rsqrt(x), rcp32(x),
          rsqrt32(x).
   Asynchronous on `stream` (a cudaStream_t; NULL = the legacy default stream).
   Returns 0 on success, 1 for a bad argument, 3 on a launch error. */
int fs_eval_reciprocals(const double* x, int n, double* out, void* stream);

/* The bounded device-side wait of the single-pass classification, made to run out:
   `blocks` (1..64) blocks arrive at a barrier whose target is blocks + 1, so no wait is
   ever satisfied, and each gives up after `polls` (1..2^20) polls of about 64 ns and
   counts a timeout.  *timeouts receives the count (blocks when the limit works).
   Synchronous on the current device; allocates and frees a few bytes.  Returns 0 on
   success, 1 for a bad argument, 2 if allocation fails, 3 on a CUDA error.  The paper
   has no counterpart. */
int fs_check_bounded_wait(int blocks, unsigned polls, long long* timeouts);

#ifdef __cplusplus
}
#endif

#endif /* FLATLAYER_PEAKS_H */
