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

#ifdef __cplusplus
}
#endif

#endif /* FLATLAYER_PEAKS_H */
