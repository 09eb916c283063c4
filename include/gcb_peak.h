/*
 * gcb_peak.h -- measured arithmetic peaks of the GPU (libgcb_peak.so).
 *
 * A measurement helper of the benchmark, not part of the method: the paper
 * has no counterpart.  The pushes are reported against the HBM roofline and,
 * where arithmetic bounds them, against these measured fused multiply-add
 * rates (the Kerr-Schild push against the FP64 rate, the flat pushes'
 * FP32 work against the FP32 rate), and the current deposition against the
 * measured rate of scattered atomic additions.
 */
#ifndef GCB_PEAK_H
#define GCB_PEAK_H

#ifdef __cplusplus
extern "C" {
#endif

enum { GCB_PEAK_FP32 = 0, GCB_PEAK_FP32X2 = 1, GCB_PEAK_FP64 = 2 };

/*
 * Fused multiply-add throughput of the current device, in TFLOP/s (one FMA =
 * 2 flops; a packed FP32x2 FMA = 4): kind GCB_PEAK_FP32 (scalar FP32 FMA),
 * GCB_PEAK_FP32X2 (packed two-lane FP32 FMA) or GCB_PEAK_FP64.  Every thread
 * of 16 blocks of 256 per SM runs 8 independent FMA chains of `iters` rounds;
 * the second of two launches is timed with CUDA events on cuda_stream (NULL:
 * the default stream).  Allocates and frees a 2 KB device buffer; changes no
 * device setting.
 * Returns 0 and writes *tflops; 1 for invalid arguments (iters < 1, unknown
 * kind, NULL tflops); 2 for a CUDA error.
 */
int gcb_peak_fma(int kind, int iters, void *cuda_stream, double *tflops);

/*
 * Rate of atomic additions without return, in G operations/s: dtype 0 FP32,
 * 1 FP64; pattern 0 coalesced (the 32 lanes of a warp add to 32 consecutive
 * elements), 1 scattered (to 32 different 32-byte sectors).  8 blocks of 256
 * threads per SM each add `iters` times into a 2^23-element buffer
 * (L2-resident); the second of two launches is timed with CUDA events on
 * cuda_stream.  Allocates and frees the buffer; changes no device setting.
 * Returns 0 and writes *gops; 1 for invalid arguments; 2 for a CUDA error.
 */
int gcb_peak_red(int dtype, int pattern, int iters, void *cuda_stream, double *gops);

#ifdef __cplusplus
}
#endif
#endif /* GCB_PEAK_H */
