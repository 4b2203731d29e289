/*
 * nsrhs_probe — machine-peak probes used to state the roofline of the
 * assembly kernels. The paper measures its machines' FP peaks with
 * microbenchmarks (Sec. III-B, III-C: likwid-bench peakflops, 9.7 TF/s FP64
 * on the A100) and places its kernels on that roofline (Sec. V-D, Fig. 4).
 * The FP64 element kernels here are bound by the FP64 pipe (no tensor
 * cores). Their roofline denominator is that pipe's issue rate (2 FP64 FMA
 * lanes per SM per clock x 2 flops x SMs x the SM clock sampled while they
 * run); this probe's measured FMA rate is reported beside it, and its FP32
 * rate is the denominator of the mixed-precision kernels.
 */
#ifndef NSRHS_PROBE_H
#define NSRHS_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Launch an FMA-throughput kernel on `stream`: `blocks` blocks of 256
 * threads, each thread running 16 independent dependent chains of `iters`
 * fused multiply-adds in double (fp64 != 0) or float (fp64 == 0), then
 * writing one value per thread to sink[blocks * 256] (device memory, double)
 * so that the work cannot be removed. FLOPs per launch =
 * blocks * 256 * 16 * iters * 2. Time it with events on the same stream.
 * Returns 0, or a nonzero nsrhs_status value (1 bad argument, 4 CUDA error).
 */
int nsrhs_probe_fma(int fp64, int64_t blocks, int64_t iters, double* sink, void* stream);

/*
 * Evaluate this library's double-precision special functions beside CUDA's
 * on n device values x: which = 0 reciprocal (x > 0), 1 square root
 * (x >= 0), 2 reciprocal cube root (x > 0), 3 float -> double widening of
 * float(x). ours[i] / ref[i] (device arrays of n doubles) receive the
 * library's and CUDA's results. Used by the tests to bound the error of the
 * kernels' special functions. Returns 0, 1 (bad argument) or 4 (CUDA error).
 */
int nsrhs_probe_special(int which, int64_t n, const double* x, double* ours, double* ref,
                        void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NSRHS_PROBE_H */
