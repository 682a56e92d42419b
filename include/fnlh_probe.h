/*
 * fnlh_probe.h -- measurement helper shipped beside the FNLH library (not part
 * of the solver): a multiply-add throughput probe that gives the FP64 and
 * FP32 arithmetic peaks the sweeps' rooflines are reported against.
 */
#ifndef FNLH_PROBE_H
#define FNLH_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runs `iters` steps of `chains` (4, 8 or 16) x `reuse` (1, 2 or 4)
 * independent multiply-add accumulators per thread, acc[k][r] += j[k] x[r]
 * (every j[k] feeds `reuse` consecutive multiply-adds), on `blocks` x
 * `threads` threads (threads a multiple of 32, at most 1024), in FP64
 * (precision 0) or FP32 (precision 1), and returns the kernel's duration in
 * milliseconds (CUDA events on `stream`, a cudaStream_t; synchronises on it).
 * Work done: 2 flops x chains x reuse x iters x threads x blocks.  sink:
 * caller-owned device memory of one double per thread (blocks x threads x 8
 * bytes), written.  Returns 0, -1 on a bad argument (checked before anything
 * is launched), -2 on a CUDA error. */
int fnlh_probe_fma(int32_t precision, int32_t chains, int32_t reuse, int32_t blocks, int32_t threads, int32_t iters,
                   double *sink, float *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FNLH_PROBE_H */
