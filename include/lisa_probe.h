/*
 * lisa_probe.h -- pipe-throughput microbenchmark of the current device, for the roofline
 * denominators of the likelihood kernels (FP64 for the dense FP64 path, FP32 for the split
 * path, MUFU for the special-function unit).  Not part of the method.
 *
 * lisa_probe_pipes runs three short kernels on every SM with independent dependency
 * chains per thread (8 per thread, enough to cover the pipe latencies): FP64 FMA, FP32 FMA
 * and MUFU sine, each timed with CUDA events after a warm-up launch, and returns the
 * achieved rates per second for the whole device: out[0] FP64 FMA/s, out[1] FP32 FMA/s,
 * out[2] MUFU sin/s, out[3] the SM clock the driver reports [Hz].  Takes about 50 ms.
 * Synchronous; LISA_ERR_CUDA on a CUDA failure.
 */
#ifndef LISA_PROBE_H
#define LISA_PROBE_H

#include "lisa_like.h"

#ifdef __cplusplus
extern "C" {
#endif

lisa_status lisa_probe_pipes(int device, double *out);

#ifdef __cplusplus
}
#endif
#endif
