// split.h -- split-precision segment records and launchers (internal).
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace lisa {

// FP32 staged data per bin: s_A, s_E, s_T (sqrt(w) 2^-64), then sqrt(w) d for A, E, T
// (re, im); 36 bytes.
constexpr int kBinFloats = 9;

// One spline segment of one (walker, mode) in the split-precision form, 192 bytes:
// c[4 q + k] is the t^k coefficient (t = (j - kb0) / W over the segment's W bins) of
// series q = A 2^64, Re T^A, Im T^A, Re T^E, Im T^E, Re T^T, Im T^T; ph[] is the
// fixed-point phase record of the segment (see kernels.h).
struct __align__(16) SegRec {
    float c[28];
    unsigned long long ph[kPhaseWords];
    int kb0;
    float invw;
    int pad[2];
};
static_assert(sizeof(SegRec) == 192, "segment record is 192 bytes");

cudaError_t launch_prep_split(const double *bins, int N, float *out, cudaStream_t s);
cudaError_t launch_segprep(const StageDims &d, const StageBufs &b, SegRec *segs, cudaStream_t s);
cudaError_t launch_dense_split(const StageDims &d, const StageBufs &b, const SegRec *segs,
                               const float *bins, const DenseTune &t, cudaStream_t s);

}  // namespace lisa
