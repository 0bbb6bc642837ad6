// split.h -- split-precision segment records and launchers (internal).
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace lisa {

// FP32 staged data per bin: s_A, s_E, s_T (s_X = sqrt(w_X) 2^-64), then -2 sqrt(w_X) d_X
// for X = A, E, T (re, im); 36 bytes, so that a tile of 1024 bins takes 36 KB of shared
// memory and four blocks per SM leave L1 room for the segment records.
constexpr int kBinFloats = 9;

// One spline segment of one (walker, mode) in the split-precision form, 192 bytes.
// With t = (j - kb0) / W over the segment's W bins: c[k] is the t^k coefficient of
// A 2^64, and for channel x = 0, 1, 2 (A, E, T) c[4 + 8 x + 2 k] and c[4 + 8 x + 2 k + 1]
// are the t^k coefficients of Re T^X and Im T^X, interleaved so that the pair is one
// packed f32x2 operand.  ph[] is the fixed-point phase record of the segment (see
// kernels.h).  pad[] is zero except in segment 0, where it holds the FP32 bit patterns
// of the segment-guess constants: sc log2 f_lo and sc = (K - 1) / log2(f_hi / f_lo).
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
