// kernels.h -- launchers of the device stages (internal to liblisalike.so).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lisa {

constexpr int kScratchRows = 11;  // rows of K doubles per (walker, mode) in mscratch

// Device layout of one bin of the uploaded data: the FP64 dense kernel reads the
// nine doubles w_A, w_E, w_T, (w d)_A re/im, (w d)_E re/im, (w d)_T re/im
// (w = 4 df / S, Eqs. (3) and (11)); 72 bytes, 16-byte aligned rows of 2 bins.
constexpr int kBinDoubles = 9;

struct StageDims {
    int B;       // walkers in this call
    int L;       // modes
    int K;       // knots per mode
    int N;       // dense bins
    double f0, df, t0;
    int ml[6], mm[6];  // (l, m) of each mode
};

// Per-call device buffers (sized for max_batch by the host).
struct StageBufs {
    const double *params;  // [B][11]
    int *valid;            // [B]
    double *tc;            // [B]
    double *xpk;           // [B] peak of f^2 A_22 in M f
    int *band;             // [B][L][3]: active, j_lo, j_hi
    double *fedge;         // [B][L][2]
    double *fk;            // [B][L][K]
    int *kb;               // [B][L][K]: first dense bin with f_j >= f_k
    double *vals;          // [B][L][8][K]
    double *mscratch;      // [B][L][11][K]: spline second derivatives of the 8 series, then
                           // the shared factorisation: 1/h (row 8) and the normalised
                           // super-diagonal (row 10); row 9 is spare
    double *coef;          // [B][L][K-1][8][4]
    int *wrange;           // [B][2] union of the walker's active mode ranges
    int *order;            // [B] walkers sorted by band (groups are runs of G entries)
    int *slot_of;          // [B] position of each walker in `order`
    int *grange;           // [groups][2] union range of each group (start a multiple of 4)
    int *item_start;       // [groups+1] exclusive prefix of the dense work items
    int *counter;          // dense work-queue counter
    int *err;              // set by a device wait that gave up
    double *part;          // [items][G][2] per-item, per-slot partial sums
    // Test only (0 in normal operation): when > 0 the dense kernels arm each tile's
    // barrier for the tile's bytes but issue no copy, so every wait on it gives up after
    // this many polls, with no copy in flight, and takes the error path.
    unsigned wait_test_polls = 0;
};

// Split precision keeps the phase series in FP64 (row 1 of vals and of the second
// derivatives in mscratch, as in FP64) and the seven other series in FP32 inside the same
// per-(walker, mode) storage: series q' = 0 (A 2^64) and 1..6 (Re, Im of T^A, T^E, T^T)
// as FP32 rows of K values from double row 2 of vals (knot values) and of mscratch
// (second derivatives), and FP32 copies of 1/h, h, 1/pivot and the normalised
// super-diagonal as four FP32 rows from double row 6 of mscratch.
constexpr int kSplitSeries32 = 7;
__host__ __device__ inline float *split_vals32(double *vals, size_t wm, int K) {
    return reinterpret_cast<float *>(vals + (wm * 8 + 2) * (size_t)K);
}
__host__ __device__ inline float *split_m32(double *mscratch, size_t wm, int K) {
    return reinterpret_cast<float *>(mscratch + (wm * kScratchRows + 2) * (size_t)K);
}
__host__ __device__ inline float *split_fac32(double *mscratch, size_t wm, int K) {
    return reinterpret_cast<float *>(mscratch + (wm * kScratchRows + 6) * (size_t)K);
}

struct DenseTune {
    int threads;     // threads per block
    int per_thread;  // consecutive bins per thread
    int blocks;      // persistent grid size
    int group;       // walkers sharing one staged data tile
};

// groups of a call with B walkers
__host__ __device__ inline int n_groups(int B, int G) { return (B + G - 1) / G; }

cudaError_t launch_knots(const StageDims &d, const StageBufs &b, cudaStream_t s);
// the band kernel alone (walker constants, peak, bands; no knots)
cudaError_t launch_band(const StageDims &d, const StageBufs &b, cudaStream_t s);
cudaError_t launch_spline(const StageDims &d, const StageBufs &b, cudaStream_t s);
// split precision: FP64 phase, FP32 amplitude and transfer (layout above)
cudaError_t launch_knots_split(const StageDims &d, const StageBufs &b, cudaStream_t s);
cudaError_t launch_spline_split(const StageDims &d, const StageBufs &b, cudaStream_t s);
cudaError_t launch_plan(const StageDims &d, const StageBufs &b, int tile_bins, int group,
                        cudaStream_t s);
// Fixed-point phase record of one spline segment (kPhaseWords words): the full phase
// phi - 2 pi f t_coal and its first three forward differences over one bin at the
// segment's first bin, as fractions of a turn scaled by 2^64 (words 0..3), and the next
// 64 fractional bits of the three differences (words 4..6), which keep anchors deep
// inside long segments exact to the FP64 value of the differences; the low 32 bits of
// word 7 hold the first bin of the next segment (0x7fffffff for the last one).
constexpr int kPhaseWords = 8;

// FP64 path: the phase records of all segments ([B][L][K-1][kPhaseWords]).
cudaError_t launch_phaseprep(const StageDims &d, const StageBufs &b, unsigned long long *phases,
                             cudaStream_t s);
cudaError_t launch_dense_f64(const StageDims &d, const StageBufs &b,
                             const unsigned long long *phases, const double *bins,
                             const DenseTune &t, cudaStream_t s);
// split = 0: parts hold (<d|h>, <h|h>); split = 1: (sum |h|^2 - 2 Re(d h*), <h|h>)
cudaError_t launch_finish(const StageDims &d, const StageBufs &b, int group, int split, double dd,
                          double *lnL, double *dh, double *hh, cudaStream_t s);
cudaError_t launch_template(const StageDims &d, const StageBufs &b, double *out,
                            cudaStream_t s);
cudaError_t launch_prep(const double *d, const double *psd, int N, double df, double *bins,
                        double *ddpart, int *bad, cudaStream_t s);
int prep_blocks(int N);

// Resident blocks per SM of a dense-kernel variant (0 if the variant does not exist).
int dense_f64_occupancy(int per_thread, int group);
int dense_split_occupancy(int per_thread, int group);

// Largest number of (item, slot) partial-sum pairs a call with B walkers can produce.
int64_t max_items(int B, int N, int tile_bins);
// Bytes of dynamic shared memory the planning kernel needs for B walkers.
size_t plan_smem(int B);

}  // namespace lisa
