// plan.cu -- work planning and finishing of the dense stage (Katz et al. 2020, Sec. II.A).
//
// Walkers are sorted by their band (the union of their modes' dense-bin ranges) and cut
// into groups of G consecutive walkers; the group's union range is split into tiles of
// tile_bins bins, and each (group, tile) is one work item: one bulk copy stages the
// tile's data in shared memory and every walker of the group reuses it.  Masses that
// span decades give bands of very different lengths; sorting keeps a group's bands
// alike, and the persistent dense blocks pull items from a counter, so the uneven
// batch stays balanced.  Everything runs on the device (no host round trip), so a
// whole call can be captured in a CUDA graph.
#include "kernels.h"
#include "model.cuh"

namespace lisa {

constexpr int kSortMax = 8192;  // walkers sorted in shared memory; larger batches keep their order

size_t plan_smem(int B) {
    if (B > kSortMax) return 0;
    int P = 1;
    while (P < B) P <<= 1;
    return sizeof(unsigned long long) * (size_t)P;
}

int64_t max_items(int B, int N, int tile_bins) {
    // groups of at most 8 walkers: (B + 7) slots, and a group range of at most N + 3 bins
    return (int64_t)(B + 7) * (((int64_t)N + 3 + tile_bins - 1) / tile_bins + 1);
}

// block-wide exclusive scan of one int per thread; returns the exclusive prefix and
// leaves the block total in *total (blockDim.x a multiple of 32, at most 1024)
__device__ int block_scan(int v, int *warp_tot, int *total) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int excl = (wid > 0 ? warp_tot[wid - 1] : 0) + x - v;
    *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(1024) plan_kernel(StageDims d, StageBufs b, int tile_bins,
                                                    int G) {
    extern __shared__ unsigned long long keys[];
    __shared__ int warp_tot[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool sort = d.B <= kSortMax;
    int P = 1;
    while (P < d.B) P <<= 1;
    if (tid == 0) {
        *b.counter = 0;
        *b.err = 0;
    }
    for (int w = tid; w < d.B; w += nt) {
        int lo = 0x7fffffff, hi = -1;
        if (b.valid[w])
            for (int mi = 0; mi < d.L; mi++) {
                const int *bd = b.band + ((size_t)w * d.L + mi) * 3;
                if (bd[0]) {
                    lo = min(lo, bd[1]);
                    hi = max(hi, bd[2]);
                }
            }
        const bool empty = hi < lo;
        b.wrange[2 * w] = empty ? 0 : lo;
        b.wrange[2 * w + 1] = empty ? -1 : hi;
        if (sort) {
            const unsigned long long klo = empty ? 0x1fffffull : (unsigned long long)(lo >> 10);
            const unsigned long long khi = empty ? 0x1fffffull : (unsigned long long)(hi >> 10);
            keys[w] = (klo << 41) | (khi << 20) | (unsigned long long)w;
        }
    }
    if (sort) {
        for (int i = d.B + tid; i < P; i += nt) keys[i] = ~0ull;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < P; i += nt) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long a = keys[i], c = keys[ixj];
                        if ((a > c) == ((i & k) == 0)) {
                            keys[i] = c;
                            keys[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = tid; i < d.B; i += nt) b.order[i] = (int)(keys[i] & 0xfffffull);
    } else {
        for (int i = tid; i < d.B; i += nt) b.order[i] = i;
    }
    __syncthreads();
    for (int i = tid; i < d.B; i += nt) b.slot_of[b.order[i]] = i;
    __syncthreads();

    const int ng = n_groups(d.B, G);
    int carry = 0;
    for (int base = 0; base < ng; base += nt) {
        const int g = base + tid;
        int cnt = 0;
        if (g < ng) {
            int lo = 0x7fffffff, hi = -1;
            for (int k = 0; k < G; k++) {
                const int i = g * G + k;
                if (i >= d.B) break;
                const int w = b.order[i];
                if (b.wrange[2 * w + 1] >= b.wrange[2 * w]) {
                    lo = min(lo, b.wrange[2 * w]);
                    hi = max(hi, b.wrange[2 * w + 1]);
                }
            }
            if (hi >= lo) {
                lo &= ~3;  // 16-byte aligned bulk copies of the staged data
                cnt = (hi - lo + tile_bins) / tile_bins;
            } else {
                lo = 0;
                hi = -1;
            }
            b.grange[2 * g] = lo;
            b.grange[2 * g + 1] = hi;
        }
        int total;
        const int excl = block_scan(cnt, warp_tot, &total);
        if (g < ng) b.item_start[g] = carry + excl;
        carry += total;
    }
    if (tid == 0) b.item_start[ng] = carry;
}

cudaError_t launch_plan(const StageDims &d, const StageBufs &b, int tile_bins, int group,
                        cudaStream_t s) {
    const size_t smem = plan_smem(d.B);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    plan_kernel<<<1, 1024, smem, s>>>(d, b, tile_bins, group);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- finish
// Per walker, the sums of its slot over its group's items, taken in item order so the
// result does not depend on which block ran which item.  FP64: ln L = <d|h> - <h|h>/2 -
// <d|d>/2 (Eq. (2)).  Split: the parts hold sum (|h|^2 - 2 Re(d h*)) and <h|h>, and
// ln L = -sum/2 - <d|d>/2.  A device wait that gave up poisons every output with NaN.
__global__ void finish_kernel(StageDims d, StageBufs b, int G, int split, double dd, double *lnL,
                              double *dh, double *hh) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= d.B) return;
    double a = 0.0, c = 0.0;
    double out;
    if (b.valid[w]) {
        const int i = b.slot_of[w], g = i / G, k = i % G;
        for (int it = b.item_start[g]; it < b.item_start[g + 1]; it++) {
            a += b.part[2 * ((size_t)it * G + k)];
            c += b.part[2 * ((size_t)it * G + k) + 1];
        }
        out = split ? -0.5 * a - 0.5 * dd : a - 0.5 * c - 0.5 * dd;
    } else {
        out = -INFINITY;
    }
    double dhv = split ? 0.5 * (c - a) : a;
    if (*b.err) {
        out = NAN;
        dhv = NAN;
        c = NAN;
    }
    lnL[w] = out;
    if (dh) dh[w] = dhv;
    if (hh) hh[w] = c;
}

cudaError_t launch_finish(const StageDims &d, const StageBufs &b, int group, int split, double dd,
                          double *lnL, double *dh, double *hh, cudaStream_t s) {
    finish_kernel<<<(d.B + 127) / 128, 128, 0, s>>>(d, b, group, split, dd, lnL, dh, hh);
    return cudaGetLastError();
}

}  // namespace lisa
