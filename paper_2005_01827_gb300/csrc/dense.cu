// dense.cu -- the fused dense kernel of the batched LISA likelihood (Katz et al. 2020,
// Sec. II.A): spline interpolation of A, phase and T onto the dense bins, the mode
// sum, and the noise-weighted inner products of Eqs. (3) and (11), reduced to one
// <d|h>, <h|h> pair per work item.  The dense template is never stored.
//
// Work item = (walker, tile of consecutive bins inside the union of the walker's
// active mode ranges).  Blocks are persistent and pull items from a counter, so
// walkers with very different bands (masses spanning decades) load-balance.
#include "kernels.h"
#include "model.cuh"

namespace lisa {

__device__ __forceinline__ double bin_freq_d(double f0, double df, int j) {
    return __dadd_rn(f0, __dmul_rn((double)j, df));
}

__device__ __forceinline__ int segment_of(const int *__restrict__ kb, int K, int j) {
    int lo = 0, hi = K - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(kb + mid) <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Horner evaluation of the 8 cubics of one segment at offset x.
__device__ __forceinline__ void eval_segment(const double *__restrict__ c, double x,
                                             double v[kNSeries]) {
    const double2 *c2 = reinterpret_cast<const double2 *>(c);
#pragma unroll
    for (int q = 0; q < kNSeries; q++) {
        const double2 lo = __ldg(c2 + 2 * q);
        const double2 hi = __ldg(c2 + 2 * q + 1);
        v[q] = fma(x, fma(x, fma(x, hi.y, hi.x), lo.y), lo.x);
    }
}

template <int C>
__global__ void __launch_bounds__(128) dense_f64_kernel(StageDims d, StageBufs b,
                                                        const double *__restrict__ bins,
                                                        int tile_bins) {
    __shared__ int s_item;
    __shared__ double red[2][4];
    const int total = b.item_start[d.B];
    const int K = d.K;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;

        int lo = 0, hi = d.B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.item_start[mid] <= item)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int w = lo;
        const int J0 = b.wrange[2 * w] + (item - b.item_start[w]) * tile_bins;
        const int Jend = min(J0 + tile_bins, b.wrange[2 * w + 1] + 1);
        const int j0 = J0 + (int)threadIdx.x * C;
        const double wtc = kTwoPi * b.tc[w];

        int seg[kMaxModes], jlo[kMaxModes], jhi[kMaxModes];
#pragma unroll
        for (int mi = 0; mi < kMaxModes; mi++) {
            jlo[mi] = 1;
            jhi[mi] = 0;
            seg[mi] = 0;
            if (mi < d.L) {
                const int *bd = b.band + ((size_t)w * d.L + mi) * 3;
                if (bd[0]) {
                    jlo[mi] = bd[1];
                    jhi[mi] = bd[2];
                }
                const int jj = max(j0, jlo[mi]);
                if (jj <= jhi[mi] && jj < min(j0 + C, Jend))
                    seg[mi] = segment_of(b.kb + ((size_t)w * d.L + mi) * K, K, jj);
            }
        }

        double dh = 0.0, hh = 0.0;
        for (int i = 0; i < C; i++) {
            const int j = j0 + i;
            if (j >= Jend) break;
            const double f = bin_freq_d(d.f0, d.df, j);
            double hr0 = 0.0, hi0 = 0.0, hr1 = 0.0, hi1 = 0.0, hr2 = 0.0, hi2 = 0.0;
#pragma unroll
            for (int mi = 0; mi < kMaxModes; mi++) {
                if (mi >= d.L || j < jlo[mi] || j > jhi[mi]) continue;
                const size_t wm = (size_t)w * d.L + mi;
                const int *kbm = b.kb + wm * K;
                int s = seg[mi];
                while (s < K - 2 && j >= __ldg(kbm + s + 1)) s++;
                seg[mi] = s;
                const double x = f - __ldg(b.fk + wm * K + s);
                double v[kNSeries];
                eval_segment(b.coef + (wm * (K - 1) + s) * 32, x, v);
                double sn, cs;
                sincos(fma(-wtc, f, v[1]), &sn, &cs);
                const double zr = v[0] * cs, zi = v[0] * sn;
                hr0 = fma(v[2], zr, fma(-v[3], zi, hr0));
                hi0 = fma(v[2], zi, fma(v[3], zr, hi0));
                hr1 = fma(v[4], zr, fma(-v[5], zi, hr1));
                hi1 = fma(v[4], zi, fma(v[5], zr, hi1));
                hr2 = fma(v[6], zr, fma(-v[7], zi, hr2));
                hi2 = fma(v[6], zi, fma(v[7], zr, hi2));
            }
            const double *o = bins + (size_t)j * kBinDoubles;
            hh = fma(__ldg(o + 0), fma(hr0, hr0, hi0 * hi0), hh);
            hh = fma(__ldg(o + 1), fma(hr1, hr1, hi1 * hi1), hh);
            hh = fma(__ldg(o + 2), fma(hr2, hr2, hi2 * hi2), hh);
            dh = fma(__ldg(o + 3), hr0, fma(__ldg(o + 4), hi0, dh));
            dh = fma(__ldg(o + 5), hr1, fma(__ldg(o + 6), hi1, dh));
            dh = fma(__ldg(o + 7), hr2, fma(__ldg(o + 8), hi2, dh));
        }

        for (int o = 16; o > 0; o >>= 1) {
            dh += __shfl_down_sync(0xffffffffu, dh, o);
            hh += __shfl_down_sync(0xffffffffu, hh, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = dh;
            red[1][threadIdx.x >> 5] = hh;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, c = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
                a += red[0][k];
                c += red[1][k];
            }
            b.part[2 * (size_t)item] = a;
            b.part[2 * (size_t)item + 1] = c;
        }
    }
}

cudaError_t launch_dense_f64(const StageDims &d, const StageBufs &b, const double *bins,
                             const DenseTune &t, cudaStream_t s) {
    if (t.threads != 128) return cudaErrorInvalidValue;
    const int tile = t.threads * t.per_thread;
    switch (t.per_thread) {
        case 4:
            dense_f64_kernel<4><<<t.blocks, 128, 0, s>>>(d, b, bins, tile);
            break;
        case 8:
            dense_f64_kernel<8><<<t.blocks, 128, 0, s>>>(d, b, bins, tile);
            break;
        case 16:
            dense_f64_kernel<16><<<t.blocks, 128, 0, s>>>(d, b, bins, tile);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lisa
