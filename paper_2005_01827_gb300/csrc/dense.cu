// dense.cu -- the fused FP64 dense kernel of the batched LISA likelihood (Katz et al.
// 2020, Sec. II.A): spline interpolation of A, phase and T onto the dense bins, the mode
// sum, and the noise-weighted inner products of Eqs. (3) and (11), reduced to one
// (<d|h>, <h|h>) pair per (work item, walker).  The dense template is never stored.
//
// Work item = (walker group, tile of consecutive bins inside the group's union band).
// One bulk copy (TMA) stages the tile's w and w d (72 bytes per bin) in shared memory;
// every walker of the group then reads them from there.  Blocks are persistent and pull
// items from a counter.
//
// The phase phi - 2 pi f t_coal of each mode advances from bin to bin by exact 64-bit
// fixed-point forward differences (anchored per spline segment by an FP64 prologue),
// and e^{i phase} is a 1024-entry FP64 table entry rotated by a short polynomial in the
// remaining angle (< 2 pi / 1024): every floating-point operation stays FP64.
#include "kernels.h"
#include "model.cuh"
#include "tma.cuh"

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

// Horner evaluation of the amplitude and transfer cubics (series 0, 2..7) of one segment
// at offset x; the phase series is carried by the fixed-point recurrence instead.
__device__ __forceinline__ void eval_segment(const double *__restrict__ c, double x,
                                             double v[kNSeries]) {
    const double2 *c2 = reinterpret_cast<const double2 *>(c);
#pragma unroll
    for (int q = 0; q < kNSeries; q++) {
        if (q == 1) continue;
        const double2 lo = __ldg(c2 + 2 * q);
        const double2 hi = __ldg(c2 + 2 * q + 1);
        v[q] = fma(x, fma(x, fma(x, hi.y, hi.x), lo.y), lo.x);
    }
}

struct Phase64 {
    unsigned long long ph, d1, d2, d3;
};

// fixed-point forward differences of a segment's phase moved to bin n of the segment
// (Newton's forward-difference formula in modular arithmetic; for n > 0 the low words
// add the carries of the 128-bit products)
__device__ __forceinline__ Phase64 phase64_at(const unsigned long long *__restrict__ r, int n) {
    const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(r));
    const ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2 *>(r) + 1);
    const long long nn = n;
    const unsigned long long c1 = (unsigned long long)nn;
    const unsigned long long c2 = (unsigned long long)(nn * (nn - 1)) >> 1;
    const unsigned long long c3 = (c2 * (unsigned long long)(nn - 2)) * 0xAAAAAAAAAAAAAAABull;
    Phase64 p;
    p.ph = a.x + c1 * a.y + c2 * b.x + c3 * b.y;
    p.d1 = a.y + c1 * b.x + c2 * b.y;
    p.d2 = b.x + c1 * b.y;
    p.d3 = b.y;
    if (n > 0) {
        const ulonglong2 c = __ldg(reinterpret_cast<const ulonglong2 *>(r) + 2);
        const ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2 *>(r) + 3);
        p.ph += __umul64hi(c1, c.x) + __umul64hi(c2, c.y) + __umul64hi(c3, e.x);
        p.d1 += __umul64hi(c1, c.y) + __umul64hi(c2, e.x);
        p.d2 += __umul64hi(c1, e.x);
    }
    return p;
}

// e^{2 pi i ph / 2^64} in FP64: the top 10 bits select e^{2 pi i k / 1024}, the next 52
// bits give r < 2 pi / 1024 = R, sin r is its Taylor polynomial to r^5 (truncation below
// 1e-19) and cos r = 1 - s/2 + c s^2 with s = r^2: the s^3 term of the Taylor series is
// absorbed into c, chosen so that the error c s^2 - (1/24 - s/720 + ...) s^2 equioscillates
// over s in [0, R^2] (c = 1/24 - k R^2 with 76800 k^3 + k = 1/720; truncation below 8e-18)
constexpr double kStep64 = 6.1359231515425647e-03;  // 2 pi / 1024
constexpr double kCos2 = 0.041666619912852754;

__device__ __forceinline__ void phasor64(unsigned long long ph, const double2 *__restrict__ tab,
                                         double &zr, double &zi) {
    const double2 t = tab[ph >> 54];
    // x in [1, 2) carries the next 52 bits; fma(x, step, -step) = (x - 1) step exactly
    // rounded once, as (x - 1) is exact
    const double x = __longlong_as_double(0x3ff0000000000000ull | ((ph << 10) >> 12));
    const double r = fma(x, kStep64, -kStep64);
    const double r2 = r * r;
    const double sn = r * fma(r2, fma(r2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    const double cs = fma(r2, fma(r2, kCos2, -0.5), 1.0);
    zr = fma(t.x, cs, -t.y * sn);
    zi = fma(t.x, sn, t.y * cs);
}

// group of a work item: largest g with item_start[g] <= item
__device__ __forceinline__ int group_of(const int *__restrict__ item_start, int ng, int item) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

constexpr int kTab64 = 1024;

template <int C, int G>
__global__ void __launch_bounds__(128) dense_f64_kernel(StageDims d, StageBufs b,
                                                        const unsigned long long *__restrict__ segs,
                                                        const double *__restrict__ bins,
                                                        int tile_bins) {
    extern __shared__ __align__(128) unsigned char smem[];
    double2 *tab = reinterpret_cast<double2 *>(smem);                       // [1024]
    double *sbin = reinterpret_cast<double *>(smem + sizeof(double2) * kTab64);  // [tile][9]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + sizeof(double2) * kTab64 +
                                                 sizeof(double) * kBinDoubles * tile_bins);
    __shared__ int s_item, s_walker[G], s_lo[G][kMaxModes], s_hi[G][kMaxModes];
    __shared__ double red[2][4];
    const int tid = threadIdx.x;
    for (int k = tid; k < kTab64; k += blockDim.x) {
        double sn, cs;
        sincospi((double)k / (kTab64 / 2), &sn, &cs);
        tab[k] = make_double2(cs, sn);
    }
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    const int ng = n_groups(d.B, G);
    const int total = b.item_start[ng];
    const int K = d.K;
    uint32_t parity = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;
        const int g = group_of(b.item_start, ng, item);
        const int J0 = b.grange[2 * g] + (item - b.item_start[g]) * tile_bins;
        const int Jend = min(J0 + tile_bins, b.grange[2 * g + 1] + 1);
        // whole groups of 4 rows (16-byte multiples) by one bulk copy, the last <= 3 rows
        // by plain loads, so nothing past the end of the data is read
        const int full = (Jend - J0) & ~3, tail = Jend - J0 - full;
        if (tid == 0 && full > 0) {
            const uint32_t bytes = (uint32_t)(full * kBinDoubles * sizeof(double));
            fence_proxy_async();
            if (b.wait_test_polls == 0)
                tma_load_1d(sbin, bins + (size_t)J0 * kBinDoubles, bytes, bar);
            else
                mbar_expect_tx(bar, bytes);  // test of the give-up path: no copy is issued
        }
        if (tid < tail * kBinDoubles)
            sbin[full * kBinDoubles + tid] = bins[((size_t)J0 + full) * kBinDoubles + tid];
        if (tid < G) {
            const int i = g * G + tid;
            s_walker[tid] = i < d.B ? b.order[i] : -1;
        }
        if (tid < G * kMaxModes) {
            const int k = tid / kMaxModes, mi = tid % kMaxModes;
            const int i = g * G + k;
            int lo = 1, hi = 0;
            if (i < d.B && mi < d.L) {
                const int w = b.order[i];
                const int *bd = b.band + ((size_t)w * d.L + mi) * 3;
                if (b.valid[w] && bd[0]) {
                    lo = bd[1];
                    hi = bd[2];
                }
            }
            s_lo[k][mi] = lo;
            s_hi[k][mi] = hi;
        }
        __syncthreads();
        if (full > 0) {
            // every thread waits; the block leaves together if the copy never completed
            const uint32_t polls = b.wait_test_polls ? b.wait_test_polls : kWaitPolls;
            if (!__syncthreads_and(mbar_wait_bounded(bar, parity, b.err, polls))) return;
            parity ^= 1u;
        }

        for (int k = 0; k < G; k++) {
            const int w = s_walker[k];
            if (w < 0) continue;
            const size_t slot = (size_t)item * G + k;
            if (b.wrange[2 * w + 1] < J0 || b.wrange[2 * w] >= Jend) {
                if (tid == 0) {
                    b.part[2 * slot] = 0.0;
                    b.part[2 * slot + 1] = 0.0;
                }
                continue;
            }
            const int j0 = J0 + tid * C;
            int seg[kMaxModes], knext[kMaxModes];
            Phase64 ph[kMaxModes];
#pragma unroll
            for (int mi = 0; mi < kMaxModes; mi++) {
                seg[mi] = 0;
                knext[mi] = 0x7fffffff;
                ph[mi] = Phase64{0, 0, 0, 0};
                const int jj = max(j0, s_lo[k][mi]);
                if (mi < d.L && jj <= s_hi[k][mi] && jj < min(j0 + C, Jend)) {
                    const size_t wm = (size_t)w * d.L + mi;
                    const int *kbm = b.kb + wm * K;
                    const int s = segment_of(kbm, K, jj);
                    seg[mi] = s;
                    knext[mi] = (s < K - 2) ? __ldg(kbm + s + 1) : 0x7fffffff;
                    ph[mi] = phase64_at(segs + kPhaseWords * (wm * (K - 1) + s), jj - __ldg(kbm + s));
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
                    if (mi >= d.L || j < s_lo[k][mi] || j > s_hi[k][mi]) continue;
                    const size_t wm = (size_t)w * d.L + mi;
                    if (j >= knext[mi]) {  // into the next segment: new anchor
                        const int *kbm = b.kb + wm * K;
                        int s = seg[mi];
                        while (s < K - 2 && j >= __ldg(kbm + s + 1)) s++;
                        seg[mi] = s;
                        knext[mi] = (s < K - 2) ? __ldg(kbm + s + 1) : 0x7fffffff;
                        ph[mi] = phase64_at(segs + kPhaseWords * (wm * (K - 1) + s), j - __ldg(kbm + s));
                    }
                    const int s = seg[mi];
                    const double x = f - __ldg(b.fk + wm * K + s);
                    double v[kNSeries];
                    eval_segment(b.coef + (wm * (K - 1) + s) * 32, x, v);
                    double cs, sn;
                    phasor64(ph[mi].ph, tab, cs, sn);
                    ph[mi].ph += ph[mi].d1;
                    ph[mi].d1 += ph[mi].d2;
                    ph[mi].d2 += ph[mi].d3;
                    const double zr = v[0] * cs, zi = v[0] * sn;
                    hr0 = fma(v[2], zr, fma(-v[3], zi, hr0));
                    hi0 = fma(v[2], zi, fma(v[3], zr, hi0));
                    hr1 = fma(v[4], zr, fma(-v[5], zi, hr1));
                    hi1 = fma(v[4], zi, fma(v[5], zr, hi1));
                    hr2 = fma(v[6], zr, fma(-v[7], zi, hr2));
                    hi2 = fma(v[6], zi, fma(v[7], zr, hi2));
                }
                const double *o = sbin + (size_t)(j - J0) * kBinDoubles;
                hh = fma(o[0], fma(hr0, hr0, hi0 * hi0), hh);
                hh = fma(o[1], fma(hr1, hr1, hi1 * hi1), hh);
                hh = fma(o[2], fma(hr2, hr2, hi2 * hi2), hh);
                dh = fma(o[3], hr0, fma(o[4], hi0, dh));
                dh = fma(o[5], hr1, fma(o[6], hi1, dh));
                dh = fma(o[7], hr2, fma(o[8], hi2, dh));
            }
            for (int o = 16; o > 0; o >>= 1) {
                dh += __shfl_down_sync(0xffffffffu, dh, o);
                hh += __shfl_down_sync(0xffffffffu, hh, o);
            }
            if ((tid & 31) == 0) {
                red[0][tid >> 5] = dh;
                red[1][tid >> 5] = hh;
            }
            __syncthreads();
            if (tid == 0) {
                double a = 0.0, c = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
                    a += red[0][q];
                    c += red[1][q];
                }
                b.part[2 * slot] = a;
                b.part[2 * slot + 1] = c;
            }
            __syncthreads();
        }
    }
}

template <int C>
constexpr size_t f64_smem() {
    return sizeof(double2) * kTab64 + sizeof(double) * kBinDoubles * 128 * C + 16;
}

template <int C, int G>
cudaError_t launch_f64(const StageDims &d, const StageBufs &b, const unsigned long long *segs,
                       const double *bins, int blocks, cudaStream_t s) {
    const int tile = 128 * C;
    const size_t smem = f64_smem<C>();
    cudaError_t e = cudaFuncSetAttribute(dense_f64_kernel<C, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dense_f64_kernel<C, G><<<blocks, 128, smem, s>>>(d, b, segs, bins, tile);
    return cudaGetLastError();
}

template <int C, int G>
int occ_f64() {
    const size_t smem = f64_smem<C>();
    if (cudaFuncSetAttribute(dense_f64_kernel<C, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dense_f64_kernel<C, G>, 128, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

int dense_f64_occupancy(int per_thread, int group) {
    if (per_thread == 8 && group == 8) return occ_f64<8, 8>();
    if (per_thread == 8 && group == 1) return occ_f64<8, 1>();
    if (per_thread == 4 && group == 8) return occ_f64<4, 8>();
    if (per_thread == 4 && group == 1) return occ_f64<4, 1>();
    return 0;
}

cudaError_t launch_dense_f64(const StageDims &d, const StageBufs &b,
                             const unsigned long long *segs, const double *bins,
                             const DenseTune &t, cudaStream_t s) {
    if (t.threads != 128) return cudaErrorInvalidValue;
    if (t.per_thread == 8 && t.group == 8) return launch_f64<8, 8>(d, b, segs, bins, t.blocks, s);
    if (t.per_thread == 8 && t.group == 1) return launch_f64<8, 1>(d, b, segs, bins, t.blocks, s);
    if (t.per_thread == 4 && t.group == 8) return launch_f64<4, 8>(d, b, segs, bins, t.blocks, s);
    if (t.per_thread == 4 && t.group == 1) return launch_f64<4, 1>(d, b, segs, bins, t.blocks, s);
    return cudaErrorInvalidValue;
}

}  // namespace lisa
