// split.cu -- split-precision dense stage of the batched LISA likelihood (Katz et al.
// 2020, Sec. II.A): FP64 is kept for the knot phases (through the FP64 spline
// coefficients) and for the final cross-block sums; the in-segment evaluation, the
// sincos, amplitudes, transfer functions and per-thread partial sums run in FP32.
//
// Phase: per spline segment an FP64 prologue turns the cubic phase (including the
// -2 pi f t_coal ramp) into forward differences over one bin, Phi, D1, D2, D3, held as
// 64-bit fixed-point fractions of a turn.  Per bin the phase then advances by three
// exact modular integer additions, so no rounding accumulates along a segment; its top
// 8 bits index a table of e^{2 pi i k / 256} and the next 23 bits give a small angle
// (< 2 pi / 256) whose sine and cosine are short FP32 polynomials.
#include "kernels.h"
#include "model.cuh"
#include "split.h"

namespace lisa {

namespace {
constexpr double kTwoPiHi = 6.2831854820251465;        // FP32-exact leading part of 2 pi
constexpr double kTwoPiMid = -1.748455600074497e-07;   // 2 pi - hi
constexpr double kTwoPiLo = -1.0687562935444062e-23;   // 2 pi - hi - mid
constexpr double kInvTwoPi = 0.15915494309189535;
constexpr double kAmpScale = 18446744073709551616.0;    // 2^64: keeps A in FP32 range
}  // namespace

// fraction of a turn of x radians as a 64-bit two's-complement fixed-point number
__device__ __forceinline__ unsigned long long turns_fixed(double x) {
    const double k = rint(x * kInvTwoPi);
    double r = fma(-k, kTwoPiHi, x);
    r = fma(-k, kTwoPiMid, r);
    r = fma(-k, kTwoPiLo, r);
    double fr = r * kInvTwoPi;  // in about [-0.5, 0.5]
    if (fr >= 0.5) fr -= 1.0;
    if (fr < -0.5) fr += 1.0;
    return (unsigned long long)__double2ll_rn(ldexp(fr, 64));
}

__device__ __forceinline__ double bin_freq_s(double f0, double df, int j) {
    return __dadd_rn(f0, __dmul_rn((double)j, df));
}

// ------------------------------------------------------------------------ data prep
// Whitened FP32 data: s = sqrt(w) 2^-64 and d_hat = sqrt(w) d per channel, w = 4 df / S.
__global__ void __launch_bounds__(256) prep_split_kernel(const double *__restrict__ bins, int N,
                                                         float *__restrict__ out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double *b = bins + (size_t)j * kBinDoubles;
        float *o = out + (size_t)j * kBinFloats;
        for (int c = 0; c < 3; c++) {
            const double w = b[c];
            const double sw = sqrt(w);
            o[c] = (float)(sw * 5.421010862427522e-20);
            // (w d) / sqrt(w) = sqrt(w) d
            o[3 + 2 * c] = (float)(b[3 + 2 * c] / sw);
            o[4 + 2 * c] = (float)(b[4 + 2 * c] / sw);
        }
    }
}

cudaError_t launch_prep_split(const double *bins, int N, float *out, cudaStream_t s) {
    const int blocks = min((N + 255) / 256, 4096);
    prep_split_kernel<<<blocks, 256, 0, s>>>(bins, N, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ segments
// One thread per (walker, mode, segment): FP32 cubics of A 2^64 and the six transfer
// components in t = (j - kb_s) / W_s over the segment's W_s bins, and the fixed-point
// forward differences of the full phase at its first bin.
__global__ void __launch_bounds__(256) segprep_kernel(StageDims d, StageBufs b, SegRec *segs) {
    const int K = d.K;
    const long long total = (long long)d.B * d.L * (K - 1);
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(g % (K - 1));
        const long long wm = g / (K - 1);
        const int w = (int)(wm / d.L);
        const int *bd = b.band + wm * 3;
        if (!bd[0] || !b.valid[w]) continue;
        const int *kb = b.kb + wm * K;
        const int kb0 = kb[s];
        const int kb1 = (s < K - 2) ? kb[s + 1] : bd[2] + 1;
        const int W = max(kb1 - kb0, 1);
        const double fs = b.fk[wm * K + s];
        const double fj0 = bin_freq_s(d.f0, d.df, kb0);
        const double a = fj0 - fs;
        const double wd = (double)W * d.df;
        const double *cf = b.coef + ((size_t)wm * (K - 1) + s) * 32;
        SegRec r;
        int slot = 0;
        for (int q = 0; q < kNSeries; q++) {
            const double c0 = cf[4 * q], c1 = cf[4 * q + 1], c2 = cf[4 * q + 2], c3 = cf[4 * q + 3];
            const double y = fma(a, fma(a, fma(a, c3, c2), c1), c0);
            const double y1 = fma(a, fma(3.0 * a, c3, 2.0 * c2), c1);
            const double y2 = fma(3.0 * a, c3, c2);  // y''/2
            if (q == 1) {
                const double tw = kTwoPi * b.tc[w];
                const double p0 = fma(-tw, fj0, y);
                const double p1 = (y1 - tw) * d.df;
                const double p2 = y2 * d.df * d.df;
                const double p3 = c3 * d.df * d.df * d.df;
                r.p[0] = turns_fixed(p0);
                r.p[1] = turns_fixed(p1 + p2 + p3);
                r.p[2] = turns_fixed(2.0 * p2 + 6.0 * p3);
                r.p[3] = turns_fixed(6.0 * p3);
                continue;
            }
            const double sc = (q == 0) ? kAmpScale : 1.0;
            r.c[4 * slot + 0] = (float)(sc * y);
            r.c[4 * slot + 1] = (float)(sc * y1 * wd);
            r.c[4 * slot + 2] = (float)(sc * y2 * wd * wd);
            r.c[4 * slot + 3] = (float)(sc * c3 * wd * wd * wd);
            slot++;
        }
        r.kb0 = kb0;
        r.invw = 1.0f / (float)W;
        r.pad0 = 0;
        r.pad1 = 0;
        segs[g] = r;
    }
}

cudaError_t launch_segprep(const StageDims &d, const StageBufs &b, SegRec *segs, cudaStream_t s) {
    const long long total = (long long)d.B * d.L * (d.K - 1);
    const int blocks = (int)min((total + 255) / 256, (long long)152 * 32);
    segprep_kernel<<<blocks, 256, 0, s>>>(d, b, segs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ dense
__device__ __forceinline__ int seg_of(const int *__restrict__ kb, int K, int j) {
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

struct PhaseState {
    unsigned long long ph, d1, d2, d3;
};

// forward differences of the segment's phase moved from its first bin to bin n
// (Newton's forward-difference formula, exact in modular integer arithmetic)
__device__ __forceinline__ PhaseState phase_at(const SegRec &r, int n) {
    const long long nn = n;
    const unsigned long long c1 = (unsigned long long)nn;
    const unsigned long long c2 = (unsigned long long)(nn * (nn - 1) / 2);
    const unsigned long long c3 = (unsigned long long)(nn * (nn - 1) * (nn - 2) / 6);
    PhaseState p;
    p.ph = r.p[0] + c1 * r.p[1] + c2 * r.p[2] + c3 * r.p[3];
    p.d1 = r.p[1] + c1 * r.p[2] + c2 * r.p[3];
    p.d2 = r.p[2] + c1 * r.p[3];
    p.d3 = r.p[3];
    return p;
}

// e^{2 pi i ph / 2^64}: table entry of the top 8 bits times a short polynomial in the
// next 23 bits (angle below 2 pi / 256)
__device__ __forceinline__ void phasor(unsigned long long ph, const float2 *__restrict__ tab,
                                       float &zr, float &zi) {
    const unsigned int hi = (unsigned int)(ph >> 32);
    const float2 t = tab[hi >> 24];
    const float u = __uint_as_float(0x3f800000u | ((hi << 8) >> 9)) - 1.0f;  // 23 bits in [0,1)
    const float r = u * 0.024543692606170259f;                              // 2 pi / 256
    const float r2 = r * r;
    const float sn = r * fmaf(r2, -0.16666666666666666f, 1.0f);
    const float cs = fmaf(r2, fmaf(r2, 0.041666666666666664f, -0.5f), 1.0f);
    zr = t.x * cs - t.y * sn;
    zi = fmaf(t.x, sn, t.y * cs);
}

template <int C>
__global__ void __launch_bounds__(128) dense_split_kernel(StageDims d, StageBufs b,
                                                          const SegRec *__restrict__ segs,
                                                          const float *__restrict__ bins,
                                                          int tile_bins) {
    __shared__ float2 tab[256];
    __shared__ int s_item;
    __shared__ double red[2][4];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        double sn, cs;
        sincospi((double)k / 128.0, &sn, &cs);
        tab[k] = make_float2((float)cs, (float)sn);
    }
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

        float hr[C][3], hm[C][3];
#pragma unroll
        for (int i = 0; i < C; i++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                hr[i][c] = 0.0f;
                hm[i][c] = 0.0f;
            }

        for (int mi = 0; mi < d.L; mi++) {
            const size_t wm = (size_t)w * d.L + mi;
            const int *bd = b.band + wm * 3;
            if (!bd[0]) continue;
            const int ja = max(j0, bd[1]);
            const int jb = min(min(j0 + C, Jend), bd[2] + 1);
            if (ja >= jb) continue;
            const int *kb = b.kb + wm * K;
            const SegRec *sg = segs + wm * (K - 1);
            int s = seg_of(kb, K, ja);
            SegRec r = sg[s];
            int knext = (s < K - 2) ? __ldg(kb + s + 1) : 0x7fffffff;
            PhaseState p = phase_at(r, ja - r.kb0);
            float t = (float)(ja - r.kb0) * r.invw;
#pragma unroll
            for (int i = 0; i < C; i++) {
                const int j = j0 + i;
                if (j < ja || j >= jb) continue;
                if (j >= knext) {  // the chunk crosses into the next segment
                    s++;
                    r = sg[s];
                    knext = (s < K - 2) ? __ldg(kb + s + 1) : 0x7fffffff;
                    p = phase_at(r, j - r.kb0);
                    t = (float)(j - r.kb0) * r.invw;
                }
                float v[7];
#pragma unroll
                for (int q = 0; q < 7; q++)
                    v[q] = fmaf(t, fmaf(t, fmaf(t, r.c[4 * q + 3], r.c[4 * q + 2]), r.c[4 * q + 1]),
                                r.c[4 * q]);
                float zr, zi;
                phasor(p.ph, tab, zr, zi);
                zr *= v[0];
                zi *= v[0];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float tr = v[1 + 2 * c], ti = v[2 + 2 * c];
                    hr[i][c] = fmaf(tr, zr, fmaf(-ti, zi, hr[i][c]));
                    hm[i][c] = fmaf(tr, zi, fmaf(ti, zr, hm[i][c]));
                }
                p.ph += p.d1;
                p.d1 += p.d2;
                p.d2 += p.d3;
                t += r.invw;
            }
        }

        // per-bin integrand |h|^2 - 2 Re(d h*) and |h|^2 in whitened units, compensated
        float rs = 0.0f, rc = 0.0f, hs = 0.0f, hc = 0.0f;
#pragma unroll
        for (int i = 0; i < C; i++) {
            const int j = j0 + i;
            if (j >= Jend) continue;
            const float *o = bins + (size_t)j * kBinFloats;
            float ri = 0.0f, hi2 = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float sw = __ldg(o + c);
                const float xr = sw * hr[i][c], xi = sw * hm[i][c];
                const float er = fmaf(-2.0f, __ldg(o + 3 + 2 * c), xr);
                const float ei = fmaf(-2.0f, __ldg(o + 4 + 2 * c), xi);
                ri = fmaf(xr, er, fmaf(xi, ei, ri));
                hi2 = fmaf(xr, xr, fmaf(xi, xi, hi2));
            }
            // Kahan-Babuska compensated accumulation
            float y = ri - rc;
            float tt = rs + y;
            rc = (tt - rs) - y;
            rs = tt;
            y = hi2 - hc;
            tt = hs + y;
            hc = (tt - hs) - y;
            hs = tt;
        }
        double R = (double)rs - (double)rc, H = (double)hs - (double)hc;
        for (int o = 16; o > 0; o >>= 1) {
            R += __shfl_down_sync(0xffffffffu, R, o);
            H += __shfl_down_sync(0xffffffffu, H, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = R;
            red[1][threadIdx.x >> 5] = H;
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

cudaError_t launch_dense_split(const StageDims &d, const StageBufs &b, const SegRec *segs,
                               const float *bins, const DenseTune &t, cudaStream_t s) {
    if (t.threads != 128) return cudaErrorInvalidValue;
    const int tile = t.threads * t.per_thread;
    switch (t.per_thread) {
        case 8:
            dense_split_kernel<8><<<t.blocks, 128, 0, s>>>(d, b, segs, bins, tile);
            break;
        case 16:
            dense_split_kernel<16><<<t.blocks, 128, 0, s>>>(d, b, segs, bins, tile);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ln L = -(sum of |h|^2 - 2 Re(d h*))/2 - <d|d>/2; <h|h> and <d|h> follow from the sums
__global__ void finish_split_kernel(StageDims d, StageBufs b, double dd, double *lnL, double *dh,
                                    double *hh) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= d.B) return;
    double R = 0.0, H = 0.0;
    if (b.valid[w]) {
        for (int i = b.item_start[w]; i < b.item_start[w + 1]; i++) {
            R += b.part[2 * (size_t)i];
            H += b.part[2 * (size_t)i + 1];
        }
        lnL[w] = -0.5 * R - 0.5 * dd;
    } else {
        lnL[w] = -INFINITY;
    }
    if (dh) dh[w] = 0.5 * (H - R);
    if (hh) hh[w] = H;
}

cudaError_t launch_finish_split(const StageDims &d, const StageBufs &b, double dd, double *lnL,
                                double *dh, double *hh, cudaStream_t s) {
    finish_split_kernel<<<(d.B + 127) / 128, 128, 0, s>>>(d, b, dd, lnL, dh, hh);
    return cudaGetLastError();
}

}  // namespace lisa
