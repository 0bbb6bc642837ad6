// stages.cu -- knot, spline, planning, finishing, data-preparation and template
// kernels of the batched LISA likelihood (Katz et al. 2020, Sec. II.A).
#include "kernels.h"
#include "model.cuh"

namespace lisa {

// f_j = f0 + j df, rounded as a separate product and sum (no fused multiply-add) so
// that band edges and knot-to-bin boundaries are decided exactly as written.
__device__ __forceinline__ double bin_freq(double f0, double df, int j) {
    return __dadd_rn(f0, __dmul_rn((double)j, df));
}

// ---------------------------------------------------------------------------- bands
// One thread per (walker, mode): the walker constants, the peak of f^2 A_22 (thread of
// mode 0 stores it), and the band (Sec. II: the cut where t_lm(f) < 0, and the
// ringdown cut) with its integer dense-bin range.
__global__ void __launch_bounds__(128) band_kernel(StageDims d, StageBufs b) {
    const int wm = blockIdx.x * blockDim.x + threadIdx.x;
    if (wm >= d.B * d.L) return;
    const int w = wm / d.L, mi = wm % d.L;
    const Mode md = {d.ml[mi], d.mm[mi]};
    Source src;
    const bool ok = make_source(b.params + (size_t)w * kNPar, d.t0, src);
    int act = 0;
    double lo = 0.0, hi = 0.0;
    int jl = 0, jh = -1;
    if (ok) {
        const double fmn = d.f0;
        const double fmx = bin_freq(d.f0, d.df, d.N - 1);
        const double fcut = 0.5 * md.m * kXCut / src.M;
        hi = fmx < fcut ? fmx : fcut;
        if (hi > fmn * (1.0 + 1e-12)) {
            act = 1;
            if (mode_time(src, md, fmn) >= 0.0) {
                lo = fmn;
            } else if (mode_time(src, md, hi) < 0.0) {
                act = 0;  // the mode ends before the observation starts
            } else {
                double a = fmn, c = hi;
                for (int it = 0; it < 200 && c - a > 1e-14 * c; it++) {
                    const double mid = 0.5 * (a + c);
                    if (mode_time(src, md, mid) < 0.0)
                        a = mid;
                    else
                        c = mid;
                }
                lo = c;
            }
            if (act && !(hi > lo * (1.0 + 1e-12))) act = 0;
            if (act) {
                const double gl = ceil((lo - d.f0) / d.df - 1e-9);
                const double gh = floor((hi - d.f0) / d.df + 1e-9);
                jl = gl < 0.0 ? 0 : (int)gl;
                jh = gh > (double)(d.N - 1) ? d.N - 1 : (int)gh;
                if (jl > jh) act = 0;
            }
        }
    }
    if (!act) {
        jl = 0;
        jh = -1;
    }
    int *bd = b.band + (size_t)wm * 3;
    bd[0] = act;
    bd[1] = jl;
    bd[2] = jh;
    b.fedge[(size_t)wm * 2] = lo;
    b.fedge[(size_t)wm * 2 + 1] = hi;
    if (mi == 0) {
        b.valid[w] = ok ? 1 : 0;
        b.tc[w] = ok ? src.tc : 0.0;
        b.xpk[w] = ok ? src.xpk : 0.0;
    }
}

// ---------------------------------------------------------------------------- knots
// One block per (walker, mode): thread 0 rebuilds the walker constants (the stored peak
// spares the bisection) and the source frame; all threads then fill the K log-spaced
// knots (Sec. II.A: ~2^10 points) with A, phase + delay, and T.
__global__ void __launch_bounds__(128) knot_kernel(StageDims d, StageBufs b) {
    const int wm = blockIdx.x;
    const int w = wm / d.L, mi = wm % d.L;
    const Mode md = {d.ml[mi], d.mm[mi]};
    __shared__ Source src;
    __shared__ Frame frame;
    __shared__ cplx kp, kc;
    if (!b.band[(size_t)wm * 3]) return;  // inactive modes (and invalid walkers) have no knots
    if (threadIdx.x == 0) {
        make_source_core(b.params + (size_t)w * kNPar, d.t0, src);
        set_peak(src, b.xpk[w]);
        make_frame(src, frame);
        pol_weights(src, md, kp, kc);
    }
    __syncthreads();

    const int K = d.K;
    const double flo = b.fedge[(size_t)wm * 2], fhi = b.fedge[(size_t)wm * 2 + 1];
    const double r = log(fhi / flo);
    const double idf = 1.0 / d.df;
    double *fkm = b.fk + (size_t)wm * K;
    int *kbm = b.kb + (size_t)wm * K;
    double *vm = b.vals + (size_t)wm * kNSeries * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double f = (k == K - 1) ? fhi : flo * exp(r * (double)k / (double)(K - 1));
        fkm[k] = f;
        // first dense bin at or above this knot: a guess from 1/df, then exact by the
        // bin frequencies themselves
        double g = ceil((f - d.f0) * idf);
        int j = g <= 0.0 ? 0 : (g >= (double)d.N ? d.N : (int)g);
        while (j > 0 && bin_freq(d.f0, d.df, j - 1) >= f) j--;
        while (j < d.N && bin_freq(d.f0, d.df, j) < f) j++;
        kbm[k] = j;
        double amp, ph, t;
        mode_all(src, md, f, amp, ph, t);
        cplx T[3];
        double dly;
        tdi_transfer(frame, kp, kc, f, t, T, &dly);
        vm[0 * K + k] = amp;
        vm[1 * K + k] = ph + dly;
        vm[2 * K + k] = T[0].re;
        vm[3 * K + k] = T[0].im;
        vm[4 * K + k] = T[1].re;
        vm[5 * K + k] = T[1].im;
        vm[6 * K + k] = T[2].re;
        vm[7 * K + k] = T[2].im;
    }
}

cudaError_t launch_band(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    band_kernel<<<(d.B * d.L + 127) / 128, 128, 0, s>>>(d, b);
    return cudaGetLastError();
}

cudaError_t launch_knots(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    band_kernel<<<(d.B * d.L + 127) / 128, 128, 0, s>>>(d, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    knot_kernel<<<d.B * d.L, 128, 0, s>>>(d, b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- splines
// Not-a-knot cubic splines (the Scipy-type tridiagonal solve of Sec. II.A).  Unknowns
// are the second derivatives M_1..M_{K-2}; not-a-knot eliminates M_0 and M_{K-1}.  The
// 8 series of one (walker, mode) share the matrix.  A block owns 32 systems and every
// lane one system, so the serial recurrences keep all 32 lanes busy (GB300's FP64 pipe
// spends a full warp's time on every FP64 instruction whatever the active mask): warp 0
// factorises the 32 matrices, warp q sweeps series q of the 32 systems; a second,
// grid-stride kernel emits the per-segment coefficients.  The factorisation lives in
// global scratch rows next to the second derivatives.
constexpr int kSplineSystems = 32;

// The three serial recurrences (factorisation, forward and backward sweeps) load their
// inputs in chunks of kChunk knots ahead of the dependent arithmetic, so that the loads of
// a chunk are in flight together instead of one per step; the arithmetic is unchanged.
constexpr int kChunk = 8;

__global__ void __launch_bounds__(256) spline_kernel(StageDims d, StageBufs b) {
    const int K = d.K, n = K;
    const int nsys = d.B * d.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = blockIdx.x * kSplineSystems + lane;
    const bool mine = wm < nsys && b.band[(size_t)wm * 3];
    const double *__restrict__ x = b.fk + (size_t)wm * K;
    double *Mv = b.mscratch + (size_t)wm * kScratchRows * K;
    double *__restrict__ ih = Mv + (size_t)kNSeries * K;  // 1 / h
    double *__restrict__ dinv = ih + K;                   // 1 / pivot
    double *__restrict__ cpr = dinv + K;                  // normalised super-diagonal
    if (warp == 0 && mine) {
        double hprev = x[1] - x[0], hcur;
        const double ih0 = 1.0 / hprev;
        ih[0] = ih0;
        double cprev = 0.0;
        double ihprev = ih0;  // 1 / h_{i-1}
        double xi = x[1];
        for (int i0 = 1; i0 <= n - 2; i0 += kChunk) {
            double xn[kChunk];
#pragma unroll
            for (int k = 0; k < kChunk; k++) xn[k] = (i0 + k <= n - 2) ? x[i0 + k + 1] : 0.0;
#pragma unroll
            for (int k = 0; k < kChunk; k++) {
                const int i = i0 + k;
                if (i > n - 2) break;
                hcur = xn[k] - xi;
                xi = xn[k];
                const double ihc = 1.0 / hcur;
                ih[i] = ihc;
                double dia = 2.0 * (hprev + hcur);
                double sup = hcur;
                double sb = hprev;
                if (i == 1) {
                    dia += hprev * (hprev + hcur) * ihc;
                    sup -= hprev * hprev * ihc;
                }
                if (i == n - 2) {
                    dia += hcur * (hprev + hcur) * ihprev;
                    sb -= hcur * hcur * ihprev;
                }
                const double pv = (i == 1) ? dia : dia - sb * cprev;
                const double inv = 1.0 / pv;
                dinv[i] = inv;
                cprev = sup * inv;
                cpr[i] = cprev;
                hprev = hcur;
                ihprev = ihc;
            }
        }
    }
    __syncthreads();
    if (mine) {
        const int q = warp;  // series
        const double *__restrict__ yq = b.vals + ((size_t)wm * kNSeries + q) * K;
        double *__restrict__ Mq = Mv + (size_t)q * K;
        double prev = 0.0;
        double dprev = (yq[1] - yq[0]) * ih[0];
        double ylast = yq[1];
        double xprev = x[0];  // x[i - 1]
        const double hb_end = x[n - 1] - x[n - 2];
        const double ih_end = ih[n - 3];
        for (int i0 = 1; i0 <= n - 2; i0 += kChunk) {
            double yn[kChunk], ihv[kChunk], dv[kChunk], xv[kChunk];
#pragma unroll
            for (int k = 0; k < kChunk; k++) {
                const int i = i0 + k;
                const bool in = i <= n - 2;
                yn[k] = in ? yq[i + 1] : 0.0;
                ihv[k] = in ? ih[i] : 0.0;
                dv[k] = in ? dinv[i] : 0.0;
                xv[k] = in ? x[i] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < kChunk; k++) {
                const int i = i0 + k;
                if (i > n - 2) break;
                const double ynext = yn[k];
                const double dcur = (ynext - ylast) * ihv[k];
                ylast = ynext;
                const double rhs = 6.0 * (dcur - dprev);
                dprev = dcur;
                double sb = xv[k] - xprev;
                xprev = xv[k];
                if (i == n - 2) sb -= hb_end * hb_end * ih_end;
                const double rp = (i == 1) ? rhs * dv[k] : (rhs - sb * prev) * dv[k];
                Mq[i] = rp;
                prev = rp;
            }
        }
        double nxt = Mq[n - 2];
        for (int i0 = n - 3; i0 >= 1; i0 -= kChunk) {
            double mv[kChunk], cv[kChunk];
#pragma unroll
            for (int k = 0; k < kChunk; k++) {
                const int i = i0 - k;
                mv[k] = i >= 1 ? Mq[i] : 0.0;
                cv[k] = i >= 1 ? cpr[i] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < kChunk; k++) {
                const int i = i0 - k;
                if (i < 1) break;
                nxt = mv[k] - cv[k] * nxt;
                Mq[i] = nxt;
            }
        }
        const double h0 = x[1] - x[0], h1 = x[2] - x[1];
        const double ha = x[n - 2] - x[n - 3], hb = x[n - 1] - x[n - 2];
        Mq[0] = ((h0 + h1) * Mq[1] - h0 * Mq[2]) * ih[1];
        Mq[n - 1] = ((ha + hb) * Mq[n - 2] - hb * Mq[n - 3]) * ih[n - 3];
    }
}

// Cubic coefficients of every (system, segment, series) from the second derivatives, as
// a grid-stride kernel of its own: the blocks of the solve do not divide evenly over the
// SMs, this FP64 work does.
__global__ void __launch_bounds__(256) spline_coef_kernel(StageDims d, StageBufs b) {
    const int K = d.K;
    const long long per_sys = (long long)(K - 1) * kNSeries;
    const long long total = (long long)d.B * d.L * per_sys;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long w2 = t / per_sys;
        const int rem = (int)(t - w2 * per_sys);
        if (!b.band[w2 * 3]) continue;
        const int sgm = rem / kNSeries, q = rem % kNSeries;
        const double *x2 = b.fk + (size_t)w2 * K;
        const double *M2 = b.mscratch + (size_t)w2 * kScratchRows * K;
        const double *yq = b.vals + ((size_t)w2 * kNSeries + q) * K;
        const double *Mq = M2 + (size_t)q * K;
        const double h = x2[sgm + 1] - x2[sgm], hi = M2[(size_t)kNSeries * K + sgm];
        const double m0 = Mq[sgm], m1 = Mq[sgm + 1];
        double *c = b.coef + ((size_t)w2 * (K - 1) + sgm) * 32 + q * 4;
        c[0] = yq[sgm];
        c[1] = (yq[sgm + 1] - yq[sgm]) * hi - h * (2.0 * m0 + m1) * (1.0 / 6.0);
        c[2] = 0.5 * m0;
        c[3] = (m1 - m0) * hi * (1.0 / 6.0);
    }
}

cudaError_t launch_spline(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    const int nsys = d.B * d.L;
    spline_kernel<<<(nsys + kSplineSystems - 1) / kSplineSystems, 256, 0, s>>>(d, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long total = (long long)nsys * (d.K - 1) * kNSeries;
    const long long want = (total + 255) / 256, cap = 152LL * 8;  // 8 blocks per SM
    const int blocks = (int)(want < cap ? want : cap);
    spline_coef_kernel<<<blocks, 256, 0, s>>>(d, b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- data prep
// w = 4 df / S and w d per bin and channel (Eq. (3)), the partial sums of <d|d>, and a
// flag for a non-positive or non-finite PSD value or a non-finite data value.
__global__ void __launch_bounds__(256) prep_kernel(const double *d, const double *psd, int N,
                                                   double df, double *bins, double *ddpart,
                                                   int *bad) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        double *o = bins + (size_t)j * kBinDoubles;
        for (int c = 0; c < 3; c++) {
            const double S = psd[(size_t)c * N + j];
            const double dr = d ? d[2 * ((size_t)c * N + j)] : 0.0;
            const double di = d ? d[2 * ((size_t)c * N + j) + 1] : 0.0;
            if (!(S > 0.0) || !isfinite(S) || !isfinite(dr) || !isfinite(di)) atomicExch(bad, 1);
            const double wgt = 4.0 * df / S;
            o[c] = wgt;
            o[3 + 2 * c] = wgt * dr;
            o[4 + 2 * c] = wgt * di;
            acc += wgt * (dr * dr + di * di);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
        ddpart[blockIdx.x] = t;
    }
}

int prep_blocks(int N) {
    const int b = (N + 255) / 256;
    return b < 4096 ? b : 4096;
}

cudaError_t launch_prep(const double *d, const double *psd, int N, double df, double *bins,
                        double *ddpart, int *bad, cudaStream_t s) {
    prep_kernel<<<prep_blocks(N), 256, 0, s>>>(d, psd, N, df, bins, ddpart, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- template
// Materialise the dense template of walker 0 (injections and element-wise checks):
// one thread per bin, the same segment rule and evaluation as the fused kernel.
__device__ __forceinline__ int find_segment(const int *kb, int K, int j) {
    int lo = 0, hi = K - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (kb[mid] <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) template_kernel(StageDims d, StageBufs b, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.N) return;
    const double f = bin_freq(d.f0, d.df, j);
    double h[6] = {0, 0, 0, 0, 0, 0};
    if (b.valid[0]) {
        const double wt = kTwoPi * b.tc[0];
        for (int mi = 0; mi < d.L; mi++) {
            const int *bd = b.band + (size_t)mi * 3;
            if (!bd[0] || j < bd[1] || j > bd[2]) continue;
            const int s = find_segment(b.kb + (size_t)mi * d.K, d.K, j);
            const double x = f - b.fk[(size_t)mi * d.K + s];
            const double *c = b.coef + ((size_t)mi * (d.K - 1) + s) * 32;
            double v[kNSeries];
            for (int q = 0; q < kNSeries; q++)
                v[q] = c[4 * q] + x * (c[4 * q + 1] + x * (c[4 * q + 2] + x * c[4 * q + 3]));
            double sn, cs;
            sincos(fma(-wt, f, v[1]), &sn, &cs);
            const double zr = v[0] * cs, zi = v[0] * sn;
            for (int ch = 0; ch < 3; ch++) {
                const double tr = v[2 + 2 * ch], ti = v[3 + 2 * ch];
                h[2 * ch] += tr * zr - ti * zi;
                h[2 * ch + 1] += tr * zi + ti * zr;
            }
        }
    }
    for (int ch = 0; ch < 3; ch++) {
        out[2 * ((size_t)ch * d.N + j)] = h[2 * ch];
        out[2 * ((size_t)ch * d.N + j) + 1] = h[2 * ch + 1];
    }
}

cudaError_t launch_template(const StageDims &d, const StageBufs &b, double *out, cudaStream_t s) {
    template_kernel<<<(d.N + 255) / 256, 256, 0, s>>>(d, b, out);
    return cudaGetLastError();
}

}  // namespace lisa
