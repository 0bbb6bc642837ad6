// split.cu -- split-precision dense stage of the batched LISA likelihood (Katz et al.
// 2020, Sec. II.A): FP64 is kept for the knot phases (through the FP64 spline
// coefficients) and for the final cross-block sums; the in-segment evaluation, the
// sincos, amplitudes, transfer functions and per-thread partial sums run in FP32.
//
// Phase: per spline segment an FP64 prologue turns the cubic phase (including the
// -2 pi f t_coal ramp) into forward differences over one bin, Phi, D1, D2, D3, held as
// 64-bit fixed-point fractions of a turn (with extra low words for the differences).
// Each thread moves them to the first bin of its 8-bin chunk by Newton's formula in
// modular integer arithmetic, so no rounding accumulates along a segment, rounds them
// to 32-bit words and advances the phase by three 32-bit additions per bin; the top 8
// bits of the phase index a table of e^{2 pi i k / 256} (the nearest entry) and the
// next 23 bits give a small signed angle (|r| <= pi / 256) whose sine and cosine are
// short FP32 polynomials.
//
// Packed FP32: each channel's (Re, Im) transfer pair is one Horner evaluation in
// Blackwell's f32x2 FMA (one instruction for both lanes, each rounded as the scalar
// FMA), and the per-bin integrand runs on (re, im) pairs the same way.
#include "kernels.h"
#include "model.cuh"
#include "split.h"
#include "tma.cuh"

namespace lisa {

namespace {
// Cody-Waite three-part split of 2 pi for the exact reduction of a knot phase to a
// fraction of a turn: a head with few significant bits (so k x head is exact for the
// multiples k that occur), then the FP64 middle and tail of the remainder.
constexpr double kTwoPiHi = 6.2831854820251465;        // FP32-exact leading part of 2 pi
constexpr double kTwoPiMid = -1.748455600074497e-07;   // 2 pi - hi
constexpr double kTwoPiLo = -1.0687562935444062e-23;   // 2 pi - hi - mid
constexpr double kInvTwoPi = 0.15915494309189535;
}  // namespace

// fraction of a turn of x radians as a 128-bit two's-complement fixed-point number:
// hi holds the turns scaled by 2^64 (modulo 2^64), lo the next 64 fractional bits
__device__ __forceinline__ void turns_fixed(double x, unsigned long long &hi,
                                            unsigned long long &lo) {
    const double k = rint(x * kInvTwoPi);
    double r = fma(-k, kTwoPiHi, x);
    r = fma(-k, kTwoPiMid, r);
    r = fma(-k, kTwoPiLo, r);
    double fr = r * kInvTwoPi;  // in about [-0.5, 0.5]
    if (fr >= 0.5) fr -= 1.0;
    if (fr < -0.5) fr += 1.0;
    const double t = ldexp(fr, 64);  // exact scaling
    const double ft = floor(t);      // exact
    hi = (unsigned long long)(long long)ft;
    lo = (unsigned long long)ldexp(t - ft, 64);  // t - ft in [0, 1), exact
}

__device__ __forceinline__ double bin_freq_s(double f0, double df, int j) {
    return __dadd_rn(f0, __dmul_rn((double)j, df));
}

// ------------------------------------------------------------------------ data prep
// Whitened FP32 data: s = sqrt(w) 2^-64 and -2 d_hat = -2 sqrt(w) d per channel,
// w = 4 df / S.
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
            o[3 + 2 * c] = (float)(-2.0 * b[3 + 2 * c] / sw);
            o[4 + 2 * c] = (float)(-2.0 * b[4 + 2 * c] / sw);
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
// forward differences of the full phase at its first bin.  With kFull (split precision)
// the amplitude and transfer cubics come from their FP32 knot values and second
// derivatives, the phase from its FP64 spline coefficients; without it (the FP64 path)
// only the phase record is made.
template <bool kFull>
__global__ void __launch_bounds__(256) segprep_kernel(StageDims d, StageBufs b, SegRec *segs,
                                                      unsigned long long *phases) {
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
            if (!kFull && q != 1) continue;
            if (q != 1) {
                // FP32 cubic of series q in t from its knot values and second derivatives:
                // the spline's x-polynomial on [f_s, f_s+1) re-expanded at x = a and scaled
                // to t (x = a + t W df)
                const int q32 = (q == 0) ? 0 : q - 1;
                const float *yv = split_vals32(b.vals, wm, K) + (size_t)q32 * K;
                const float *Mv = split_m32(b.mscratch, wm, K) + (size_t)q32 * K;
                const float *f32 = split_fac32(b.mscratch, wm, K);
                const float ihs = f32[s], hs = f32[K + s];
                const float ys = yv[s], ys1 = yv[s + 1], ms = Mv[s], ms1 = Mv[s + 1];
                const float e1 = (ys1 - ys) * ihs - hs * fmaf(2.0f, ms, ms1) * (1.0f / 6.0f);
                const float e2 = 0.5f * ms;
                const float e3 = (ms1 - ms) * ihs * (1.0f / 6.0f);
                const float af = (float)a, wf = (float)wd;
                const int base = slot == 0 ? 0 : 4 + 8 * ((slot - 1) >> 1) + ((slot - 1) & 1);
                const int step = slot == 0 ? 1 : 2;
                r.c[base] = fmaf(af, fmaf(af, fmaf(af, e3, e2), e1), ys);
                r.c[base + step] = fmaf(af, fmaf(3.0f * af, e3, 2.0f * e2), e1) * wf;
                r.c[base + 2 * step] = fmaf(3.0f * af, e3, e2) * wf * wf;
                r.c[base + 3 * step] = e3 * wf * wf * wf;
                slot++;
                continue;
            }
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
                unsigned long long dummy;
                turns_fixed(p0, r.ph[0], dummy);
                turns_fixed(p1 + p2 + p3, r.ph[1], r.ph[4]);
                turns_fixed(2.0 * p2 + 6.0 * p3, r.ph[2], r.ph[5]);
                turns_fixed(6.0 * p3, r.ph[3], r.ph[6]);
                r.ph[7] = (unsigned int)((s < K - 2) ? kb[s + 1] : 0x7fffffff);
            }
        }
        if (kFull) {
            r.kb0 = kb0;
            r.invw = 1.0f / (float)W;
            r.pad[0] = r.pad[1] = 0;
            if (s == 0) {  // the (walker, mode)'s segment-guess constants, read once per tile
                const double f_lo = b.fedge[2 * wm], f_hi = b.fedge[2 * wm + 1];
                const double scl = (double)(K - 1) / log2(f_hi / f_lo);
                r.pad[0] = __float_as_int((float)(log2(f_lo) * scl));
                r.pad[1] = __float_as_int((float)scl);
            }
            segs[g] = r;
        } else {
            ulonglong2 *o = reinterpret_cast<ulonglong2 *>(phases + (size_t)kPhaseWords * g);
            for (int q = 0; q < kPhaseWords / 2; q++)
                o[q] = make_ulonglong2(r.ph[2 * q], r.ph[2 * q + 1]);
        }
    }
}

cudaError_t launch_segprep(const StageDims &d, const StageBufs &b, SegRec *segs, cudaStream_t s) {
    const long long total = (long long)d.B * d.L * (d.K - 1);
    const int blocks = (int)min((total + 255) / 256, (long long)152 * 32);
    segprep_kernel<true><<<blocks, 256, 0, s>>>(d, b, segs, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_phaseprep(const StageDims &d, const StageBufs &b, unsigned long long *phases,
                             cudaStream_t s) {
    const long long total = (long long)d.B * d.L * (d.K - 1);
    const int blocks = (int)min((total + 255) / 256, (long long)152 * 32);
    segprep_kernel<false><<<blocks, 256, 0, s>>>(d, b, nullptr, phases);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ dense
// segment of bin j from the log spacing of the knots: (log2 f - log2 f_lo) (K - 1) /
// log2(f_hi / f_lo) by one MUFU log2 and one FMA (l0 = scale log2 f_lo)
__device__ __forceinline__ int seg_index_guess(float fjf, float l0, float scale) {
    return (int)fmaf(__log2f(fjf), scale, -l0);
}

// the guess moved by the integer knot-to-bin boundaries so that kb[s] <= j < kb[s + 1]
__device__ __forceinline__ int seg_guess(const int *__restrict__ kb, int K, int j, float fjf,
                                         float l0, float scale) {
    int s = seg_index_guess(fjf, l0, scale);
    s = min(max(s, 0), K - 2);
    while (s > 0 && __ldg(kb + s) > j) s--;
    while (s < K - 2 && __ldg(kb + s + 1) <= j) s++;
    return s;
}

// packed FP32 pairs (Blackwell f32x2): one instruction, each lane rounded as its scalar
// counterpart
#define LISA_F32X2(op, ...)                                                                  \
    asm("{\n.reg .b64 ra, rb, rc, rd;\n"                                                      \
        "mov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\nmov.b64 rc, {%6, %7};\n" op         \
        "\nmov.b64 {%0, %1}, rd;\n}"                                                          \
        : "=f"(d.x), "=f"(d.y)                                                              \
        : __VA_ARGS__)

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    LISA_F32X2("fma.rn.f32x2 rd, ra, rb, rc;", "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x),
               "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    LISA_F32X2("mul.rn.f32x2 rd, ra, rb;", "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(0.0f),
               "f"(0.0f));
    return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    LISA_F32X2("add.rn.f32x2 rd, ra, rb;", "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(0.0f),
               "f"(0.0f));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    LISA_F32X2("sub.rn.f32x2 rd, ra, rb;", "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(0.0f),
               "f"(0.0f));
    return d;
}
#undef LISA_F32X2

// phase and forward differences at one bin as 32-bit fractions of a turn; the phase is
// offset by half a table cell so that its top 8 bits name the nearest table entry
struct PhaseState {
    unsigned int ph, d1, d2, d3;
};

// x / 2^32 rounded to the nearest integer (modulo 2^32)
__device__ __forceinline__ unsigned int top_rn(unsigned long long x) {
    return (unsigned int)(x >> 32) + ((unsigned int)x >> 31);
}

// floor(c L / 2^64) from the top 32 bits of L: low by less than c / 2^32 + 2 (c < 2^63)
__device__ __forceinline__ unsigned long long mulhi_top32(unsigned long long c,
                                                          unsigned long long L) {
    const unsigned int lh = (unsigned int)(L >> 32);
    return (c >> 32) * lh + (((unsigned long long)(unsigned int)c * lh) >> 32);
}

// the fixed-point phase words of a segment record (the last one holds the next
// segment's first bin), loaded together with its cubics so that one round trip to
// memory serves a guessed segment
struct SegPhase {
    ulonglong2 a, b, c, e;
};

__device__ __forceinline__ SegPhase seg_phase(const SegRec *__restrict__ rp) {
    const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(rp->ph);
    return SegPhase{__ldg(w), __ldg(w + 1), __ldg(w + 2), __ldg(w + 3)};
}

__device__ __forceinline__ int seg_next(const SegPhase &q) { return (int)(unsigned int)q.e.y; }

// forward differences of the segment's phase moved from its first bin to bin n >= 0
// (Newton's forward-difference formula in modular integer arithmetic).  The carries of
// the low words into the phase and the first difference are taken from their top 32
// bits and the ones multiplied by n are dropped: the 64-bit anchor is low by at most a
// few n units of 2^-64 turn for n < 2^21.  It is then rounded to 32-bit words, with
// which a thread advances its chunk: after i steps the phase is off by at most
// (1 + i + i(i-1)/2 + i(i-1)(i-2)/6) / 2 units of 2^-32 turn (32 units, 4.7e-8 rad, at
// i = 7), and every chunk starts again from the exact record.
__device__ __forceinline__ PhaseState phase_at(const SegPhase &q, int n) {
    const ulonglong2 a = q.a, b = q.b;
    const unsigned int un = (unsigned int)n;
    // n(n-1)/2 and n(n-1)(n-2)/6 (the product of three consecutive integers divided by 2
    // is a multiple of 3: multiplying by the inverse of 3 modulo 2^64 divides it exactly)
    const unsigned long long c2 = ((unsigned long long)un * (un - 1u)) >> 1;
    const unsigned long long c3 = (c2 * (unsigned long long)(un - 2u)) * 0xAAAAAAAAAAAAAAABull;
    unsigned long long ph = a.x + a.y * un + c2 * b.x + c3 * b.y;
    unsigned long long d1 = a.y + b.x * un + c2 * b.y;
    if (n >= 2) {
        ph += mulhi_top32(c2, q.c.y) + mulhi_top32(c3, q.e.x);
        d1 += mulhi_top32(c2, q.e.x);
    }
    PhaseState p;
    p.ph = top_rn(ph) + (1u << 23);  // + half a cell of the 256-entry table
    p.d1 = top_rn(d1);
    p.d2 = top_rn(b.x + b.y * un);
    p.d3 = top_rn(b.y);
    return p;
}

// the FP32 cubic coefficients, first bin and 1/width of a segment record
struct SegCoef {
    float c[28];
    int kb0;
    float invw;
};

__device__ __forceinline__ SegCoef seg_coef(const SegRec *__restrict__ rp) {
    SegCoef r;
    const float4 *v = reinterpret_cast<const float4 *>(rp->c);
#pragma unroll
    for (int q = 0; q < 7; q++) {
        const float4 x = __ldg(v + q);
        r.c[4 * q] = x.x;
        r.c[4 * q + 1] = x.y;
        r.c[4 * q + 2] = x.z;
        r.c[4 * q + 3] = x.w;
    }
    r.kb0 = __ldg(&rp->kb0);
    r.invw = __ldg(&rp->invw);
    return r;
}

// e^{2 pi i (ph - 2^23) / 2^32} for a phase word ph offset by half a cell: the table
// entry k = ph >> 24 (the nearest multiple of 2 pi / 256) times the rotation by the
// remaining signed angle r, |r| <= pi / 256, whose cosine 1 - r^2/2 is off by r^4/24 <
// 1e-9 and sine r - r^3/6 by r^5/120 < 3e-12
__device__ __forceinline__ void phasor(unsigned int ph, const float2 *__restrict__ tab,
                                       float &zr, float &zi) {
    const float2 t = tab[ph >> 24];
    // x = 1 + (ph mod 2^24) / 2^24 from the next 23 bits; x - 1.5 is exact, and so is
    // 1.5 kStep (kStep is 2 pi / 256 rounded to 23 significant bits), so the FMA
    // rounds (x - 1.5) kStep once
    const float x = __uint_as_float(0x3f800000u | ((ph << 8) >> 9));
    const float r = fmaf(x, 0.02454369142651558f, -0.03681553713977337f);
    const float r2 = r * r;
    const float sn = r * fmaf(r2, -0.16666666666666666f, 1.0f);
    const float cs = fmaf(r2, -0.5f, 1.0f);
    zr = t.x * cs - t.y * sn;
    zi = fmaf(t.x, sn, t.y * cs);
}

__device__ __forceinline__ int group_of_s(const int *__restrict__ item_start, int ng, int item) {
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

// error-free sum of two floats: a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// warp sum of FP32 (value, compensation) pairs, kept as an unevaluated hi + lo pair
__device__ __forceinline__ void warp_sum_pair(float &hi, float &lo) {
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo = lo + l2 + e;
    }
}

// the seven FP32 series of a record at in-segment coordinate tt = (t, t): the amplitude
// by scalar Horner, each channel's (Re, Im) transfer pair by packed Horner
__device__ __forceinline__ void eval_series(const SegCoef &r, float2 tt, float &amp,
                                            float2 tr[3]) {
    const float t = tt.x;
    amp = fmaf(t, fmaf(t, fmaf(t, r.c[3], r.c[2]), r.c[1]), r.c[0]);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *k = r.c + 4 + 8 * c;
        float2 x = fma2(tt, make_float2(k[6], k[7]), make_float2(k[4], k[5]));
        x = fma2(tt, x, make_float2(k[2], k[3]));
        tr[c] = fma2(tt, x, make_float2(k[0], k[1]));
    }
}

// h += T A e^{i phi} for the three channels of one bin
__device__ __forceinline__ void add_mode(const PhaseState &p, const float2 *__restrict__ tab,
                                         float amp, const float2 tr[3], float hr[3],
                                         float hm[3]) {
    float zr, zi;
    phasor(p.ph, tab, zr, zi);
    zr *= amp;
    zi *= amp;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        hr[c] = fmaf(tr[c].x, zr, fmaf(-tr[c].y, zi, hr[c]));
        hm[c] = fmaf(tr[c].x, zi, fmaf(tr[c].y, zr, hm[c]));
    }
}

template <int C, int G>
__global__ void __launch_bounds__(128, 4) dense_split_kernel(StageDims d, StageBufs b,
                                                          const SegRec *__restrict__ segs,
                                                          const float *__restrict__ bins,
                                                          int tile_bins) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *sbin = reinterpret_cast<float *>(smem);  // [tile_bins][9]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + sizeof(float) * kBinFloats * tile_bins);
    __shared__ float2 tab[256];
    __shared__ int s_item, s_walker[G], s_lo[G][kMaxModes], s_hi[G][kMaxModes];
    __shared__ float s_flo[G][kMaxModes], s_scl[G][kMaxModes];
    __shared__ float4 red[G][4];  // per slot, per warp: (ri, ri comp, hh, hh comp)
    // groups of 8 walkers: every thread's (ri, ri comp, hh, hh comp) per slot, reduced
    // once per item below instead of by warp shuffles per walker
    __shared__ float4 part_s[G == 8 ? G * 128 : 1];
    __shared__ int s_skip[G];
    const int tid = threadIdx.x;
    for (int k = tid; k < 256; k += blockDim.x) {
        double sn, cs;
        sincospi((double)k / 128.0, &sn, &cs);
        tab[k] = make_float2((float)cs, (float)sn);
    }
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    const int ng = n_groups(d.B, G);
    const int total = b.item_start[ng];
    const int K = d.K;
    const float f0f = (float)d.f0, dff = (float)d.df;
    uint32_t parity = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;
        const int g = group_of_s(b.item_start, ng, item);
        const int J0 = b.grange[2 * g] + (item - b.item_start[g]) * tile_bins;
        const int Jend = min(J0 + tile_bins, b.grange[2 * g + 1] + 1);
        // whole groups of 4 rows (16-byte multiples) by one bulk copy, the last <= 3 rows
        // by plain loads, so nothing past the end of the data is read
        const int full = (Jend - J0) & ~3, tail = Jend - J0 - full;
        if (tid == 0 && full > 0) {
            const uint32_t bytes = (uint32_t)(full * kBinFloats * sizeof(float));
            fence_proxy_async();
            if (b.wait_test_polls == 0)
                tma_load_1d(sbin, bins + (size_t)J0 * kBinFloats, bytes, bar);
            else
                mbar_expect_tx(bar, bytes);  // test of the give-up path: no copy is issued
        }
        if (tid < tail * kBinFloats)
            sbin[full * kBinFloats + tid] = bins[((size_t)J0 + full) * kBinFloats + tid];
        if (tid < G) {
            const int i = g * G + tid;
            s_walker[tid] = i < d.B ? b.order[i] : -1;
        }
        if (tid < G * kMaxModes) {
            const int k = tid / kMaxModes, mi = tid % kMaxModes;
            const int i = g * G + k;
            int lo = 1, hi = 0;
            float flo = 0.0f, scl = 0.0f;  // scale log2 f_lo and the guess scale
            if (i < d.B && mi < d.L) {
                const int w = b.order[i];
                const size_t wm = (size_t)w * d.L + mi;
                const int *bd = b.band + wm * 3;
                if (b.valid[w] && bd[0]) {
                    lo = bd[1];
                    hi = bd[2];
                    const int2 pv = __ldg(reinterpret_cast<const int2 *>(segs[wm * (K - 1)].pad));
                    flo = __int_as_float(pv.x);
                    scl = __int_as_float(pv.y);
                }
            }
            s_lo[k][mi] = lo;
            s_hi[k][mi] = hi;
            s_flo[k][mi] = flo;
            s_scl[k][mi] = scl;
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
            if (w < 0 || b.wrange[2 * w + 1] < J0 || b.wrange[2 * w] >= Jend) {
                if (tid == 0) s_skip[k] = 1;  // empty slot or band outside the tile
                continue;
            }
            if (tid == 0) s_skip[k] = 0;
            const int j0 = J0 + tid * C;
            float hr[C][3], hm[C][3];
#pragma unroll
            for (int i = 0; i < C; i++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    hr[i][c] = 0.0f;
                    hm[i][c] = 0.0f;
                }
            for (int mi = 0; mi < d.L; mi++) {
                const int ja = max(j0, s_lo[k][mi]);
                const int jb = min(min(j0 + C, Jend), s_hi[k][mi] + 1);
                if (ja >= jb) continue;
                const size_t wm = (size_t)w * d.L + mi;
                const int *kb = b.kb + wm * K;
                const SegRec *sg = segs + wm * (K - 1);
                int s = seg_index_guess(fmaf((float)ja, dff, f0f), s_flo[k][mi], s_scl[k][mi]);
                s = min(max(s, 0), K - 2);
                SegCoef r = seg_coef(sg + s);
                SegPhase q = seg_phase(sg + s);
                int knext = seg_next(q);
                // the record of the guessed segment is loaded with the bounds that check it,
                // so a right guess (the usual case) costs no dependent load
                if ((s > 0 && r.kb0 > ja) || knext <= ja) {  // the guess missed: search
                    s = seg_guess(kb, K, ja, fmaf((float)ja, dff, f0f), s_flo[k][mi], s_scl[k][mi]);
                    r = seg_coef(sg + s);
                    q = seg_phase(sg + s);
                    knext = seg_next(q);
                }
                PhaseState p = phase_at(q, ja - r.kb0);
                const float ta = (float)(ja - r.kb0) * r.invw;
                float2 tt = make_float2(ta, ta);  // (t, t): the packed Horner operand
                if (ja == j0 && jb == j0 + C && knext >= j0 + C) {
                    // the whole chunk lies in one segment and in the band: no predicates
#pragma unroll
                    for (int i = 0; i < C; i++) {
                        float amp;
                        float2 tr[3];
                        eval_series(r, tt, amp, tr);
                        add_mode(p, tab, amp, tr, hr[i], hm[i]);
                        p.ph += p.d1;
                        p.d1 += p.d2;
                        p.d2 += p.d3;
                        tt = add2(tt, make_float2(r.invw, r.invw));
                    }
                    continue;
                }
#pragma unroll
                for (int i = 0; i < C; i++) {
                    const int j = j0 + i;
                    if (j < ja || j >= jb) continue;
                    if (j >= knext) {  // the chunk crosses into the next segment
                        s++;
                        r = seg_coef(sg + s);
                        q = seg_phase(sg + s);
                        knext = seg_next(q);
                        p = phase_at(q, j - r.kb0);
                        const float tj = (float)(j - r.kb0) * r.invw;
                        tt = make_float2(tj, tj);
                    }
                    float amp;
                    float2 tr[3];
                    eval_series(r, tt, amp, tr);
                    add_mode(p, tab, amp, tr, hr[i], hm[i]);
                    p.ph += p.d1;
                    p.d1 += p.d2;
                    p.d2 += p.d3;
                    tt = add2(tt, make_float2(r.invw, r.invw));
                }
            }

            // per-bin integrand |h|^2 - 2 Re(d h*) and |h|^2 in whitened units, packed as
            // (re, im) pairs per channel, then compensated (Kahan) sums over the chunk of
            // the pair (integrand, |h|^2)
            float2 sum = make_float2(0.0f, 0.0f), comp = make_float2(0.0f, 0.0f);
            auto bin_term = [&](const float *o, int i) {
                float2 ri = make_float2(0.0f, 0.0f), hh = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float sw = o[c];
                    const float2 x = mul2(make_float2(sw, sw), make_float2(hr[i][c], hm[i][c]));
                    const float2 e = add2(x, make_float2(o[3 + 2 * c], o[4 + 2 * c]));
                    ri = fma2(x, e, ri);
                    hh = fma2(x, x, hh);
                }
                const float2 y = sub2(make_float2(ri.x + ri.y, hh.x + hh.y), comp);
                const float2 t2 = add2(sum, y);
                comp = sub2(sub2(t2, sum), y);
                sum = t2;
            };
            if (j0 + C <= Jend) {
                // the chunk's C rows start on a 16-byte boundary ((j0 - J0) 36 bytes =
                // tid C 36): four rows at a time by nine 16-byte loads
                const float4 *o4 = reinterpret_cast<const float4 *>(sbin + (j0 - J0) * kBinFloats);
#pragma unroll
                for (int h4 = 0; h4 < C / 4; h4++) {
                    float rows[4 * kBinFloats];
#pragma unroll
                    for (int q = 0; q < kBinFloats; q++) {
                        const float4 v = o4[kBinFloats * h4 + q];
                        rows[4 * q] = v.x;
                        rows[4 * q + 1] = v.y;
                        rows[4 * q + 2] = v.z;
                        rows[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int i = 0; i < 4; i++) bin_term(rows + kBinFloats * i, 4 * h4 + i);
                }
            } else {
#pragma unroll
                for (int i = 0; i < C; i++) {
                    const int j = j0 + i;
                    if (j >= Jend) continue;
                    bin_term(sbin + (j - J0) * kBinFloats, i);
                }
            }
            // FP32 (value, compensation) pairs summed error-free across the block below;
            // FP64 from the block's partial up
            if constexpr (G == 8) {
                part_s[k * 128 + tid] = make_float4(sum.x, -comp.x, sum.y, -comp.y);
            } else {
                float rs = sum.x, hs = sum.y, rl = -comp.x, hl = -comp.y;
                warp_sum_pair(rs, rl);
                warp_sum_pair(hs, hl);
                if ((tid & 31) == 0) red[k][tid >> 5] = make_float4(rs, rl, hs, hl);
            }
        }
        // one block barrier per item, then error-free FP32 sums (two-sum of the values,
        // compensations added) of every slot, once to FP64
        __syncthreads();
        if constexpr (G == 8) {
            // 16 sums (slot k, quantity q) of the 128 thread pairs, 8 threads each: 16
            // pairs per thread, then the 8 threads' pairs by shuffles
            const int grp = tid >> 3, j = tid & 7, k = grp >> 1, q = grp & 1;
            float ps = 0.0f, pe = 0.0f;
            if (s_walker[k] >= 0 && !s_skip[k]) {
                for (int i = 0; i < 16; i++) {
                    const float4 v = part_s[k * 128 + i * 8 + j];
                    float t, r;
                    two_sum(ps, q ? v.z : v.x, t, r);
                    ps = t;
                    pe += r + (q ? v.w : v.y);
                }
            }
            for (int o = 4; o > 0; o >>= 1) {
                const float s2 = __shfl_down_sync(0xffffffffu, ps, o, 8);
                const float e2 = __shfl_down_sync(0xffffffffu, pe, o, 8);
                float t, r;
                two_sum(ps, s2, t, r);
                ps = t;
                pe = pe + e2 + r;
            }
            if (j == 0 && s_walker[k] >= 0)
                b.part[2 * ((size_t)item * G + k) + q] = (double)ps + (double)pe;
        } else if (tid < G && s_walker[tid] >= 0) {
            const size_t slot = (size_t)item * G + tid;
            double a = 0.0, c = 0.0;
            if (!s_skip[tid]) {
                float4 v = red[tid][0];
                float as = v.x, ae = v.y, cs = v.z, ce = v.w;
                for (int q = 1; q < (int)(blockDim.x >> 5); q++) {
                    v = red[tid][q];
                    float t, e;
                    two_sum(as, v.x, t, e);
                    as = t;
                    ae += e + v.y;
                    two_sum(cs, v.z, t, e);
                    cs = t;
                    ce += e + v.w;
                }
                a = (double)as + (double)ae;
                c = (double)cs + (double)ce;
            }
            b.part[2 * slot] = a;
            b.part[2 * slot + 1] = c;
        }
    }
}

template <int C, int G>
cudaError_t launch_split(const StageDims &d, const StageBufs &b, const SegRec *segs,
                         const float *bins, int blocks, cudaStream_t s) {
    const int tile = 128 * C;
    const size_t smem = sizeof(float) * kBinFloats * tile + 16;
    cudaError_t e = cudaFuncSetAttribute(dense_split_kernel<C, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dense_split_kernel<C, G><<<blocks, 128, smem, s>>>(d, b, segs, bins, tile);
    return cudaGetLastError();
}

template <int C, int G>
int occ_split() {
    const size_t smem = sizeof(float) * kBinFloats * 128 * C + 16;
    if (cudaFuncSetAttribute(dense_split_kernel<C, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dense_split_kernel<C, G>, 128, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

int dense_split_occupancy(int per_thread, int group) {
    if (per_thread == 8 && group == 8) return occ_split<8, 8>();
    if (per_thread == 8 && group == 1) return occ_split<8, 1>();
    if (per_thread == 16 && group == 8) return occ_split<16, 8>();
    if (per_thread == 4 && group == 8) return occ_split<4, 8>();
    return 0;
}

cudaError_t launch_dense_split(const StageDims &d, const StageBufs &b, const SegRec *segs,
                               const float *bins, const DenseTune &t, cudaStream_t s) {
    if (t.threads != 128) return cudaErrorInvalidValue;
    if (t.per_thread == 8 && t.group == 8) return launch_split<8, 8>(d, b, segs, bins, t.blocks, s);
    if (t.per_thread == 8 && t.group == 1) return launch_split<8, 1>(d, b, segs, bins, t.blocks, s);
    if (t.per_thread == 16 && t.group == 8)
        return launch_split<16, 8>(d, b, segs, bins, t.blocks, s);
    if (t.per_thread == 4 && t.group == 8) return launch_split<4, 8>(d, b, segs, bins, t.blocks, s);
    return cudaErrorInvalidValue;
}

}  // namespace lisa
