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
// knots (Sec. II.A: ~2^10 points) with A, phase + delay, and T.  kSplit: the same FP64
// values, A (times 2^64) and T stored as FP32 (the split-precision layout).
template <bool kSplit>
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
        if (kSplit) {
            double amp, ph, t, dly;
            mode_all(src, md, f, amp, ph, t);
            cplx T[3];
            tdi_transfer(frame, kp, kc, f, t, T, &dly);
            vm[1 * K + k] = ph + dly;
            float *v32 = split_vals32(b.vals, wm, K);
            v32[k] = (float)(amp * kAmpScale64);
            for (int c = 0; c < 3; c++) {
                v32[(1 + 2 * c) * K + k] = (float)T[c].re;
                v32[(2 + 2 * c) * K + k] = (float)T[c].im;
            }
            continue;
        }
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
    knot_kernel<false><<<d.B * d.L, 128, 0, s>>>(d, b);
    return cudaGetLastError();
}

cudaError_t launch_knots_split(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    band_kernel<<<(d.B * d.L + 127) / 128, 128, 0, s>>>(d, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    knot_kernel<true><<<d.B * d.L, 128, 0, s>>>(d, b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- splines
// Not-a-knot cubic splines (the Scipy-type tridiagonal solve of Sec. II.A).  Unknowns
// are the second derivatives M_1..M_{K-2}; not-a-knot eliminates M_0 and M_{K-1}.  The
// 8 series of one (walker, mode) share the matrix.  A block owns 32 systems and every
// lane one system, so the serial recurrences keep all 32 lanes busy (GB300's FP64 pipe
// spends a full warp's time on every FP64 instruction whatever the active mask): warp 0
// factorises the 32 matrices, warp q sweeps series q of the 32 systems.
//
// The recurrences run over chunks of kCh knots staged in shared memory: the whole block
// loads a chunk of every input row of its 32 systems with coalesced accesses (threads
// walk consecutive knots of one row), transposed so that lane s reads system s; warp 0
// factorises the chunk, the eight warps sweep it, and the block writes the chunk's
// outputs back the same coalesced way.  (Walking each system's rows directly from
// global memory made every warp access touch 32 rows, and the solve waited on memory.)
// The arithmetic and its order are those of the plain recurrences.  A second,
// grid-stride kernel emits the per-segment coefficients.  The factorisation lives in
// global scratch rows next to the second derivatives.
constexpr int kSplineSystems = 32;
constexpr int kCh = 16;                     // knots per staged chunk
constexpr int kPad = kSplineSystems + 1;    // row pitch of a transposed tile
constexpr int kTile = kCh * kPad;           // elements of one [kCh][kPad] tile

// Shared memory of the solve: x, the 8 FP64 series values (outputs written in place)
// and the factorisation chunk (1/h, h, 1/pivot, normalised super-diagonal) in FP64; in
// split precision also 7 FP32 series tiles and the FP32 copies of the factorisation.
template <bool kSplit>
constexpr size_t spline_smem() {
    return sizeof(double) * kTile * (1 + kNSeries + 4) +
           (kSplit ? sizeof(float) * kTile * (kSplitSeries32 + 4) : 0);
}

// Coalesced transposed copies between kCh consecutive entries [i0, i0 + kCh) of one row
// per system and a [kCh][kPad] tile (entry k of system s at tile[k * kPad + s]); rows of
// systems outside the call or inactive are skipped, and so are indices >= iend.
template <typename T>
__device__ __forceinline__ void tile_load(T *tile, const T *base, size_t pitch, int i0, int iend,
                                          const int *act) {
    for (int e = threadIdx.x; e < kSplineSystems * kCh; e += blockDim.x) {
        const int s = e / kCh, k = e % kCh, i = i0 + k;
        if (act[s] && i < iend) tile[k * kPad + s] = base[s * pitch + i];
    }
}

// The two tile entries of this thread (blockDim.x = 256 threads, 512 entries), fetched
// into registers ahead of use and put into the tile later.
template <typename T>
__device__ __forceinline__ void tile_fetch(T r[2], const T *base, size_t pitch, int i0, int iend,
                                           const int *act) {
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const int e = threadIdx.x + j * 256;
        const int s = e / kCh, k = e % kCh, i = i0 + k;
        r[j] = (act[s] && i < iend) ? base[s * pitch + i] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void tile_put(T *tile, const T r[2]) {
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const int e = threadIdx.x + j * 256;
        tile[(e % kCh) * kPad + e / kCh] = r[j];
    }
}

template <typename T>
__device__ __forceinline__ void tile_store(const T *tile, T *base, size_t pitch, int i0, int iend,
                                           const int *act) {
    for (int e = threadIdx.x; e < kSplineSystems * kCh; e += blockDim.x) {
        const int s = e / kCh, k = e % kCh, i = i0 + k;
        if (act[s] && i < iend) base[s * pitch + i] = tile[k * kPad + s];
    }
}

// kSplit: warp 0 also writes FP32 copies of the factorisation; series 1 (the phase) is
// swept in FP64, the other seven in FP32 (the split-precision layout).  FP32 sweeps: the
// second differences lose bits in FP32, but the interpolant depends on M only through
// terms of order h^2 M, far below the values.
template <bool kSplit>
__global__ void __launch_bounds__(256) spline_kernel(StageDims d, StageBufs b) {
    extern __shared__ __align__(16) unsigned char spl_sm[];
    const int K = d.K, n = K;
    const size_t KK = (size_t)K;
    const int nsys = d.B * d.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t wm0 = (size_t)blockIdx.x * kSplineSystems;
    const size_t wm = wm0 + lane;
    __shared__ int act[kSplineSystems];
    if (threadIdx.x < kSplineSystems) {
        const size_t w2 = wm0 + threadIdx.x;
        act[threadIdx.x] = (w2 < (size_t)nsys && b.band[w2 * 3]) ? 1 : 0;
    }
    double *xs = reinterpret_cast<double *>(spl_sm);         // x[i + 1]
    double *ys = xs + kTile;                                  // [8] y[i + 1], then M[i]
    double *fs = ys + kNSeries * kTile;                       // [4] 1/h, h, 1/pivot, cpr
    float *ys32 = reinterpret_cast<float *>(fs + 4 * kTile);  // split: [7]
    float *fs32 = ys32 + kSplitSeries32 * kTile;              // split: [4]
    __syncthreads();
    const bool mine = act[lane] != 0;
    const int q = warp;  // series swept by this warp
    const bool f32s = kSplit && q != 1;
    const int q32 = (q == 0) ? 0 : q - 1;
    // row bases of the block's first system and the pitches between systems
    const double *xg = b.fk + wm0 * KK;
    const double *yg = b.vals + wm0 * kNSeries * KK;
    double *Mg = b.mscratch + wm0 * kScratchRows * KK;
    const size_t pY = kNSeries * KK, pM = kScratchRows * KK;
    const float *y32g = kSplit ? split_vals32(b.vals, wm0, K) : nullptr;
    float *M32g = kSplit ? split_m32(b.mscratch, wm0, K) : nullptr;
    float *F32g = kSplit ? split_fac32(b.mscratch, wm0, K) : nullptr;
    const size_t pY32 = 2 * pY, pM32 = 2 * pM;  // the same pitches in floats

    // per-lane set-up from the lane's own rows
    double hprev = 0.0, ihp = 0.0, cprev = 0.0;                     // factorisation
    double prev = 0.0, dprev = 0.0, ylast = 0.0, hlast = 0.0, ihl = 0.0;
    float prevf = 0.0f, dprevf = 0.0f, ylastf = 0.0f, hlastf = 0.0f, ihlf = 0.0f;
    if (mine) {
        const double *x = b.fk + wm * KK;
        const double h0 = x[1] - x[0];
        const double ih0 = 1.0 / h0;
        if (warp == 0) {
            hprev = h0;
            ihp = ih0;
            Mg[lane * pM + kNSeries * KK] = ih0;
            if (kSplit) {
                F32g[lane * pM32] = (float)ih0;
                F32g[lane * pM32 + KK] = (float)h0;
            }
        }
        if (f32s) {
            const float *yq = y32g + lane * pY32 + q32 * KK;
            dprevf = (yq[1] - yq[0]) * (float)ih0;
            ylastf = yq[1];
            hlastf = (float)h0;
        } else {
            const double *yq = b.vals + (wm * kNSeries + q) * KK;
            dprev = (yq[1] - yq[0]) * ih0;
            ylast = yq[1];
            hlast = h0;
        }
    }

    // factorisation and forward sweeps, chunk by chunk (steps i = 1 .. n - 2).  The next
    // chunk's inputs are fetched into registers while the current chunk is computed;
    // h_i = x[i+1] - x[i] and 1/h_i of a chunk are formed by all threads at once, so that
    // the serial factorisation only carries the pivots.
    __shared__ double xlast[kSplineSystems];  // x[i0] of the current chunk, per system
    if (warp == 0 && mine) xlast[lane] = b.fk[wm * KK + 1];
    double rx[2], ry[kNSeries][2];
    float ry32[kSplitSeries32][2];
    auto fetch = [&](int i1) {
        tile_fetch(rx, xg, KK, i1 + 1, n, act);
#pragma unroll
        for (int qq = 0; qq < kNSeries; qq++)
            if (!kSplit || qq == 1) tile_fetch(ry[qq], yg + qq * KK, pY, i1 + 1, n, act);
        if (kSplit)
#pragma unroll
            for (int r = 0; r < kSplitSeries32; r++)
                tile_fetch(ry32[r], y32g + r * KK, pY32, i1 + 1, n, act);
    };
    fetch(1);
    for (int i0 = 1; i0 <= n - 2; i0 += kCh) {
        const int nk = min(kCh, n - 1 - i0);
        __syncthreads();
        tile_put(xs, rx);
#pragma unroll
        for (int qq = 0; qq < kNSeries; qq++)
            if (!kSplit || qq == 1) tile_put(ys + qq * kTile, ry[qq]);
        if (kSplit)
#pragma unroll
            for (int r = 0; r < kSplitSeries32; r++) tile_put(ys32 + r * kTile, ry32[r]);
        __syncthreads();
        if (i0 + kCh <= n - 2) fetch(i0 + kCh);
        for (int e = threadIdx.x; e < kSplineSystems * kCh; e += blockDim.x) {
            const int s = e / kCh, k = e % kCh;
            if (!act[s] || k >= nk) continue;
            const int o = k * kPad + s;
            const double h = xs[o] - (k == 0 ? xlast[s] : xs[o - kPad]);
            const double ih = 1.0 / h;
            fs[o] = ih;
            fs[kTile + o] = h;
            if (kSplit) {
                fs32[o] = (float)ih;
                fs32[kTile + o] = (float)h;
            }
        }
        __syncthreads();
        if (warp == 0 && mine) {
            for (int k = 0; k < nk; k++) {
                const int i = i0 + k, o = k * kPad + lane;
                const double hcur = fs[kTile + o];
                const double ihc = fs[o];
                double dia = 2.0 * (hprev + hcur);
                double sup = hcur;
                double sb = hprev;
                if (i == 1) {
                    dia += hprev * (hprev + hcur) * ihc;
                    sup -= hprev * hprev * ihc;
                }
                if (i == n - 2) {
                    dia += hcur * (hprev + hcur) * ihp;
                    sb -= hcur * hcur * ihp;
                }
                const double pv = (i == 1) ? dia : dia - sb * cprev;
                const double inv = 1.0 / pv;
                cprev = sup * inv;
                hprev = hcur;
                ihp = ihc;
                fs[2 * kTile + o] = inv;
                fs[3 * kTile + o] = cprev;
                if (kSplit) {
                    fs32[2 * kTile + o] = (float)inv;
                    fs32[3 * kTile + o] = (float)cprev;
                }
            }
        }
        if (warp == 1 && act[lane]) xlast[lane] = xs[(nk - 1) * kPad + lane];
        __syncthreads();
        if (mine && f32s) {
            float *yt = ys32 + q32 * kTile;
            for (int k = 0; k < nk; k++) {
                const int i = i0 + k, o = k * kPad + lane;
                const float ihv = fs32[o], hv = fs32[kTile + o], dv = fs32[2 * kTile + o];
                const float yn = yt[o];
                const float dcur = (yn - ylastf) * ihv;
                ylastf = yn;
                const float rhs = 6.0f * (dcur - dprevf);
                dprevf = dcur;
                float sb = hlastf;
                if (i == n - 2) sb -= hv * hv * ihlf;
                const float rp = (i == 1) ? rhs * dv : (rhs - sb * prevf) * dv;
                yt[o] = rp;
                prevf = rp;
                hlastf = hv;
                ihlf = ihv;
            }
        } else if (mine) {
            double *yt = ys + q * kTile;
            for (int k = 0; k < nk; k++) {
                const int i = i0 + k, o = k * kPad + lane;
                const double ihv = fs[o], hv = fs[kTile + o], dv = fs[2 * kTile + o];
                const double yn = yt[o];
                const double dcur = (yn - ylast) * ihv;
                ylast = yn;
                const double rhs = 6.0 * (dcur - dprev);
                dprev = dcur;
                double sb = hlast;
                if (i == n - 2) sb -= hv * hv * ihl;
                const double rp = (i == 1) ? rhs * dv : (rhs - sb * prev) * dv;
                yt[o] = rp;
                prev = rp;
                hlast = hv;
                ihl = ihv;
            }
        }
        __syncthreads();
        // the chunk's forward values and factorisation rows (tile entry k is step i0 + k)
        for (int qq = 0; qq < kNSeries; qq++)
            if (!kSplit || qq == 1) tile_store(ys + qq * kTile, Mg + qq * KK, pM, i0, n - 1, act);
        tile_store(fs, Mg + kNSeries * KK, pM, i0, n - 1, act);                 // 1/h
        tile_store(fs + 3 * kTile, Mg + (kNSeries + 2) * KK, pM, i0, n - 1, act);  // cpr
        if (kSplit) {
            for (int r = 0; r < kSplitSeries32; r++)
                tile_store(ys32 + r * kTile, M32g + r * KK, pM32, i0, n - 1, act);
            tile_store(fs32, F32g, pM32, i0, n - 1, act);                      // 1/h
            tile_store(fs32 + kTile, F32g + KK, pM32, i0, n - 1, act);         // h
            tile_store(fs32 + 3 * kTile, F32g + 3 * KK, pM32, i0, n - 1, act); // cpr
        }
    }

    // backward sweeps, chunk by chunk from the top (steps i = n - 3 .. 1)
    __syncthreads();
    double nxt = 0.0;
    float nxtf = 0.0f;
    if (mine) {
        if (f32s)
            nxtf = M32g[lane * pM32 + q32 * KK + (n - 2)];
        else
            nxt = Mg[lane * pM + q * KK + (n - 2)];
    }
    for (int i1 = n - 3; i1 >= 1; i1 -= kCh) {
        const int lo = max(1, i1 - kCh + 1);  // tile entry k is step lo + k
        __syncthreads();
        for (int qq = 0; qq < kNSeries; qq++)
            if (!kSplit || qq == 1) tile_load(ys + qq * kTile, Mg + qq * KK, pM, lo, i1 + 1, act);
        tile_load(fs + 3 * kTile, Mg + (kNSeries + 2) * KK, pM, lo, i1 + 1, act);
        if (kSplit) {
            for (int r = 0; r < kSplitSeries32; r++)
                tile_load(ys32 + r * kTile, M32g + r * KK, pM32, lo, i1 + 1, act);
            tile_load(fs32 + 3 * kTile, F32g + 3 * KK, pM32, lo, i1 + 1, act);
        }
        __syncthreads();
        if (mine && f32s) {
            float *yt = ys32 + q32 * kTile;
            for (int i = i1; i >= lo; i--) {
                const int o = (i - lo) * kPad + lane;
                nxtf = yt[o] - fs32[3 * kTile + o] * nxtf;
                yt[o] = nxtf;
            }
        } else if (mine) {
            double *yt = ys + q * kTile;
            for (int i = i1; i >= lo; i--) {
                const int o = (i - lo) * kPad + lane;
                nxt = yt[o] - fs[3 * kTile + o] * nxt;
                yt[o] = nxt;
            }
        }
        __syncthreads();
        for (int qq = 0; qq < kNSeries; qq++)
            if (!kSplit || qq == 1) tile_store(ys + qq * kTile, Mg + qq * KK, pM, lo, i1 + 1, act);
        if (kSplit)
            for (int r = 0; r < kSplitSeries32; r++)
                tile_store(ys32 + r * kTile, M32g + r * KK, pM32, lo, i1 + 1, act);
    }
    __syncthreads();

    // not-a-knot ends: M_0 and M_{n-1} from their neighbours
    if (mine) {
        const double *x = b.fk + wm * KK;
        if (f32s) {
            float *Mq = M32g + lane * pM32 + q32 * KK;
            const float *F = F32g + lane * pM32;  // 1/h, then h
            const float h0 = F[KK], h1 = F[KK + 1], ha = F[KK + n - 3], hb = F[KK + n - 2];
            Mq[0] = ((h0 + h1) * Mq[1] - h0 * Mq[2]) * F[1];
            Mq[n - 1] = ((ha + hb) * Mq[n - 2] - hb * Mq[n - 3]) * F[n - 3];
        } else {
            double *Mq = Mg + lane * pM + q * KK;
            const double *ih = Mg + lane * pM + kNSeries * KK;
            const double h0 = x[1] - x[0], h1 = x[2] - x[1];
            const double ha = x[n - 2] - x[n - 3], hb = x[n - 1] - x[n - 2];
            Mq[0] = ((h0 + h1) * Mq[1] - h0 * Mq[2]) * ih[1];
            Mq[n - 1] = ((ha + hb) * Mq[n - 2] - hb * Mq[n - 3]) * ih[n - 3];
        }
    }
}

// Cubic coefficients of every (system, segment, series) from the second derivatives, as
// a grid-stride kernel of its own: the blocks of the solve do not divide evenly over the
// SMs, this FP64 work does.
// kSplit: only the FP64 phase series (the others stay as FP32 values and second
// derivatives for the segment records).
template <bool kSplit>
__global__ void __launch_bounds__(256) spline_coef_kernel(StageDims d, StageBufs b) {
    const int K = d.K;
    const long long per_sys = (long long)(K - 1) * (kSplit ? 1 : kNSeries);
    const long long total = (long long)d.B * d.L * per_sys;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long w2 = t / per_sys;
        const int rem = (int)(t - w2 * per_sys);
        if (!b.band[w2 * 3]) continue;
        const int sgm = kSplit ? rem : rem / kNSeries, q = kSplit ? 1 : rem % kNSeries;
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

template <bool kSplit>
cudaError_t launch_spline_t(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    const int nsys = d.B * d.L;
    const size_t smem = spline_smem<kSplit>();
    cudaError_t e = cudaFuncSetAttribute(spline_kernel<kSplit>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spline_kernel<kSplit><<<(nsys + kSplineSystems - 1) / kSplineSystems, 256, smem, s>>>(d, b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long total = (long long)nsys * (d.K - 1) * (kSplit ? 1 : kNSeries);
    const long long want = (total + 255) / 256, cap = 152LL * 8;  // 8 blocks per SM
    const int blocks = (int)(want < cap ? want : cap);
    spline_coef_kernel<kSplit><<<blocks, 256, 0, s>>>(d, b);
    return cudaGetLastError();
}

cudaError_t launch_spline(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    return launch_spline_t<false>(d, b, s);
}

cudaError_t launch_spline_split(const StageDims &d, const StageBufs &b, cudaStream_t s) {
    return launch_spline_t<true>(d, b, s);
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
