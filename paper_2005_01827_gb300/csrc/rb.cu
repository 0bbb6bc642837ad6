// rb.cu -- the relative-binning (heterodyned) likelihood of include/lisa_like.h
// (lisa_like_set_fiducial, lisa_like_loglike_rb*): the paper leaves cheaper
// approximations of its likelihood as future work (Sec. II.A); this one follows Zackay,
// Dai & Venumadhav (2018) and Cornish (2010).  A fiducial waveform h0 near the posterior
// turns the dense sums into per-bin summary data; a template then needs its modes only
// at the bin edges, where its ratio to h0 is taken as linear across each bin.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lisa_like.h"
#include "internal.h"
#include "kernels.h"
#include "model.cuh"

namespace lisa {

constexpr int kRbMaxBins = 256;
constexpr int kRbThreads = 256;
constexpr int kRbTile = 256;  // grid bins per tile of the summary kernel

struct RbState {
    int ne = 0, nb = 0, L = 0, P = 0;
    int *edges = nullptr;    // [ne] grid indices
    double *fe = nullptr;    // [ne] edge frequencies
    double *h0e = nullptr;   // [L][3][ne] complex: the fiducial's modes at the edges
    double *A = nullptr;     // [2][L][3][nb] complex: A0, A1
    double *Bs = nullptr;    // [2][P][3][nb] complex: B0, B1 for the mode pairs a <= a2
    double *fid = nullptr;   // [11] fiducial parameters
    double *flo = nullptr;   // [L] fiducial band edges
    double *fhi = nullptr;
    double xpk = 0.0;
    std::vector<int> h_edges;
};

void rb_free(RbState *r) {
    if (!r) return;
    for (void *p : {(void *)r->edges, (void *)r->fe, (void *)r->h0e, (void *)r->A, (void *)r->Bs,
                    (void *)r->fid, (void *)r->flo, (void *)r->fhi})
        if (p) cudaFree(p);
    delete r;
}

namespace {

struct RbDev {
    int ne, nb, L, P;
    const int *edges;
    const double *fe, *h0e, *A, *Bs;
    double f0, df, t0, dd;
    int ml[6], mm[6];
};

// mode pair p (a <= a2) in row order
__host__ __device__ inline void pair_of(int p, int L, int &a, int &a2) {
    a = 0;
    while (p >= L - a) {
        p -= L - a;
        a++;
    }
    a2 = a + p;
}

// one mode's A, E, T response at f (the template of the dense path before splining)
__device__ inline void response(const Source &src, const Frame &fr, const Mode &md, cplx kp,
                                cplx kc, double f, cplx out[3]) {
    double amp, ph, t;
    mode_all(src, md, f, amp, ph, t);
    cplx T[3];
    double dly;
    tdi_transfer(fr, kp, kc, f, t, T, &dly);
    const double phase = ph + dly - 2.0 * kPi * f * src.tc;
    double sn, cs;
    sincos(phase, &sn, &cs);
    for (int c = 0; c < 3; c++) {
        out[c].re = amp * (T[c].re * cs - T[c].im * sn);
        out[c].im = amp * (T[c].re * sn + T[c].im * cs);
    }
}

// the fiducial's modes at the edges: one block per mode
__global__ void rb_fid_kernel(RbDev r, const double *fid, double xpk, const double *flo,
                              const double *fhi, double *h0e) {
    const int a = blockIdx.x;
    const Mode md = {r.ml[a], r.mm[a]};
    __shared__ Source src;
    __shared__ Frame fr;
    __shared__ cplx kp, kc;
    if (threadIdx.x == 0) {
        make_source_core(fid, r.t0, src);
        set_peak(src, xpk);
        make_frame(src, fr);
        pol_weights(src, md, kp, kc);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r.ne; e += blockDim.x) {
        const double f = r.fe[e];
        cplx h[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        if (f >= flo[a] && f <= fhi[a]) response(src, fr, md, kp, kc, f, h);
        for (int c = 0; c < 3; c++) {
            h0e[2 * ((a * 3 + c) * r.ne + e)] = h[c].re;
            h0e[2 * ((a * 3 + c) * r.ne + e) + 1] = h[c].im;
        }
    }
}

// Summary data of one coarse bin: tiles of grid bins evaluate the fiducial's modes into
// shared memory, then one thread per summary quantity accumulates the tile.
__global__ void __launch_bounds__(kRbThreads) rb_summary_kernel(RbDev r, const double *fid,
                                                                double xpk, const double *flo,
                                                                const double *fhi,
                                                                const double *bins, double *A,
                                                                double *Bs) {
    extern __shared__ double sm[];
    const int L = r.L, b = blockIdx.x;
    double *h0t = sm;                          // [tile][L][3] complex
    double *wt = h0t + kRbTile * L * 6;        // [tile][3]
    double *wdt = wt + kRbTile * 3;            // [tile][3] complex
    double *dft = wdt + kRbTile * 6;           // [tile]
    __shared__ Source src;
    __shared__ Frame fr;
    __shared__ cplx kp[6], kc[6];
    if (threadIdx.x == 0) {
        make_source_core(fid, r.t0, src);
        set_peak(src, xpk);
        make_frame(src, fr);
    }
    __syncthreads();
    if (threadIdx.x < L) pol_weights(src, Mode{r.ml[threadIdx.x], r.mm[threadIdx.x]}, kp[threadIdx.x], kc[threadIdx.x]);
    __syncthreads();
    const int j_begin = r.edges[b], j_end = r.edges[b + 1];
    const double fb = __dadd_rn(r.f0, __dmul_rn((double)j_begin, r.df));
    const int Q = 6 * L + 6 * r.P;
    const int q = threadIdx.x;
    double accr = 0.0, acci = 0.0;
    int kind = 0, a = 0, a2 = 0, c = 0;
    if (q < 6 * L) {
        kind = q / (3 * L);
        a = (q % (3 * L)) / 3;
        c = q % 3;
    } else if (q < Q) {
        const int qq = q - 6 * L;
        kind = qq / (3 * r.P);
        pair_of((qq % (3 * r.P)) / 3, L, a, a2);
        c = qq % 3;
    }
    for (int j0 = j_begin; j0 < j_end; j0 += kRbTile) {
        const int cnt = min(kRbTile, j_end - j0);
        const int i = threadIdx.x;
        if (i < cnt) {
            const int j = j0 + i;
            const double f = __dadd_rn(r.f0, __dmul_rn((double)j, r.df));
            for (int m = 0; m < L; m++) {
                cplx h[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
                if (f >= flo[m] && f <= fhi[m])
                    response(src, fr, Mode{r.ml[m], r.mm[m]}, kp[m], kc[m], f, h);
                for (int ch = 0; ch < 3; ch++) {
                    h0t[((size_t)i * L + m) * 6 + 2 * ch] = h[ch].re;
                    h0t[((size_t)i * L + m) * 6 + 2 * ch + 1] = h[ch].im;
                }
            }
            const double *bj = bins + (size_t)j * kBinDoubles;
            for (int ch = 0; ch < 3; ch++) {
                wt[i * 3 + ch] = bj[ch];
                wdt[i * 6 + 2 * ch] = bj[3 + 2 * ch];
                wdt[i * 6 + 2 * ch + 1] = bj[4 + 2 * ch];
            }
            dft[i] = f - fb;
        }
        __syncthreads();
        if (q < 6 * L) {
            for (int k = 0; k < cnt; k++) {
                const double hr = h0t[((size_t)k * L + a) * 6 + 2 * c];
                const double hi = h0t[((size_t)k * L + a) * 6 + 2 * c + 1];
                const double dr = wdt[k * 6 + 2 * c], di = wdt[k * 6 + 2 * c + 1];
                const double s = kind ? dft[k] : 1.0;
                accr += s * (dr * hr + di * hi);  // (w d) conj(h0)
                acci += s * (di * hr - dr * hi);
            }
        } else if (q < Q) {
            for (int k = 0; k < cnt; k++) {
                const double xr = h0t[((size_t)k * L + a) * 6 + 2 * c];
                const double xi = h0t[((size_t)k * L + a) * 6 + 2 * c + 1];
                const double yr = h0t[((size_t)k * L + a2) * 6 + 2 * c];
                const double yi = h0t[((size_t)k * L + a2) * 6 + 2 * c + 1];
                const double s = wt[k * 3 + c] * (kind ? dft[k] : 1.0);
                accr += s * (xr * yr + xi * yi);  // w h0_a conj(h0_a2)
                acci += s * (xi * yr - xr * yi);
            }
        }
        __syncthreads();
    }
    if (q < 6 * L) {
        double *o = A + 2 * (((size_t)(kind * L + a) * 3 + c) * r.nb + b);
        o[0] = accr;
        o[1] = acci;
    } else if (q < Q) {
        const int p = ((q - 6 * L) % (3 * r.P)) / 3;
        double *o = Bs + 2 * (((size_t)(kind * r.P + p) * 3 + c) * r.nb + b);
        o[0] = accr;
        o[1] = acci;
    }
}

__device__ inline double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    return s;
}

// ln L of one walker per block
__global__ void __launch_bounds__(kRbThreads) rb_walker_kernel(RbDev r, StageDims d, StageBufs b,
                                                               double *lnL, double *dh, double *hh) {
    extern __shared__ double sm[];
    const int w = blockIdx.x, L = r.L, ne = r.ne, nb = r.nb;
    double *rr = sm;                                               // [L][3][ne] complex
    unsigned char *ok = reinterpret_cast<unsigned char *>(rr + (size_t)L * 3 * ne * 2);  // [L][3][ne]
    __shared__ Source src;
    __shared__ Frame fr;
    __shared__ cplx kp[6], kc[6];
    __shared__ double red[32];
    if (!b.valid[w]) {
        if (threadIdx.x == 0) {
            lnL[w] = -INFINITY;
            if (dh) dh[w] = 0.0;
            if (hh) hh[w] = 0.0;
        }
        return;
    }
    if (threadIdx.x == 0) {
        make_source_core(b.params + (size_t)w * kNPar, d.t0, src);
        set_peak(src, b.xpk[w]);
        make_frame(src, fr);
    }
    __syncthreads();
    if (threadIdx.x < L) pol_weights(src, Mode{r.ml[threadIdx.x], r.mm[threadIdx.x]}, kp[threadIdx.x], kc[threadIdx.x]);
    __syncthreads();
    for (int i = threadIdx.x; i < L * ne; i += blockDim.x) {
        const int a = i / ne, e = i % ne;
        const int *bd = b.band + ((size_t)w * L + a) * 3;
        const double flo = b.fedge[((size_t)w * L + a) * 2], fhi = b.fedge[((size_t)w * L + a) * 2 + 1];
        const double f = r.fe[e];
        cplx h[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        if (bd[0] && f >= flo && f <= fhi) response(src, fr, Mode{r.ml[a], r.mm[a]}, kp[a], kc[a], f, h);
        for (int c = 0; c < 3; c++) {
            const double *g = r.h0e + 2 * ((size_t)(a * 3 + c) * ne + e);
            const bool nz = g[0] != 0.0 || g[1] != 0.0;
            double qr = 0.0, qi = 0.0;
            if (nz) {  // h / h0
                const double den = g[0] * g[0] + g[1] * g[1];
                qr = (h[c].re * g[0] + h[c].im * g[1]) / den;
                qi = (h[c].im * g[0] - h[c].re * g[1]) / den;
            }
            rr[2 * ((size_t)(a * 3 + c) * ne + e)] = qr;
            rr[2 * ((size_t)(a * 3 + c) * ne + e) + 1] = qi;
            ok[(a * 3 + c) * ne + e] = nz ? 1 : 0;
        }
    }
    __syncthreads();
    // r0, r1 of (mode a, channel c, bin k) by the edge rule
    auto ratios = [&](int a, int c, int k, double &r0r, double &r0i, double &r1r, double &r1i) {
        const int base = (a * 3 + c) * ne;
        const bool okL = ok[base + k], okR = ok[base + k + 1];
        const double *pL = rr + 2 * ((size_t)base + k), *pR = pL + 2;
        r1r = r1i = 0.0;
        if (okL) {
            r0r = pL[0];
            r0i = pL[1];
            if (okR) {
                const double inv = 1.0 / (r.fe[k + 1] - r.fe[k]);
                r1r = (pR[0] - pL[0]) * inv;
                r1i = (pR[1] - pL[1]) * inv;
            }
        } else if (okR) {
            r0r = pR[0];
            r0i = pR[1];
        } else {
            r0r = r0i = 0.0;
        }
    };
    double sdh = 0.0, shh = 0.0;
    for (int i = threadIdx.x; i < L * 3 * nb; i += blockDim.x) {
        const int a = i / (3 * nb), c = (i / nb) % 3, k = i % nb;
        double r0r, r0i, r1r, r1i;
        ratios(a, c, k, r0r, r0i, r1r, r1i);
        const double *A0 = r.A + 2 * (((size_t)a * 3 + c) * nb + k);
        const double *A1 = r.A + 2 * (((size_t)(L + a) * 3 + c) * nb + k);
        sdh += A0[0] * r0r + A0[1] * r0i + A1[0] * r1r + A1[1] * r1i;  // Re(A conj(r))
    }
    for (int i = threadIdx.x; i < r.P * 3 * nb; i += blockDim.x) {
        const int p = i / (3 * nb), c = (i / nb) % 3, k = i % nb;
        int a, a2;
        pair_of(p, L, a, a2);
        double x0r, x0i, x1r, x1i, y0r, y0i, y1r, y1i;
        ratios(a, c, k, x0r, x0i, x1r, x1i);
        ratios(a2, c, k, y0r, y0i, y1r, y1i);
        const double *B0 = r.Bs + 2 * (((size_t)p * 3 + c) * nb + k);
        const double *B1 = r.Bs + 2 * (((size_t)(r.P + p) * 3 + c) * nb + k);
        // Re(B0 x0 conj(y0) + B1 (x0 conj(y1) + x1 conj(y0)))
        const double u0r = x0r * y0r + x0i * y0i, u0i = x0i * y0r - x0r * y0i;
        const double u1r = x0r * y1r + x0i * y1i + x1r * y0r + x1i * y0i;
        const double u1i = x0i * y1r - x0r * y1i + x1i * y0r - x1r * y0i;
        const double t = B0[0] * u0r - B0[1] * u0i + B1[0] * u1r - B1[1] * u1i;
        shh += (a == a2) ? t : 2.0 * t;
    }
    const double tdh = block_sum(sdh, red);
    const double thh = block_sum(shh, red);
    if (threadIdx.x == 0) {
        lnL[w] = tdh - 0.5 * thh - 0.5 * r.dd;
        if (dh) dh[w] = tdh;
        if (hh) hh[w] = thh;
    }
}

RbDev dev_of(const LikeCore &c, const RbState *s) {
    RbDev r;
    r.ne = s->ne;
    r.nb = s->nb;
    r.L = s->L;
    r.P = s->P;
    r.edges = s->edges;
    r.fe = s->fe;
    r.h0e = s->h0e;
    r.A = s->A;
    r.Bs = s->Bs;
    r.f0 = c.f0;
    r.df = c.df;
    r.t0 = c.t0;
    r.dd = c.dd;
    for (int i = 0; i < 6; i++) {
        r.ml[i] = c.ml[i];
        r.mm[i] = c.mm[i];
    }
    return r;
}

StageDims dims_of(const LikeCore &c, int B) {
    StageDims d;
    d.B = B;
    d.L = c.L;
    d.K = c.K;
    d.N = c.N;
    d.f0 = c.f0;
    d.df = c.df;
    d.t0 = c.t0;
    for (int i = 0; i < 6; i++) {
        d.ml[i] = c.ml[i];
        d.mm[i] = c.mm[i];
    }
    return d;
}

size_t walker_smem(const RbState *s) {
    return sizeof(double) * 2 * s->L * 3 * s->ne + (size_t)s->L * 3 * s->ne + 16;
}

size_t summary_smem(int L) { return sizeof(double) * kRbTile * (L * 6 + 3 + 6 + 1); }

lisa_status enqueue_rb(lisa_like_t *h, const RbState *s, const double *d_params, int B, double *lnL,
                       double *dh, double *hh, cudaStream_t st) {
    const LikeCore c = like_core(h);
    StageBufs b = c.stage;
    b.params = d_params;
    const StageDims d = dims_of(c, B);
    cudaError_t e = launch_band(d, b, st);
    if (e == cudaSuccess) {
        rb_walker_kernel<<<B, kRbThreads, walker_smem(s), st>>>(dev_of(c, s), d, b, lnL, dh, hh);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return like_fail(h, LISA_ERR_CUDA, std::string("relative-binning launch: ") + cudaGetErrorString(e));
    return LISA_OK;
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" {

lisa_status lisa_like_set_fiducial(lisa_like_t *h, const double *params, int n_rb) {
    if (!h) return LISA_ERR_ARG;
    LikeCore c = like_core(h);
    if (!c.have_data) return like_fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (!params) return like_fail(h, LISA_ERR_ARG, "NULL fiducial");
    if (n_rb < 8 || n_rb > kRbMaxBins) return like_fail(h, LISA_ERR_ARG, "n_rb must be in [8, 256]");
    cudaError_t e = cudaSetDevice(c.device);
    cudaStream_t s = c.stream;
    // the fiducial's bands (walker 0 of the handle's buffers)
    std::memcpy(c.h_params, params, sizeof(double) * kNPar);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.params, c.h_params, sizeof(double) * kNPar, cudaMemcpyHostToDevice, s);
    const StageDims d1 = dims_of(c, 1);
    if (e == cudaSuccess) e = launch_band(d1, c.stage, s);
    std::vector<int> band(3 * c.L);
    std::vector<double> fedge(2 * c.L);
    int valid = 0;
    double xpk = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(band.data(), c.stage.band, sizeof(int) * 3 * c.L, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fedge.data(), c.stage.fedge, sizeof(double) * 2 * c.L, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&valid, c.stage.valid, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&xpk, c.stage.xpk, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return like_fail(h, LISA_ERR_CUDA, std::string("fiducial bands: ") + cudaGetErrorString(e));
    lisa_status st = like_wait(h, s);
    if (st != LISA_OK) return st;
    if (!valid) return like_fail(h, LISA_ERR_ARG, "invalid fiducial parameters");
    // edges: n_rb + 1 log-spaced frequencies across the union band snapped to the grid,
    // plus every mode's band start and end + 1
    int lo = -1, hi = -1;
    std::vector<int> ed;
    for (int a = 0; a < c.L; a++) {
        if (!band[3 * a]) continue;
        const int jl = band[3 * a + 1], jh = band[3 * a + 2];
        lo = lo < 0 ? jl : std::min(lo, jl);
        hi = hi < 0 ? jh : std::max(hi, jh);
        ed.push_back(jl);
        ed.push_back(jh + 1);
    }
    if (lo < 0) return like_fail(h, LISA_ERR_ARG, "the fiducial has no active mode on this grid");
    const double f_lo = c.f0 + (double)lo * c.df, f_hi = c.f0 + (double)(hi + 1) * c.df;
    const double ya = std::log(f_lo), yb = std::log(f_hi), step = (yb - ya) / (double)n_rb;
    for (int i = 0; i <= n_rb; i++) {
        const double y = i == n_rb ? yb : (double)i * step + ya;
        double j = std::nearbyint((std::exp(y) - c.f0) / c.df);
        j = std::min(std::max(j, (double)lo), (double)(hi + 1));
        ed.push_back((int)j);
    }
    ed.push_back(lo);
    ed.push_back(hi + 1);
    std::sort(ed.begin(), ed.end());
    ed.erase(std::unique(ed.begin(), ed.end()), ed.end());
    RbState *r = new RbState();
    r->h_edges = ed;
    r->ne = (int)ed.size();
    r->nb = r->ne - 1;
    r->L = c.L;
    r->P = c.L * (c.L + 1) / 2;
    r->xpk = xpk;
    std::vector<double> fe(r->ne);
    for (int i = 0; i < r->ne; i++) fe[i] = c.f0 + (double)ed[i] * c.df;
    std::vector<double> flo(c.L), fhi(c.L);
    for (int a = 0; a < c.L; a++) {
        flo[a] = band[3 * a] ? fedge[2 * a] : 1.0;   // inactive: an empty interval
        fhi[a] = band[3 * a] ? fedge[2 * a + 1] : 0.0;
    }
    const size_t nA = (size_t)2 * r->L * 3 * r->nb * 2, nB = (size_t)2 * r->P * 3 * r->nb * 2;
    if ((e = cudaMalloc(&r->edges, sizeof(int) * r->ne)) != cudaSuccess ||
        (e = cudaMalloc(&r->fe, sizeof(double) * r->ne)) != cudaSuccess ||
        (e = cudaMalloc(&r->h0e, sizeof(double) * r->L * 3 * r->ne * 2)) != cudaSuccess ||
        (e = cudaMalloc(&r->A, sizeof(double) * nA)) != cudaSuccess ||
        (e = cudaMalloc(&r->Bs, sizeof(double) * nB)) != cudaSuccess ||
        (e = cudaMalloc(&r->fid, sizeof(double) * kNPar)) != cudaSuccess ||
        (e = cudaMalloc(&r->flo, sizeof(double) * c.L)) != cudaSuccess ||
        (e = cudaMalloc(&r->fhi, sizeof(double) * c.L)) != cudaSuccess) {
        rb_free(r);
        return like_fail(h, e == cudaErrorMemoryAllocation ? LISA_ERR_OOM : LISA_ERR_CUDA,
                         std::string("relative-binning allocation: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(r->edges, ed.data(), sizeof(int) * r->ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->fe, fe.data(), sizeof(double) * r->ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->fid, params, sizeof(double) * kNPar, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->flo, flo.data(), sizeof(double) * c.L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->fhi, fhi.data(), sizeof(double) * c.L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rb_summary_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)summary_smem(c.L));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rb_walker_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)walker_smem(r));
    if (e == cudaSuccess) {
        const RbDev rd = dev_of(c, r);
        rb_fid_kernel<<<c.L, 128, 0, s>>>(rd, r->fid, xpk, r->flo, r->fhi, r->h0e);
        rb_summary_kernel<<<r->nb, kRbThreads, summary_smem(c.L), s>>>(rd, r->fid, xpk, r->flo, r->fhi, c.bins, r->A, r->Bs);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        rb_free(r);
        return like_fail(h, LISA_ERR_CUDA, std::string("relative-binning set-up: ") + cudaGetErrorString(e));
    }
    st = like_wait(h, s);
    if (st != LISA_OK) {
        rb_free(r);
        return st;
    }
    rb_free(like_rb(h));
    like_rb(h) = r;
    return LISA_OK;
}

lisa_status lisa_like_rb_edges(lisa_like_t *h, int64_t *edges, int *n_edges) {
    if (!h || !n_edges) return LISA_ERR_ARG;
    const RbState *r = like_rb(h);
    if (!r) return like_fail(h, LISA_ERR_STATE, "lisa_like_set_fiducial must be called first");
    *n_edges = r->ne;
    if (edges)
        for (int i = 0; i < r->ne; i++) edges[i] = r->h_edges[i];
    return LISA_OK;
}

lisa_status lisa_like_loglike_rb_device(lisa_like_t *h, const double *d_params, int B, double *d_lnL,
                                        double *d_dh, double *d_hh, void *stream) {
    if (!h) return LISA_ERR_ARG;
    const LikeCore c = like_core(h);
    const RbState *r = like_rb(h);
    if (!r) return like_fail(h, LISA_ERR_STATE, "lisa_like_set_fiducial must be called first");
    if (B < 1 || B > c.max_batch) return like_fail(h, LISA_ERR_ARG, "B must be in [1, max_batch]");
    if (!d_params || !d_lnL) return like_fail(h, LISA_ERR_ARG, "NULL parameter or output pointer");
    if (cudaSetDevice(c.device) != cudaSuccess) return like_fail(h, LISA_ERR_CUDA, "cudaSetDevice");
    return enqueue_rb(h, r, d_params, B, d_lnL, d_dh, d_hh, (cudaStream_t)stream);
}

lisa_status lisa_like_loglike_rb(lisa_like_t *h, const double *params, int B, double *lnL,
                                 double *dh, double *hh) {
    if (!h) return LISA_ERR_ARG;
    const LikeCore c = like_core(h);
    const RbState *r = like_rb(h);
    if (!r) return like_fail(h, LISA_ERR_STATE, "lisa_like_set_fiducial must be called first");
    if (B < 1 || B > c.max_batch) return like_fail(h, LISA_ERR_ARG, "B must be in [1, max_batch]");
    if (!params || !lnL) return like_fail(h, LISA_ERR_ARG, "NULL parameter or output pointer");
    if (cudaSetDevice(c.device) != cudaSuccess) return like_fail(h, LISA_ERR_CUDA, "cudaSetDevice");
    cudaStream_t s = c.stream;
    std::memcpy(c.h_params, params, sizeof(double) * kNPar * B);
    cudaError_t e = cudaMemcpyAsync(c.params, c.h_params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return like_fail(h, LISA_ERR_CUDA, "parameter upload");
    lisa_status st = enqueue_rb(h, r, c.params, B, c.out, c.out + B, c.out + 2 * B, s);
    if (st != LISA_OK) return st;
    e = cudaMemcpyAsync(c.h_out, c.out, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return like_fail(h, LISA_ERR_CUDA, "result download");
    st = like_wait(h, s);
    if (st != LISA_OK) return st;
    std::memcpy(lnL, c.h_out, sizeof(double) * B);
    if (dh) std::memcpy(dh, c.h_out + B, sizeof(double) * B);
    if (hh) std::memcpy(hh, c.h_out + 2 * B, sizeof(double) * B);
    return LISA_OK;
}

}  // extern "C"
