// sampler.cu -- the parallel-tempered affine-invariant ensemble sampler of Katz et al.
// (2020), Sec. III, on the device: stretch proposals, tempered Metropolis-Hastings
// acceptance, temperature swaps and the adaptive ladder as CUDA kernels around the
// batched likelihood, one CUDA graph per step.  C ABI: include/lisa_sampler.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lisa_sampler.h"
#include "flow.h"
#include "internal.h"
#include "sampler_dev.cuh"

using namespace lisa_smp;

namespace {

constexpr int kThreads = 128;
constexpr int kSwapThreads = 256;
constexpr int kMaxT = LISA_SAMPLER_MAX_TEMPS;

// ------------------------------------------------------------------ device state
struct RecCtl {
    double *chain;  // [n][W][D] or NULL
    double *lnl;    // [n][W] or NULL
    int i;          // next row
    int pad;
};

struct Dev {
    int T, W, H, target, lisa_frame, adaptive;
    uint32_t k0, k1;
    double a, t0, lag, nu;
    double lo[D], hi[D], mean[D], sig[D];
    double *x, *lnl, *lnp, *betas;       // [T][W][D], [T][W], [T][W], [T]
    double *y, *pth, *ly, *z, *py;       // [T*H][D], [T*H][D], [T*H] x3
    unsigned long long *acc, *swaps;     // [T][2]
    unsigned *step;
    int *err;                            // sticky: a likelihood call gave up
    const int *like_err;                 // the likelihood's flag of its last call (or NULL)
    RecCtl *rec;
    double *ring;                        // [R][W][D] recent coldest states (flow training) or NULL
    int ring_rows;                       // R
};

// ------------------------------------------------------------------ kernels
// ln pi and the likelihood input (or the Gaussian ln L) of walkers c*T*H .. (c+1)*T*H-1
__global__ void init_kernel(Dev s, int c) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.T * s.H) return;
    const int i = c * s.T * s.H + p;
    const double *x = s.x + (size_t)i * D;
    const double lp = ln_prior(x, s.lo, s.hi);
    s.lnp[i] = lp;
    if (s.target == LISA_TARGET_GAUSSIAN) {
        s.lnl[i] = gauss_lnl(x, s.mean, s.sig);
    } else if (isfinite(lp)) {
        to_physical(x, s.lisa_frame, s.t0, s.pth + (size_t)p * D);
    } else {
        invalid_params(s.pth + (size_t)p * D);
    }
}

// stretch proposals (Eqs. (14)-(15)) for the walkers of half h of every temperature
__global__ void propose_kernel(Dev s, int h) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.T * s.H) return;
    const int t = p / s.H, kk = p - t * s.H, k = h * s.H + kk;
    const U4 r = philox(*s.step, (uint32_t)h, (uint32_t)t, (uint32_t)k, s.k0, s.k1);
    int jj = (int)__dmul_rn(unit(r.v[0]), (double)s.H);
    if (jj > s.H - 1) jj = s.H - 1;
    const int j = (1 - h) * s.H + jj;
    // z = (1 + (a - 1) u)^2 / a: the inverse CDF of g(z) ~ 1/sqrt(z) on [1/a, a]
    const double g = __dadd_rn(__dmul_rn(__dsub_rn(s.a, 1.0), unit(r.v[1])), 1.0);
    const double z = __ddiv_rn(__dmul_rn(g, g), s.a);
    const double *xk = s.x + ((size_t)t * s.W + k) * D;
    const double *xj = s.x + ((size_t)t * s.W + j) * D;
    double y[D];
    for (int q = 0; q < D; q++) y[q] = __dadd_rn(xj[q], __dmul_rn(z, __dsub_rn(xk[q], xj[q])));
    const double lp = ln_prior(y, s.lo, s.hi);
    double *yo = s.y + (size_t)p * D;
    for (int q = 0; q < D; q++) yo[q] = y[q];
    s.z[p] = z;
    s.py[p] = lp;
    if (s.target == LISA_TARGET_GAUSSIAN)
        s.ly[p] = gauss_lnl(y, s.mean, s.sig);
    else if (isfinite(lp))
        to_physical(y, s.lisa_frame, s.t0, s.pth + (size_t)p * D);
    else
        invalid_params(s.pth + (size_t)p * D);
}

// tempered Metropolis-Hastings acceptance of the stretch move (Eq. (16), Sec. III.B)
__global__ void accept_kernel(Dev s, int h) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.T * s.H) return;
    if (*s.err) return;
    if (s.like_err && *s.like_err) {
        atomicOr(s.err, 1);
        return;
    }
    const int t = p / s.H, kk = p - t * s.H, k = h * s.H + kk;
    const size_t i = (size_t)t * s.W + k;
    const U4 r = philox(*s.step, (uint32_t)h, (uint32_t)t, (uint32_t)k, s.k0, s.k1);
    const double py = s.py[p], ly = s.ly[p], beta = s.betas[t];
    double lr = __dsub_rn(__dadd_rn(__dmul_rn((double)(D - 1), log(s.z[p])), py), s.lnp[i]);
    if (beta > 0.0) lr = __dadd_rn(lr, __dmul_rn(beta, __dsub_rn(ly, s.lnl[i])));
    if (isfinite(py) && log(unit(r.v[2])) < lr) {
        const double *yo = s.y + (size_t)p * D;
        double *xo = s.x + i * D;
        for (int q = 0; q < D; q++) xo[q] = yo[q];
        s.lnl[i] = ly;
        s.lnp[i] = py;
        atomicAdd(s.acc + 2 * t, 1ULL);
    }
}

// temperature swaps (Eq. (17)) from the hottest pair down, the ladder update of Vousden,
// Farr & Mandel (2016), the chain record and the step counter; one block
__global__ void __launch_bounds__(kSwapThreads) swap_kernel(Dev s) {
    __shared__ int cnt[kMaxT];
    const int tid = threadIdx.x;
    for (int t = tid; t < kMaxT; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    const unsigned step = *s.step;
    for (int w = tid; w < s.W; w += blockDim.x) {
        for (int t = s.T - 2; t >= 0; t--) {
            const U4 r = philox(step, 2u, (uint32_t)t, (uint32_t)w, s.k0, s.k1);
            const size_t i = (size_t)t * s.W + w, j = (size_t)(t + 1) * s.W + w;
            const double la =
                __dmul_rn(__dsub_rn(s.betas[t], s.betas[t + 1]), __dsub_rn(s.lnl[j], s.lnl[i]));
            if (log(unit(r.v[0])) < la) {
                double *xi = s.x + i * D, *xj = s.x + j * D;
                for (int q = 0; q < D; q++) {
                    const double v = xi[q];
                    xi[q] = xj[q];
                    xj[q] = v;
                }
                double v = s.lnl[i];
                s.lnl[i] = s.lnl[j];
                s.lnl[j] = v;
                v = s.lnp[i];
                s.lnp[i] = s.lnp[j];
                s.lnp[j] = v;
                atomicAdd(&cnt[t], 1);
            }
        }
    }
    __syncthreads();
    RecCtl *rc = s.rec;
    const int row = rc->i;
    if (s.ring) {
        double *dst = s.ring + (size_t)(step % (unsigned)s.ring_rows) * s.W * D;
        for (int i = tid; i < s.W * D; i += blockDim.x) dst[i] = s.x[i];
    }
    if (rc->chain || rc->lnl) {
        for (int w = tid; w < s.W; w += blockDim.x) {
            if (rc->chain)
                for (int q = 0; q < D; q++)
                    rc->chain[((size_t)row * s.W + w) * D + q] = s.x[(size_t)w * D + q];
            if (rc->lnl) rc->lnl[(size_t)row * s.W + w] = s.lnl[w];
        }
    }
    if (tid == 0) {
        double A[kMaxT];
        for (int t = 0; t < s.T; t++) {
            s.acc[2 * t + 1] += (unsigned long long)s.W;
            A[t] = 0.0;
        }
        for (int t = 0; t + 1 < s.T; t++) {
            s.swaps[2 * t] += (unsigned long long)cnt[t];
            s.swaps[2 * t + 1] += (unsigned long long)s.W;
            A[t] = __ddiv_rn((double)cnt[t], (double)s.W);
        }
        if (s.adaptive && s.T >= 3) {
            // S_g = ln(T_{g+1} - T_g) moves by kappa (A_g - A_{g+1}); T_0 and T_{T-1} fixed
            const double kappa = __ddiv_rn(s.lag, __dmul_rn(s.nu, __dadd_rn((double)step, s.lag)));
            double gap[kMaxT];
            for (int g = 0; g + 1 < s.T - 1; g++) {
                const double dS = __dmul_rn(kappa, __dsub_rn(A[g], A[g + 1]));
                gap[g] = __dmul_rn(__dsub_rn(__ddiv_rn(1.0, s.betas[g + 1]), __ddiv_rn(1.0, s.betas[g])),
                                   exp(dS));
            }
            double Tacc = __ddiv_rn(1.0, s.betas[0]);
            for (int g = 0; g + 1 < s.T - 1; g++) {
                Tacc = __dadd_rn(Tacc, gap[g]);
                s.betas[g + 1] = __ddiv_rn(1.0, Tacc);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        rc->i = row + 1;
        *s.step = step + 1;
    }
}

__global__ void to_physical_kernel(const double *x, int n, int lisa_frame, double t0, double *th) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[D], o[D];
    for (int q = 0; q < D; q++) xi[q] = x[(size_t)i * D + q];
    to_physical(xi, lisa_frame, t0, o);
    for (int q = 0; q < D; q++) th[(size_t)i * D + q] = o[q];
}

// per-walker mean and lag-0 autocovariance (Eqs. (20)-(21))
__global__ void acf_stats_kernel(const double *c, int n, int W, int stride, int off, double *mu,
                                 double *c0) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    double m = 0.0;
    for (int i = 0; i < n; i++) m += c[((size_t)i * W + w) * stride + off];
    m /= n;
    double v = 0.0;
    for (int i = 0; i < n; i++) {
        const double e = c[((size_t)i * W + w) * stride + off] - m;
        v += e * e;
    }
    mu[w] = m;
    c0[w] = v / n;
}

// rho_w(lag) = c_w(lag) / c_w(0) for lags lag0 .. lag0 + gridDim.y - 1 (Eq. (19))
__global__ void acf_lag_kernel(const double *c, int n, int W, int stride, int off, int lag0,
                               const double *mu, const double *c0, double *rho) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int lag = lag0 + blockIdx.y;
    if (w >= W || lag >= n) return;
    const double m = mu[w];
    double acc = 0.0;
    for (int i = 0; i + lag < n; i++)
        acc += (c[((size_t)i * W + w) * stride + off] - m) *
               (c[((size_t)(i + lag) * W + w) * stride + off] - m);
    rho[(size_t)blockIdx.y * W + w] = c0[w] > 0.0 ? acc / (double)(n - lag) / c0[w] : 0.0;
}

int blocks_for(int n) { return (n + kThreads - 1) / kThreads; }

}  // namespace

// ------------------------------------------------------------------ host handle
struct lisa_sampler {
    lisa_sampler_config cfg;
    lisa_like_t *like = nullptr;
    lisa::LikeInfo li{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    Dev dev{};
    RecCtl *h_rec = nullptr;  // pinned staging
    int *h_err = nullptr;
    double timeout_s = 60.0;
    bool have_state = false;
    int launches = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_launches = 0;
    cudaEvent_t done = nullptr;
    std::vector<void *> bufs;
    std::string err;
    // flow proposal
    lisa_flow_t *flow = nullptr;
    lisa_flow_schedule fs{};
    bool flow_on = false;        // enabled
    bool flow_active = false;    // proposals are being made (trained or forced)
    int trainings = 0;
    int64_t since_train = 0;     // steps recorded in the ring since the last training
    int64_t steps_run = 0;       // steps since set_state
    lisa_flowint::FStep fst{};
    lisa_like_t *flow_like = nullptr;  // likelihood of the flow moves (default: like)
    cudaGraphExec_t gexec_flow = nullptr;
    int g_launches_flow = 0;
};

namespace {

lisa_status sfail(lisa_sampler_t *s, lisa_status st, const std::string &m) {
    if (s) s->err = m;
    return st;
}

lisa_status scuda(lisa_sampler_t *s, cudaError_t e, const char *what) {
    return sfail(s, e == cudaErrorMemoryAllocation ? LISA_ERR_OOM : LISA_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define SCK(call, what)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return scuda(s, e_, what);    \
    } while (0)

template <typename T>
cudaError_t salloc(lisa_sampler_t *s, T **p, size_t n) {
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
    if (e == cudaSuccess) s->bufs.push_back(*p);
    return e;
}

lisa_status wait_done(lisa_sampler_t *s, double limit_s) {
    SCK(cudaEventRecord(s->done, s->stream), "cudaEventRecord");
    const auto t0 = std::chrono::steady_clock::now();
    int polls = 0;
    for (;;) {
        const cudaError_t e = cudaEventQuery(s->done);
        if (e == cudaSuccess) return LISA_OK;
        if (e != cudaErrorNotReady) return scuda(s, e, "device work failed");
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit_s) return sfail(s, LISA_ERR_TIMEOUT, "sampler did not finish within the timeout");
        if (++polls > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// the kernels of one step on the sampler's stream
lisa_status enqueue_step(lisa_sampler_t *s, bool with_flow, int *nl) {
    const int n = s->dev.T * s->dev.H;
    int count = 0;
    if (with_flow) {
        SCK(lisa_flowint::launch_flow_propose(s->flow, s->fst, s->stream), "flow proposal launch");
        count++;
        if (s->dev.target == LISA_TARGET_LIKELIHOOD && s->flow_like && s->fst.margin > 0.0) {
            // screened: the sampler's likelihood on every proposal, then the second
            // likelihood on the ones the screen sends on
            int l1 = 0, l2 = 0;
            lisa_status st = lisa::like_enqueue(s->like, s->fst.fpth, s->fst.W, s->fst.fly, s->stream, &l1);
            if (st != LISA_OK) return sfail(s, st, std::string("likelihood: ") + lisa_like_last_error(s->like));
            SCK(lisa_flowint::launch_flow_screen(s->fst, s->stream), "flow screen launch");
            st = lisa::like_enqueue(s->flow_like, s->fst.fpth2, s->fst.W, s->fst.fly2, s->stream, &l2);
            if (st != LISA_OK)
                return sfail(s, st, std::string("likelihood: ") + lisa_like_last_error(s->flow_like));
            count += l1 + 1 + l2;
        } else if (s->dev.target == LISA_TARGET_LIKELIHOOD) {
            int l = 0;
            lisa_like_t *fl = s->flow_like ? s->flow_like : s->like;
            lisa_status st = lisa::like_enqueue(fl, s->fst.fpth, s->fst.W, s->fst.fly, s->stream, &l);
            if (st != LISA_OK) return sfail(s, st, std::string("likelihood: ") + lisa_like_last_error(fl));
            count += l;
        }
        SCK(lisa_flowint::launch_flow_accept(s->fst, s->stream), "flow acceptance launch");
        count++;
        if (s->fs.flow_only) {
            swap_kernel<<<1, kSwapThreads, 0, s->stream>>>(s->dev);
            SCK(cudaGetLastError(), "swap kernel launch");
            *nl = count + 1;
            return LISA_OK;
        }
    }
    for (int h = 0; h < 2; h++) {
        propose_kernel<<<blocks_for(n), kThreads, 0, s->stream>>>(s->dev, h);
        SCK(cudaGetLastError(), "proposal kernel launch");
        count++;
        if (s->dev.target == LISA_TARGET_LIKELIHOOD) {
            int l = 0;
            lisa_status st = lisa::like_enqueue(s->like, s->dev.pth, n, s->dev.ly, s->stream, &l);
            if (st != LISA_OK) return sfail(s, st, std::string("likelihood: ") + lisa_like_last_error(s->like));
            count += l;
        }
        accept_kernel<<<blocks_for(n), kThreads, 0, s->stream>>>(s->dev, h);
        SCK(cudaGetLastError(), "acceptance kernel launch");
        count++;
    }
    swap_kernel<<<1, kSwapThreads, 0, s->stream>>>(s->dev);
    SCK(cudaGetLastError(), "swap kernel launch");
    count++;
    *nl = count;
    return LISA_OK;
}

void drop_graph(lisa_sampler_t *s) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->gexec_flow) cudaGraphExecDestroy(s->gexec_flow);
    s->gexec = nullptr;
    s->gexec_flow = nullptr;
}

lisa_status capture_one(lisa_sampler_t *s, bool with_flow, cudaGraphExec_t *out, int *launches) {
    cudaGraph_t g = nullptr;
    SCK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    int nl = 0;
    lisa_status st = enqueue_step(s, with_flow, &nl);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (st != LISA_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return scuda(s, e, "graph capture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return scuda(s, e, "graph instantiation");
    }
    *launches = nl;
    return LISA_OK;
}

lisa_status capture(lisa_sampler_t *s) {
    drop_graph(s);
    lisa_status st = capture_one(s, false, &s->gexec, &s->g_launches);
    if (st == LISA_OK && s->flow_on) st = capture_one(s, true, &s->gexec_flow, &s->g_launches_flow);
    return st;
}

// steps [i0, i0 + k) with or without the flow proposal
lisa_status launch_steps(lisa_sampler_t *s, int k, bool with_flow) {
    if (s->cfg.use_graphs) {
        cudaGraphExec_t ge = with_flow ? s->gexec_flow : s->gexec;
        for (int i = 0; i < k; i++) SCK(cudaGraphLaunch(ge, s->stream), "cudaGraphLaunch");
        s->launches = with_flow ? s->g_launches_flow : s->g_launches;
    } else {
        for (int i = 0; i < k; i++) {
            int nl = 0;
            lisa_status st = enqueue_step(s, with_flow, &nl);
            if (st != LISA_OK) return st;
            s->launches = nl;
        }
    }
    return LISA_OK;
}

bool valid_box(const double *lo, const double *hi) {
    for (int q = 0; q < D; q++)
        if (!(std::isfinite(lo[q]) && std::isfinite(hi[q]) && lo[q] < hi[q])) return false;
    return true;
}

}  // namespace

extern "C" {

void lisa_sampler_default_config(lisa_sampler_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->n_temps = 8;
    c->n_walkers = 256;
    c->a = 1.15;
    c->ladder_ratio = 2.04807;
    c->t_max_inf = 1;
    c->adaptive = 1;
    c->adapt_lag = 10000.0;
    c->adapt_time = 100.0;
    c->seed = 1;
    // Table I
    const double lo[D] = {std::log(1e3), 0.05, -0.99, -0.99, std::log(0.044), 0.0, -1.0, 0.0,
                          -1.0, 0.0, 0.0};
    const double hi[D] = {std::log(1e9), 1.0, 0.99, 0.99, std::log(1298.0), 2.0 * kPi, 1.0,
                          2.0 * kPi, 1.0, kPi, std::log(3.15576e8)};
    std::memcpy(c->lower, lo, sizeof(lo));
    std::memcpy(c->upper, hi, sizeof(hi));
    c->lisa_frame = 1;
    c->target = LISA_TARGET_LIKELIHOOD;
    for (int q = 0; q < D; q++) c->gauss_sigma[q] = 1.0;
    c->use_graphs = 1;
}

lisa_status lisa_sampler_create(lisa_like_t *like, const lisa_sampler_config *cfg,
                                lisa_sampler_t **out) {
    lisa::set_thread_error("");
    auto bad = [](const char *m) {
        lisa::set_thread_error(m);
        return LISA_ERR_ARG;
    };
    if (!cfg || !out) return bad("NULL config or output pointer");
    *out = nullptr;
    const int T = cfg->n_temps, W = cfg->n_walkers;
    if (T < 1 || T > kMaxT) return bad("n_temps must be in [1, 64]");
    if (W < 4 || (W & 1) || W > (1 << 16)) return bad("n_walkers must be even and in [4, 65536]");
    if (!(cfg->a > 1.0) || !std::isfinite(cfg->a)) return bad("stretch scale a must be > 1");
    if (!(cfg->ladder_ratio > 1.0) || !std::isfinite(cfg->ladder_ratio))
        return bad("ladder_ratio must be > 1");
    if (cfg->adaptive && !(cfg->adapt_lag > 0.0 && cfg->adapt_time > 0.0))
        return bad("adapt_lag and adapt_time must be > 0");
    if (!valid_box(cfg->lower, cfg->upper)) return bad("prior bounds must be finite with lower < upper");
    if (cfg->target != LISA_TARGET_LIKELIHOOD && cfg->target != LISA_TARGET_GAUSSIAN)
        return bad("unknown target");
    if (cfg->target == LISA_TARGET_GAUSSIAN)
        for (int q = 0; q < D; q++)
            if (!(cfg->gauss_sigma[q] > 0.0) || !std::isfinite(cfg->gauss_mean[q]))
                return bad("Gaussian target needs finite means and sigma > 0");
    lisa::LikeInfo li{};
    if (cfg->target == LISA_TARGET_LIKELIHOOD) {
        if (!like) return bad("the likelihood target needs a lisa_like handle");
        li = lisa::like_info(like);
        if (!li.have_data) {
            lisa::set_thread_error("lisa_like_set_data must be called before creating the sampler");
            return LISA_ERR_STATE;
        }
        if ((int64_t)T * (W / 2) > li.max_batch)
            return bad("the likelihood's max_batch must be >= n_temps * n_walkers / 2");
    }
    lisa_sampler_t *s = new lisa_sampler();
    s->cfg = *cfg;
    s->like = cfg->target == LISA_TARGET_LIKELIHOOD ? like : nullptr;
    s->li = li;
    lisa_status st = LISA_OK;
    do {
        int dev = 0;
        cudaError_t e = cudaSuccess;
        if (s->like) {
            dev = li.device;
            s->stream = li.stream;
            s->timeout_s = cfg->timeout_s > 0.0 ? cfg->timeout_s : li.timeout_s;
            e = cudaSetDevice(dev);
        } else {
            e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = e == cudaSuccess;
            s->timeout_s = cfg->timeout_s > 0.0 ? cfg->timeout_s : 60.0;
        }
        if (e != cudaSuccess) {
            st = scuda(s, e, "device setup");
            break;
        }
        s->device = dev;
        Dev &d = s->dev;
        d.T = T;
        d.W = W;
        d.H = W / 2;
        d.target = cfg->target;
        d.lisa_frame = cfg->lisa_frame ? 1 : 0;
        d.adaptive = cfg->adaptive ? 1 : 0;
        d.k0 = (uint32_t)cfg->seed;
        d.k1 = (uint32_t)(cfg->seed >> 32);
        d.a = cfg->a;
        d.t0 = li.t0;
        d.lag = cfg->adapt_lag;
        d.nu = cfg->adapt_time;
        for (int q = 0; q < D; q++) {
            d.lo[q] = cfg->lower[q];
            d.hi[q] = cfg->upper[q];
            d.mean[q] = cfg->gauss_mean[q];
            d.sig[q] = cfg->gauss_sigma[q];
        }
        const size_t TW = (size_t)T * W, TH = (size_t)T * d.H;
        if ((e = salloc(s, &d.x, TW * D)) != cudaSuccess || (e = salloc(s, &d.lnl, TW)) != cudaSuccess ||
            (e = salloc(s, &d.lnp, TW)) != cudaSuccess || (e = salloc(s, &d.betas, (size_t)T)) != cudaSuccess ||
            (e = salloc(s, &d.y, TH * D)) != cudaSuccess || (e = salloc(s, &d.pth, TH * D)) != cudaSuccess ||
            (e = salloc(s, &d.ly, TH)) != cudaSuccess || (e = salloc(s, &d.z, TH)) != cudaSuccess ||
            (e = salloc(s, &d.py, TH)) != cudaSuccess || (e = salloc(s, &d.acc, 2 * (size_t)T)) != cudaSuccess ||
            (e = salloc(s, &d.swaps, 2 * (size_t)T)) != cudaSuccess || (e = salloc(s, &d.step, 1)) != cudaSuccess ||
            (e = salloc(s, &d.err, 1)) != cudaSuccess || (e = salloc(s, &d.rec, 1)) != cudaSuccess) {
            st = scuda(s, e, "device allocation (sampler state)");
            break;
        }
        d.like_err = s->like ? li.err_flag : nullptr;
        if ((e = cudaMallocHost(&s->h_rec, sizeof(RecCtl))) != cudaSuccess ||
            (e = cudaMallocHost(&s->h_err, sizeof(int))) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming)) != cudaSuccess) {
            st = scuda(s, e, "host staging");
            break;
        }
        std::memset(s->h_rec, 0, sizeof(RecCtl));
        if ((e = cudaMemsetAsync(d.rec, 0, sizeof(RecCtl), s->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(d.err, 0, sizeof(int), s->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(d.step, 0, sizeof(unsigned), s->stream)) != cudaSuccess) {
            st = scuda(s, e, "cudaMemsetAsync");
            break;
        }
        std::vector<double> b(T);
        for (int t = 0; t < T; t++) b[t] = 1.0 / std::pow(cfg->ladder_ratio, (double)t);
        if (cfg->t_max_inf && T > 1) b[T - 1] = 0.0;
        st = lisa_sampler_set_ladder(s, b.data());
    } while (0);
    if (st != LISA_OK) {
        lisa::set_thread_error(s->err);
        lisa_sampler_destroy(s);
        return st;
    }
    *out = s;
    return LISA_OK;
}

lisa_status lisa_sampler_set_ladder(lisa_sampler_t *s, const double *betas) {
    if (!s) return LISA_ERR_ARG;
    if (!betas) return sfail(s, LISA_ERR_ARG, "NULL ladder");
    const int T = s->dev.T;
    for (int t = 0; t < T; t++) {
        if (!(betas[t] >= 0.0 && betas[t] <= 1.0)) return sfail(s, LISA_ERR_ARG, "betas must be in [0, 1]");
        if (t > 0 && !(betas[t] <= betas[t - 1]))
            return sfail(s, LISA_ERR_ARG, "betas must not increase with the temperature index");
    }
    if (T > 1 && s->dev.adaptive && T >= 3 && !(betas[T - 2] > 0.0))
        return sfail(s, LISA_ERR_ARG, "only the hottest beta may be 0");
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    SCK(cudaMemcpyAsync(s->dev.betas, betas, sizeof(double) * T, cudaMemcpyHostToDevice, s->stream),
        "ladder upload");
    return wait_done(s, s->timeout_s);
}

lisa_status lisa_sampler_set_state(lisa_sampler_t *s, const double *x, uint32_t step) {
    if (!s) return LISA_ERR_ARG;
    if (!x) return sfail(s, LISA_ERR_ARG, "NULL state");
    Dev &d = s->dev;
    const size_t TW = (size_t)d.T * d.W;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    SCK(cudaMemcpyAsync(d.x, x, sizeof(double) * TW * D, cudaMemcpyHostToDevice, s->stream),
        "state upload");
    *s->h_err = (int)step;
    SCK(cudaMemcpyAsync(d.step, s->h_err, sizeof(unsigned), cudaMemcpyHostToDevice, s->stream),
        "step upload");
    SCK(cudaMemsetAsync(d.acc, 0, sizeof(unsigned long long) * 2 * d.T, s->stream), "cudaMemsetAsync");
    SCK(cudaMemsetAsync(d.swaps, 0, sizeof(unsigned long long) * 2 * d.T, s->stream), "cudaMemsetAsync");
    SCK(cudaMemsetAsync(d.err, 0, sizeof(int), s->stream), "cudaMemsetAsync");
    if (s->flow_on)
        SCK(cudaMemsetAsync(s->fst.facc, 0, sizeof(unsigned long long) * 3, s->stream), "cudaMemsetAsync");
    const int n = d.T * d.H;
    for (int c = 0; c < 2; c++) {
        init_kernel<<<blocks_for(n), kThreads, 0, s->stream>>>(d, c);
        SCK(cudaGetLastError(), "init kernel launch");
        if (d.target == LISA_TARGET_LIKELIHOOD) {
            lisa_status st = lisa::like_enqueue(s->like, d.pth, n, d.lnl + (size_t)c * n, s->stream, nullptr);
            if (st != LISA_OK) return sfail(s, st, std::string("likelihood: ") + lisa_like_last_error(s->like));
            // the likelihood's own flag of this call
            SCK(cudaMemcpyAsync(s->h_err, s->li.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
                "flag download");
            lisa_status w = wait_done(s, s->timeout_s);
            if (w != LISA_OK) return w;
            if (*s->h_err)
                return sfail(s, LISA_ERR_TIMEOUT, "a likelihood wait gave up while evaluating the state");
        }
    }
    lisa_status w = wait_done(s, s->timeout_s);
    if (w != LISA_OK) return w;
    s->have_state = true;
    s->steps_run = 0;
    s->since_train = 0;
    return LISA_OK;
}

lisa_status lisa_sampler_run(lisa_sampler_t *s, int n_steps, double *d_chain, double *d_lnl) {
    if (!s) return LISA_ERR_ARG;
    if (!s->have_state) return sfail(s, LISA_ERR_STATE, "set_state must be called first");
    if (n_steps < 1) return sfail(s, LISA_ERR_ARG, "n_steps must be >= 1");
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    s->h_rec->chain = d_chain;
    s->h_rec->lnl = d_lnl;
    s->h_rec->i = 0;
    SCK(cudaMemcpyAsync(s->dev.rec, s->h_rec, sizeof(RecCtl), cudaMemcpyHostToDevice, s->stream),
        "record upload");
    if (s->cfg.use_graphs) {
        // likelihood buffers can change with set_data or a new tile shape: capture afresh
        lisa_status st = capture(s);
        if (st != LISA_OK) return st;
    }
    const bool may_train = s->flow_on && s->fs.train_every > 0;
    for (int done = 0; done < n_steps;) {
        int k = n_steps - done;
        const bool frozen = s->fs.freeze_after > 0 && s->steps_run >= s->fs.freeze_after;
        if (may_train && !frozen) {
            const int64_t to_train = s->fs.train_every - s->since_train;
            if (to_train > 0 && to_train < k) k = (int)to_train;
        }
        lisa_status st = launch_steps(s, k, s->flow_active);
        if (st != LISA_OK) return st;
        done += k;
        s->steps_run += k;
        s->since_train += k;
        if (may_train && !frozen && s->since_train >= s->fs.train_every) {
            // the ring holds the coldest walkers of the last train_every steps
            st = lisa_flowint::flow_train_async(s->flow, s->dev.ring,
                                                (int64_t)s->fs.train_every * s->dev.W,
                                                s->fs.train_iters, s->fs.batch, s->fs.lr,
                                                s->fs.seed, (uint32_t)s->trainings, s->stream);
            if (st != LISA_OK) return sfail(s, st, std::string("flow training: ") + lisa_flow_last_error(s->flow));
            s->trainings++;
            s->since_train = 0;
            s->flow_active = true;
        }
    }
    SCK(cudaMemcpyAsync(s->h_err, s->dev.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
        "flag download");
    lisa_status w = wait_done(s, s->timeout_s * n_steps);
    if (w != LISA_OK) return w;
    if (*s->h_err)
        return sfail(s, LISA_ERR_TIMEOUT,
                     "a likelihood wait gave up during the run; the state stopped changing there");
    return LISA_OK;
}

lisa_status lisa_sampler_get_state(lisa_sampler_t *s, double *x, double *lnl, double *betas,
                                   uint32_t *step) {
    if (!s) return LISA_ERR_ARG;
    const Dev &d = s->dev;
    const size_t TW = (size_t)d.T * d.W;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    if (x) SCK(cudaMemcpyAsync(x, d.x, sizeof(double) * TW * D, cudaMemcpyDeviceToHost, s->stream), "download");
    if (lnl) SCK(cudaMemcpyAsync(lnl, d.lnl, sizeof(double) * TW, cudaMemcpyDeviceToHost, s->stream), "download");
    if (betas) SCK(cudaMemcpyAsync(betas, d.betas, sizeof(double) * d.T, cudaMemcpyDeviceToHost, s->stream), "download");
    SCK(cudaMemcpyAsync(s->h_err, d.step, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream), "download");
    lisa_status w = wait_done(s, s->timeout_s);
    if (w != LISA_OK) return w;
    if (step) *step = (uint32_t)*s->h_err;
    return LISA_OK;
}

lisa_status lisa_sampler_get_counts(lisa_sampler_t *s, int64_t *acc, int64_t *swaps) {
    if (!s) return LISA_ERR_ARG;
    const Dev &d = s->dev;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    if (acc) SCK(cudaMemcpyAsync(acc, d.acc, sizeof(int64_t) * 2 * d.T, cudaMemcpyDeviceToHost, s->stream), "download");
    if (swaps) SCK(cudaMemcpyAsync(swaps, d.swaps, sizeof(int64_t) * 2 * d.T, cudaMemcpyDeviceToHost, s->stream), "download");
    return wait_done(s, s->timeout_s);
}

int lisa_sampler_step_launches(const lisa_sampler_t *s) { return s ? s->launches : 0; }

void lisa_flow_default_schedule(lisa_flow_schedule *fs) {
    if (!fs) return;
    std::memset(fs, 0, sizeof(*fs));
    fs->train_every = 500;
    fs->train_iters = 400;
    fs->batch = 1024;
    fs->lr = 1e-3;
    fs->freeze_after = 0;
    fs->seed = 1;
    fs->flow_only = 0;
}

lisa_status lisa_sampler_enable_flow(lisa_sampler_t *s, const lisa_flow_schedule *fs) {
    if (!s) return LISA_ERR_ARG;
    if (!fs) return sfail(s, LISA_ERR_ARG, "NULL schedule");
    if (fs->train_every < 0 || (fs->train_every > 0 && (fs->train_iters < 1 || fs->batch < 64 ||
                                                        fs->batch % 64 || !(fs->lr > 0.0))))
        return sfail(s, LISA_ERR_ARG, "train_every >= 0; when training: iters >= 1, batch a multiple of 64, lr > 0");
    if (s->flow_on) return sfail(s, LISA_ERR_STATE, "the flow is already enabled");
    Dev &d = s->dev;
    if (s->like && d.W > s->li.max_batch)
        return sfail(s, LISA_ERR_ARG, "the likelihood's max_batch must be >= n_walkers for flow proposals");
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    lisa_status st = lisa_flow_create(fs->seed, &s->flow);
    if (st != LISA_OK) return sfail(s, st, std::string("flow: ") + lisa_flow_last_error(nullptr));
    const size_t W = d.W;
    lisa_flowint::FStep &a = s->fst;
    cudaError_t e;
    if ((e = salloc(s, &a.fy, W * D)) != cudaSuccess || (e = salloc(s, &a.fpth, W * D)) != cudaSuccess ||
        (e = salloc(s, &a.fly, W)) != cudaSuccess || (e = salloc(s, &a.fq, W)) != cudaSuccess ||
        (e = salloc(s, &a.fpy, W)) != cudaSuccess || (e = salloc(s, &a.facc, 3)) != cudaSuccess)
        return scuda(s, e, "device allocation (flow step)");
    if (fs->train_every > 0) {
        if ((e = salloc(s, &d.ring, (size_t)fs->train_every * W * D)) != cudaSuccess)
            return scuda(s, e, "device allocation (training ring)");
        d.ring_rows = fs->train_every;
    }
    SCK(cudaMemsetAsync(a.facc, 0, sizeof(unsigned long long) * 3, s->stream), "cudaMemsetAsync");
    a.W = d.W;
    a.k0 = d.k0;
    a.k1 = d.k1;
    a.step = d.step;
    a.x = d.x;
    a.lnl = d.lnl;
    a.lnp = d.lnp;
    a.betas = d.betas;
    for (int q = 0; q < D; q++) {
        a.lo[q] = d.lo[q];
        a.hi[q] = d.hi[q];
        a.mean[q] = d.mean[q];
        a.sig[q] = d.sig[q];
    }
    a.lisa_frame = d.lisa_frame;
    a.target = d.target;
    a.t0 = d.t0;
    a.err = d.err;
    a.like_err = d.like_err;
    s->fs = *fs;
    s->flow_on = true;
    s->flow_active = fs->train_every == 0;  // no training: the caller's weights propose at once
    drop_graph(s);
    return wait_done(s, s->timeout_s);
}

lisa_flow_t *lisa_sampler_get_flow(lisa_sampler_t *s) { return s ? s->flow : nullptr; }

lisa_status lisa_sampler_set_flow_likelihood(lisa_sampler_t *s, lisa_like_t *like2) {
    if (!s) return LISA_ERR_ARG;
    if (!s->flow_on) return sfail(s, LISA_ERR_STATE, "enable the flow first");
    if (s->dev.target != LISA_TARGET_LIKELIHOOD)
        return sfail(s, LISA_ERR_STATE, "the Gaussian target has no likelihood handle");
    if (like2) {
        const lisa::LikeInfo li2 = lisa::like_info(like2);
        if (!li2.have_data) return sfail(s, LISA_ERR_STATE, "the flow's likelihood has no data");
        if (li2.device != s->device) return sfail(s, LISA_ERR_ARG, "the flow's likelihood is on another device");
        if (li2.max_batch < s->dev.W) return sfail(s, LISA_ERR_ARG, "the flow's likelihood needs max_batch >= n_walkers");
        if (li2.t0 != s->li.t0) return sfail(s, LISA_ERR_ARG, "the flow's likelihood has another t0");
        s->fst.like_err = s->fst.margin > 0.0 ? s->li.err_flag : li2.err_flag;
        s->fst.like_err2 = s->fst.margin > 0.0 ? li2.err_flag : nullptr;
    } else {
        s->fst.like_err = s->li.err_flag;
        s->fst.like_err2 = nullptr;
        s->fst.margin = 0.0;
    }
    s->flow_like = like2;
    drop_graph(s);
    return LISA_OK;
}

lisa_status lisa_sampler_set_flow_screen(lisa_sampler_t *s, double margin) {
    if (!s) return LISA_ERR_ARG;
    if (!s->flow_on || !s->flow_like)
        return sfail(s, LISA_ERR_STATE, "set the flow's second likelihood first");
    if (!(margin >= 0.0) || !std::isfinite(margin)) return sfail(s, LISA_ERR_ARG, "margin must be finite and >= 0");
    lisa_flowint::FStep &a = s->fst;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    if (margin > 0.0 && !a.fpth2) {
        const size_t W = s->dev.W;
        cudaError_t e;
        if ((e = salloc(s, &a.fpth2, W * D)) != cudaSuccess || (e = salloc(s, &a.fly2, W)) != cudaSuccess ||
            (e = salloc(s, &a.fsent, W)) != cudaSuccess)
            return scuda(s, e, "device allocation (flow screen)");
    }
    const lisa::LikeInfo li2 = lisa::like_info(s->flow_like);
    a.margin = margin;
    a.like_err = margin > 0.0 ? s->li.err_flag : li2.err_flag;
    a.like_err2 = margin > 0.0 ? li2.err_flag : nullptr;
    drop_graph(s);
    return LISA_OK;
}

lisa_status lisa_sampler_flow_screen_count(lisa_sampler_t *s, int64_t *sent) {
    if (!s || !sent) return LISA_ERR_ARG;
    if (!s->flow_on) return sfail(s, LISA_ERR_STATE, "the flow is not enabled");
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    SCK(cudaMemcpyAsync(sent, s->fst.facc + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream), "download");
    return wait_done(s, s->timeout_s);
}

lisa_status lisa_sampler_flow_stats(lisa_sampler_t *s, int64_t *acc, int *trainings, double *last_loss) {
    if (!s) return LISA_ERR_ARG;
    if (!s->flow_on) return sfail(s, LISA_ERR_STATE, "the flow is not enabled");
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    if (acc) SCK(cudaMemcpyAsync(acc, s->fst.facc, sizeof(int64_t) * 2, cudaMemcpyDeviceToHost, s->stream), "download");
    if (last_loss) {
        lisa_status st = lisa_flowint::flow_last_loss(s->flow, last_loss, s->stream);
        if (st != LISA_OK) return sfail(s, st, lisa_flow_last_error(s->flow));
    }
    if (trainings) *trainings = s->trainings;
    return wait_done(s, s->timeout_s);
}

void lisa_sampler_destroy(lisa_sampler_t *s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    if (s->flow) lisa_flow_destroy(s->flow);
    for (void *p : s->bufs) cudaFree(p);
    if (s->h_rec) cudaFreeHost(s->h_rec);
    if (s->h_err) cudaFreeHost(s->h_err);
    if (s->done) cudaEventDestroy(s->done);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char *lisa_sampler_last_error(const lisa_sampler_t *s) {
    return s ? s->err.c_str() : lisa::thread_error();
}

lisa_status lisa_sampler_to_physical(const double *d_x, int n, int lisa_frame, double t0,
                                     double *d_th, void *stream) {
    lisa::set_thread_error("");
    if (!d_x || !d_th || n < 0 || !std::isfinite(t0)) {
        lisa::set_thread_error("NULL pointer, negative n or non-finite t0");
        return LISA_ERR_ARG;
    }
    if (n == 0) return LISA_OK;
    to_physical_kernel<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(d_x, n, lisa_frame, t0, d_th);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        lisa::set_thread_error(std::string("conversion kernel launch: ") + cudaGetErrorString(e));
        return LISA_ERR_CUDA;
    }
    return LISA_OK;
}

lisa_status lisa_sampler_from_physical(const double *th, int n, int lisa_frame, double t0,
                                       double *x) {
    lisa::set_thread_error("");
    if (!th || !x || n < 0 || !std::isfinite(t0)) {
        lisa::set_thread_error("NULL pointer, negative n or non-finite t0");
        return LISA_ERR_ARG;
    }
    for (int i = 0; i < n; i++) {
        const double *p = th + (size_t)i * D;
        double *o = x + (size_t)i * D;
        if (!(p[0] > 0.0) || !(p[4] > 0.0)) {
            lisa::set_thread_error("M_T and D_L must be positive");
            return LISA_ERR_ARG;
        }
        o[0] = std::log(p[0]);
        o[1] = p[1];
        o[2] = p[2];
        o[3] = p[3];
        o[4] = std::log(p[4]);
        o[5] = p[5];
        o[6] = std::cos(p[6]);
        double lam = p[7], sb = std::sin(p[8]), psi = p[9], tref = p[10];
        if (lisa_frame) {
            const double cl = std::cos(p[7]), sl = std::sin(p[7]), cb = std::cos(p[8]);
            const double cp = std::cos(p[9]), sp = std::sin(p[9]);
            const double nv[3] = {cb * cl, cb * sl, sb};
            const double pv[3] = {cp * sl - sp * sb * cl, -cp * cl - sp * sb * sl, sp * cb};
            const double t = p[10] + t0;
            const double al = 2.0 * kPi * t / kYearS;
            const double tL = t - kAuS * (nv[0] * std::cos(al) + nv[1] * std::sin(al));
            const double a2 = 2.0 * kPi * tL / kYearS, ca = std::cos(a2), sa = std::sin(a2);
            const double h = 0.8660254037844386467637231707529362;
            const double Q[3][3] = {{0.5 * ca * ca + sa * sa, -0.5 * ca * sa, -h * ca},
                                    {-0.5 * ca * sa, 0.5 * sa * sa + ca * ca, -h * sa},
                                    {h * ca, h * sa, 0.5}};
            double nL[3], pL[3];
            for (int r = 0; r < 3; r++) {  // Q^T: constellation frame components
                nL[r] = Q[0][r] * nv[0] + Q[1][r] * nv[1] + Q[2][r] * nv[2];
                pL[r] = Q[0][r] * pv[0] + Q[1][r] * pv[1] + Q[2][r] * pv[2];
            }
            lam = std::atan2(nL[1], nL[0]);
            if (lam < 0.0) lam += 2.0 * kPi;
            sb = std::fmin(1.0, std::fmax(-1.0, nL[2]));
            const double rho2 = nL[0] * nL[0] + nL[1] * nL[1];
            psi = std::atan2(-sb * (pL[0] * nL[0] + pL[1] * nL[1]) + pL[2] * rho2,
                             pL[0] * nL[1] - pL[1] * nL[0]);
            psi = std::fmod(psi, kPi);
            if (psi < 0.0) psi += kPi;
            tref = tL - t0;
        }
        if (!(tref > 0.0)) {
            lisa::set_thread_error("the reference time must be positive in the sampling frame");
            return LISA_ERR_ARG;
        }
        o[7] = lam;
        o[8] = sb;
        o[9] = psi;
        o[10] = std::log(tref);
    }
    return LISA_OK;
}

lisa_status lisa_sampler_sky_mode_init(const double *xc, const double *scale, const double *lower,
                                       const double *upper, int T, int W, uint64_t seed,
                                       double *x_out) {
    lisa::set_thread_error("");
    if (!xc || !scale || !lower || !upper || !x_out || T < 1 || W < 8 || W % 8) {
        lisa::set_thread_error("NULL pointer, T < 1, or W not a positive multiple of 8");
        return LISA_ERR_ARG;
    }
    if (!valid_box(lower, upper)) {
        lisa::set_thread_error("prior bounds must be finite with lower < upper");
        return LISA_ERR_ARG;
    }
    // a key of its own, so that the jitter is independent of the sampler's draws
    const uint32_t k0 = (uint32_t)seed ^ 0x5BD1E995u, k1 = (uint32_t)(seed >> 32) ^ 0x1B873593u;
    for (int t = 0; t < T; t++)
        for (int w = 0; w < W; w++) {
            double g[12];
            for (int blk = 0; blk < 3; blk++) {
                // Box-Muller on two Philox pairs
                const U4 r = philox((uint32_t)t, (uint32_t)w, 0x51u, (uint32_t)blk, k0, k1);
                for (int pr = 0; pr < 2; pr++) {
                    const double u1 = unit(r.v[2 * pr]), u2 = unit(r.v[2 * pr + 1]);
                    const double rad = std::sqrt(-2.0 * std::log(u1));
                    g[4 * blk + 2 * pr] = rad * std::cos(2.0 * kPi * u2);
                    g[4 * blk + 2 * pr + 1] = rad * std::sin(2.0 * kPi * u2);
                }
            }
            double *x = x_out + ((size_t)t * W + w) * D;
            const int mode = w % 8;
            for (int q = 0; q < D; q++) {
                double v = xc[q] + scale[q] * g[q];
                if (q == 7) v += (mode % 4) * 0.5 * kPi;
                if (q == 8 && mode >= 4) v = -xc[q] + scale[q] * g[q];
                const double lo = lower[q], hi = upper[q];
                if (q == 7) {  // longitude: periodic
                    const double span = hi - lo;
                    v = lo + std::fmod(v - lo, span);
                    if (v < lo) v += span;
                    if (v >= hi) v = lo;
                } else {
                    for (int it = 0; it < 64 && (v < lo || v > hi); it++) v = v < lo ? 2.0 * lo - v : 2.0 * hi - v;
                    v = std::fmin(hi, std::fmax(lo, v));
                }
                x[q] = v;
            }
        }
    return LISA_OK;
}

lisa_status lisa_autocorr_time(const double *d_chain, int n, int W, int stride, int offset,
                               double *tau, double *rho, void *stream) {
    lisa::set_thread_error("");
    if (!d_chain || !tau || n < 2 || W < 1 || stride < 1 || offset < 0 || offset >= stride) {
        lisa::set_thread_error("need a chain, n >= 2, W >= 1 and 0 <= offset < stride");
        return LISA_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int kLags = 256;
    double *mu = nullptr, *c0 = nullptr, *rb = nullptr;
    std::vector<double> h_c0(W), h_rho((size_t)kLags * W);
    std::string msg;
    cudaError_t e = cudaMalloc(&mu, sizeof(double) * W);
    if (e == cudaSuccess) e = cudaMalloc(&c0, sizeof(double) * W);
    if (e == cudaSuccess) e = cudaMalloc(&rb, sizeof(double) * kLags * W);
    if (e == cudaSuccess) {
        acf_stats_kernel<<<blocks_for(W), kThreads, 0, st>>>(d_chain, n, W, stride, offset, mu, c0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_c0.data(), c0, sizeof(double) * W, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int used = 0;
    for (int w = 0; w < W && e == cudaSuccess; w++) used += h_c0[w] > 0.0;
    double t_est = NAN;
    if (rho) std::memset(rho, 0, sizeof(double) * n);
    if (e == cudaSuccess && used > 0) {
        if (rho) rho[0] = 1.0;
        t_est = 1.0;
        bool done = false;
        for (int lag0 = 1; lag0 < n && !done && e == cudaSuccess; lag0 += kLags) {
            const int nl = std::min(kLags, n - lag0);
            acf_lag_kernel<<<dim3(blocks_for(W), nl), kThreads, 0, st>>>(d_chain, n, W, stride, offset,
                                                                         lag0, mu, c0, rb);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_rho.data(), rb, sizeof(double) * nl * W, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            for (int l = 0; l < nl && e == cudaSuccess; l++) {
                double r = 0.0;
                for (int w = 0; w < W; w++) r += h_rho[(size_t)l * W + w];
                r /= used;
                const int M = lag0 + l;
                if (rho) rho[M] = r;
                t_est += 2.0 * r;
                if ((double)M >= 5.0 * t_est) {
                    done = true;
                    break;
                }
            }
        }
    }
    if (mu) cudaFree(mu);
    if (c0) cudaFree(c0);
    if (rb) cudaFree(rb);
    if (e != cudaSuccess) {
        lisa::set_thread_error(std::string("autocorrelation: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LISA_ERR_OOM : LISA_ERR_CUDA;
    }
    *tau = t_est;
    return LISA_OK;
}

}  // extern "C"
