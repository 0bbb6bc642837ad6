// lisa_like.cu -- host side of the C ABI in include/lisa_like.h: handle, device
// buffers, data upload, and the per-call stage sequence of the batched LISA
// likelihood (Katz et al. 2020, Sec. II.A): knots -> splines -> fused dense ln L.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <map>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/lisa_like.h"
#include "internal.h"
#include "kernels.h"
#include "model.cuh"
#include "split.h"

using namespace lisa;

namespace {
thread_local std::string g_create_error;
}

namespace lisa {
// failure text of handle-free entry points, read back by lisa_like_last_error(NULL)
void set_thread_error(const std::string &msg) { g_create_error = msg; }
const char *thread_error() { return g_create_error.c_str(); }
}  // namespace lisa

struct lisa_like {
    int L = 0, K = 0, precision = 0, device = 0, max_batch = 0;
    int ml[6] = {0}, mm[6] = {0};
    double t0 = 0.0, timeout_s = 60.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t done = nullptr;
    int n_sm = 0;
    DenseTune tune = {128, 8, 0, 8};
    int min_tile = 512;  // smallest tile the dense kernels use (sizes the partial sums)

    // data
    bool have_data = false;
    double f0 = 0.0, df = 0.0, dd = 0.0;
    int N = 0;
    double *bins = nullptr;   // [N][9] FP64 staged data
    float *bins32 = nullptr;  // [N][kBinFloats] FP32 whitened data (split precision)
    SegRec *segs = nullptr;   // [max_batch][L][K-1] split-precision segment records
    unsigned long long *phases = nullptr;  // [max_batch][L][K-1][8] FP64-path phase records

    // per-call buffers
    double *params = nullptr, *tc = nullptr, *xpk = nullptr, *fedge = nullptr, *fk = nullptr;
    double *vals = nullptr;
    double *mscr = nullptr, *coef = nullptr, *part = nullptr, *out = nullptr;
    int *valid = nullptr, *band = nullptr, *kb = nullptr, *wrange = nullptr;
    int *order = nullptr, *slot_of = nullptr, *grange = nullptr;
    int *item_start = nullptr, *counter = nullptr, *err_flag = nullptr;
    int64_t part_items = 0;
    double *h_params = nullptr, *h_out = nullptr;  // pinned staging
    int *h_err = nullptr;
    int last_launches = 0;
    std::vector<void *> deferred;  // device buffers that in-flight work may still touch
    // CUDA graphs: one cached executable for the last (B, pointers) key
    bool use_graphs = false;
    cudaGraphExec_t gexec = nullptr;
    int g_B = 0;
    const void *g_key[4] = {nullptr, nullptr, nullptr, nullptr};
    int g_launches = 0;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // tile shapes chosen by lisa_like_autotune, per (n_bins, K, precision)
    std::map<std::tuple<int, int, int>, DenseTune> tuned;
    bool profiling = false;
    unsigned wait_test_polls = 0;      // lisa_like_test_device_wait
    lisa::RbState *rb = nullptr;       // relative binning (lisa_like_set_fiducial)
    std::vector<cudaEvent_t> prof_ev;  // kProfEvents events per profiled call
    int prof_calls = 0;
    std::string err;
};

namespace {

constexpr int kStages = 6;  // knots, splines, segment prep, plan, dense, finish
constexpr int kProfEvents = kStages + 1;

lisa_status fail(lisa_like_t *h, lisa_status st, const std::string &msg) {
    if (h) h->err = msg;
    return st;
}

lisa_status cuda_fail(lisa_like_t *h, cudaError_t e, const char *what) {
    const lisa_status st = (e == cudaErrorMemoryAllocation) ? LISA_ERR_OOM : LISA_ERR_CUDA;
    return fail(h, st, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LCK(call, what)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    if (getenv("LISA_LIKE_INJECT_OOM")) return cudaErrorMemoryAllocation;
    return cudaMalloc((void **)p, n * sizeof(T) + 16);
}

void free_batch(lisa_like_t *h) {
    void *ptrs[] = {h->params, h->tc,    h->xpk,    h->fedge,  h->fk,  h->vals,  h->mscr,
                    h->coef,   h->out,   h->valid,  h->band,   h->kb,         h->wrange,
                    h->order,  h->slot_of, h->grange, h->item_start, h->counter, h->err_flag};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    h->order = h->slot_of = h->grange = h->err_flag = nullptr;
    h->xpk = nullptr;
    if (h->segs) cudaFree(h->segs);
    if (h->phases) cudaFree(h->phases);
    h->segs = nullptr;
    h->phases = nullptr;
    h->params = h->tc = h->fedge = h->fk = h->vals = h->mscr = h->coef = h->out = nullptr;
    h->valid = h->band = h->kb = h->wrange = h->item_start = h->counter = nullptr;
    if (h->h_params) cudaFreeHost(h->h_params);
    if (h->h_out) cudaFreeHost(h->h_out);
    if (h->h_err) cudaFreeHost(h->h_err);
    h->h_params = h->h_out = nullptr;
    h->h_err = nullptr;
}

lisa_status alloc_batch(lisa_like_t *h) {
    const size_t B = h->max_batch, L = h->L, K = h->K;
    LCK(dalloc(&h->params, B * kNPar), "device allocation (params)");
    LCK(dalloc(&h->tc, B), "device allocation (tc)");
    LCK(dalloc(&h->xpk, B), "device allocation (peaks)");
    LCK(dalloc(&h->valid, B), "device allocation (valid)");
    LCK(dalloc(&h->band, B * L * 3), "device allocation (band)");
    LCK(dalloc(&h->fedge, B * L * 2), "device allocation (fedge)");
    LCK(dalloc(&h->fk, B * L * K), "device allocation (knots)");
    LCK(dalloc(&h->kb, B * L * K), "device allocation (knot bins)");
    LCK(dalloc(&h->vals, B * L * kNSeries * K), "device allocation (knot values)");
    LCK(dalloc(&h->mscr, B * L * kScratchRows * K), "device allocation (spline scratch)");
    LCK(dalloc(&h->coef, B * L * (K - 1) * 32), "device allocation (spline coefficients)");
    LCK(dalloc(&h->wrange, 2 * B), "device allocation (ranges)");
    LCK(dalloc(&h->order, B), "device allocation (order)");
    LCK(dalloc(&h->slot_of, B), "device allocation (slots)");
    LCK(dalloc(&h->grange, 2 * B), "device allocation (group ranges)");
    LCK(dalloc(&h->item_start, B + 1), "device allocation (items)");
    LCK(dalloc(&h->counter, 1), "device allocation (counter)");
    LCK(dalloc(&h->err_flag, 1), "device allocation (error flag)");
    LCK(cudaMemset(h->err_flag, 0, sizeof(int)), "cudaMemset");
    LCK(dalloc(&h->out, 3 * B), "device allocation (outputs)");
    if (h->precision == LISA_PREC_SPLIT)
        LCK(dalloc(&h->segs, B * L * (K - 1)), "device allocation (split segments)");
    else
        LCK(dalloc(&h->phases, B * L * (K - 1) * kPhaseWords), "device allocation (phase anchors)");
    LCK(cudaMallocHost(&h->h_params, sizeof(double) * B * kNPar), "pinned allocation");
    LCK(cudaMallocHost(&h->h_out, sizeof(double) * 3 * B), "pinned allocation");
    LCK(cudaMallocHost(&h->h_err, sizeof(int)), "pinned allocation");
    return LISA_OK;
}

StageBufs bufs_of(const lisa_like_t *h, const double *params) {
    StageBufs b;
    b.params = params;
    b.valid = h->valid;
    b.tc = h->tc;
    b.xpk = h->xpk;
    b.band = h->band;
    b.fedge = h->fedge;
    b.fk = h->fk;
    b.kb = h->kb;
    b.vals = h->vals;
    b.mscratch = h->mscr;
    b.coef = h->coef;
    b.wrange = h->wrange;
    b.order = h->order;
    b.slot_of = h->slot_of;
    b.grange = h->grange;
    b.item_start = h->item_start;
    b.counter = h->counter;
    b.err = h->err_flag;
    b.part = h->part;
    b.wait_test_polls = h->wait_test_polls;
    return b;
}

StageDims dims_of(const lisa_like_t *h, int B) {
    StageDims d;
    d.B = B;
    d.L = h->L;
    d.K = h->K;
    d.N = h->N;
    d.f0 = h->f0;
    d.df = h->df;
    d.t0 = h->t0;
    for (int i = 0; i < 6; i++) {
        d.ml[i] = h->ml[i];
        d.mm[i] = h->mm[i];
    }
    return d;
}

lisa_status wait_for(lisa_like_t *h, cudaStream_t s) {
    LCK(cudaEventRecord(h->done, s), "cudaEventRecord");
    const auto t0 = std::chrono::steady_clock::now();
    int polls = 0;
    for (;;) {
        const cudaError_t e = cudaEventQuery(h->done);
        if (e == cudaSuccess) return LISA_OK;
        if (e != cudaErrorNotReady) return cuda_fail(h, e, "device work failed");
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > h->timeout_s)
            return fail(h, LISA_ERR_TIMEOUT, "device did not finish within the timeout");
        if (++polls > 2000) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// knots -> splines (steps 1-3 of the header)
lisa_status run_front(lisa_like_t *h, const double *dparams, int B, cudaStream_t s, int *nl) {
    const StageDims d = dims_of(h, B);
    const StageBufs b = bufs_of(h, dparams);
    LCK(launch_knots(d, b, s), "knot kernel launch");
    LCK(launch_spline(d, b, s), "spline kernel launch");
    *nl += 2;
    return LISA_OK;
}

// the events of profiled call `c` (created on first use)
lisa_status prof_events(lisa_like_t *h, int c, cudaEvent_t **ev) {
    while ((int)h->prof_ev.size() < kProfEvents * (c + 1)) {
        cudaEvent_t e;
        LCK(cudaEventCreate(&e), "cudaEventCreate");
        h->prof_ev.push_back(e);
    }
    *ev = h->prof_ev.data() + kProfEvents * c;
    return LISA_OK;
}

// persistent grid of the dense kernel for a tile shape: every SM filled with resident blocks
bool make_tune(const lisa_like_t *h, int per_thread, int group, DenseTune *t) {
    const int occ = h->precision == LISA_PREC_SPLIT ? dense_split_occupancy(per_thread, group)
                                                     : dense_f64_occupancy(per_thread, group);
    if (occ <= 0) return false;
    *t = {128, per_thread, h->n_sm * occ, group};
    return true;
}

lisa_status enqueue(lisa_like_t *h, const double *dparams, int B, double *lnL, double *dh,
                    double *hh, cudaStream_t s, bool profile, unsigned mode_mask = 0);

void drop_graph(lisa_like_t *h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_B = 0;
}

lisa_status run_all(lisa_like_t *h, const double *dparams, int B, double *lnL, double *dh,
                    double *hh, cudaStream_t s) {
    if (!h->use_graphs) return enqueue(h, dparams, B, lnL, dh, hh, s, h->profiling);
    const void *key[4] = {dparams, lnL, dh, hh};
    const bool hit = h->gexec && h->g_B == B && std::equal(key, key + 4, h->g_key);
    if (!hit) {
        drop_graph(h);
        cudaGraph_t g = nullptr;
        LCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
        lisa_status st = enqueue(h, dparams, B, lnL, dh, hh, h->stream, false);
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (st != LISA_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->gexec = nullptr;
            return cuda_fail(h, e, "graph instantiation");
        }
        h->g_B = B;
        std::copy(key, key + 4, h->g_key);
        h->g_launches = h->last_launches;
    }
    // the graph runs on the handle's stream, ordered after and before the caller's stream
    if (s != h->stream) {
        LCK(cudaEventRecord(h->ev_in, s), "cudaEventRecord");
        LCK(cudaStreamWaitEvent(h->stream, h->ev_in, 0), "cudaStreamWaitEvent");
    }
    LCK(cudaGraphLaunch(h->gexec, h->stream), "cudaGraphLaunch");
    if (s != h->stream) {
        LCK(cudaEventRecord(h->ev_out, h->stream), "cudaEventRecord");
        LCK(cudaStreamWaitEvent(s, h->ev_out, 0), "cudaStreamWaitEvent");
    }
    h->last_launches = h->g_launches;
    return LISA_OK;
}

// the call's kernels on stream s; a non-zero mode_mask restricts the template to the modes
// whose bits are set (bit i = the handle's mode i)
lisa_status enqueue(lisa_like_t *h, const double *dparams, int B, double *lnL, double *dh,
                    double *hh, cudaStream_t s, bool profile, unsigned mode_mask) {
    cudaEvent_t *ev = nullptr;
    if (profile) {
        if (h->prof_calls >= 4096) return fail(h, LISA_ERR_STATE, "read the profile first");
        lisa_status st = prof_events(h, h->prof_calls, &ev);
        if (st != LISA_OK) return st;
        h->prof_calls++;
    }
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    StageDims d = dims_of(h, B);
    if (mode_mask) {
        int n = 0;
        for (int i = 0; i < h->L; i++)
            if ((mode_mask >> i) & 1u) {
                d.ml[n] = h->ml[i];
                d.mm[n] = h->mm[i];
                n++;
            }
        d.L = n;
    }
    const StageBufs b = bufs_of(h, dparams);
    const int tile = h->tune.threads * h->tune.per_thread;
    const bool split = h->precision == LISA_PREC_SPLIT;
    LCK(mark(0), "cudaEventRecord");
    LCK(split ? launch_knots_split(d, b, s) : launch_knots(d, b, s), "knot kernel launch");
    LCK(mark(1), "cudaEventRecord");
    LCK(split ? launch_spline_split(d, b, s) : launch_spline(d, b, s), "spline kernel launch");
    LCK(mark(2), "cudaEventRecord");
    if (split)
        LCK(launch_segprep(d, b, h->segs, s), "segment kernel launch");
    else
        LCK(launch_phaseprep(d, b, h->phases, s), "segment kernel launch");
    LCK(mark(3), "cudaEventRecord");
    LCK(launch_plan(d, b, tile, h->tune.group, s), "plan kernel launch");
    LCK(mark(4), "cudaEventRecord");
    if (split)
        LCK(launch_dense_split(d, b, h->segs, h->bins32, h->tune, s), "dense kernel launch");
    else
        LCK(launch_dense_f64(d, b, h->phases, h->bins, h->tune, s), "dense kernel launch");
    LCK(mark(5), "cudaEventRecord");
    LCK(launch_finish(d, b, h->tune.group, split ? 1 : 0, h->dd, lnL, dh, hh, s),
        "finish kernel launch");
    LCK(mark(6), "cudaEventRecord");
    h->last_launches = 8;  // band, knots, spline solve + coefficients, segments, plan, dense, finish
    return LISA_OK;
}

}  // namespace

namespace lisa {

LikeInfo like_info(const lisa_like_t *h) {
    LikeInfo i;
    i.stream = h->stream;
    i.device = h->device;
    i.max_batch = h->max_batch;
    i.have_data = h->have_data ? 1 : 0;
    i.t0 = h->t0;
    i.err_flag = h->err_flag;
    i.timeout_s = h->timeout_s;
    return i;
}

LikeCore like_core(lisa_like_t *h) {
    LikeCore c;
    c.stream = h->stream;
    c.device = h->device;
    c.max_batch = h->max_batch;
    c.have_data = h->have_data ? 1 : 0;
    c.N = h->N;
    c.L = h->L;
    c.K = h->K;
    c.t0 = h->t0;
    c.f0 = h->f0;
    c.df = h->df;
    c.dd = h->dd;
    c.timeout_s = h->timeout_s;
    for (int i = 0; i < 6; i++) {
        c.ml[i] = h->ml[i];
        c.mm[i] = h->mm[i];
    }
    c.bins = h->bins;
    c.params = h->params;
    c.h_params = h->h_params;
    c.out = h->out;
    c.h_out = h->h_out;
    c.stage = bufs_of(h, h->params);
    return c;
}

RbState *&like_rb(lisa_like_t *h) { return h->rb; }
lisa_status like_fail(lisa_like_t *h, lisa_status st, const std::string &msg) { return fail(h, st, msg); }
lisa_status like_wait(lisa_like_t *h, cudaStream_t s) { return wait_for(h, s); }

lisa_status like_enqueue(lisa_like_t *h, const double *d_params, int B, double *d_lnL,
                         cudaStream_t s, int *launches) {
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch) return fail(h, LISA_ERR_ARG, "B must be in [1, max_batch]");
    lisa_status st = enqueue(h, d_params, B, d_lnL, nullptr, nullptr, s, false);
    if (launches) *launches = h->last_launches;
    return st;
}

}  // namespace lisa

extern "C" {

void lisa_like_default_config(lisa_like_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    const int md[6][2] = {{2, 2}, {3, 3}, {4, 4}, {2, 1}, {3, 2}, {4, 3}};
    cfg->n_modes = 6;
    std::memcpy(cfg->modes, md, sizeof(md));
    cfg->n_knots = 1024;
    cfg->precision = LISA_PREC_FP64;
    cfg->t0_s = 3.15576e7;
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->max_batch = 1024;
    cfg->timeout_s = 60.0;
}

lisa_status lisa_like_create(const lisa_like_config *cfg, lisa_like_t **out) {
    g_create_error.clear();
    if (!cfg || !out) {
        g_create_error = "NULL config or output pointer";
        return LISA_ERR_ARG;
    }
    *out = nullptr;
    if (cfg->n_modes < 1 || cfg->n_modes > 6) {
        g_create_error = "n_modes must be 1..6";
        return LISA_ERR_ARG;
    }
    int seen = 0;
    for (int i = 0; i < cfg->n_modes; i++) {
        const int id = mode_index(cfg->modes[i][0], cfg->modes[i][1]);
        if (id < 0 || (seen >> id) & 1) {
            g_create_error = "modes must be distinct entries of (2,2),(3,3),(4,4),(2,1),(3,2),(4,3)";
            return LISA_ERR_ARG;
        }
        seen |= 1 << id;
    }
    if (cfg->n_knots < 4 || cfg->n_knots > 4096) {
        g_create_error = "n_knots must be in [4, 4096]";
        return LISA_ERR_ARG;
    }
    if (cfg->precision != LISA_PREC_FP64 && cfg->precision != LISA_PREC_SPLIT) {
        g_create_error = "precision must be LISA_PREC_FP64 or LISA_PREC_SPLIT";
        return LISA_ERR_ARG;
    }
    if (cfg->max_batch < 1 || cfg->max_batch > (1 << 20) || !std::isfinite(cfg->t0_s)) {
        g_create_error = "max_batch must be in [1, 2^20] and t0 finite";
        return LISA_ERR_ARG;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        g_create_error = std::string("no such CUDA device: ") +
                         (e != cudaSuccess ? cudaGetErrorString(e) : "ordinal out of range");
        return e != cudaSuccess ? LISA_ERR_CUDA : LISA_ERR_ARG;
    }
    lisa_like_t *h = new lisa_like();
    h->L = cfg->n_modes;
    for (int i = 0; i < h->L; i++) {
        h->ml[i] = cfg->modes[i][0];
        h->mm[i] = cfg->modes[i][1];
    }
    h->K = cfg->n_knots;
    h->precision = cfg->precision;
    h->t0 = cfg->t0_s;
    h->device = cfg->device;
    h->max_batch = cfg->max_batch;
    h->timeout_s = cfg->timeout_s > 0.0 ? cfg->timeout_s : 60.0;
    lisa_status st = LISA_OK;
    do {
        if ((e = cudaSetDevice(h->device)) != cudaSuccess) {
            st = cuda_fail(h, e, "cudaSetDevice");
            break;
        }
        cudaDeviceProp prop;
        if ((e = cudaGetDeviceProperties(&prop, h->device)) != cudaSuccess) {
            st = cuda_fail(h, e, "cudaGetDeviceProperties");
            break;
        }
        h->n_sm = prop.multiProcessorCount;
        if (cfg->stream) {
            h->stream = (cudaStream_t)cfg->stream;
        } else {
            if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) {
                st = cuda_fail(h, e, "cudaStreamCreate");
                break;
            }
            h->own_stream = true;
        }
        if ((e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming)) != cudaSuccess) {
            st = cuda_fail(h, e, "cudaEventCreate");
            break;
        }
        st = alloc_batch(h);
        if (st != LISA_OK) break;
        if ((e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming)) != cudaSuccess) {
            st = cuda_fail(h, e, "cudaEventCreate");
            break;
        }
        if (!make_tune(h, 8, 8, &h->tune)) {
            st = fail(h, LISA_ERR_CUDA, "dense kernel cannot be made resident on this device");
            break;
        }
    } while (0);
    if (st != LISA_OK) {
        g_create_error = h->err;
        lisa_like_destroy(h);
        return st;
    }
    *out = h;
    return LISA_OK;
}

lisa_status lisa_like_set_data(lisa_like_t *h, double f0, double df, int64_t n_bins,
                               const double *d, const double *psd) {
    if (!h) return LISA_ERR_ARG;
    if (!psd) return fail(h, LISA_ERR_ARG, "psd must not be NULL");
    if (!(f0 > 0.0) || !std::isfinite(f0) || !(df > 0.0) || !std::isfinite(df))
        return fail(h, LISA_ERR_ARG, "grid needs finite f0 > 0 and df > 0");
    if (n_bins < 1 || n_bins >= ((int64_t)1 << 31))
        return fail(h, LISA_ERR_ARG, "n_bins must be in [1, 2^31)");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    const int N = (int)n_bins;
    cudaStream_t s = h->stream;
    double *dd_dev = nullptr, *psd_dev = nullptr, *bins = nullptr, *ddpart = nullptr;
    int *bad = nullptr;
    const int nblk = prep_blocks(N);
    auto cleanup = [&]() {
        if (dd_dev) cudaFree(dd_dev);
        if (psd_dev) cudaFree(psd_dev);
        if (ddpart) cudaFree(ddpart);
        if (bad) cudaFree(bad);
        if (bins) cudaFree(bins);
    };
    cudaError_t e;
    if ((e = dalloc(&psd_dev, (size_t)3 * N)) != cudaSuccess ||
        (d && (e = dalloc(&dd_dev, (size_t)6 * N)) != cudaSuccess) ||
        (e = dalloc(&bins, (size_t)kBinDoubles * N)) != cudaSuccess ||
        (e = dalloc(&ddpart, (size_t)nblk)) != cudaSuccess || (e = dalloc(&bad, 1)) != cudaSuccess) {
        cleanup();
        return cuda_fail(h, e, "device allocation (data)");
    }
    double *hpart = nullptr;
    int *hbad = nullptr;
    if ((e = cudaMallocHost(&hpart, sizeof(double) * nblk)) != cudaSuccess ||
        (e = cudaMallocHost(&hbad, sizeof(int))) != cudaSuccess) {
        if (hpart) cudaFreeHost(hpart);
        cleanup();
        return cuda_fail(h, e, "pinned allocation (data)");
    }
    *hbad = 0;
    lisa_status st = LISA_OK;
    do {
        if ((e = cudaMemcpyAsync(psd_dev, psd, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s)) ||
            (d && (e = cudaMemcpyAsync(dd_dev, d, sizeof(double) * 6 * N, cudaMemcpyHostToDevice, s))) ||
            (e = cudaMemsetAsync(bad, 0, sizeof(int), s)) ||
            (e = launch_prep(dd_dev, psd_dev, N, df, bins, ddpart, bad, s)) ||
            (e = cudaMemcpyAsync(hpart, ddpart, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s))) {
            st = cuda_fail(h, e, "data upload");
            break;
        }
        st = wait_for(h, s);
    } while (0);
    if (st == LISA_OK && *hbad) st = fail(h, LISA_ERR_ARG, "psd must be finite and > 0 and d finite");
    if (st == LISA_ERR_TIMEOUT || st == LISA_ERR_CUDA) {
        // the device may still be using these: release them at destroy, after a sync
        void *keep[] = {dd_dev, psd_dev, ddpart, bad, bins, hpart, hbad};
        for (void *p : keep)
            if (p) h->deferred.push_back(p);
        return st;
    }
    if (st != LISA_OK) {
        cudaFreeHost(hpart);
        cudaFreeHost(hbad);
        cleanup();
        return st;
    }
    double ddv = 0.0;
    for (int i = 0; i < nblk; i++) ddv += hpart[i];
    cudaFreeHost(hpart);
    cudaFreeHost(hbad);
    cudaFree(psd_dev);
    if (dd_dev) cudaFree(dd_dev);
    cudaFree(ddpart);
    cudaFree(bad);
    // partial sums of the dense items, sized for the smallest tile any kernel uses
    const int64_t items = max_items(h->max_batch, N, h->min_tile);
    double *part = nullptr;
    float *bins32 = nullptr;
    if ((e = dalloc(&part, (size_t)items * 2)) != cudaSuccess ||
        (h->precision == LISA_PREC_SPLIT &&
         (e = dalloc(&bins32, (size_t)kBinFloats * N)) != cudaSuccess)) {
        if (part) cudaFree(part);
        cudaFree(bins);
        return cuda_fail(h, e, "device allocation (partial sums / FP32 data)");
    }
    if (bins32) {
        if ((e = launch_prep_split(bins, N, bins32, s)) != cudaSuccess) {
            cudaFree(part);
            cudaFree(bins32);
            cudaFree(bins);
            return cuda_fail(h, e, "FP32 data preparation");
        }
        st = wait_for(h, s);
        if (st != LISA_OK) {
            h->deferred.push_back(part);
            h->deferred.push_back(bins32);
            h->deferred.push_back(bins);
            return st;
        }
    }
    if (h->bins) cudaFree(h->bins);
    if (h->bins32) cudaFree(h->bins32);
    if (h->part) cudaFree(h->part);
    if (h->rb) {  // summary data belong to the previous data
        lisa::rb_free(h->rb);
        h->rb = nullptr;
    }
    h->bins = bins;
    h->bins32 = bins32;
    h->part = part;
    h->part_items = items;
    h->f0 = f0;
    h->df = df;
    h->N = N;
    h->dd = ddv;
    h->have_data = true;
    return LISA_OK;
}

lisa_status lisa_like_loglike_device(lisa_like_t *h, const double *d_params, int B, double *d_lnL,
                                     double *d_dh, double *d_hh, void *stream) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch) return fail(h, LISA_ERR_ARG, "B must be in [1, max_batch]");
    if (!d_params || !d_lnL) return fail(h, LISA_ERR_ARG, "NULL parameter or output pointer");
    cudaStream_t s = (cudaStream_t)stream;
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    return run_all(h, d_params, B, d_lnL, d_dh, d_hh, s);
}

lisa_status lisa_like_loglike(lisa_like_t *h, const double *params, int B, double *lnL, double *dh,
                              double *hh) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch) return fail(h, LISA_ERR_ARG, "B must be in [1, max_batch]");
    if (!params || !lnL) return fail(h, LISA_ERR_ARG, "NULL parameter or output pointer");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = h->stream;
    std::memcpy(h->h_params, params, sizeof(double) * kNPar * B);
    LCK(cudaMemcpyAsync(h->params, h->h_params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s),
        "parameter upload");
    lisa_status st = run_all(h, h->params, B, h->out, h->out + B, h->out + 2 * B, s);
    if (st != LISA_OK) return st;
    LCK(cudaMemcpyAsync(h->h_out, h->out, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s),
        "result download");
    LCK(cudaMemcpyAsync(h->h_err, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s),
        "result download");
    st = wait_for(h, s);
    if (st != LISA_OK) return st;
    if (*h->h_err)
        return fail(h, LISA_ERR_TIMEOUT, "a device wait for staged data gave up (outputs are NaN)");
    std::memcpy(lnL, h->h_out, sizeof(double) * B);
    if (dh) std::memcpy(dh, h->h_out + B, sizeof(double) * B);
    if (hh) std::memcpy(hh, h->h_out + 2 * B, sizeof(double) * B);
    return LISA_OK;
}

lisa_status lisa_like_data_inner(const lisa_like_t *h, double *dd) {
    if (!h || !dd) return LISA_ERR_ARG;
    if (!h->have_data) return LISA_ERR_STATE;
    *dd = h->dd;
    return LISA_OK;
}

lisa_status lisa_like_stage_knots(lisa_like_t *h, const double *params, int B, int64_t *band,
                                  double *fedge, double *fk, double *vals) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch || !params) return fail(h, LISA_ERR_ARG, "bad batch");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = h->stream;
    LCK(cudaMemcpyAsync(h->params, params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s),
        "parameter upload");
    const StageDims d = dims_of(h, B);
    LCK(launch_knots(d, bufs_of(h, h->params), s), "knot kernel launch");
    const size_t BL = (size_t)B * h->L, K = h->K;
    int *bandi = band ? new int[BL * 3] : nullptr;
    lisa_status st = LISA_OK;
    cudaError_t e = cudaSuccess;
    if (bandi) e = cudaMemcpyAsync(bandi, h->band, sizeof(int) * BL * 3, cudaMemcpyDeviceToHost, s);
    if (!e && fedge) e = cudaMemcpyAsync(fedge, h->fedge, sizeof(double) * BL * 2, cudaMemcpyDeviceToHost, s);
    if (!e && fk) e = cudaMemcpyAsync(fk, h->fk, sizeof(double) * BL * K, cudaMemcpyDeviceToHost, s);
    if (!e && vals) e = cudaMemcpyAsync(vals, h->vals, sizeof(double) * BL * kNSeries * K, cudaMemcpyDeviceToHost, s);
    if (e) st = cuda_fail(h, e, "stage download");
    if (st == LISA_OK) st = wait_for(h, s);
    if (st == LISA_OK && bandi)
        for (size_t i = 0; i < BL * 3; i++) band[i] = bandi[i];
    delete[] bandi;
    return st;
}

lisa_status lisa_like_stage_coeffs(lisa_like_t *h, const double *params, int B, double *coef) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch || !params || !coef) return fail(h, LISA_ERR_ARG, "bad batch");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = h->stream;
    LCK(cudaMemcpyAsync(h->params, params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s),
        "parameter upload");
    int nl = 0;
    lisa_status st = run_front(h, h->params, B, s, &nl);
    if (st != LISA_OK) return st;
    const size_t n = (size_t)B * h->L * (h->K - 1) * 32;
    LCK(cudaMemcpyAsync(coef, h->coef, sizeof(double) * n, cudaMemcpyDeviceToHost, s), "stage download");
    return wait_for(h, s);
}

lisa_status lisa_like_template(lisa_like_t *h, const double *params, double *out) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (!params || !out) return fail(h, LISA_ERR_ARG, "NULL parameter or output pointer");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = h->stream;
    LCK(cudaMemcpyAsync(h->params, params, sizeof(double) * kNPar, cudaMemcpyHostToDevice, s),
        "parameter upload");
    int nl = 0;
    lisa_status st = run_front(h, h->params, 1, s, &nl);
    if (st != LISA_OK) return st;
    double *dev = nullptr;
    LCK(dalloc(&dev, (size_t)6 * h->N), "device allocation (template)");
    cudaError_t e = launch_template(dims_of(h, 1), bufs_of(h, h->params), dev, s);
    if (!e) e = cudaMemcpyAsync(out, dev, sizeof(double) * 6 * h->N, cudaMemcpyDeviceToHost, s);
    if (e) {
        cudaFree(dev);
        return cuda_fail(h, e, "template");
    }
    st = wait_for(h, s);
    if (st == LISA_OK)
        cudaFree(dev);
    else
        h->deferred.push_back(dev);
    return st;
}

lisa_status lisa_like_set_profiling(lisa_like_t *h, int on) {
    if (!h) return LISA_ERR_ARG;
    h->profiling = on != 0;
    return LISA_OK;
}

lisa_status lisa_like_read_profile(lisa_like_t *h, double *ms, int *n_calls) {
    if (!h || !ms) return LISA_ERR_ARG;
    for (int i = 0; i < kStages; i++) ms[i] = 0.0;
    const int n = h->prof_calls;
    if (n_calls) *n_calls = n;
    if (n == 0) return LISA_OK;
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(h->prof_ev[kProfEvents * (n - 1) + kStages]);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(h, e, "device work failed");
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
            h->timeout_s)
            return fail(h, LISA_ERR_TIMEOUT, "profiled calls did not finish within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (int c = 0; c < n; c++)
        for (int i = 0; i < kStages; i++) {
            float t = 0.0f;
            LCK(cudaEventElapsedTime(&t, h->prof_ev[kProfEvents * c + i],
                                     h->prof_ev[kProfEvents * c + i + 1]),
                "cudaEventElapsedTime");
            ms[i] += t;
        }
    h->prof_calls = 0;
    return LISA_OK;
}

lisa_status lisa_like_test_device_wait(lisa_like_t *h, int polls) {
    if (!h) return LISA_ERR_ARG;
    if (polls < 0 || polls > (1 << 20)) return fail(h, LISA_ERR_ARG, "polls must be in [0, 2^20]");
    h->wait_test_polls = (unsigned)polls;
    drop_graph(h);  // a captured graph holds the previous setting
    return LISA_OK;
}

lisa_status lisa_like_set_graphs(lisa_like_t *h, int on) {
    if (!h) return LISA_ERR_ARG;
    h->use_graphs = on != 0;
    if (!h->use_graphs) drop_graph(h);
    return LISA_OK;
}

lisa_status lisa_like_set_tune(lisa_like_t *h, int per_thread, int group) {
    if (!h) return LISA_ERR_ARG;
    DenseTune t;
    if (!make_tune(h, per_thread, group, &t))
        return fail(h, LISA_ERR_ARG, "unsupported (per_thread, group) for this precision");
    h->tune = t;
    drop_graph(h);
    return LISA_OK;
}

lisa_status lisa_like_get_tune(const lisa_like_t *h, int *out) {
    if (!h || !out) return LISA_ERR_ARG;
    out[0] = h->tune.per_thread;
    out[1] = h->tune.group;
    out[2] = h->tune.blocks;
    return LISA_OK;
}

lisa_status lisa_like_autotune(lisa_like_t *h, const double *params, int B, int *out) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch || !params) return fail(h, LISA_ERR_ARG, "bad batch");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    const auto key = std::make_tuple(h->N, h->K, h->precision);
    auto it = h->tuned.find(key);
    if (it == h->tuned.end()) {
        cudaStream_t s = h->stream;
        LCK(cudaMemcpyAsync(h->params, params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s),
            "parameter upload");
        const int cand[][2] = {{8, 8}, {4, 8}, {16, 8}, {8, 1}};
        cudaEvent_t e0, e1;
        LCK(cudaEventCreate(&e0), "cudaEventCreate");
        LCK(cudaEventCreate(&e1), "cudaEventCreate");
        float best = 3.4e38f;
        DenseTune bt = h->tune;
        lisa_status st = LISA_OK;
        for (const auto &c : cand) {
            DenseTune t;
            if (!make_tune(h, c[0], c[1], &t)) continue;
            h->tune = t;
            st = enqueue(h, h->params, B, h->out, nullptr, nullptr, s, false);  // warm
            if (st != LISA_OK) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && st == LISA_OK; r++)
                st = enqueue(h, h->params, B, h->out, nullptr, nullptr, s, false);
            cudaEventRecord(e1, s);
            if (st != LISA_OK) break;
            st = wait_for(h, s);
            if (st != LISA_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt = t;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != LISA_OK) return st;
        it = h->tuned.emplace(key, bt).first;
    }
    h->tune = it->second;
    drop_graph(h);
    if (out) {
        out[0] = h->tune.per_thread;
        out[1] = h->tune.group;
        out[2] = h->tune.blocks;
    }
    return LISA_OK;
}

lisa_status lisa_like_mode_inner(lisa_like_t *h, const double *params, int B, double *dh_modes,
                                 double *hh_modes) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch || !params || (!dh_modes && !hh_modes))
        return fail(h, LISA_ERR_ARG, "bad batch or NULL outputs");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = h->stream;
    LCK(cudaMemcpyAsync(h->params, params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s),
        "parameter upload");
    const int L = h->L;
    std::vector<double> buf((size_t)2 * B * L);
    for (int mi = 0; mi < L; mi++) {
        lisa_status st = enqueue(h, h->params, B, h->out, h->out + B, h->out + 2 * B, s, false,
                                 1u << mi);
        if (st != LISA_OK) return st;
        LCK(cudaMemcpyAsync(h->h_out, h->out, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s),
            "result download");
        LCK(cudaMemcpyAsync(h->h_err, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s),
            "result download");
        st = wait_for(h, s);
        if (st != LISA_OK) return st;
        if (*h->h_err) return fail(h, LISA_ERR_TIMEOUT, "a device wait for staged data gave up");
        for (int b = 0; b < B; b++) {
            buf[(size_t)b * L + mi] = h->h_out[B + b];
            buf[(size_t)B * L + (size_t)b * L + mi] = h->h_out[2 * B + b];
        }
    }
    if (dh_modes) std::memcpy(dh_modes, buf.data(), sizeof(double) * B * L);
    if (hh_modes) std::memcpy(hh_modes, buf.data() + (size_t)B * L, sizeof(double) * B * L);
    return LISA_OK;
}

lisa_status lisa_like_mode_cross(lisa_like_t *h, const double *params, int B, double *cross) {
    if (!h) return LISA_ERR_ARG;
    if (!h->have_data) return fail(h, LISA_ERR_STATE, "set_data must be called first");
    if (B < 1 || B > h->max_batch || !params || !cross)
        return fail(h, LISA_ERR_ARG, "bad batch or NULL output");
    LCK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = h->stream;
    LCK(cudaMemcpyAsync(h->params, params, sizeof(double) * kNPar * B, cudaMemcpyHostToDevice, s),
        "parameter upload");
    const int L = h->L;
    // <h_a + h_b | h_a + h_b> for every pair (a single mode when a = b), then
    // Re<h_a|h_b> = (<h_a+b|h_a+b> - <h_a|h_a> - <h_b|h_b>) / 2
    std::vector<double> pair((size_t)L * L * B);
    for (int a = 0; a < L; a++)
        for (int b = a; b < L; b++) {
            const unsigned mask = (1u << a) | (1u << b);
            lisa_status st = enqueue(h, h->params, B, h->out, h->out + B, h->out + 2 * B, s,
                                     false, mask);
            if (st != LISA_OK) return st;
            LCK(cudaMemcpyAsync(h->h_out, h->out, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s),
                "result download");
            LCK(cudaMemcpyAsync(h->h_err, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s),
                "result download");
            st = wait_for(h, s);
            if (st != LISA_OK) return st;
            if (*h->h_err) return fail(h, LISA_ERR_TIMEOUT, "a device wait for staged data gave up");
            for (int w = 0; w < B; w++) pair[((size_t)a * L + b) * B + w] = h->h_out[2 * B + w];
        }
    for (int w = 0; w < B; w++)
        for (int a = 0; a < L; a++)
            for (int b = 0; b < L; b++) {
                const int lo = a < b ? a : b, hi = a < b ? b : a;
                double v = pair[((size_t)lo * L + hi) * B + w];
                if (lo != hi)
                    v = 0.5 * (v - pair[((size_t)lo * L + lo) * B + w] - pair[((size_t)hi * L + hi) * B + w]);
                cross[((size_t)w * L + a) * L + b] = v;
            }
    return LISA_OK;
}

int lisa_like_last_launches(const lisa_like_t *h) { return h ? h->last_launches : 0; }

void lisa_like_destroy(lisa_like_t *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_batch(h);
    for (void *p : h->deferred) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost)
            cudaFreeHost(p);
        else
            cudaFree(p);
    }
    if (h->bins) cudaFree(h->bins);
    if (h->bins32) cudaFree(h->bins32);
    if (h->part) cudaFree(h->part);
    lisa::rb_free(h->rb);
    drop_graph(h);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    if (h->done) cudaEventDestroy(h->done);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char *lisa_like_last_error(const lisa_like_t *h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

// ------------------------------------------------------------------ host-side helpers
double lisa_dl_from_z(double z) {
    // flat LambdaCDM, H0 = 67.7 km/s/Mpc, Omega_m = 0.31 (stand-in for the paper's
    // Astropy cosmology): D_L = (1+z) c/H0 int_0^z dz'/E(z'), 5-point Gauss-Legendre
    // on 400 equal panels
    if (!(z >= 0.0) || !std::isfinite(z)) return NAN;
    const double om = 0.31, hub = 299792.458 / 67.7 / 1000.0;
    static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0,
                                 0.5384693101056831, 0.9061798459386640};
    static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                                 0.4786286704993665, 0.2369268850561891};
    const int panels = 400;
    const double hw = 0.5 * z / panels;
    double acc = 0.0;
    for (int p = 0; p < panels; p++) {
        const double mid = (2 * p + 1) * hw;
        for (int k = 0; k < 5; k++) {
            const double zz = mid + hw * gx[k];
            const double a = 1.0 + zz;
            acc += gw[k] / std::sqrt(om * a * a * a + (1.0 - om));
        }
    }
    return (1.0 + z) * hub * acc * hw;
}

lisa_status lisa_psd_aet(double f0, double df, int64_t n_bins, double *out) {
    // stand-in one-sided PSD of first-generation A, E, T with equal 2.5 Gm arms:
    // optical-metrology noise 15 pm/sqrt(Hz) (with a 2 mHz knee) and acceleration noise
    // 3 fm/s^2/sqrt(Hz) (0.4 mHz and 8 mHz shaping), in fractional-frequency units
    if (!out || !(f0 > 0.0) || !(df > 0.0) || n_bins < 1) return LISA_ERR_ARG;
    const double L = kArmM / kClight;
    for (int64_t j = 0; j < n_bins; j++) {
        const double f = f0 + (double)j * df;
        const double om = kTwoPi * f;
        const double conv = (om / kClight) * (om / kClight);
        const double a = 2e-3 / f, b = 0.4e-3 / f, c = f / 8e-3;
        const double oms = 2.25e-22 * (1.0 + a * a * a * a) * conv;
        const double acc = 9e-30 * (1.0 + b * b) * (1.0 + c * c * c * c) / (om * om * om * om) * conv;
        const double x = om * L;
        const double sx = std::sin(x), cx = std::cos(x);
        const double sae = 8.0 * sx * sx * ((2.0 + cx) * oms + 2.0 * (3.0 + 2.0 * cx + std::cos(2.0 * x)) * acc);
        const double st = 16.0 * sx * sx * (1.0 - cx) * (oms + 2.0 * (1.0 - cx) * acc);
        out[j] = sae;
        out[n_bins + j] = sae;
        out[2 * n_bins + j] = st;
    }
    return LISA_OK;
}

}  // extern "C"
