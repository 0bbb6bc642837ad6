// noalloc.cu -- lisa_like_loglike_noalloc: the batched ln L for callers that cannot
// call cudaMalloc.  Such callers include code running inside a framework that owns the
// whole device heap and hands an operation only the buffers it may use (a custom op or
// foreign-function handler), and real-time loops where the implicit device
// synchronisation of an allocation is not acceptable.  The caller passes every input
// and output; all per-call scratch comes from one file-scope device array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lisa_like.h"
#include "kernels.h"
#include "model.cuh"

namespace lisa {
void set_thread_error(const std::string &msg);  // defined in lisa_like.cu
}

using namespace lisa;

namespace {

constexpr size_t kScratchBytes = LISA_NOALLOC_SCRATCH_BYTES;
// The dense kernel's fixed shape here: 128 threads x 8 bins per tile, one walker per
// group.  The item bound and the partial-sum buffer below are derived from it.
constexpr int kThreads = 128, kPerThread = 8, kGroup = 1;
constexpr int kTile = kThreads * kPerThread;
static_assert(kTile == 1024, "the limit LISA_NOALLOC_MAX_ITEMS is stated for 1024-bin tiles");
static_assert(kGroup == 1, "the item bound counts one (item, walker) slot per walker and tile");

// The scratch of every no-alloc call on this device.  It is part of the library's
// device image, so every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

struct Layout {
    size_t valid, tc, xpk, band, fedge, fk, kb, vals, mscr, coef, phases, wrange, order, slot,
        grange, items,
        counter, err, part, end;
};

Layout layout_for(size_t B, size_t L, size_t K, size_t items) {
    Layout o;
    size_t p = 0;
    auto take = [&](size_t bytes) {
        const size_t at = p;
        p += up256(bytes);
        return at;
    };
    o.valid = take(sizeof(int) * B);
    o.tc = take(sizeof(double) * B);
    o.xpk = take(sizeof(double) * B);
    o.band = take(sizeof(int) * B * L * 3);
    o.fedge = take(sizeof(double) * B * L * 2);
    o.fk = take(sizeof(double) * B * L * K);
    o.kb = take(sizeof(int) * B * L * K);
    o.vals = take(sizeof(double) * B * L * kNSeries * K);
    o.mscr = take(sizeof(double) * B * L * kScratchRows * K);
    o.coef = take(sizeof(double) * B * L * (K - 1) * 32);
    // the knot values are dead once the splines exist: the phase records reuse them
    o.phases = o.vals;
    static_assert(sizeof(unsigned long long) * kPhaseWords <= sizeof(double) * kNSeries,
                  "phase records fit in the knot-value rows");
    o.wrange = take(sizeof(int) * 2 * B);
    o.order = take(sizeof(int) * B);
    o.slot = take(sizeof(int) * B);
    o.grange = take(sizeof(int) * 2 * B);
    o.items = take(sizeof(int) * (B + 1));
    o.counter = take(sizeof(int));
    o.err = take(sizeof(int));
    o.part = take(sizeof(double) * 2 * items);
    o.end = p;
    return o;
}

lisa_status arg_error(const char *msg) {
    set_thread_error(msg);
    return LISA_ERR_ARG;
}

lisa_status cuda_error(cudaError_t e, const char *what) {
    set_thread_error(std::string(what) + ": " + cudaGetErrorString(e));
    return LISA_ERR_CUDA;
}

// Address of the scratch array on the current device, looked up once per device with
// that device current.
lisa_status scratch_on_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return arg_error("device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress (no-alloc scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LISA_OK;
}

}  // namespace

extern "C" lisa_status lisa_like_loglike_noalloc(const lisa_like_config *cfg, double f0, double df,
                                                 int64_t n_bins, const double *d_bins, double dd,
                                                 const double *d_params, int B, double *d_lnL,
                                                 double *d_dh, double *d_hh, void *stream) {
    set_thread_error("");
    if (!cfg || !d_bins || !d_params || !d_lnL) return arg_error("NULL config, data, parameter or ln L pointer");
    if (cfg->n_modes < 1 || cfg->n_modes > 6) return arg_error("n_modes must be 1..6");
    int seen = 0;
    for (int i = 0; i < cfg->n_modes; i++) {
        const int id = mode_index(cfg->modes[i][0], cfg->modes[i][1]);
        if (id < 0 || ((seen >> id) & 1))
            return arg_error("modes must be distinct entries of (2,2),(3,3),(4,4),(2,1),(3,2),(4,3)");
        seen |= 1 << id;
    }
    const int K = cfg->n_knots, L = cfg->n_modes;
    if (K < 4 || K > 4096) return arg_error("n_knots must be in [4, 4096]");
    if (!(f0 > 0.0) || !std::isfinite(f0) || !(df > 0.0) || !std::isfinite(df) ||
        !std::isfinite(cfg->t0_s) || !std::isfinite(dd))
        return arg_error("grid needs finite f0 > 0, df > 0; t0 and <d|d> must be finite");
    if (n_bins < 1 || n_bins >= ((int64_t)1 << 31)) return arg_error("n_bins must be in [1, 2^31)");
    if (B < 1) return arg_error("B must be >= 1");
    if (((uintptr_t)d_bins & 15) != 0) return arg_error("d_bins must be 16-byte aligned");
    const int64_t blk = (int64_t)B * L * K;
    // one walker per group here: (item, walker) pairs = B x tiles of at most n_bins + 3 bins
    const int64_t items = (int64_t)B * ((n_bins + 3 + kTile - 1) / kTile + 1);
    if (blk > LISA_NOALLOC_MAX_WALKER_MODE_KNOTS)
        return arg_error("B * n_modes * n_knots exceeds the no-alloc limit (8192)");
    if (items > LISA_NOALLOC_MAX_ITEMS)
        return arg_error("B * (ceil(n_bins / 1024) + 1) exceeds the no-alloc limit (16384)");
    const Layout o = layout_for(B, L, K, (size_t)items);
    if (o.end > kScratchBytes) return arg_error("request does not fit the no-alloc scratch");

    void *base = nullptr;
    lisa_status st = scratch_on_current_device(&base);
    if (st != LISA_OK) return st;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");

    unsigned char *s8 = static_cast<unsigned char *>(base);
    StageBufs b;
    b.params = d_params;
    b.valid = reinterpret_cast<int *>(s8 + o.valid);
    b.tc = reinterpret_cast<double *>(s8 + o.tc);
    b.xpk = reinterpret_cast<double *>(s8 + o.xpk);
    b.band = reinterpret_cast<int *>(s8 + o.band);
    b.fedge = reinterpret_cast<double *>(s8 + o.fedge);
    b.fk = reinterpret_cast<double *>(s8 + o.fk);
    b.kb = reinterpret_cast<int *>(s8 + o.kb);
    b.vals = reinterpret_cast<double *>(s8 + o.vals);
    b.mscratch = reinterpret_cast<double *>(s8 + o.mscr);
    b.coef = reinterpret_cast<double *>(s8 + o.coef);
    b.wrange = reinterpret_cast<int *>(s8 + o.wrange);
    b.order = reinterpret_cast<int *>(s8 + o.order);
    b.slot_of = reinterpret_cast<int *>(s8 + o.slot);
    b.grange = reinterpret_cast<int *>(s8 + o.grange);
    b.item_start = reinterpret_cast<int *>(s8 + o.items);
    b.counter = reinterpret_cast<int *>(s8 + o.counter);
    b.err = reinterpret_cast<int *>(s8 + o.err);
    b.part = reinterpret_cast<double *>(s8 + o.part);

    StageDims d;
    d.B = B;
    d.L = L;
    d.K = K;
    d.N = (int)n_bins;
    d.f0 = f0;
    d.df = df;
    d.t0 = cfg->t0_s;
    for (int i = 0; i < 6; i++) {
        d.ml[i] = i < L ? cfg->modes[i][0] : 0;
        d.mm[i] = i < L ? cfg->modes[i][1] : 0;
    }
    const DenseTune tune = {kThreads, kPerThread, nsm * 2, kGroup};
    cudaStream_t s = (cudaStream_t)stream;
    // Every buffer is written before it is read within the call; the work counter and the
    // error flag, the only values that must start at zero, are cleared by the planning
    // kernel.
    if ((e = launch_knots(d, b, s)) != cudaSuccess) return cuda_error(e, "knot kernel launch");
    if ((e = launch_spline(d, b, s)) != cudaSuccess) return cuda_error(e, "spline kernel launch");
    if ((e = launch_plan(d, b, kTile, tune.group, s)) != cudaSuccess)
        return cuda_error(e, "plan kernel launch");
    unsigned long long *phases = reinterpret_cast<unsigned long long *>(s8 + o.phases);
    if ((e = launch_phaseprep(d, b, phases, s)) != cudaSuccess)
        return cuda_error(e, "segment kernel launch");
    if ((e = launch_dense_f64(d, b, phases, d_bins, tune, s)) != cudaSuccess)
        return cuda_error(e, "dense kernel launch");
    if ((e = launch_finish(d, b, tune.group, 0, dd, d_lnL, d_dh, d_hh, s)) != cudaSuccess)
        return cuda_error(e, "finish kernel launch");
    return LISA_OK;
}
