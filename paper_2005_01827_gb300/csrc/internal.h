// internal.h -- what other parts of liblisalike.so (the sampler) need from a likelihood
// handle; not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/lisa_like.h"
#include "kernels.h"

namespace lisa {

struct LikeInfo {
    cudaStream_t stream;   // the handle's stream
    int device;
    int max_batch;
    int have_data;
    double t0;             // t_coal = t_ref + t0
    const int *err_flag;   // device flag: a dense-kernel wait gave up in the last call
    double timeout_s;
};

LikeInfo like_info(const lisa_like_t *h);

// The likelihood's kernels for B walkers on stream s (capturable: no allocation, no
// synchronisation).  d_lnL receives ln L; walkers with invalid parameters get -inf.
lisa_status like_enqueue(lisa_like_t *h, const double *d_params, int B, double *d_lnL,
                         cudaStream_t s, int *launches);

// What the relative-binning likelihood needs from a handle.
struct LikeCore {
    cudaStream_t stream;
    int device, max_batch, have_data, N, L, K;
    double t0, f0, df, dd, timeout_s;
    int ml[6], mm[6];
    const double *bins;   // [N][9] staged data: w_A, w_E, w_T, (w d) re/im per channel
    double *params;       // [max_batch][11] device staging
    double *h_params;     // pinned host staging of the same size
    double *out, *h_out;  // [3][max_batch] device outputs and their pinned copy
    StageBufs stage;      // band, edge, validity and peak buffers (params = `params`)
};
LikeCore like_core(lisa_like_t *h);

struct RbState;                 // relative-binning state of a handle (rb.cu)
RbState *&like_rb(lisa_like_t *h);
void rb_free(RbState *r);
lisa_status like_fail(lisa_like_t *h, lisa_status st, const std::string &msg);
lisa_status like_wait(lisa_like_t *h, cudaStream_t s);

// failure text of handle-free entry points (lisa_like_last_error(NULL))
void set_thread_error(const std::string &msg);
const char *thread_error();

}  // namespace lisa
