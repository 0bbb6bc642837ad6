// internal.h -- what other parts of liblisalike.so (the sampler) need from a likelihood
// handle; not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/lisa_like.h"

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

// failure text of handle-free entry points (lisa_like_last_error(NULL))
void set_thread_error(const std::string &msg);
const char *thread_error();

}  // namespace lisa
