// flow.h -- what the sampler needs from the flow (internal to liblisalike.so).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lisa_flow.h"

namespace lisa_flowint {

// One independence-proposal step for the coldest temperature's W walkers.
struct FStep {
    int W;                      // walkers of the coldest temperature (rows 0..W-1 of x)
    uint32_t k0, k1;            // Philox key
    const unsigned *step;       // step counter (device)
    double *x, *lnl, *lnp;      // the sampler's state (temperature 0 first)
    const double *betas;        // [T]
    double lo[11], hi[11];      // prior box
    int lisa_frame, target;
    double t0;
    double mean[11], sig[11];   // Gaussian test target
    double *fy;                 // [W][11] proposals
    double *fpth;               // [W][11] their physical parameters (likelihood input)
    double *fly;                // [W] their ln L (written by the likelihood or the test target)
    double *fq;                 // [W] log q(x) - log q(y)
    double *fpy;                // [W] ln prior of the proposals
    unsigned long long *facc;   // [3] accepted, proposed, sent to the second likelihood
    int *err;                   // sticky sampler error
    const int *like_err;        // the likelihood's flag of its last call (or NULL)
    // Screened flow moves (margin > 0): the sampler's own likelihood evaluates every
    // proposal (fly); those it rejects by more than margin in ln L keep that decision, the
    // others are evaluated again by the second likelihood (fly2), which decides them.
    double margin;
    double *fpth2;              // [W][11] proposals sent on; the rest carry a NaN mass
    double *fly2;               // [W] their ln L from the second likelihood
    int *fsent;                 // [W] 1 if the proposal was sent on
    const int *like_err2;       // the second likelihood's flag (or NULL)
};

cudaError_t launch_flow_propose(lisa_flow_t *f, const FStep &a, cudaStream_t s);
cudaError_t launch_flow_accept(const FStep &a, cudaStream_t s);
// screened flow moves: the first likelihood's verdict, and the proposals for the second
cudaError_t launch_flow_screen(const FStep &a, cudaStream_t s);
// training without host synchronisation (losses kept on the device)
lisa_status flow_train_async(lisa_flow_t *f, const double *d_data, int64_t n, int iters,
                             int batch, double lr, uint64_t seed, uint32_t round, cudaStream_t s);
// loss of the last iteration of the last training (host read, synchronous on s)
lisa_status flow_last_loss(lisa_flow_t *f, double *loss, cudaStream_t s);

}  // namespace lisa_flowint
