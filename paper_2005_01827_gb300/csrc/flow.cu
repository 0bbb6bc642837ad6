// flow.cu -- the normalizing-flow proposal of include/lisa_flow.h: evaluation in both
// directions, training (forward, back-propagation, Adam) and the independence
// Metropolis-Hastings step of the sampler (Eq. (13)).
//
// Every network layer is a GEMM on the tensor cores: bfloat16 operands staged in shared
// memory, FP32 accumulation, mma.sync.m16n8k16.  A block holds 64 samples; each of its
// four warps owns 16 of them for every per-sample GEMM (so a layer needs only warp
// synchronisation), and the weight-gradient GEMMs, which contract over the block's 64
// samples, run after a block barrier and add into FP32 gradients in global memory.  The
// back-propagation recomputes each layer's activations from the layer input stored in
// the forward pass (64 x 11 values per coupling) instead of keeping them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lisa_flow.h"
#include "flow.h"
#include "internal.h"
#include "sampler_dev.cuh"

using bf16 = __nv_bfloat16;

namespace {

constexpr int FD = 11, FH = 128, FC = 8, FO = 22;
constexpr int K1 = 16;   // layer-1 reduction length (11 padded)
constexpr int N3 = 24;   // layer-3 outputs (22 padded)
constexpr int R3 = 32;   // W3 rows kept (22 padded to two k-steps of the backward GEMM)
// master FP32 layout of one coupling
constexpr int OW1 = 0, OB1 = OW1 + FH * FD, OW2 = OB1 + FH, OB2 = OW2 + FH * FH, OW3 = OB2 + FH,
              OB3 = OW3 + FO * FH, PC = OB3 + FO;
static_assert(PC == LISA_FLOW_PARAMS_PER_COUPLING, "weight layout");
constexpr int NP = FC * PC;
// bfloat16 copies of one coupling: W1 [128][16], W2 [128][128], W3 [32][128]
constexpr int BW1 = 0, BW2 = BW1 + FH * K1, BW3 = BW2 + FH * FH, BC = BW3 + R3 * FH;
constexpr int TS = 64;    // samples per block
constexpr int NTH = 128;  // four warps of 16 samples
// shared-memory leading dimensions (bf16 elements), padded against bank conflicts
constexpr int LW1 = 24, LH = 136, LGO = 40, LU = 12;
constexpr float kS = 2.0f;  // s = kS tanh(o_s / kS)
constexpr double kLog2Pi = 1.8378770664093454835606594728112353;

__host__ __device__ inline bool keep(int c, int d) {
    switch (c & 3) {
        case 0: return (d & 1) == 0;
        case 1: return (d & 1) == 1;
        case 2: return d < 6;
        default: return d >= 6;
    }
}

// ------------------------------------------------------------------ shared memory
struct alignas(16) SmemNet {
    bf16 w1[FH * LW1];
    bf16 w2[FH * LH];
    bf16 w3[R3 * LH];
    float b1[FH], b2[FH], b3[N3];
    bf16 a0[TS * LW1];
    bf16 a1[TS * LH];
    bf16 a2[TS * LH];
    float o[TS * N3];
    float u[TS * LU];
};

struct alignas(16) SmemTrain {
    SmemNet n;
    bf16 go[TS * LGO];
    bf16 gz2[TS * LH];
    bf16 gz1[TS * LH];
    float ust[FC * TS * LU];  // layer inputs of the forward pass
    float gv[TS * LU];        // dL/dv of the current layer's output
    float db1[FH], db2[FH], db3[N3];
    double lsum[4];
};

// ------------------------------------------------------------------ warp GEMMs
__device__ __forceinline__ uint32_t ld2(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ uint32_t pk(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                    uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[16][8 NT] += A[16][16 KS] B with A row-major (lda) and B[k][n] = Bt[n][k] (ldb)
template <int NT, int KS>
__device__ __forceinline__ void mma_nt(const bf16 *A, int lda, const bf16 *Bt, int ldb,
                                       float (&c)[NT][4], int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < KS; ks++) {
        const int k0 = 16 * ks + 2 * t;
        const uint32_t a0 = ld2(A + g * lda + k0), a1 = ld2(A + (g + 8) * lda + k0);
        const uint32_t a2 = ld2(A + g * lda + k0 + 8), a3 = ld2(A + (g + 8) * lda + k0 + 8);
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const bf16 *bp = Bt + (nt * 8 + g) * ldb + k0;
            mma(c[nt], a0, a1, a2, a3, ld2(bp), ld2(bp + 8));
        }
    }
}

// C[16][8 NT] += A[16][16 KS] B with A row-major (lda) and B[k][n] = Bk[k][n] (ldb)
template <int NT, int KS>
__device__ __forceinline__ void mma_nn(const bf16 *A, int lda, const bf16 *Bk, int ldb,
                                       float (&c)[NT][4], int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < KS; ks++) {
        const int k0 = 16 * ks + 2 * t;
        const uint32_t a0 = ld2(A + g * lda + k0), a1 = ld2(A + (g + 8) * lda + k0);
        const uint32_t a2 = ld2(A + g * lda + k0 + 8), a3 = ld2(A + (g + 8) * lda + k0 + 8);
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int n = nt * 8 + g;
            const uint32_t b0 = pk(Bk[k0 * ldb + n], Bk[(k0 + 1) * ldb + n]);
            const uint32_t b1 = pk(Bk[(k0 + 8) * ldb + n], Bk[(k0 + 9) * ldb + n]);
            mma(c[nt], a0, a1, a2, a3, b0, b1);
        }
    }
}

// C[16][8 NT] += At^T B over the 64 samples: A[m][k] = At[k][m0 + m] (lda),
// B[k][n] = Bk[k][n0 + n] (ldb)
template <int NT>
__device__ __forceinline__ void mma_tn(const bf16 *At, int lda, int m0, const bf16 *Bk, int ldb,
                                       int n0, float (&c)[NT][4], int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < TS / 16; ks++) {
        const int k0 = 16 * ks + 2 * t;
        const int m = m0 + g;
        const uint32_t a0 = pk(At[k0 * lda + m], At[(k0 + 1) * lda + m]);
        const uint32_t a1 = pk(At[k0 * lda + m + 8], At[(k0 + 1) * lda + m + 8]);
        const uint32_t a2 = pk(At[(k0 + 8) * lda + m], At[(k0 + 9) * lda + m]);
        const uint32_t a3 = pk(At[(k0 + 8) * lda + m + 8], At[(k0 + 9) * lda + m + 8]);
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int n = n0 + nt * 8 + g;
            const uint32_t b0 = pk(Bk[k0 * ldb + n], Bk[(k0 + 1) * ldb + n]);
            const uint32_t b1 = pk(Bk[(k0 + 8) * ldb + n], Bk[(k0 + 9) * ldb + n]);
            mma(c[nt], a0, a1, a2, a3, b0, b1);
        }
    }
}

template <int NT>
__device__ __forceinline__ void zero(float (&c)[NT][4]) {
#pragma unroll
    for (int i = 0; i < NT; i++) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.0f;
}

// ------------------------------------------------------------------ network pieces
__device__ void load_coupling(SmemNet &sm, const bf16 *wb, const float *w, int c) {
    const bf16 *src = wb + (size_t)c * BC;
    const float *ws = w + (size_t)c * PC;
    for (int i = threadIdx.x; i < FH * 2; i += NTH) {
        const int r = i >> 1, q = i & 1;
        *reinterpret_cast<uint4 *>(sm.w1 + r * LW1 + q * 8) =
            *reinterpret_cast<const uint4 *>(src + BW1 + r * K1 + q * 8);
    }
    for (int i = threadIdx.x; i < FH * 16; i += NTH) {
        const int r = i >> 4, q = i & 15;
        *reinterpret_cast<uint4 *>(sm.w2 + r * LH + q * 8) =
            *reinterpret_cast<const uint4 *>(src + BW2 + r * FH + q * 8);
    }
    for (int i = threadIdx.x; i < R3 * 16; i += NTH) {
        const int r = i >> 4, q = i & 15;
        *reinterpret_cast<uint4 *>(sm.w3 + r * LH + q * 8) =
            *reinterpret_cast<const uint4 *>(src + BW3 + r * FH + q * 8);
    }
    for (int i = threadIdx.x; i < FH; i += NTH) {
        sm.b1[i] = ws[OB1 + i];
        sm.b2[i] = ws[OB2 + i];
        if (i < N3) sm.b3[i] = i < FO ? ws[OB3 + i] : 0.0f;
    }
}

// The coupling network of layer c on the warp's 16 rows r0.. of `uin` (row stride LU):
// a0 = bf16(m u), a1 = bf16(relu(W1 a0 + b1)), a2 = bf16(relu(W2 a1 + b2)), o = W3 a2 + b3.
__device__ void net_forward(SmemNet &sm, const float *uin, int c, int r0, int lane) {
    for (int i = lane; i < 16 * K1; i += 32) {
        const int r = i >> 4, k = i & 15;
        const float v = (k < FD && keep(c, k)) ? uin[(r0 + r) * LU + k] : 0.0f;
        sm.a0[(r0 + r) * LW1 + k] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    const int g = lane >> 2, t = lane & 3;
    {
        float acc[16][4];
        zero(acc);
        mma_nt<16, 1>(sm.a0 + r0 * LW1, LW1, sm.w1, LW1, acc, lane);
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            const int col = nt * 8 + 2 * t;
            const float bl = sm.b1[col], bh = sm.b1[col + 1];
            *reinterpret_cast<uint32_t *>(sm.a1 + (r0 + g) * LH + col) =
                pk(__float2bfloat16_rn(fmaxf(acc[nt][0] + bl, 0.0f)),
                   __float2bfloat16_rn(fmaxf(acc[nt][1] + bh, 0.0f)));
            *reinterpret_cast<uint32_t *>(sm.a1 + (r0 + g + 8) * LH + col) =
                pk(__float2bfloat16_rn(fmaxf(acc[nt][2] + bl, 0.0f)),
                   __float2bfloat16_rn(fmaxf(acc[nt][3] + bh, 0.0f)));
        }
    }
    __syncwarp();
    {
        float acc[16][4];
        zero(acc);
        mma_nt<16, 8>(sm.a1 + r0 * LH, LH, sm.w2, LH, acc, lane);
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            const int col = nt * 8 + 2 * t;
            const float bl = sm.b2[col], bh = sm.b2[col + 1];
            *reinterpret_cast<uint32_t *>(sm.a2 + (r0 + g) * LH + col) =
                pk(__float2bfloat16_rn(fmaxf(acc[nt][0] + bl, 0.0f)),
                   __float2bfloat16_rn(fmaxf(acc[nt][1] + bh, 0.0f)));
            *reinterpret_cast<uint32_t *>(sm.a2 + (r0 + g + 8) * LH + col) =
                pk(__float2bfloat16_rn(fmaxf(acc[nt][2] + bl, 0.0f)),
                   __float2bfloat16_rn(fmaxf(acc[nt][3] + bh, 0.0f)));
        }
    }
    __syncwarp();
    {
        float acc[3][4];
        zero(acc);
        mma_nt<3, 8>(sm.a2 + r0 * LH, LH, sm.w3, LH, acc, lane);
#pragma unroll
        for (int nt = 0; nt < 3; nt++) {
            const int col = nt * 8 + 2 * t;
            sm.o[(r0 + g) * N3 + col] = acc[nt][0] + sm.b3[col];
            sm.o[(r0 + g) * N3 + col + 1] = acc[nt][1] + sm.b3[col + 1];
            sm.o[(r0 + g + 8) * N3 + col] = acc[nt][2] + sm.b3[col];
            sm.o[(r0 + g + 8) * N3 + col + 1] = acc[nt][3] + sm.b3[col + 1];
        }
    }
    __syncwarp();
}

// the coupling update of one row: normalizing (x -> z) or generating (z -> x); returns
// the row's sum of s
__device__ float couple_row(SmemNet &sm, int c, int row, bool gen) {
    float ssum = 0.0f;
    for (int d = 0; d < FD; d++) {
        if (keep(c, d)) continue;
        const float s = kS * tanhf(sm.o[row * N3 + d] / kS);
        const float tt = sm.o[row * N3 + FD + d];
        float &u = sm.u[row * LU + d];
        u = gen ? u * expf(s) + tt : (u - tt) * expf(-s);
        ssum += s;
    }
    return ssum;
}

// ------------------------------------------------------------------ evaluation
struct FlowView {
    const float *w;
    const bf16 *wb;
    const double *mu, *L;  // mean [11], lower-triangular whitening factor [11][11]
};

// u = L^{-1} (x - mu) by forward substitution (FP64), written as FP32
__device__ inline void whiten_row(const double *x, const double *mu, const double *L, float *u) {
    double v[FD];
    for (int d = 0; d < FD; d++) {
        double acc = x[d] - mu[d];
        for (int j = 0; j < d; j++) acc -= L[d * FD + j] * v[j];
        v[d] = acc / L[d * FD + d];
        u[d] = (float)v[d];
    }
}

__device__ inline double log_det_factor(const double *L) {
    double s = 0.0;
    for (int d = 0; d < FD; d++) s += log(L[d * FD + d]);
    return s;
}

// Both directions for up to 64 rows per block.  Normalizing: in = x, out = z;
// generating: in = z, out = x.  logq = log q(x) in both cases.
__global__ void __launch_bounds__(NTH) flow_eval_kernel(FlowView f, const double *in, int n,
                                                        int gen, double *out, double *logq) {
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemNet &sm = *reinterpret_cast<SmemNet *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, r0 = warp * 16;
    const int row0 = blockIdx.x * TS;
    double lq = 0.0;  // lanes 0..15: the row r0 + lane
    if (threadIdx.x < TS) {
        const int r = threadIdx.x, row = row0 + r;
        float *u = sm.u + r * LU;
        for (int d = 0; d < LU; d++) u[d] = 0.0f;
        if (row < n) {
            if (gen)
                for (int d = 0; d < FD; d++) u[d] = (float)in[(size_t)row * FD + d];
            else
                whiten_row(in + (size_t)row * FD, f.mu, f.L, u);
        }
    }
    __syncthreads();
    if (gen && lane < 16) {
        const int row = row0 + r0 + lane;
        if (row < n) {
            double zz = 0.0;
            for (int d = 0; d < FD; d++) {
                const double zv = in[(size_t)row * FD + d];
                zz += zv * zv;
            }
            lq = -0.5 * zz - 0.5 * FD * kLog2Pi;
        }
    }
    for (int k = 0; k < FC; k++) {
        const int c = gen ? FC - 1 - k : k;
        load_coupling(sm, f.wb, f.w, c);
        __syncthreads();
        net_forward(sm, sm.u, c, r0, lane);
        if (lane < 16) lq -= (double)couple_row(sm, c, r0 + lane, gen != 0);
        __syncwarp();
        __syncthreads();
    }
    if (lane < 16) {
        const int rr = r0 + lane, row = row0 + rr;
        if (row < n) {
            const double lsig = log_det_factor(f.L);
            double zz = 0.0;
            for (int d = 0; d < FD; d++) {
                const double v = sm.u[rr * LU + d];
                if (gen) {
                    double xv = f.mu[d];  // x = mu + L v
                    for (int j = 0; j <= d; j++) xv += f.L[d * FD + j] * (double)sm.u[rr * LU + j];
                    out[(size_t)row * FD + d] = xv;
                } else {
                    zz += v * v;
                    if (out) out[(size_t)row * FD + d] = v;
                }
            }
            logq[row] = gen ? lq - lsig : -0.5 * zz - 0.5 * FD * kLog2Pi + lq - lsig;
        }
    }
}

// ------------------------------------------------------------------ training
struct TrainArgs {
    const float *w;
    const bf16 *wb;
    float *grad;            // [8][PC], accumulated
    const double *mu, *L;
    const double *data;     // [n][11]
    long long n;
    int batch;              // rows of this minibatch (multiple of 64)
    uint32_t k0, k1, round, iter;
    int random_rows;        // 1: Philox minibatch rows; 0: rows 0..batch-1 in order
    double *loss;           // accumulated mean loss of the minibatch
};

__global__ void __launch_bounds__(NTH) flow_train_kernel(TrainArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemTrain &st = *reinterpret_cast<SmemTrain *>(smraw);
    SmemNet &sm = st.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, r0 = warp * 16;
    const int g = lane >> 2, t = lane & 3;
    const float inv_n = 1.0f / (float)a.batch;
    // minibatch rows, whitened
    if (threadIdx.x < TS) {
        const int r = threadIdx.x, j = blockIdx.x * TS + r;
        long long idx = j;
        if (a.random_rows) {
            const lisa_smp::U4 q = lisa_smp::philox(a.round, 5u, a.iter, (uint32_t)(j >> 2), a.k0, a.k1);
            idx = (long long)(lisa_smp::unit(q.v[j & 3]) * (double)a.n);
            if (idx > a.n - 1) idx = a.n - 1;
        }
        sm.u[r * LU + FD] = 0.0f;
        whiten_row(a.data + idx * FD, a.mu, a.L, sm.u + r * LU);
    }
    __syncthreads();
    float ssum = 0.0f;  // lanes 0..15: the row's sum of s
    for (int c = 0; c < FC; c++) {
        load_coupling(sm, a.wb, a.w, c);
        for (int i = lane; i < 16 * LU; i += 32) st.ust[(c * TS + r0) * LU + i] = sm.u[r0 * LU + i];
        __syncthreads();
        net_forward(sm, sm.u, c, r0, lane);
        if (lane < 16) ssum += couple_row(sm, c, r0 + lane, false);
        __syncwarp();
        __syncthreads();
    }
    // loss and dL/dz = z / batch
    double lrow = 0.0;
    if (lane < 16) {
        const int rr = r0 + lane;
        float zz = 0.0f;
        for (int d = 0; d < FD; d++) {
            const float z = sm.u[rr * LU + d];
            zz += z * z;
            st.gv[rr * LU + d] = z * inv_n;
        }
        lrow = 0.5 * (double)zz + (double)ssum;
    }
    for (int o = 16; o > 0; o >>= 1) lrow += __shfl_xor_sync(0xffffffffu, lrow, o);
    if (lane == 0) st.lsum[warp] = lrow;
    __syncthreads();
    if (threadIdx.x == 0)
        atomicAdd(a.loss, (st.lsum[0] + st.lsum[1] + st.lsum[2] + st.lsum[3]) / (double)a.batch);
    for (int c = FC - 1; c >= 0; c--) {
        load_coupling(sm, a.wb, a.w, c);
        for (int i = threadIdx.x; i < FH; i += NTH) {
            st.db1[i] = 0.0f;
            st.db2[i] = 0.0f;
            if (i < N3) st.db3[i] = 0.0f;
        }
        for (int i = lane; i < 16 * LU; i += 32) sm.u[r0 * LU + i] = st.ust[(c * TS + r0) * LU + i];
        __syncthreads();
        net_forward(sm, sm.u, c, r0, lane);
        // dL/ds, dL/dt of the coupling, and dL/du through the affine map
        if (lane < 16) {
            const int rr = r0 + lane;
            for (int k = 0; k < LGO; k++) st.go[rr * LGO + k] = __float2bfloat16_rn(0.0f);
            for (int d = 0; d < FD; d++) {
                if (keep(c, d)) continue;
                const float th = tanhf(sm.o[rr * N3 + d] / kS);
                const float s = kS * th;
                const float e = expf(-s);
                const float v = (sm.u[rr * LU + d] - sm.o[rr * N3 + FD + d]) * e;
                const float gvd = st.gv[rr * LU + d];
                const float gs = (-gvd * v + inv_n) * (1.0f - th * th);
                const float gt = -gvd * e;
                st.go[rr * LGO + d] = __float2bfloat16_rn(gs);
                st.go[rr * LGO + FD + d] = __float2bfloat16_rn(gt);
                atomicAdd(&st.db3[d], gs);
                atomicAdd(&st.db3[FD + d], gt);
                st.gv[rr * LU + d] = gvd * e;
            }
        }
        __syncwarp();
        {  // dL/da2 = go W3, through the relu
            float acc[16][4];
            zero(acc);
            mma_nn<16, 2>(st.go + r0 * LGO, LGO, sm.w3, LH, acc, lane);
#pragma unroll
            for (int nt = 0; nt < 16; nt++) {
                const int col = nt * 8 + 2 * t;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int rr = r0 + g + 8 * h;
                    const float v0 = __bfloat162float(sm.a2[rr * LH + col]) > 0.0f ? acc[nt][2 * h] : 0.0f;
                    const float v1 = __bfloat162float(sm.a2[rr * LH + col + 1]) > 0.0f ? acc[nt][2 * h + 1] : 0.0f;
                    atomicAdd(&st.db2[col], v0);
                    atomicAdd(&st.db2[col + 1], v1);
                    *reinterpret_cast<uint32_t *>(st.gz2 + rr * LH + col) =
                        pk(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
                }
            }
        }
        __syncwarp();
        {  // dL/da1 = gz2 W2, through the relu
            float acc[16][4];
            zero(acc);
            mma_nn<16, 8>(st.gz2 + r0 * LH, LH, sm.w2, LH, acc, lane);
#pragma unroll
            for (int nt = 0; nt < 16; nt++) {
                const int col = nt * 8 + 2 * t;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int rr = r0 + g + 8 * h;
                    const float v0 = __bfloat162float(sm.a1[rr * LH + col]) > 0.0f ? acc[nt][2 * h] : 0.0f;
                    const float v1 = __bfloat162float(sm.a1[rr * LH + col + 1]) > 0.0f ? acc[nt][2 * h + 1] : 0.0f;
                    atomicAdd(&st.db1[col], v0);
                    atomicAdd(&st.db1[col + 1], v1);
                    *reinterpret_cast<uint32_t *>(st.gz1 + rr * LH + col) =
                        pk(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
                }
            }
        }
        __syncwarp();
        {  // dL/da0 = gz1 W1: reaches the kept coordinates of u
            float acc[2][4];
            zero(acc);
            mma_nn<2, 8>(st.gz1 + r0 * LH, LH, sm.w1, LW1, acc, lane);
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int col = nt * 8 + 2 * t + (j & 1), rr = r0 + g + 8 * (j >> 1);
                    if (col < FD && keep(c, col)) st.gv[rr * LU + col] += acc[nt][j];
                }
            }
        }
        __syncthreads();
        // weight gradients: contractions over the block's 64 samples
        float *gw = a.grad + (size_t)c * PC;
        {  // dW3 [22][128] = go^T a2: warp w takes columns 32w..32w+31
            for (int mt = 0; mt < 2; mt++) {
                float acc[4][4];
                zero(acc);
                mma_tn<4>(st.go, LGO, 16 * mt, sm.a2, LH, 32 * warp, acc, lane);
#pragma unroll
                for (int nt = 0; nt < 4; nt++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int m = 16 * mt + g + 8 * (j >> 1);
                        const int n = 32 * warp + nt * 8 + 2 * t + (j & 1);
                        if (m < FO) atomicAdd(gw + OW3 + m * FH + n, acc[nt][j]);
                    }
            }
        }
        {  // dW2 [128][128] = gz2^T a1: warp w takes rows 32w..32w+31
            for (int mt = 0; mt < 2; mt++)
                for (int nc = 0; nc < 2; nc++) {
                    float acc[8][4];
                    zero(acc);
                    mma_tn<8>(st.gz2, LH, 32 * warp + 16 * mt, sm.a1, LH, 64 * nc, acc, lane);
#pragma unroll
                    for (int nt = 0; nt < 8; nt++)
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const int m = 32 * warp + 16 * mt + g + 8 * (j >> 1);
                            const int n = 64 * nc + nt * 8 + 2 * t + (j & 1);
                            atomicAdd(gw + OW2 + m * FH + n, acc[nt][j]);
                        }
                }
        }
        {  // dW1 [128][11] = gz1^T a0
            for (int mt = 0; mt < 2; mt++) {
                float acc[2][4];
                zero(acc);
                mma_tn<2>(st.gz1, LH, 32 * warp + 16 * mt, sm.a0, LW1, 0, acc, lane);
#pragma unroll
                for (int nt = 0; nt < 2; nt++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int m = 32 * warp + 16 * mt + g + 8 * (j >> 1);
                        const int n = nt * 8 + 2 * t + (j & 1);
                        if (n < FD) atomicAdd(gw + OW1 + m * FD + n, acc[nt][j]);
                    }
            }
        }
        for (int i = threadIdx.x; i < FH; i += NTH) {
            atomicAdd(gw + OB1 + i, st.db1[i]);
            atomicAdd(gw + OB2 + i, st.db2[i]);
            if (i < FO) atomicAdd(gw + OB3 + i, st.db3[i]);
        }
        __syncthreads();
    }
}

// Adam on the FP32 master weights (Kingma & Ba 2015), then the bf16 copies
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, int n, float lr,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    if (!isfinite(gi)) gi = 0.0f;
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void pack_kernel(const float *w, bf16 *wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= FC * BC) return;
    const int c = i / BC, e = i % BC;
    const float *ws = w + (size_t)c * PC;
    float v = 0.0f;
    if (e < BW2) {
        const int r = e / K1, k = e % K1;
        v = k < FD ? ws[OW1 + r * FD + k] : 0.0f;
    } else if (e < BW3) {
        v = ws[OW2 + (e - BW2)];
    } else {
        const int r = (e - BW3) / FH, k = (e - BW3) % FH;
        v = r < FO ? ws[OW3 + r * FH + k] : 0.0f;
    }
    wb[i] = __float2bfloat16_rn(v);
}

// mean of each coordinate (one block per coordinate, FP64)
__global__ void mean_kernel(const double *x, long long n, double *mu) {
    __shared__ double red[256];
    const int d = blockIdx.x;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += x[i * FD + d];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu[d] = red[0] / (double)n;
}

// covariance entry (i, j), i >= j, one block each (population normalisation)
__global__ void cov_kernel(const double *x, long long n, const double *mu, double *cov) {
    __shared__ double red[256];
    int b = blockIdx.x, i = 0;
    while (b > i) {
        b -= i + 1;
        i++;
    }
    const int j = b;
    double s = 0.0;
    for (long long r = threadIdx.x; r < n; r += blockDim.x)
        s += (x[r * FD + i] - mu[i]) * (x[r * FD + j] - mu[j]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cov[i * FD + j] = red[0] / (double)n;
        cov[j * FD + i] = red[0] / (double)n;
    }
}

// Cholesky factor of the covariance, each pivot floored at 1e-12 of its diagonal entry
__global__ void cholesky_kernel(const double *cov, double *L) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < FD * FD; i++) L[i] = 0.0;
    for (int i = 0; i < FD; i++)
        for (int j = 0; j <= i; j++) {
            double acc = cov[i * FD + j];
            for (int k = 0; k < j; k++) acc -= L[i * FD + k] * L[j * FD + k];
            if (i == j) {
                const double cii = cov[i * FD + i];
                const double floor = cii > 0.0 ? 1e-12 * cii : 1e-300;
                L[i * FD + i] = sqrt(fmax(acc, floor));
            } else {
                L[i * FD + j] = acc / L[j * FD + j];
            }
        }
}

// ------------------------------------------------------------------ sampler step
// Independence proposals for the coldest temperature: y = flow(z) with z from Philox
// counters (step, 3, blk, w) by Box-Muller, and log q(x) - log q(y).
__global__ void __launch_bounds__(NTH) flow_propose_kernel(FlowView f, lisa_flowint::FStep a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemNet &sm = *reinterpret_cast<SmemNet *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, r0 = warp * 16;
    const int w0 = blockIdx.x * TS;
    const unsigned step = *a.step;
    __shared__ double zlat[TS * FD];
    __shared__ double qy[TS];
    // latent draws
    if (threadIdx.x < TS) {
        const int w = w0 + threadIdx.x;
        double nrm[12];
        for (int blk = 0; blk < 3; blk++) {
            const lisa_smp::U4 q = lisa_smp::philox(step, 3u, (uint32_t)blk, (uint32_t)w, a.k0, a.k1);
            for (int p = 0; p < 2; p++) {
                const double u1 = lisa_smp::unit(q.v[2 * p]), u2 = lisa_smp::unit(q.v[2 * p + 1]);
                const double r = sqrt(-2.0 * log(u1));
                double sn, cs;
                sincos(2.0 * lisa_smp::kPi * u2, &sn, &cs);
                nrm[4 * blk + 2 * p] = r * cs;
                nrm[4 * blk + 2 * p + 1] = r * sn;
            }
        }
        double zz = 0.0;
        for (int d = 0; d < FD; d++) {
            zlat[threadIdx.x * FD + d] = nrm[d];
            zz += nrm[d] * nrm[d];
        }
        qy[threadIdx.x] = -0.5 * zz - 0.5 * FD * kLog2Pi;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TS * LU; i += NTH) {
        const int r = i / LU, d = i % LU;
        sm.u[i] = d < FD ? (float)zlat[r * FD + d] : 0.0f;
    }
    __syncthreads();
    double lq = 0.0;
    for (int k = 0; k < FC; k++) {  // generate
        const int c = FC - 1 - k;
        load_coupling(sm, f.wb, f.w, c);
        __syncthreads();
        net_forward(sm, sm.u, c, r0, lane);
        if (lane < 16) lq -= (double)couple_row(sm, c, r0 + lane, true);
        __syncwarp();
        __syncthreads();
    }
    const double lsig = log_det_factor(f.L);
    if (lane < 16) {
        const int rr = r0 + lane, w = w0 + rr;
        if (w < a.W) {
            for (int d = 0; d < FD; d++) {
                double xv = f.mu[d];  // y = mu + L v
                for (int j = 0; j <= d; j++) xv += f.L[d * FD + j] * (double)sm.u[rr * LU + j];
                a.fy[(size_t)w * FD + d] = xv;
            }
            qy[rr] += lq - lsig;
        }
    }
    __syncthreads();
    // log q of the current walkers
    if (threadIdx.x < TS) {
        const int r = threadIdx.x, w = w0 + r;
        float *u = sm.u + r * LU;
        for (int d = 0; d < LU; d++) u[d] = 0.0f;
        if (w < a.W) whiten_row(a.x + (size_t)w * FD, f.mu, f.L, u);
    }
    __syncthreads();
    lq = 0.0;
    for (int c = 0; c < FC; c++) {
        load_coupling(sm, f.wb, f.w, c);
        __syncthreads();
        net_forward(sm, sm.u, c, r0, lane);
        if (lane < 16) lq -= (double)couple_row(sm, c, r0 + lane, false);
        __syncwarp();
        __syncthreads();
    }
    if (lane < 16) {
        const int rr = r0 + lane, w = w0 + rr;
        if (w < a.W) {
            double zz = 0.0;
            for (int d = 0; d < FD; d++) {
                const double v = sm.u[rr * LU + d];
                zz += v * v;
            }
            const double qx = -0.5 * zz - 0.5 * FD * kLog2Pi + lq - lsig;
            a.fq[w] = qx - qy[rr];
            double y[FD];
            for (int d = 0; d < FD; d++) y[d] = a.fy[(size_t)w * FD + d];
            const double py = lisa_smp::ln_prior(y, a.lo, a.hi);
            a.fpy[w] = py;
            if (a.target == LISA_TARGET_GAUSSIAN)
                a.fly[w] = lisa_smp::gauss_lnl(y, a.mean, a.sig);
            else if (isfinite(py))
                lisa_smp::to_physical(y, a.lisa_frame, a.t0, a.fpth + (size_t)w * FD);
            else
                lisa_smp::invalid_params(a.fpth + (size_t)w * FD);
        }
    }
}

// Metropolis-Hastings acceptance of Eq. (13) with the tempered likelihood of the
// coldest temperature and the prior
// log of the MH ratio of flow proposal w with ln L ly (Eq. (13) with the proposal density)
__device__ __forceinline__ double flow_log_ratio(const lisa_flowint::FStep &a, int w, double ly) {
    const double beta = a.betas[0], py = a.fpy[w];
    const double lt = beta > 0.0 ? __dmul_rn(beta, __dsub_rn(ly, a.lnl[w])) : 0.0;
    return __dadd_rn(__dadd_rn(lt, __dsub_rn(py, a.lnp[w])), a.fq[w]);
}

// Screened flow moves: with the first likelihood's ln L, a proposal whose log ratio falls
// below log u by more than beta margin is rejected here (a second likelihood within
// margin of the first would reject it too); every other one, accepted or undecided, is
// sent to the second likelihood, which decides it.  Proposals not sent on get a NaN
// mass, so the second likelihood spends no dense work on them.
__global__ void flow_screen_kernel(lisa_flowint::FStep a) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= a.W) return;
    const lisa_smp::U4 q = lisa_smp::philox(*a.step, 4u, 0u, (uint32_t)w, a.k0, a.k1);
    const double py = a.fpy[w];
    const double lr = flow_log_ratio(a, w, a.fly[w]);
    const double lu = log(lisa_smp::unit(q.v[0]));
    const bool send = isfinite(py) && !(lu >= lr + a.betas[0] * a.margin);
    a.fsent[w] = send ? 1 : 0;
    for (int d = 0; d < FD; d++)
        a.fpth2[(size_t)w * FD + d] = (send || d > 0) ? a.fpth[(size_t)w * FD + d] : NAN;
    if (send) atomicAdd(a.facc + 2, 1ULL);
}

__global__ void flow_accept_kernel(lisa_flowint::FStep a) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= a.W) return;
    if (*a.err) return;
    if ((a.like_err && *a.like_err) || (a.like_err2 && *a.like_err2)) {
        atomicOr(a.err, 1);
        return;
    }
    if (w == 0) atomicAdd(a.facc + 1, (unsigned long long)a.W);
    const lisa_smp::U4 q = lisa_smp::philox(*a.step, 4u, 0u, (uint32_t)w, a.k0, a.k1);
    if (a.margin > 0.0 && !a.fsent[w]) return;  // rejected by the screen
    const double beta = a.betas[0], py = a.fpy[w];
    const double ly = a.margin > 0.0 ? a.fly2[w] : a.fly[w];
    const double lt = beta > 0.0 ? __dmul_rn(beta, __dsub_rn(ly, a.lnl[w])) : 0.0;
    const double lr = __dadd_rn(__dadd_rn(lt, __dsub_rn(py, a.lnp[w])), a.fq[w]);
    if (isfinite(py) && log(lisa_smp::unit(q.v[0])) < lr) {
        for (int d = 0; d < FD; d++) a.x[(size_t)w * FD + d] = a.fy[(size_t)w * FD + d];
        a.lnl[w] = ly;
        a.lnp[w] = py;
        atomicAdd(a.facc, 1ULL);
    }
}

int eval_smem() { return (int)sizeof(SmemNet); }
int train_smem() { return (int)sizeof(SmemTrain); }

}  // namespace

// ------------------------------------------------------------------ host handle
struct lisa_flow {
    int device = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wb = nullptr;
    double *mu = nullptr, *L = nullptr, *cov = nullptr, *loss = nullptr;
    int loss_cap = 0, last_iters = 0;
    float *h_grad = nullptr;
    std::string err;
};

namespace {

lisa_status ffail(lisa_flow_t *f, lisa_status st, const std::string &m) {
    if (f) f->err = m;
    else lisa::set_thread_error(m);
    return st;
}

lisa_status fcuda(lisa_flow_t *f, cudaError_t e, const char *what) {
    return ffail(f, e == cudaErrorMemoryAllocation ? LISA_ERR_OOM : LISA_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define FCK(call, what)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fcuda(f, e_, what); \
    } while (0)

FlowView view(const lisa_flow_t *f) { return {f->w, f->wb, f->mu, f->L}; }

cudaError_t set_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(flow_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, eval_smem());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flow_propose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, eval_smem());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flow_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, train_smem());
    return e;
}

lisa_status pack(lisa_flow_t *f, cudaStream_t s) {
    pack_kernel<<<(FC * BC + 255) / 256, 256, 0, s>>>(f->w, f->wb);
    FCK(cudaGetLastError(), "pack kernel launch");
    return LISA_OK;
}

lisa_status ensure_loss(lisa_flow_t *f, int iters) {
    if (iters <= f->loss_cap) return LISA_OK;
    if (f->loss) cudaFree(f->loss);
    f->loss = nullptr;
    FCK(cudaMalloc(&f->loss, sizeof(double) * iters), "device allocation (loss history)");
    f->loss_cap = iters;
    return LISA_OK;
}

lisa_status train_iters(lisa_flow_t *f, const double *d_data, int64_t n, int iters, int batch,
                        double lr, uint64_t seed, uint32_t round, cudaStream_t s, int random_rows) {
    lisa_status st = ensure_loss(f, iters);
    if (st != LISA_OK) return st;
    FCK(cudaMemsetAsync(f->loss, 0, sizeof(double) * iters, s), "cudaMemsetAsync");
    for (int it = 0; it < iters; it++) {
        FCK(cudaMemsetAsync(f->g, 0, sizeof(float) * NP, s), "cudaMemsetAsync");
        TrainArgs a;
        a.w = f->w;
        a.wb = f->wb;
        a.grad = f->g;
        a.mu = f->mu;
        a.L = f->L;
        a.data = d_data;
        a.n = n;
        a.batch = batch;
        a.k0 = (uint32_t)seed;
        a.k1 = (uint32_t)(seed >> 32);
        a.round = round;
        a.iter = (uint32_t)it;
        a.random_rows = random_rows;
        a.loss = f->loss + it;
        flow_train_kernel<<<batch / TS, NTH, train_smem(), s>>>(a);
        FCK(cudaGetLastError(), "flow training kernel launch");
        if (lr > 0.0) {
            const int t = it + 1;
            adam_kernel<<<(NP + 255) / 256, 256, 0, s>>>(f->w, f->g, f->m, f->v, NP, (float)lr,
                                                         (float)(1.0 - std::pow(0.9, t)),
                                                         (float)(1.0 - std::pow(0.999, t)));
            FCK(cudaGetLastError(), "Adam kernel launch");
            st = pack(f, s);
            if (st != LISA_OK) return st;
        }
    }
    f->last_iters = iters;
    return LISA_OK;
}

}  // namespace

namespace lisa_flowint {

cudaError_t launch_flow_propose(lisa_flow_t *f, const FStep &a, cudaStream_t s) {
    flow_propose_kernel<<<(a.W + TS - 1) / TS, NTH, eval_smem(), s>>>(view(f), a);
    return cudaGetLastError();
}

cudaError_t launch_flow_screen(const FStep &a, cudaStream_t s) {
    flow_screen_kernel<<<(a.W + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flow_accept(const FStep &a, cudaStream_t s) {
    flow_accept_kernel<<<(a.W + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

lisa_status flow_train_async(lisa_flow_t *f, const double *d_data, int64_t n, int iters,
                             int batch, double lr, uint64_t seed, uint32_t round, cudaStream_t s) {
    mean_kernel<<<FD, 256, 0, s>>>(d_data, n, f->mu);
    cov_kernel<<<FD * (FD + 1) / 2, 256, 0, s>>>(d_data, n, f->mu, f->cov);
    cholesky_kernel<<<1, 32, 0, s>>>(f->cov, f->L);
    FCK(cudaGetLastError(), "whitening kernel launch");
    FCK(cudaMemsetAsync(f->m, 0, sizeof(float) * NP, s), "cudaMemsetAsync");
    FCK(cudaMemsetAsync(f->v, 0, sizeof(float) * NP, s), "cudaMemsetAsync");
    return train_iters(f, d_data, n, iters, batch, lr, seed, round, s, 1);
}

lisa_status flow_last_loss(lisa_flow_t *f, double *loss, cudaStream_t s) {
    if (f->last_iters < 1) {
        *loss = NAN;
        return LISA_OK;
    }
    FCK(cudaMemcpyAsync(loss, f->loss + f->last_iters - 1, sizeof(double), cudaMemcpyDeviceToHost, s),
        "loss download");
    FCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return LISA_OK;
}

}  // namespace lisa_flowint

extern "C" {

lisa_status lisa_flow_create(uint64_t seed, lisa_flow_t **out) {
    lisa::set_thread_error("");
    if (!out) return ffail(nullptr, LISA_ERR_ARG, "NULL output pointer");
    *out = nullptr;
    lisa_flow_t *f = new lisa_flow();
    lisa_status st = LISA_OK;
    do {
        cudaError_t e = cudaGetDevice(&f->device);
        if (e == cudaSuccess) e = set_smem_limits();
        if (e == cudaSuccess) e = cudaMalloc(&f->w, sizeof(float) * NP);
        if (e == cudaSuccess) e = cudaMalloc(&f->g, sizeof(float) * NP);
        if (e == cudaSuccess) e = cudaMalloc(&f->m, sizeof(float) * NP);
        if (e == cudaSuccess) e = cudaMalloc(&f->v, sizeof(float) * NP);
        if (e == cudaSuccess) e = cudaMalloc(&f->wb, sizeof(bf16) * FC * BC);
        if (e == cudaSuccess) e = cudaMalloc(&f->mu, sizeof(double) * FD);
        if (e == cudaSuccess) e = cudaMalloc(&f->L, sizeof(double) * FD * FD);
        if (e == cudaSuccess) e = cudaMalloc(&f->cov, sizeof(double) * FD * FD);
        if (e == cudaSuccess) e = cudaMallocHost(&f->h_grad, sizeof(float) * NP);
        if (e != cudaSuccess) {
            st = fcuda(f, e, "flow allocation");
            break;
        }
        // hidden layers uniform in +-sqrt(6 / fan_in) from Philox, zero output layer
        std::vector<float> w(NP, 0.0f);
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        for (int c = 0; c < FC; c++) {
            float *ws = w.data() + (size_t)c * PC;
            const double lim1 = std::sqrt(6.0 / FD), lim2 = std::sqrt(6.0 / FH);
            for (int i = 0; i < FH * FD; i++) {
                const lisa_smp::U4 q = lisa_smp::philox((uint32_t)c, 1u, (uint32_t)(i >> 2), 0x1Fu, k0, k1);
                ws[OW1 + i] = (float)(lim1 * (2.0 * lisa_smp::unit(q.v[i & 3]) - 1.0));
            }
            for (int i = 0; i < FH * FH; i++) {
                const lisa_smp::U4 q = lisa_smp::philox((uint32_t)c, 2u, (uint32_t)(i >> 2), 0x1Fu, k0, k1);
                ws[OW2 + i] = (float)(lim2 * (2.0 * lisa_smp::unit(q.v[i & 3]) - 1.0));
            }
        }
        st = lisa_flow_set_weights(f, w.data());
        if (st != LISA_OK) break;
        std::vector<double> mu(FD, 0.0), L(FD * FD, 0.0);
        for (int d = 0; d < FD; d++) L[d * FD + d] = 1.0;
        st = lisa_flow_set_whitening(f, mu.data(), L.data());
    } while (0);
    if (st != LISA_OK) {
        lisa::set_thread_error(f->err);
        lisa_flow_destroy(f);
        return st;
    }
    *out = f;
    return LISA_OK;
}

void lisa_flow_destroy(lisa_flow_t *f) {
    if (!f) return;
    cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)f->w, (void *)f->g, (void *)f->m, (void *)f->v, (void *)f->wb,
                    (void *)f->mu, (void *)f->L, (void *)f->cov, (void *)f->loss})
        if (p) cudaFree(p);
    if (f->h_grad) cudaFreeHost(f->h_grad);
    delete f;
}

const char *lisa_flow_last_error(const lisa_flow_t *f) { return f ? f->err.c_str() : lisa::thread_error(); }

lisa_status lisa_flow_set_weights(lisa_flow_t *f, const float *w) {
    if (!f) return LISA_ERR_ARG;
    if (!w) return ffail(f, LISA_ERR_ARG, "NULL weights");
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    FCK(cudaMemcpy(f->w, w, sizeof(float) * NP, cudaMemcpyHostToDevice), "weight upload");
    lisa_status st = pack(f, nullptr);
    if (st != LISA_OK) return st;
    FCK(cudaDeviceSynchronize(), "weight packing");
    return LISA_OK;
}

lisa_status lisa_flow_get_weights(lisa_flow_t *f, float *w) {
    if (!f) return LISA_ERR_ARG;
    if (!w) return ffail(f, LISA_ERR_ARG, "NULL weights");
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    FCK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    FCK(cudaMemcpy(w, f->w, sizeof(float) * NP, cudaMemcpyDeviceToHost), "weight download");
    return LISA_OK;
}

lisa_status lisa_flow_set_whitening(lisa_flow_t *f, const double *mu, const double *L) {
    if (!f) return LISA_ERR_ARG;
    if (!mu || !L) return ffail(f, LISA_ERR_ARG, "NULL whitening");
    double Lc[FD * FD];
    for (int i = 0; i < FD; i++) {
        if (!std::isfinite(mu[i])) return ffail(f, LISA_ERR_ARG, "mu must be finite");
        for (int j = 0; j < FD; j++) {
            const double v = j <= i ? L[i * FD + j] : 0.0;
            if (!std::isfinite(v)) return ffail(f, LISA_ERR_ARG, "L must be finite");
            Lc[i * FD + j] = v;
        }
        if (!(Lc[i * FD + i] > 0.0)) return ffail(f, LISA_ERR_ARG, "L needs a positive diagonal");
    }
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    FCK(cudaMemcpy(f->mu, mu, sizeof(double) * FD, cudaMemcpyHostToDevice), "upload");
    FCK(cudaMemcpy(f->L, Lc, sizeof(double) * FD * FD, cudaMemcpyHostToDevice), "upload");
    return LISA_OK;
}

lisa_status lisa_flow_get_whitening(lisa_flow_t *f, double *mu, double *L) {
    if (!f) return LISA_ERR_ARG;
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    FCK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    if (mu) FCK(cudaMemcpy(mu, f->mu, sizeof(double) * FD, cudaMemcpyDeviceToHost), "download");
    if (L) FCK(cudaMemcpy(L, f->L, sizeof(double) * FD * FD, cudaMemcpyDeviceToHost), "download");
    return LISA_OK;
}

static lisa_status eval(lisa_flow_t *f, const double *in, int n, int gen, double *out,
                        double *logq, void *stream) {
    if (!f) return LISA_ERR_ARG;
    if (!in || !logq || n < 0 || (gen && !out)) return ffail(f, LISA_ERR_ARG, "NULL pointer or n < 0");
    if (n == 0) return LISA_OK;
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    flow_eval_kernel<<<(n + TS - 1) / TS, NTH, eval_smem(), (cudaStream_t)stream>>>(view(f), in, n, gen, out, logq);
    FCK(cudaGetLastError(), "flow kernel launch");
    return LISA_OK;
}

lisa_status lisa_flow_normalize(lisa_flow_t *f, const double *d_x, int n, double *d_z,
                                double *d_logq, void *stream) {
    return eval(f, d_x, n, 0, d_z, d_logq, stream);
}

lisa_status lisa_flow_generate(lisa_flow_t *f, const double *d_z, int n, double *d_x,
                               double *d_logq, void *stream) {
    return eval(f, d_z, n, 1, d_x, d_logq, stream);
}

lisa_status lisa_flow_gradients(lisa_flow_t *f, const double *d_x, int n, float *grad,
                                double *loss, void *stream) {
    if (!f) return LISA_ERR_ARG;
    if (!d_x || n < TS || n % TS) return ffail(f, LISA_ERR_ARG, "n must be a positive multiple of 64");
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    lisa_status st = train_iters(f, d_x, n, 1, n, 0.0, 0, 0, s, 0);
    if (st != LISA_OK) return st;
    if (grad) FCK(cudaMemcpyAsync(f->h_grad, f->g, sizeof(float) * NP, cudaMemcpyDeviceToHost, s), "download");
    double l = 0.0;
    FCK(cudaMemcpyAsync(&l, f->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "download");
    FCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (grad) std::memcpy(grad, f->h_grad, sizeof(float) * NP);
    if (loss) *loss = l;
    return LISA_OK;
}

lisa_status lisa_flow_train(lisa_flow_t *f, const double *d_data, int64_t n, int iters,
                            int batch, double lr, uint64_t seed, uint32_t round, double *loss,
                            void *stream) {
    if (!f) return LISA_ERR_ARG;
    if (!d_data || n < 2 || iters < 1 || batch < TS || batch % TS || !(lr > 0.0))
        return ffail(f, LISA_ERR_ARG, "need data (n >= 2), iters >= 1, batch a multiple of 64, lr > 0");
    FCK(cudaSetDevice(f->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    lisa_status st = lisa_flowint::flow_train_async(f, d_data, n, iters, batch, lr, seed, round, s);
    if (st != LISA_OK) return st;
    if (loss) FCK(cudaMemcpyAsync(loss, f->loss, sizeof(double) * iters, cudaMemcpyDeviceToHost, s), "download");
    FCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return LISA_OK;
}

}  // extern "C"
