// Dense CP backup: E_a[V] = sum_r lambda_{a,r} (V x_1 U_{a,r,1} ... x_D U_{a,r,D})
// (the CP form of the background section applied to each action's
// transition tensor, mode products as in Kolda and Bader), followed by
// Eq. 1's + R, x gamma and max over actions, and the residual.
//
// SIMT path: one tiled mode-product kernel per (action, rank, mode). The
// mode-d product of X (viewed as L x N_d x Rt, Rt = prod of the later mode
// sizes) with U is the batched matrix product Y[l, i, r] = sum_j U[i, j]
// X[l, j, r]; columns c = (l, r) are tiled 64 at a time, rows i 64 at a
// time, the contraction j 16 at a time through shared memory. The last
// mode's kernel carries the fused epilogue: lambda-weighted accumulation
// over ranks, Q = R + gamma E, running max/argmax over actions and, after
// the last action, V', the policy and the max |V' - V| residual.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace cpmdp {

enum DenseMode : int { DM_VI = 0, DM_EVAL = 1, DM_IMPROVE = 2, DM_GREEDY = 3, DM_STORE_E = 4 };

struct Epilogue {
    int enabled;           // 0: plain store of Y (intermediate mode)
    int first_rank, last_rank, first_action, last_action;
    int action;
    int mode;
    double lambda, gamma, margin;
    void *E;               // rank accumulator (TA)
    void *best;            // running max over actions (TA)
    uint8_t *arg;          // running argmax
    void *qold;            // IMPROVE: Q of the current policy's action (TA)
    const void *R;         // rewards (TA)
    const void *Vin;       // input values (for the residual)
    void *Vout;            // output values (nullptr: not written)
    uint8_t *pi;           // policy output / input (EVAL, IMPROVE)
    unsigned long long *res;   // residual (bits of a non-negative double)
    unsigned *changed;     // policy changes (IMPROVE)
};

constexpr int TI = 64, TC = 64, TK = 16;

// Y = X x_d U for X viewed as (L, N, Rt). 256 threads, 4x4 outputs each.
template <typename T>
__global__ void __launch_bounds__(256) mode_product_kernel(const T *__restrict__ X, T *__restrict__ Y,
                                                           const T *__restrict__ U, int N, long long Rt,
                                                           long long ncols, Epilogue ep) {
    __shared__ T sU[TK][TI + 1];   // sU[jj][ii] = U[i0+ii, j0+jj]
    __shared__ T sX[TK][TC + 1];   // sX[jj][cc] = X[addr(j0+jj, c0+cc)]
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int i0 = blockIdx.y * TI;
    const long long c0 = (long long)blockIdx.x * TC;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0;
    // The columns this thread loads are the same in every K step: their
    // offsets (l N Rt + r for column c = l Rt + r) are computed once, with no
    // 64-bit division inside the loop. Rt > 1: one column (tid % TC), rows
    // tid / TC + 4 m; Rt == 1: rows tid % TK, columns tid / TK + 16 m.
    constexpr int kLd = TK * TC / 256;   // X elements a thread loads per K step
    long long xoff[kLd];
    bool xok[kLd];
#pragma unroll
    for (int m = 0; m < kLd; m++) {
        const int cc = Rt == 1 ? tid / TK + (256 / TK) * m : tid % TC;
        const long long c = c0 + cc;
        xok[m] = c < ncols;
        if (Rt == 1) {
            xoff[m] = c * N;
        } else {
            const long long l = c / Rt, r = c - l * Rt;
            xoff[m] = l * N * Rt + r;
        }
        if (Rt != 1) break;   // one column: xoff[0]
    }

    for (int j0 = 0; j0 < N; j0 += TK) {
        // U tile: 64 rows x 16 columns, loaded along j
        for (int e = tid; e < TI * TK; e += 256) {
            const int ii = e / TK, jj = e % TK;
            const int i = i0 + ii, j = j0 + jj;
            sU[jj][ii] = (i < N && j < N) ? U[(long long)i * N + j] : (T)0;
        }
        // X tile: 16 x 64; coalesce along r when Rt > 1, along j when Rt == 1
#pragma unroll
        for (int m = 0; m < kLd; m++) {
            const int jj = Rt == 1 ? tid % TK : tid / TC + (256 / TC) * m;
            const int cc = Rt == 1 ? tid / TK + (256 / TK) * m : tid % TC;
            const int j = j0 + jj;
            const int mi = Rt == 1 ? m : 0;
            T v = 0;
            if (j < N && xok[mi]) v = X[xoff[mi] + (long long)j * (Rt == 1 ? 1 : Rt)];
            sX[jj][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < TK; jj++) {
            T u[4], x[4];
#pragma unroll
            for (int a = 0; a < 4; a++) u[a] = sU[jj][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; b++) x[b] = sX[jj][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] += u[a] * x[b];
        }
        __syncthreads();
    }

    double local_res = 0.0;
    unsigned local_chg = 0;
    long long sbase[4];   // state of (i = 0, column c): l N Rt + r
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const long long c = c0 + tx + 16 * b;
        const long long l = Rt == 1 ? c : c / Rt, r = c - l * Rt;
        sbase[b] = l * N * Rt + r;
    }
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = i0 + ty + 16 * a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const long long c = c0 + tx + 16 * b;
            if (c >= ncols) continue;
            const long long s = sbase[b] + (long long)i * Rt;
            if (!ep.enabled) { Y[s] = acc[a][b]; continue; }
            T *E = (T *)ep.E;
            const T e = (ep.first_rank ? (T)0 : E[s]) + (T)ep.lambda * acc[a][b];
            if (!ep.last_rank) { E[s] = e; continue; }
            if (ep.mode == DM_STORE_E) {
                // E_a in the tensor-core pass-B layout (64^4): [a][(i3,i4)][(i1,i2)]
                ((T *)ep.Vout)[(long long)ep.action * ncols * N + (s % 4096) * 4096 + s / 4096] = e;
                continue;
            }
            const T q = ((const T *)ep.R)[s] + (T)ep.gamma * e;
            T *best = (T *)ep.best;
            T b0;
            int arg;
            if (ep.mode == DM_EVAL) {
                // keep the value of the fixed action pi(s)
                b0 = ep.first_action ? q : best[s];
                if (ep.pi[s] == ep.action) b0 = q;
                arg = 0;
            } else if (ep.first_action) {
                b0 = q; arg = 0;
            } else {
                b0 = best[s]; arg = ep.arg[s];
                if (q > b0) { b0 = q; arg = ep.action; }
            }
            if (ep.mode == DM_IMPROVE && ep.pi[s] == ep.action) ((T *)ep.qold)[s] = q;
            if (!ep.last_action) {
                best[s] = b0;
                if (ep.mode != DM_EVAL) ep.arg[s] = (uint8_t)arg;
                continue;
            }
            const T vin = ((const T *)ep.Vin)[s];
            if (ep.mode == DM_VI || ep.mode == DM_EVAL) {
                if (ep.Vout) ((T *)ep.Vout)[s] = b0;
                if (ep.pi && ep.mode == DM_VI) ep.pi[s] = (uint8_t)arg;
                local_res = fmax(local_res, fabs((double)b0 - (double)vin));
            } else if (ep.mode == DM_GREEDY) {
                ep.pi[s] = (uint8_t)arg;
            } else {  // improve
                const T qold = ((const T *)ep.qold)[s];
                const T thr = (T)ep.margin * ((T)1 + (qold < 0 ? -qold : qold));
                if ((int)ep.pi[s] != arg && b0 > qold + thr) { ep.pi[s] = (uint8_t)arg; local_chg++; }
            }
        }
    }
    if (ep.enabled && ep.last_rank && ep.last_action && ep.mode != DM_STORE_E) {
        __shared__ double shd[8];
        __shared__ unsigned shc[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            local_res = fmax(local_res, __shfl_xor_sync(0xFFFFFFFFu, local_res, o));
            local_chg += __shfl_xor_sync(0xFFFFFFFFu, local_chg, o);
        }
        if ((tid & 31) == 0) { shd[tid >> 5] = local_res; shc[tid >> 5] = local_chg; }
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            unsigned c = 0;
            for (int w = 0; w < 8; w++) { m = fmax(m, shd[w]); c += shc[w]; }
            if (ep.res && m > 0.0) atomicMax(ep.res, (unsigned long long)__double_as_longlong(m));
            if (ep.changed && c) atomicAdd(ep.changed, c);
        }
    }
}

cpmdp_status dense_prepare(Factors &F) {
    const size_t nf = F.dense_factors.size();
    std::vector<float> u32(nf);
    for (size_t i = 0; i < nf; i++) u32[i] = (float)F.dense_factors[i];
    CPMDP_CUDA(cudaMalloc(&F.d_U32, nf * sizeof(float)));
    CPMDP_CUDA(cudaMalloc(&F.d_U64, nf * sizeof(double)));
    CPMDP_CUDA(cudaMemcpy(F.d_U32, u32.data(), nf * sizeof(float), cudaMemcpyHostToDevice));
    CPMDP_CUDA(cudaMemcpy(F.d_U64, F.dense_factors.data(), nf * sizeof(double), cudaMemcpyHostToDevice));
    const size_t S = (size_t)F.nstates;
    // chain ping-pong (2), rank accumulator, running best, Q of the current
    // action: 5 x |S| doubles; argmax |S| bytes
    F.dense_work_bytes = 5 * S * sizeof(double) + S + 256;
    CPMDP_CUDA(cudaMalloc(&F.d_dense_work, F.dense_work_bytes));
    return CPMDP_OK;
}

template <typename T>
static cpmdp_status dense_sweep(const Factors &F, const T *Vin, T *Vout, uint8_t *pi, int mode,
                                double margin, unsigned long long *res, unsigned *chg, cudaStream_t st) {
    const size_t S = (size_t)F.nstates;
    T *work = (T *)F.d_dense_work;
    T *buf0 = work, *buf1 = work + S, *E = work + 2 * S, *best = work + 3 * S, *qold = work + 4 * S;
    uint8_t *arg = (uint8_t *)(work + 5 * S);
    const T *U = std::is_same<T, double>::value ? (const T *)F.d_U64 : (const T *)F.d_U32;
    const T *R = std::is_same<T, double>::value ? (const T *)F.d_R64 : (const T *)F.d_R32;
    const int D = F.ndim;
    for (int a = 0; a < F.nactions; a++) {
        for (int r = 0; r < F.rank; r++) {
            const T *X = Vin;
            for (int d = 0; d < D; d++) {
                const int N = (int)F.shape[d];
                long long Rt = 1;
                for (int e = d + 1; e < D; e++) Rt *= F.shape[e];
                const long long ncols = (long long)S / N;
                const T *Ud = U + F.factor_off[((size_t)a * F.rank + r) * D + d];
                Epilogue ep;
                memset(&ep, 0, sizeof(ep));
                T *Y = (d % 2 == 0) ? buf0 : buf1;
                if (d == D - 1) {
                    ep.enabled = 1;
                    ep.first_rank = r == 0;
                    ep.last_rank = r == F.rank - 1;
                    ep.first_action = a == 0;
                    ep.last_action = a == F.nactions - 1;
                    ep.action = a;
                    ep.mode = mode;
                    ep.lambda = F.lambda[(size_t)a * F.rank + r];
                    ep.gamma = F.gamma;
                    ep.margin = margin;
                    ep.E = E;
                    ep.best = best;
                    ep.arg = arg;
                    ep.qold = qold;
                    ep.R = R;
                    ep.Vin = Vin;
                    ep.Vout = Vout;
                    ep.pi = pi;
                    ep.res = res;
                    ep.changed = chg;
                    Y = nullptr;
                }
                dim3 grid((unsigned)((ncols + TC - 1) / TC), (unsigned)((N + TI - 1) / TI));
                mode_product_kernel<T><<<grid, 256, 0, st>>>(X, Y, Ud, N, Rt, ncols, ep);
                X = Y;
            }
        }
    }
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status dense_store_expectation(const Factors &F, const float *V, float *EB, cudaStream_t st) {
    return dense_sweep<float>(F, V, EB, nullptr, DM_STORE_E, 0.0, nullptr, nullptr, st);
}

__global__ void widen_kernel(const float *__restrict__ x, double *__restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// FP64 backup of a float value tensor: certified residual and FP64 argmax.
cpmdp_status dense_certify(const Factors &F, const float *V, uint8_t *pi, double *res, cudaStream_t st) {
    Factors &Fm = const_cast<Factors &>(F);
    if (!Fm.d_Vd) CPMDP_CUDA(cudaMalloc(&Fm.d_Vd, (size_t)F.nstates * sizeof(double)));
    widen_kernel<<<1024, 256, 0, st>>>(V, Fm.d_Vd, F.nstates);
    CPMDP_CUDA(cudaGetLastError());
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    return dense_sweep<double>(F, Fm.d_Vd, nullptr, pi, DM_VI, 0.0, rb, nullptr, st);
}

cpmdp_status dense_backup(const Factors &F, cpmdp_precision prec, const void *Vin, void *Vout, uint8_t *pi,
                          double *res, cudaStream_t st) {
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    if (rb) CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    if (prec == CPMDP_F64)
        return dense_sweep<double>(F, (const double *)Vin, (double *)Vout, pi, DM_VI, 0.0, rb, nullptr, st);
    if (prec == CPMDP_F32)
        return dense_sweep<float>(F, (const float *)Vin, (float *)Vout, pi, DM_VI, 0.0, rb, nullptr, st);
    return dense_tc_backup(F, (const float *)Vin, (float *)Vout, pi, res, st);
}

// Value / policy iteration for dense models: each sweep is A*R*D launches
// of milliseconds of work, so the loop runs on the host and reads the
// residual (8 bytes) back once per sweep.
// ---------------------------------------------------------------------------
// The SIMT loops as one CUDA graph launch each (conditional nodes; the same
// sweeps and stop rules as a host-driven loop, no residual read back per
// sweep). Value iteration: WHILE { sweep V -> W, control, IF(second: sweep
// W -> V, control) }, IF(odd count: copy W -> V), greedy policy. Policy
// iteration: greedy start, WHILE(round) { start, WHILE(eval) { evaluation
// sweeps as above }, IF(odd: copy), improvement sweep, round end }.

// After value-iteration sweep `step` (0: V -> W, 1: W -> V).
__global__ void simt_vi_ctl_kernel(DensePiCtl *c, unsigned long long *res_slot, double tol, int max_iter,
                                   double *trace, int step, cudaGraphConditionalHandle h_loop,
                                   cudaGraphConditionalHandle h_second) {
    double r;
    memcpy(&r, res_slot, sizeof(r));
    *res_slot = 0ull;
    if (trace) trace[c->total] = r;
    c->total++;
    c->res = r;
    c->which = step == 0 ? 1 : 0;
    if (r < tol) {
        c->conv = 1;
        c->stop = 1;
    } else if (c->total >= max_iter) {
        c->stop = 1;
    }
    if (step == 0) cudaGraphSetConditional(h_second, c->stop ? 0u : 1u);
    cudaGraphSetConditional(h_loop, c->stop ? 0u : 1u);
}

template <typename T>
static cpmdp_status record_simt(Factors &F, bool pim, T *V, uint8_t *pi, const SolveOpts &o, cudaGraph_t *out) {
    T *W = (T *)F.d_scratch;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    unsigned *cb = &F.d_ctrl->changed_slot[0];
    const double margin = std::is_same<T, double>::value ? 1e-12 : 1e-6;
    DensePiCtl *c = reinterpret_cast<DensePiCtl *>(F.d_dense_loop);
    const int *err = F.d_tc_err;
    cudaGraph_t G = nullptr;
    cudaStream_t cap = nullptr;
    cpmdp_status s = CPMDP_OK;
    cudaError_t e = cudaGraphCreate(&G, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraphConditionalHandle h_outer = 0, h_eval = 0, h_second = 0, h_odd = 0;
    cudaGraph_t lbody = nullptr, sbody = nullptr, obody = nullptr, rbody = nullptr;
    cudaGraph_t host = nullptr;   // graph holding the evaluation WHILE and the odd-count copy
    cudaGraphNode_t n_outer, n_loop, n_odd;
    std::vector<cudaGraphNode_t> leaves;
    auto capture = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, auto &&fn) -> cpmdp_status {
        cudaError_t ce = cudaStreamBeginCaptureToGraph(cap, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                                       deps.size(), cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return cuda_fail(ce, "begin capture");
        cpmdp_status cs = fn();
        cudaGraph_t gg = g;
        ce = cudaStreamEndCapture(cap, &gg);
        if (cs != CPMDP_OK) return cs;
        if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
        return CPMDP_OK;
    };
    auto launched = [&](const char *what) -> cpmdp_status {
        cudaError_t ce = cudaGetLastError();
        return ce == cudaSuccess ? CPMDP_OK : cuda_fail(ce, what);
    };
    // one sweep from `in` to `outv` with its residual, then the step's control kernel
    auto sweep_ctl = [&](T *in, T *outv, int step) -> cpmdp_status {
        cudaError_t ce = cudaMemsetAsync(rb, 0, sizeof(*rb), cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "memset");
        cpmdp_status cs = dense_sweep<T>(F, in, outv, pi, pim ? DM_EVAL : DM_VI, margin, rb, nullptr, cap);
        if (cs != CPMDP_OK) return cs;
        if (pim) pi_eval_ctl_kernel<<<1, 1, 0, cap>>>(c, rb, err, o.eval_tol, step, 0, h_eval, 0, h_second);
        else simt_vi_ctl_kernel<<<1, 1, 0, cap>>>(c, rb, o.tol, o.max_iter, o.trace, step, h_eval, h_second);
        return launched("control kernel");
    };
    if (e != cudaSuccess) { s = cuda_fail(e, "graph setup"); goto done; }
    if (pim) {
        // root: greedy start, stop test, WHILE(round)
        if ((e = cudaGraphConditionalHandleCreate(&h_outer, G, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
        if ((s = capture(G, {}, [&]() -> cpmdp_status {
                 cpmdp_status cs = dense_sweep<T>(F, V, nullptr, pi, DM_GREEDY, margin, nullptr, nullptr, cap);
                 if (cs != CPMDP_OK) return cs;
                 pi_init_kernel<<<1, 1, 0, cap>>>(c, err, o.max_rounds, h_outer);
                 return launched("init kernel");
             })) != CPMDP_OK)
            goto done;
        if ((e = graph_leaves(G, leaves)) != cudaSuccess) goto fail;
        if ((e = add_conditional(G, leaves, h_outer, cudaGraphCondTypeWhile, &n_outer, &rbody)) != cudaSuccess) goto fail;
        host = rbody;
        if ((e = cudaGraphConditionalHandleCreate(&h_eval, host, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
        if ((s = capture(host, {}, [&]() -> cpmdp_status {
                 pi_round_start_kernel<<<1, 1, 0, cap>>>(c, o.partial_eval, o.max_eval_iter, h_eval);
                 return launched("round start kernel");
             })) != CPMDP_OK)
            goto done;
    } else {
        host = G;
        if ((e = cudaGraphConditionalHandleCreate(&h_eval, host, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
        if ((s = capture(host, {}, [&]() -> cpmdp_status {
                 pi_init_kernel<<<1, 1, 0, cap>>>(c, err, o.max_iter, h_eval);
                 return launched("init kernel");
             })) != CPMDP_OK)
            goto done;
    }
    // the sweep loop, then IF(odd count: copy W -> V)
    if ((e = cudaGraphConditionalHandleCreate(&h_odd, host, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = graph_leaves(host, leaves)) != cudaSuccess) goto fail;
    if ((e = add_conditional(host, leaves, h_eval, cudaGraphCondTypeWhile, &n_loop, &lbody)) != cudaSuccess) goto fail;
    if ((s = capture(host, {n_loop}, [&]() -> cpmdp_status {
             pi_after_eval_kernel<<<1, 1, 0, cap>>>(c, h_odd);
             return launched("after-loop kernel");
         })) != CPMDP_OK)
        goto done;
    if ((e = graph_leaves(host, leaves)) != cudaSuccess) goto fail;
    if ((e = add_conditional(host, leaves, h_odd, cudaGraphCondTypeIf, &n_odd, &obody)) != cudaSuccess) goto fail;
    if ((s = capture(obody, {}, [&]() -> cpmdp_status {
             cudaError_t ce = cudaMemcpyAsync(V, W, sizeof(T) * F.nstates, cudaMemcpyDeviceToDevice, cap);
             return ce == cudaSuccess ? CPMDP_OK : cuda_fail(ce, "iterate copy");
         })) != CPMDP_OK)
        goto done;
    if (pim) {
        // improvement at the evaluated values, then the round's stop rules
        if ((s = capture(host, {n_odd}, [&]() -> cpmdp_status {
                 cudaError_t ce = cudaMemsetAsync(cb, 0, sizeof(*cb), cap);
                 if (ce != cudaSuccess) return cuda_fail(ce, "memset");
                 cpmdp_status cs = dense_sweep<T>(F, V, nullptr, pi, DM_IMPROVE, margin, nullptr, cb, cap);
                 if (cs != CPMDP_OK) return cs;
                 pi_round_end_kernel<<<1, 1, 0, cap>>>(c, cb, err, o.max_rounds, h_outer);
                 return launched("round end kernel");
             })) != CPMDP_OK)
            goto done;
    } else if (pi) {
        // greedy policy of the returned values
        if ((s = capture(host, {n_odd}, [&]() -> cpmdp_status {
                 return dense_sweep<T>(F, V, nullptr, pi, DM_GREEDY, margin, nullptr, nullptr, cap);
             })) != CPMDP_OK)
            goto done;
    }
    // loop body: sweep V -> W, control, IF(second: sweep W -> V, control)
    if ((e = cudaGraphConditionalHandleCreate(&h_second, lbody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((s = capture(lbody, {}, [&] { return sweep_ctl(V, W, 0); })) != CPMDP_OK) goto done;
    {
        cudaGraphNode_t n2;
        if ((e = graph_leaves(lbody, leaves)) != cudaSuccess) goto fail;
        if ((e = add_conditional(lbody, leaves, h_second, cudaGraphCondTypeIf, &n2, &sbody)) != cudaSuccess) goto fail;
    }
    if ((s = capture(sbody, {}, [&] { return sweep_ctl(W, V, 1); })) != CPMDP_OK) goto done;
    goto done;
fail:
    s = cuda_fail(e, "recording the dense solve graph");
done:
    if (cap) cudaStreamDestroy(cap);
    if (s != CPMDP_OK) {
        if (G) cudaGraphDestroy(G);
        return s;
    }
    *out = G;
    return CPMDP_OK;
}

template <typename T>
static cpmdp_status dense_solve_t(const Factors &F, bool pim, T *V, uint8_t *pi, const SolveOpts &o,
                                  Ctrl *hc, cudaStream_t st) {
    Factors &M = const_cast<Factors &>(F);
    // buffers the recorded graph uses must exist before the recording
    if (!M.d_dense_loop) CPMDP_CUDA(cudaMalloc(&M.d_dense_loop, kLoopCtlBytes));
    if (!M.d_tc_err) CPMDP_CUDA(cudaMalloc(&M.d_tc_err, sizeof(int)));
    const int prec = std::is_same<T, double>::value ? 1 : 0;
    const bool same = M.simt_graph && M.simt_graph_V == (void *)V && M.simt_graph_pi == (void *)pi &&
                      M.simt_graph_pim == (int)pim && M.simt_graph_prec == prec && M.simt_graph_tol == o.tol &&
                      M.simt_graph_eval_tol == o.eval_tol && M.simt_graph_max_iter == o.max_iter &&
                      M.simt_graph_rounds == o.max_rounds && M.simt_graph_eval_iter == o.max_eval_iter &&
                      M.simt_graph_partial == o.partial_eval && M.simt_graph_trace == (void *)o.trace;
    if (!same) {
        if (M.simt_graph) { cudaGraphExecDestroy(M.simt_graph); M.simt_graph = nullptr; }
        cudaGraph_t g = nullptr;
        cpmdp_status s = record_simt<T>(M, pim, V, pi, o, &g);
        if (s != CPMDP_OK) return s;
        cudaError_t e = cudaGraphInstantiate(&M.simt_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { M.simt_graph = nullptr; CPMDP_CUDA(e); }
        M.simt_graph_V = (void *)V;
        M.simt_graph_pi = (void *)pi;
        M.simt_graph_pim = (int)pim;
        M.simt_graph_prec = prec;
        M.simt_graph_tol = o.tol;
        M.simt_graph_eval_tol = o.eval_tol;
        M.simt_graph_max_iter = o.max_iter;
        M.simt_graph_rounds = o.max_rounds;
        M.simt_graph_eval_iter = o.max_eval_iter;
        M.simt_graph_partial = o.partial_eval;
        M.simt_graph_trace = (void *)o.trace;
    }
    DensePiCtl c0;
    memset(&c0, 0, sizeof(c0));
    if (pim) {
        c0.full = o.partial_eval <= 0;
        c0.total = 1;   // the greedy start
    }
    CPMDP_CUDA(cudaMemcpyAsync(M.d_dense_loop, &c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    CPMDP_CUDA(cudaMemsetAsync(&F.d_ctrl->res_slot[0], 0, sizeof(unsigned long long), st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_tc_err, 0, sizeof(int), st));
    CPMDP_CUDA(cudaGraphLaunch(M.simt_graph, st));
    DensePiCtl c;
    CPMDP_CUDA(cudaMemcpyAsync(&c, M.d_dense_loop, sizeof(c), cudaMemcpyDeviceToHost, st));
    CPMDP_CUDA(cudaStreamSynchronize(st));
    hc->iterations = c.total;
    hc->rounds = c.rounds;
    hc->eval_sweeps = c.evals;
    hc->converged = c.conv;
    hc->last_residual = c.total > (pim ? 1 : 0) ? c.res : INFINITY;
    hc->backups = (long long)c.total * F.nstates * F.nactions;
    return CPMDP_OK;
}

cpmdp_status dense_solve(const Factors &F, cpmdp_precision prec, bool pim, void *V, uint8_t *pi,
                         const SolveOpts &o, Ctrl *hc, cudaStream_t st) {
    if (prec == CPMDP_F64) return dense_solve_t<double>(F, pim, (double *)V, pi, o, hc, st);
    if (prec == CPMDP_F32) return dense_solve_t<float>(F, pim, (float *)V, pi, o, hc, st);
    if (pim) return dense_tc_policy_iteration(F, (float *)V, pi, o, hc, st);
    return dense_tc_solve(F, (float *)V, pi, o, hc, st);
}

}  // namespace cpmdp
