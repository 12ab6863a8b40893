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

    for (int j0 = 0; j0 < N; j0 += TK) {
        // U tile: 64 rows x 16 columns, loaded along j
        for (int e = tid; e < TI * TK; e += 256) {
            const int ii = e / TK, jj = e % TK;
            const int i = i0 + ii, j = j0 + jj;
            sU[jj][ii] = (i < N && j < N) ? U[(long long)i * N + j] : (T)0;
        }
        // X tile: 16 x 64; coalesce along r when Rt > 1, along j when Rt == 1
        for (int e = tid; e < TK * TC; e += 256) {
            int jj, cc;
            if (Rt == 1) { jj = e % TK; cc = e / TK; }
            else { cc = e % TC; jj = e / TC; }
            const int j = j0 + jj;
            const long long c = c0 + cc;
            T v = 0;
            if (j < N && c < ncols) {
                const long long l = c / Rt, r = c - l * Rt;
                v = X[(l * N + j) * Rt + r];
            }
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
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = i0 + ty + 16 * a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const long long c = c0 + tx + 16 * b;
            if (c >= ncols) continue;
            const long long l = c / Rt, r = c - l * Rt;
            const long long s = (l * N + i) * Rt + r;
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
template <typename T>
static cpmdp_status dense_solve_t(const Factors &F, bool pim, T *V, uint8_t *pi, const SolveOpts &o,
                                  Ctrl *hc, cudaStream_t st) {
    T *W = (T *)F.d_scratch;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    unsigned *cb = &F.d_ctrl->changed_slot[0];
    const double margin = std::is_same<T, double>::value ? 1e-12 : 1e-6;
    T *cur = V, *nxt = W;
    int total = 0, conv = 0, rounds = 0, evals = 0;
    long long backups = 0;
    double res = INFINITY;
    const long long SA = (long long)F.nstates * F.nactions;
    auto sweep_res = [&](int mode) -> cpmdp_status {
        CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(*rb), st));
        cpmdp_status s2 = dense_sweep<T>(F, cur, nxt, pi, mode, margin, rb, nullptr, st);
        if (s2 != CPMDP_OK) return s2;
        unsigned long long bits = 0;
        CPMDP_CUDA(cudaMemcpyAsync(&bits, rb, sizeof(bits), cudaMemcpyDeviceToHost, st));
        CPMDP_CUDA(cudaStreamSynchronize(st));
        memcpy(&res, &bits, sizeof(res));
        T *t = cur; cur = nxt; nxt = t;
        total++;
        backups += SA;
        return CPMDP_OK;
    };
    cpmdp_status s2;
    if (!pim) {
        while (total < o.max_iter) {
            if ((s2 = sweep_res(DM_VI)) != CPMDP_OK) return s2;
            if (o.trace) CPMDP_CUDA(cudaMemcpyAsync(o.trace + total - 1, &res, sizeof(double), cudaMemcpyHostToDevice, st));
            if (res < o.tol) { conv = 1; break; }
        }
    } else {
        if ((s2 = dense_sweep<T>(F, cur, nullptr, pi, DM_GREEDY, margin, nullptr, nullptr, st)) != CPMDP_OK) return s2;
        total++;
        backups += SA;
        // modified policy iteration, as the GridWorld solvers
        bool full = o.partial_eval <= 0;
        while (rounds < o.max_rounds) {
            const int cap = full ? o.max_eval_iter : std::min(o.partial_eval, o.max_eval_iter);
            int e = 0, ok = 0;
            while (e < cap) {
                if ((s2 = sweep_res(DM_EVAL)) != CPMDP_OK) return s2;
                e++;
                if (res < o.eval_tol) { ok = 1; break; }
            }
            evals += e;
            CPMDP_CUDA(cudaMemsetAsync(cb, 0, sizeof(*cb), st));
            if ((s2 = dense_sweep<T>(F, cur, nullptr, pi, DM_IMPROVE, margin, nullptr, cb, st)) != CPMDP_OK) return s2;
            unsigned nchg = 0;
            CPMDP_CUDA(cudaMemcpyAsync(&nchg, cb, sizeof(nchg), cudaMemcpyDeviceToHost, st));
            CPMDP_CUDA(cudaStreamSynchronize(st));
            total++;
            rounds++;
            backups += SA;
            if (nchg == 0) {
                if (ok) { conv = 1; break; }
                if (full) break;
                full = true;
                continue;
            }
            if (!ok && full) break;
        }
    }
    if (cur != V) CPMDP_CUDA(cudaMemcpyAsync(V, cur, sizeof(T) * F.nstates, cudaMemcpyDeviceToDevice, st));
    if (!pim && pi) {
        if ((s2 = dense_sweep<T>(F, V, nullptr, pi, DM_GREEDY, margin, nullptr, nullptr, st)) != CPMDP_OK) return s2;
    }
    hc->iterations = total;
    hc->rounds = rounds;
    hc->eval_sweeps = evals;
    hc->converged = conv;
    hc->last_residual = res;
    hc->backups = backups;
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
