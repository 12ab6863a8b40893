// Banded (GridWorld) backup: the single-sweep kernel behind
// cpmdp_bellman_backup and the FP64 certifying sweep, and the plain unfused
// baseline. The device code of the fused backup is in banded_common.cuh,
// the persistent solvers in banded_solve.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <type_traits>

#include "banded_common.cuh"
#include "march.h"

namespace cpmdp {

// One fused value-iteration sweep, non-persistent. res_out: atomic max of
// the residual (bits of a non-negative double), may be null.
template <typename T, typename TA, int D, int VEC, bool WITH_PI>
__global__ void __launch_bounds__(256) sweep_kernel(BandArgs a, const T *__restrict__ V,
                                                    T *__restrict__ W, uint8_t *pi,
                                                    unsigned long long *res_out) {
    __shared__ unsigned shm[64];
    unsigned dummy = 0;
    const TA r = sweep_all<T, TA, D, VEC, M_VI, WITH_PI>(a, V, W, pi, (TA)0, dummy);
    if (res_out) {
        const unsigned long long mb = block_max_bits(r, shm);
        if (threadIdx.x == 0 && mb) atomicMax(res_out, mb);
    }
}

// ---------------------------------------------------------------------------
// plain (unfused) baseline: one kernel per action, then max, then residual.
// Each thread handles one state, walks the action's rank-1 terms one by one
// from the cell codes and coordinates (no shared pair sums, no packing).

struct PlainArgs {
    int nstates, ndim;
    int shape[kMaxDim], stride[kMaxDim];
    double w_move, w_perp, w_stay, gamma;
    const uint8_t *cell;
};

template <typename T>
__global__ void plain_q_kernel(PlainArgs a, const T *__restrict__ V, const T *__restrict__ R,
                               T *__restrict__ Q, int act, const int *stop) {
    if (stop && *(volatile const int *)stop) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.nstates || a.cell[s] != CPMDP_CELL_FREE) return;
    int c[kMaxDim], rem = s;
    for (int d = 0; d < a.ndim; d++) { c[d] = rem / a.stride[d]; rem -= c[d] * a.stride[d]; }
    auto value_after = [&](int d, int step) -> T {
        const int x = c[d] + step;
        if (x < 0 || x >= a.shape[d]) return V[s];
        const int t = s + step * a.stride[d];
        return a.cell[t] == CPMDP_CELL_OBSTACLE ? V[s] : V[t];
    };
    const int d0 = act / 2, sg = (act & 1) ? 1 : -1;
    T e = (T)a.w_move * value_after(d0, sg);
    if (a.ndim == 1) {
        e += (T)a.w_stay * V[s];
    } else {
        for (int d = 0; d < a.ndim; d++) {
            if (d == d0) continue;
            e += (T)a.w_perp * value_after(d, -1);
            e += (T)a.w_perp * value_after(d, +1);
        }
    }
    Q[(size_t)act * a.nstates + s] = R[s] + (T)a.gamma * e;
}

template <typename T>
__global__ void plain_max_kernel(PlainArgs a, const T *__restrict__ Q, const T *__restrict__ R,
                                 T *__restrict__ W, uint8_t *pi, int nact, const int *stop) {
    if (stop && *(volatile const int *)stop) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.nstates) return;
    const uint8_t k = a.cell[s];
    if (k != CPMDP_CELL_FREE) {
        W[s] = (k == CPMDP_CELL_TERMINAL) ? R[s] : (T)0;
        if (pi) pi[s] = 255;
        return;
    }
    T best = Q[s];
    int arg = 0;
    for (int j = 1; j < nact; j++) {
        const T q = Q[(size_t)j * a.nstates + s];
        if (q > best) { best = q; arg = j; }
    }
    W[s] = best;
    if (pi) pi[s] = (uint8_t)arg;
}

template <typename T>
__global__ void plain_residual_kernel(int n, const uint8_t *__restrict__ cell, const T *__restrict__ V,
                                      const T *__restrict__ W, unsigned long long *res, const int *stop) {
    __shared__ double shd[32];
    if (stop && *(volatile const int *)stop) return;
    double m = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        if (cell[s] != CPMDP_CELL_OBSTACLE) m = fmax(m, fabs((double)W[s] - (double)V[s]));
    m = block_max(m, shd);
    if (threadIdx.x == 0 && m > 0.0) atomicMax(res, (unsigned long long)__double_as_longlong(m));
}

// Device-side stopping rule of the plain baseline's graph variant: after
// each sweep one thread reads the sweep's residual, clears its slot for the
// next sweep, counts the sweep and raises stop when the residual is below
// tol or max_iter sweeps are done; every kernel of a later sweep then
// returns at once.
__global__ void plain_check_kernel(Ctrl *c, double tol, int max_iter) {
    if (c->plain_stop) return;
    double r;
    memcpy(&r, &c->res_slot[0], sizeof(r));
    c->res_slot[0] = 0ull;
    c->iterations += 1;
    c->last_residual = r;
    if (r < tol) {
        c->converged = 1;
        c->plain_stop = 1;
    } else if (c->iterations >= max_iter) {
        c->plain_stop = 1;
    }
}

// ---------------------------------------------------------------------------
// host side

BandArgs make_band_args(const Factors &F) {
    BandArgs a;
    a.nstates = (int)F.nstates;
    a.nlast = (int)F.shape[F.ndim - 1];
    for (int d = 0; d < kMaxDim; d++) a.stride[d] = d < F.ndim ? (int)F.stride[d] : 0;
    a.w_move = F.w_move;
    a.w_perp = F.w_perp;
    a.w_stay = F.w_stay;
    a.gamma = F.gamma;
    a.wf_move = (float)F.w_move;
    a.wf_perp = (float)F.w_perp;
    a.wf_stay = (float)F.w_stay;
    a.wf_gamma = (float)F.gamma;
    a.code = F.d_code;
    a.R32 = F.d_R32;
    a.R64 = F.d_R64;
    return a;
}

static bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

// Widest segment length usable for this row length, element size and pointers.
int band_pick_vec(const Factors &F, size_t elem, const void *p0, const void *p1) {
    const int64_t n = F.shape[F.ndim - 1];
    const int v = (int)(16 / elem);  // 4 floats or 2 doubles
    if (n % v == 0 && aligned16(p0) && aligned16(p1)) return v;
    return 1;
}

// Grid of co-resident blocks (at most one block per 256 segments).
template <typename K>
static int resident_grid(K kern, const Factors &F, int nitems, int &cache) {
    if (cache <= 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 256, 0) != cudaSuccess || o < 1) o = 1;
        cache = o;
    }
    int grid = cache * (F.num_sms > 0 ? F.num_sms : 148);
    const int need = (nitems + 255) / 256;
    if (grid > need) grid = need;
    return grid < 1 ? 1 : grid;
}

template <typename T, typename TA, int D, int VEC, bool WITH_PI>
static cudaError_t launch_sweep(const Factors &F, const T *V, T *W, uint8_t *pi, unsigned long long *res,
                                cudaStream_t st) {
    static int occ = 0;
    BandArgs a = make_band_args(F);
    const int nitems = (int)(F.nstates / VEC);
    auto kern = sweep_kernel<T, TA, D, VEC, WITH_PI>;
    const int grid = resident_grid(kern, F, nitems, occ);
    kern<<<grid, 256, 0, st>>>(a, V, W, pi, res);
    return cudaGetLastError();
}

template <typename T, typename TA>
static cudaError_t sweep_any(const Factors &F, const T *V, T *W, uint8_t *pi, unsigned long long *res,
                             cudaStream_t st) {
    // large 3-D float grids: the plane-marching sweep (same arithmetic)
    if (std::is_same<T, float>::value && march_eligible(F, V, W, pi))
        return march_sweep(F, (const float *)V, (float *)W, pi, res, std::is_same<TA, double>::value, st);
    const int vec = band_pick_vec(F, sizeof(T), V, W);
    constexpr int V2 = (int)(16 / sizeof(T));
    cudaError_t e = cudaErrorInvalidValue;
    if (pi) {
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_sweep<T, TA, DD, 1, true>(F, V, W, pi, res, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_sweep<T, TA, DD, V2, true>(F, V, W, pi, res, st))); }
    } else {
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_sweep<T, TA, DD, 1, false>(F, V, W, pi, res, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_sweep<T, TA, DD, V2, false>(F, V, W, pi, res, st))); }
    }
    return e;
}

cpmdp_status banded_backup(const Factors &F, cpmdp_precision prec, const void *Vin, void *Vout,
                           uint8_t *pi, double *res, cudaStream_t st) {
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    if (rb) CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    cudaError_t e;
    if (prec == CPMDP_F64)
        e = sweep_any<double, double>(F, (const double *)Vin, (double *)Vout, pi, rb, st);
    else
        e = sweep_any<float, float>(F, (const float *)Vin, (float *)Vout, pi, rb, st);
    CPMDP_CUDA(e);
    return CPMDP_OK;
}

// FP64 sweep of a float value tensor: certified residual and FP64 argmax.
cpmdp_status banded_certify(const Factors &F, const float *V, uint8_t *pi, double *res, cudaStream_t st) {
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    CPMDP_CUDA((sweep_any<float, double>(F, V, (float *)nullptr, pi, rb, st)));
    return CPMDP_OK;
}

// Plain baseline, second variant (fused = 3): the same unfused kernels,
// but the stopping rule is taken on the device (plain_check_kernel) and the
// host looks at it once per chunk of kPlainChunk sweeps. A chunk (an even
// number of sweeps, so it starts and ends in V) is recorded once into a
// CUDA graph and replayed until the stop flag is up; the sweeps of a chunk
// after the stopping sweep launch and return at once. The result is in V
// after an even number of sweeps and in the scratch buffer after an odd
// number.
constexpr int kPlainChunk = 32;

template <typename T>
static cpmdp_status plain_vi_graph(const Factors &F, const PlainArgs &a, T *V, const SolveOpts &o, Ctrl *hc,
                                   cudaStream_t st) {
    Factors &M = const_cast<Factors &>(F);
    const T *R = std::is_same<T, double>::value ? (const T *)F.d_R64 : (const T *)F.d_R32;
    T *Q = (T *)F.d_q;
    T *W = (T *)F.d_scratch;
    const int n = (int)F.nstates;
    const int grid = (n + 255) / 256;
    int rgrid = grid > F.num_sms * 8 ? F.num_sms * 8 : grid;
    if (rgrid < 1) rgrid = 1;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    const int *stop = &F.d_ctrl->plain_stop;
    const int prec = std::is_same<T, double>::value ? 1 : 0;
    const bool same = M.plain_graph && M.plain_graph_V == (void *)V && M.plain_graph_tol == o.tol &&
                      M.plain_graph_max_iter == o.max_iter && M.plain_graph_prec == prec;
    if (!same) {
        if (M.plain_graph) { cudaGraphExecDestroy(M.plain_graph); M.plain_graph = nullptr; }
        cudaStream_t cap;
        CPMDP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < kPlainChunk && e == cudaSuccess; k++) {
            const T *cur = (k & 1) ? W : V;
            T *nxt = (k & 1) ? V : W;
            for (int act = 0; act < F.nactions; act++) plain_q_kernel<T><<<grid, 256, 0, cap>>>(a, cur, R, Q, act, stop);
            plain_max_kernel<T><<<grid, 256, 0, cap>>>(a, Q, R, nxt, nullptr, F.nactions, stop);
            plain_residual_kernel<T><<<rgrid, 256, 0, cap>>>(n, F.d_cell, cur, nxt, rb, stop);
            plain_check_kernel<<<1, 1, 0, cap>>>(F.d_ctrl, o.tol, o.max_iter);
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&M.plain_graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) { M.plain_graph = nullptr; CPMDP_CUDA(e); }
        M.plain_graph_V = (void *)V;
        M.plain_graph_tol = o.tol;
        M.plain_graph_max_iter = o.max_iter;
        M.plain_graph_prec = prec;
    }
    // stop = 0, iterations = 0, residual slot 0
    CPMDP_CUDA(cudaMemsetAsync(F.d_ctrl, 0, sizeof(Ctrl), st));
    Ctrl h;
    for (;;) {
        CPMDP_CUDA(cudaGraphLaunch(M.plain_graph, st));
        CPMDP_CUDA(cudaMemcpyAsync(&h, F.d_ctrl, sizeof(h), cudaMemcpyDeviceToHost, st));
        CPMDP_CUDA(cudaStreamSynchronize(st));
        if (h.plain_stop || h.status) break;
    }
    if (h.iterations & 1) CPMDP_CUDA(cudaMemcpyAsync(V, W, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    hc->iterations = h.iterations;
    hc->converged = h.converged;
    hc->last_residual = h.last_residual;
    hc->backups = (long long)h.iterations * F.nstates * F.nactions;
    return CPMDP_OK;
}

// Plain baseline value iteration: per sweep |A| Q kernels, a max kernel, a
// residual kernel and a device-to-host copy of the residual checked on the
// host (fused = 0), or the same kernels with the stopping rule taken on the
// device and checked by the host once per chunk of sweeps (fused = 3).
// Fills host_ctrl (iterations, converged, residual, backups).
template <typename T>
static cpmdp_status plain_vi_impl(const Factors &F, T *V, uint8_t *pi, const SolveOpts &o, Ctrl *hc,
                                  cudaStream_t st) {
    PlainArgs a;
    a.nstates = (int)F.nstates;
    a.ndim = F.ndim;
    for (int d = 0; d < kMaxDim; d++) {
        a.shape[d] = d < F.ndim ? (int)F.shape[d] : 1;
        a.stride[d] = d < F.ndim ? (int)F.stride[d] : 0;
    }
    a.w_move = F.w_move; a.w_perp = F.w_perp; a.w_stay = F.w_stay; a.gamma = F.gamma;
    a.cell = F.d_cell;
    const T *R = std::is_same<T, double>::value ? (const T *)F.d_R64 : (const T *)F.d_R32;
    T *Q = (T *)F.d_q;
    T *cur = V, *nxt = (T *)F.d_scratch;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    unsigned long long hres_bits = 0;
    const int n = (int)F.nstates;
    const int grid = (n + 255) / 256;
    int rgrid = grid > F.num_sms * 8 ? F.num_sms * 8 : grid;
    if (rgrid < 1) rgrid = 1;
    if (o.fused == 3) {
        cpmdp_status s3 = plain_vi_graph<T>(F, a, V, o, hc, st);
        if (s3 != CPMDP_OK || !pi) return s3;
        T *spare = (T *)F.d_scratch;
        for (int act = 0; act < F.nactions; act++) plain_q_kernel<T><<<grid, 256, 0, st>>>(a, V, R, Q, act, nullptr);
        plain_max_kernel<T><<<grid, 256, 0, st>>>(a, Q, R, spare, pi, F.nactions, nullptr);
        CPMDP_CUDA(cudaGetLastError());
        return CPMDP_OK;
    }
    int k = 0, conv = 0;
    double res = INFINITY;
    while (k < o.max_iter) {
        CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(unsigned long long), st));
        for (int act = 0; act < F.nactions; act++) plain_q_kernel<T><<<grid, 256, 0, st>>>(a, cur, R, Q, act, nullptr);
        plain_max_kernel<T><<<grid, 256, 0, st>>>(a, Q, R, nxt, nullptr, F.nactions, nullptr);
        plain_residual_kernel<T><<<rgrid, 256, 0, st>>>(n, F.d_cell, cur, nxt, rb, nullptr);
        CPMDP_CUDA(cudaGetLastError());
        CPMDP_CUDA(cudaMemcpyAsync(&hres_bits, rb, sizeof(hres_bits), cudaMemcpyDeviceToHost, st));
        CPMDP_CUDA(cudaStreamSynchronize(st));
        memcpy(&res, &hres_bits, sizeof(res));
        T *t = cur; cur = nxt; nxt = t;
        k++;
        if (res < o.tol) { conv = 1; break; }
    }
    if (cur != V) CPMDP_CUDA(cudaMemcpyAsync(V, cur, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    if (pi) {
        // policy of the returned V; the max goes to the scratch buffer (V is the result)
        T *spare = (T *)F.d_scratch;
        for (int act = 0; act < F.nactions; act++) plain_q_kernel<T><<<grid, 256, 0, st>>>(a, V, R, Q, act, nullptr);
        plain_max_kernel<T><<<grid, 256, 0, st>>>(a, Q, R, spare, pi, F.nactions, nullptr);
        CPMDP_CUDA(cudaGetLastError());
    }
    hc->iterations = k;
    hc->converged = conv;
    hc->last_residual = res;
    hc->backups = (long long)k * F.nstates * F.nactions;
    return CPMDP_OK;
}

cpmdp_status banded_plain_vi(const Factors &F, cpmdp_precision prec, void *V, uint8_t *pi,
                             const SolveOpts &o, Ctrl *hc, cudaStream_t st) {
    if (prec == CPMDP_F64) return plain_vi_impl<double>(F, (double *)V, pi, o, hc, st);
    return plain_vi_impl<float>(F, (float *)V, pi, o, hc, st);
}

}  // namespace cpmdp
