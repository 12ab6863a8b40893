// Device-resident value iteration and policy iteration for GridWorld
// factors (background section: value iteration repeats Eq. 1 until it
// converges; policy iteration alternates evaluation of a fixed policy with
// greedy improvement until no action changes).
//
// Each solve is one cooperative launch of co-resident blocks. Every sweep
// ends in a grid barrier whose arrival atomic also reports whether the
// block's residual is still >= tol (VI, evaluation) or whether the block
// changed an action (improvement): every block learns the stopping decision
// from the barrier itself, with no extra round trip (an improvement sweep,
// which also writes the new policy's first evaluation step, adds its
// residual through the slot below, read after the barrier). The residual value goes
// to res_slot[k % 3] by atomic max (slot k+1 is cleared by block 0 during
// sweep k, after every block has passed the barrier of sweep k-1, so nobody
// still reads it); it is read for the trace and at the end. The host reads
// back the control block once, after the launch.
#include <cuda_runtime.h>
#include <math.h>

#include "banded_common.cuh"
#include "flow.h"
#include "march.h"

namespace cpmdp {

template <typename T, int D, int VEC>
__global__ void __launch_bounds__(256) solve_vi_kernel(BandArgs a, T *V, T *Wbuf, SolveParams sp, Ctrl *ctrl,
                                                       double *trace) {
    typedef T TA;
    __shared__ unsigned shm[64];
    const unsigned nb = gridDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const bool stall = sp.inject_stall && blockIdx.x == 0;
    T *cur = V, *nxt = Wbuf;
    int k = 0, converged = 0;
    unsigned dummy = 0;
    unsigned long long ph0 = 0ull, ph1 = 0ull;
    while (k < sp.max_iter) {
        const TA r = sweep_all<T, TA, D, VEC, M_VI, false>(a, cur, nxt, nullptr, (TA)0, dummy);
        const unsigned long long mb = block_max_bits(r, shm);
        int flag = 0;
        if (threadIdx.x == 0) {
            if (mb) atomicMax(&ctrl->res_slot[k % 3], mb);
            flag = !below_tol(mb, sp.tol);
        }
        if (lead) ctrl->res_slot[(k + 1) % 3] = 0ull;
        const long long open = grid_sync_count(ctrl, k, nb, flag, sp.timeout_ns, ph0, ph1, stall && k == 0);
        if (open < 0) return;
        if (trace && lead)
            trace[k] = __longlong_as_double((long long)*(volatile unsigned long long *)&ctrl->res_slot[k % 3]);
        k++;
        T *t = cur; cur = nxt; nxt = t;
        if (open == 0) { converged = 1; break; }
    }
    if (cur != V) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nstates; i += gridDim.x * blockDim.x) V[i] = cur[i];
    }
    if (lead) {
        ctrl->iterations = k;
        ctrl->converged = converged;
        ctrl->last_residual =
            k > 0 ? __longlong_as_double((long long)*(volatile unsigned long long *)&ctrl->res_slot[(k - 1) % 3]) : 0.0;
        ctrl->backups = (long long)k * a.nstates * sp.nactions;
    }
}

template <typename T, int D, int VEC>
__global__ void __launch_bounds__(256) solve_pi_kernel(BandArgs a, T *V, T *Wbuf, uint8_t *pi, SolveParams sp,
                                                       Ctrl *ctrl) {
    typedef T TA;
    __shared__ unsigned shm[64];
    __shared__ unsigned shu[32];
    const unsigned nb = gridDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const bool stall = sp.inject_stall && blockIdx.x == 0;
    T *cur = V, *nxt = Wbuf;
    int ks = 0, total = 0, nbar = 0, round = 0, evals = 0, converged = 0;
    long long backups = 0;
    unsigned dummy = 0;
    unsigned long long ph0 = 0ull, ph1 = 0ull;

    // initial policy: greedy with respect to the input V
    sweep_all<T, TA, D, VEC, M_GREEDY, true>(a, cur, nullptr, pi, (TA)0, dummy);
    if (grid_sync_count(ctrl, nbar++, nb, 0, sp.timeout_ns, ph0, ph1, stall) < 0) return;
    total++;
    backups += (long long)a.nstates * sp.nactions;
    // modified policy iteration: evaluations of exactly partial_eval sweeps
    // until an improvement changes no action, evaluations to eval_tol after that
    bool full = sp.partial_eval <= 0;
    while (round < sp.max_rounds) {
        const int cap = full ? sp.max_eval_iter : min(sp.partial_eval, sp.max_eval_iter);
        int e = 0, eval_ok = 0;
        while (e < cap) {
            const TA r = sweep_all<T, TA, D, VEC, M_EVAL, true>(a, cur, nxt, pi, (TA)0, dummy);
            const unsigned long long mb = block_max_bits(r, shm);
            int flag = 0;
            if (threadIdx.x == 0) {
                if (mb) atomicMax(&ctrl->res_slot[ks % 3], mb);
                flag = !below_tol(mb, sp.eval_tol);
            }
            if (lead) ctrl->res_slot[(ks + 1) % 3] = 0ull;
            const long long open = grid_sync_count(ctrl, nbar++, nb, flag, sp.timeout_ns, ph0, ph1, false);
            if (open < 0) return;
            ks++; e++; total++;
            backups += a.nstates;
            T *t = cur; cur = nxt; nxt = t;
            // a capped evaluation runs all its sweeps; one to eval_tol stops there
            if (open == 0 && full) { eval_ok = 1; break; }
        }
        evals += e;
        // improvement, and the new policy's first evaluation step V' = Q of
        // the action kept or taken (modified policy iteration)
        unsigned changed = 0;
        const TA r = sweep_all<T, TA, D, VEC, M_IMPROVE, true>(a, cur, nxt, pi, (TA)sp.margin, changed);
        const unsigned c = block_sum(changed, shu);
        const unsigned long long mb = block_max_bits(r, shm);
        if (threadIdx.x == 0) {
            if (c) atomicAdd(&ctrl->changed_total, c);
            if (mb) atomicMax(&ctrl->res_slot[ks % 3], mb);
        }
        if (lead) ctrl->res_slot[(ks + 1) % 3] = 0ull;
        const long long moved = grid_sync_count(ctrl, nbar++, nb, threadIdx.x == 0 && c > 0, sp.timeout_ns,
                                                ph0, ph1, false);
        if (moved < 0) return;
        const bool open =
            !below_tol(*(volatile unsigned long long *)&ctrl->res_slot[ks % 3], sp.eval_tol);
        ks++;
        total++;
        round++;
        backups += (long long)a.nstates * sp.nactions;
        T *t = cur; cur = nxt; nxt = t;
        if (moved == 0) {
            if (!open) { converged = 1; break; }   // stable policy, V' within eval_tol of V
            if (!eval_ok) {
                if (full) break;   // the evaluation limit ran out
                full = true;       // evaluate this policy to eval_tol before deciding
            }
            continue;
        }
        if (!eval_ok && full) break;
    }
    if (cur != V) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nstates; i += gridDim.x * blockDim.x) V[i] = cur[i];
    }
    if (lead) {
        ctrl->rounds = round;
        ctrl->eval_sweeps = evals;
        ctrl->iterations = total;
        ctrl->converged = converged;
        ctrl->last_residual =
            ks > 0 ? __longlong_as_double((long long)*(volatile unsigned long long *)&ctrl->res_slot[(ks - 1) % 3]) : 0.0;
        ctrl->backups = backups;
    }
}


// Grids that one block covers (at most 256 segments, where the kernels
// above run a single block anyway): the same solvers with the value
// ping-pong in shared memory and each sweep's residual and stop decision
// taken in shared memory (one block barrier per sweep, no global atomics or
// control-block round trips). Same per-state arithmetic and stopping rules,
// so the same values, sweep counts and residuals as the kernels above.
constexpr int kSmallMaxItems = 256;

template <typename T, int D, int VEC>
__global__ void __launch_bounds__(256) small_vi_kernel(BandArgs a, T *V, SolveParams sp, Ctrl *ctrl,
                                                       double *trace) {
    typedef T TA;
    extern __shared__ __align__(16) unsigned char small_raw[];
    __shared__ unsigned shm[64];
    __shared__ unsigned long long s_mb;
    T *cur = reinterpret_cast<T *>(small_raw), *nxt = cur + a.nstates;
    const int nitems = a.nstates / VEC;
    for (int i = threadIdx.x; i < a.nstates; i += blockDim.x) cur[i] = V[i];
    __syncthreads();
    int k = 0, converged = 0;
    unsigned long long last = 0ull;
    while (k < sp.max_iter) {
        TA r = 0;
        for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
            Segment<T, TA, D, VEC> sg;
            sg.template load<M_VI>(a, cur, nullptr, i * VEC);
            const TA x = sg.template finish_vi<false>(a, nxt, nullptr, i * VEC);
            r = x > r ? x : r;
        }
        const unsigned long long mb = block_max_bits(r, shm);
        if (threadIdx.x == 0) s_mb = mb;
        __syncthreads();   // the sweep's writes and its residual, for every thread
        const unsigned long long m = s_mb;
        if (trace && threadIdx.x == 0) trace[k] = __longlong_as_double((long long)m);
        last = m;
        k++;
        T *t = cur; cur = nxt; nxt = t;
        if (below_tol(m, sp.tol)) { converged = 1; break; }
    }
    for (int i = threadIdx.x; i < a.nstates; i += blockDim.x) V[i] = cur[i];
    if (threadIdx.x == 0) {
        ctrl->iterations = k;
        ctrl->converged = converged;
        ctrl->last_residual = __longlong_as_double((long long)last);
        ctrl->backups = (long long)k * a.nstates * sp.nactions;
    }
}

template <typename T, int D, int VEC>
__global__ void __launch_bounds__(256) small_pi_kernel(BandArgs a, T *V, uint8_t *pi, SolveParams sp, Ctrl *ctrl) {
    typedef T TA;
    extern __shared__ __align__(16) unsigned char small_raw[];
    __shared__ unsigned shm[64];
    __shared__ unsigned shu[32];
    __shared__ unsigned long long s_mb;
    __shared__ unsigned s_c;
    T *cur = reinterpret_cast<T *>(small_raw), *nxt = cur + a.nstates;
    const int nitems = a.nstates / VEC;
    for (int i = threadIdx.x; i < a.nstates; i += blockDim.x) cur[i] = V[i];
    __syncthreads();
    int total = 0, round = 0, evals = 0, converged = 0;
    long long backups = 0;
    unsigned long long last = 0ull;
    unsigned changed_total = 0, dummy = 0;
    // initial policy: greedy with respect to the input V
    for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
        Segment<T, TA, D, VEC> sg;
        sg.template load<M_GREEDY>(a, cur, pi, i * VEC);
        sg.template finish_pi<M_GREEDY>(a, nullptr, pi, (TA)0, i * VEC, dummy);
    }
    __syncthreads();
    total++;
    backups += (long long)a.nstates * sp.nactions;
    // modified policy iteration: evaluations of exactly partial_eval sweeps
    // until an improvement changes no action, evaluations to eval_tol after that
    bool full = sp.partial_eval <= 0;
    while (round < sp.max_rounds) {
        const int cap = full ? sp.max_eval_iter : min(sp.partial_eval, sp.max_eval_iter);
        int e = 0, eval_ok = 0;
        while (e < cap) {
            TA r = 0;
            for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
                Segment<T, TA, D, VEC> sg;
                sg.template load<M_EVAL>(a, cur, pi, i * VEC);
                const TA x = sg.template finish_pi<M_EVAL>(a, nxt, pi, (TA)0, i * VEC, dummy);
                r = x > r ? x : r;
            }
            const unsigned long long mb = block_max_bits(r, shm);
            if (threadIdx.x == 0) s_mb = mb;
            __syncthreads();
            const unsigned long long m = s_mb;
            last = m;
            e++;
            total++;
            backups += a.nstates;
            T *t = cur; cur = nxt; nxt = t;
            // a capped evaluation runs all its sweeps; one to eval_tol stops there
            if (full && below_tol(m, sp.eval_tol)) { eval_ok = 1; break; }
        }
        evals += e;
        // improvement, and the new policy's first evaluation step V' = Q of
        // the action kept or taken (modified policy iteration)
        unsigned changed = 0;
        TA r = 0;
        for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
            Segment<T, TA, D, VEC> sg;
            sg.template load<M_IMPROVE>(a, cur, pi, i * VEC);
            const TA x = sg.template finish_pi<M_IMPROVE>(a, nxt, pi, (TA)sp.margin, i * VEC, changed);
            r = x > r ? x : r;
        }
        const unsigned c0 = block_sum(changed, shu);
        const unsigned long long mb = block_max_bits(r, shm);
        if (threadIdx.x == 0) {
            s_c = c0;
            s_mb = mb;
        }
        __syncthreads();   // the policy changes, their count and V', for every thread
        const unsigned c = s_c;
        const unsigned long long m = s_mb;
        last = m;
        changed_total += c;
        total++;
        round++;
        backups += (long long)a.nstates * sp.nactions;
        T *t = cur; cur = nxt; nxt = t;
        if (c == 0) {
            if (below_tol(m, sp.eval_tol)) { converged = 1; break; }   // stable policy, V' within eval_tol
            if (!eval_ok) {
                if (full) break;   // the evaluation limit ran out
                full = true;       // evaluate this policy to eval_tol before deciding
            }
            continue;
        }
        if (!eval_ok && full) break;
    }
    for (int i = threadIdx.x; i < a.nstates; i += blockDim.x) V[i] = cur[i];
    if (threadIdx.x == 0) {
        ctrl->rounds = round;
        ctrl->eval_sweeps = evals;
        ctrl->iterations = total;
        ctrl->converged = converged;
        ctrl->last_residual = __longlong_as_double((long long)last);
        ctrl->backups = backups;
        ctrl->changed_total = changed_total;
    }
}

template <typename K>
static cudaError_t coop_grid(K kern, const Factors &F, int nitems, int &cache, int &grid) {
    if (cache <= 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 256, 0);
        if (e != cudaSuccess) return e;
        cache = o;
    }
    // Barrier cost grows with the number of blocks: use one block per SM as
    // long as two segments per thread cover the grid, more only for large
    // (bandwidth-bound) grids, never more than can be co-resident.
    const int cap = cache * F.num_sms;
    if (cap < 1) return cudaErrorCooperativeLaunchTooLarge;
    grid = (nitems + 511) / 512;
    if (grid < F.num_sms) grid = F.num_sms;
    if (grid > (nitems + 255) / 256) grid = (nitems + 255) / 256;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    return cudaSuccess;
}

template <typename T, int D, int VEC>
static cudaError_t launch_vi(const Factors &F, T *V, T *W, const SolveParams &sp, double *trace, cudaStream_t st) {
    static int occ = 0;
    BandArgs a = make_band_args(F);
    auto kern = solve_vi_kernel<T, D, VEC>;
    int grid = 1;
    cudaError_t e = coop_grid(kern, F, (int)(F.nstates / VEC), occ, grid);
    if (e != cudaSuccess) return e;
    Ctrl *ctrl = F.d_ctrl;
    SolveParams spc = sp;
    void *args[] = {(void *)&a, (void *)&V, (void *)&W, (void *)&spc, (void *)&ctrl, (void *)&trace};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(256), args, 0, st);
}

template <typename T, int D, int VEC>
static cudaError_t launch_pi(const Factors &F, T *V, T *W, uint8_t *pi, const SolveParams &sp, cudaStream_t st) {
    static int occ = 0;
    BandArgs a = make_band_args(F);
    auto kern = solve_pi_kernel<T, D, VEC>;
    int grid = 1;
    cudaError_t e = coop_grid(kern, F, (int)(F.nstates / VEC), occ, grid);
    if (e != cudaSuccess) return e;
    Ctrl *ctrl = F.d_ctrl;
    SolveParams spc = sp;
    void *args[] = {(void *)&a, (void *)&V, (void *)&W, (void *)&pi, (void *)&spc, (void *)&ctrl};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(256), args, 0, st);
}


template <typename T, int D, int VEC>
static cudaError_t launch_small(const Factors &F, bool pim, T *V, uint8_t *pi, const SolveParams &sp, double *trace,
                                cudaStream_t st) {
    BandArgs a = make_band_args(F);
    const size_t smem = 2 * (size_t)F.nstates * sizeof(T);
    if (pim) small_pi_kernel<T, D, VEC><<<1, 256, smem, st>>>(a, V, pi, sp, F.d_ctrl);
    else small_vi_kernel<T, D, VEC><<<1, 256, smem, st>>>(a, V, sp, F.d_ctrl, trace);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t solve_t(const Factors &F, bool pim, T *V, uint8_t *pi, const SolveParams &sp, double *trace,
                           bool small_ok, cudaStream_t st) {
    T *W = (T *)F.d_scratch;
    const int vec = band_pick_vec(F, sizeof(T), V, W);
    constexpr int V2 = (int)(16 / sizeof(T));
    cudaError_t e = cudaErrorInvalidValue;
    // one block's worth of segments, values within the default 48 KB of shared memory
    if (small_ok && F.nstates / vec <= kSmallMaxItems && 2 * (size_t)F.nstates * sizeof(T) <= 48 * 1024) {
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_small<T, DD, 1>(F, pim, V, pi, sp, trace, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_small<T, DD, V2>(F, pim, V, pi, sp, trace, st))); }
        return e;
    }
    if (pim) {
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_pi<T, DD, 1>(F, V, W, pi, sp, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_pi<T, DD, V2>(F, V, W, pi, sp, st))); }
    } else {
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_vi<T, DD, 1>(F, V, W, sp, trace, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_vi<T, DD, V2>(F, V, W, sp, trace, st))); }
    }
    return e;
}

cpmdp_status banded_solve(const Factors &F, cpmdp_precision prec, bool policy_iteration, void *V,
                          uint8_t *pi, const SolveOpts &o, cudaStream_t st) {
    SolveParams sp;
    sp.max_iter = o.max_iter;
    sp.max_eval_iter = o.max_eval_iter;
    sp.max_rounds = o.max_rounds;
    sp.tol = o.tol;
    sp.eval_tol = o.eval_tol;
    sp.margin = prec == CPMDP_F64 ? 1e-12 : 1e-6;
    sp.timeout_ns = (unsigned long long)(o.timeout_s * 1e9);
    sp.nactions = F.nactions;
    sp.inject_stall = o.inject_stall;
    sp.partial_eval = o.partial_eval;
    CPMDP_CUDA(cudaMemsetAsync(F.d_ctrl, 0, sizeof(Ctrl), st));
    // FP32 solves that fit one co-resident grid at one thread per 4 states
    // run on the barrier-free solver (fused = 2 asks for this file's
    // grid-barrier kernels instead).
    if (prec == CPMDP_F32 && o.fused == 1 && flow_eligible(F, policy_iteration, V, pi, o)) {
        Factors &M = const_cast<Factors &>(F);
        if (!M.d_flow) {
            CPMDP_CUDA(cudaMalloc(&M.d_flow, flow_bytes(F)));
            CPMDP_CUDA(cudaMemsetAsync(static_cast<char *>(M.d_flow) + flow_counter_bytes(), 0xFF,
                                       flow_bytes(F) - flow_counter_bytes(), st));
            M.flow_base = 0;
        }
        M.flow_pending = true;
        return flow_solve(F, policy_iteration, (float *)V, pi, sp, o.trace, st);
    }
    // FP32 value iteration of large 3-D grids: recorded graphs of the
    // plane-marching sweep (DRAM read about once per sweep)
    Factors &M2 = const_cast<Factors &>(F);
    M2.march_pending = false;
    if (prec == CPMDP_F32 && o.fused == 1 && !policy_iteration && !o.inject_stall &&
        march_eligible(F, V, F.d_scratch, nullptr)) {
        M2.march_pending = true;
        CPMDP_CUDA(march_solve(F, (float *)V, o.tol, o.max_iter, o.trace, st));
        return CPMDP_OK;
    }
    // grids one block covers: the shared-memory single-block kernels
    // (fused = 2 keeps the grid-barrier kernels; the stall aid needs their barrier)
    const bool small_ok = o.fused == 1 && !o.inject_stall;
    cudaError_t e;
    if (prec == CPMDP_F64) e = solve_t<double>(F, policy_iteration, (double *)V, pi, sp, o.trace, small_ok, st);
    else e = solve_t<float>(F, policy_iteration, (float *)V, pi, sp, o.trace, small_ok, st);
    CPMDP_CUDA(e);
    return CPMDP_OK;
}

cpmdp_status banded_solve_finished(const Factors &F, const Ctrl &dc, cudaStream_t st) {
    Factors &M = const_cast<Factors &>(F);
    if (!M.flow_pending) return CPMDP_OK;
    M.flow_pending = false;
    // Tags only grow, so a ring word can never look like one of a later
    // sweep. After a failed launch (which may have left words with any tag
    // above the base) and long before the tags wrap, the rings are cleared
    // to the tag 0xFFFFFFFF, which is never used.
    M.flow_base += dc.flow_tags + 2u;
    if (dc.status != 0 || dc.flow_tags == 0 || M.flow_base > 0x40000000u) {
        CPMDP_CUDA(cudaMemsetAsync(static_cast<char *>(M.d_flow) + flow_counter_bytes(), 0xFF,
                                   flow_bytes(F) - flow_counter_bytes(), st));
        CPMDP_CUDA(cudaStreamSynchronize(st));
        M.flow_base = 0;
    }
    return CPMDP_OK;
}

}  // namespace cpmdp
