// Banded (GridWorld) CP backup: fused stencil kernels and device-resident
// value / policy iteration.
//
// For a GridWorld every rank-1 CP term of an action is an outer product of
// identity factors and one shift factor (a unit move along one dimension,
// reflecting at the walls). E_a[V](s) therefore needs only the 2D face
// neighbours of s: with N_j the value reached by the unit move in direction
// j (V(s) itself when the move is blocked by a wall or an obstacle, which is
// the non-separable correction) and P_d = N_{2d} + N_{2d+1},
//     E_a = w_move * N_a + w_perp * sum_{d != d(a)} P_d + w_stay * V(s)
// (w_move = p, w_perp = (1-p)/(2(D-1)), w_stay = 1-p only for D = 1).
// Eq. 1 then gives Q_a = R(s) + gamma * E_a, V'(s) = max_a Q_a. The kernel
// fuses the neighbour gather, the CP-term sum, + R, x gamma, max/argmax
// and the infinity-norm residual. Work is O(|S| |C(s)| |A|) as in the
// paper's complexity section, with the shared pair sums.
//
// Layout: V, R, the per-state code and the policy are flat C-order arrays
// (Definition 2). A thread takes VEC consecutive states of one row of the
// last (contiguous) dimension: one 16-byte load per row neighbour, the two
// in-row halo values with scalar loads, codes as one packed load.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <type_traits>

#include "internal.h"

namespace cpmdp {

template <int D> struct CodeType { using type = uint32_t; };
template <> struct CodeType<1> { using type = uint8_t; };
template <> struct CodeType<2> { using type = uint8_t; };
template <> struct CodeType<3> { using type = uint8_t; };
template <> struct CodeType<4> { using type = uint16_t; };
template <> struct CodeType<5> { using type = uint16_t; };
template <> struct CodeType<6> { using type = uint16_t; };
template <> struct CodeType<7> { using type = uint16_t; };

struct BandArgs {
    int nstates;
    int nlast;
    int stride[kMaxDim];
    double w_move, w_perp, w_stay, gamma;
    const void *code;
    const float *R32;
    const double *R64;
};

enum Mode : int { M_VI = 0, M_EVAL = 1, M_IMPROVE = 2, M_GREEDY = 3 };

template <typename T, int VEC> struct alignas(sizeof(T) * VEC) VPack { T v[VEC]; };

template <typename T, int VEC>
__device__ __forceinline__ void load_pack(const T *p, T (&out)[VEC]) {
    VPack<T, VEC> pk = *reinterpret_cast<const VPack<T, VEC> *>(p);
#pragma unroll
    for (int k = 0; k < VEC; k++) out[k] = pk.v[k];
}

template <typename T, int VEC>
__device__ __forceinline__ void store_pack(T *p, const T (&in)[VEC]) {
    VPack<T, VEC> pk;
#pragma unroll
    for (int k = 0; k < VEC; k++) pk.v[k] = in[k];
    *reinterpret_cast<VPack<T, VEC> *>(p) = pk;
}

template <typename TA> __device__ __forceinline__ TA rew(const BandArgs &a, int s);
template <> __device__ __forceinline__ float rew<float>(const BandArgs &a, int s) { return a.R32[s]; }
template <> __device__ __forceinline__ double rew<double>(const BandArgs &a, int s) { return a.R64[s]; }

// One row segment: states s0 .. s0+VEC-1 of a row of the last dimension.
// load() issues every global load of the segment at once: the neighbour
// addresses are clamped into [0, |S|) arithmetically instead of being chosen
// from the per-state code, so no load waits for another. A clamped address
// only differs from the true neighbour where that neighbour does not exist,
// and there the code marks the move as blocked and finish() uses V(s).
// finish() applies the codes, forms Q for every action and stores.
template <typename T, typename TA, int D, int VEC>
struct Segment {
    using C = typename CodeType<D>::type;
    static constexpr int NB = 2 * D;
    C code[VEC];
    T vs[VEC];
    T rows[D > 1 ? 2 * (D - 1) : 1][VEC];
    T halo_m, halo_p;
    TA r[VEC];
    uint8_t act[VEC];

    __device__ __forceinline__ void load(const BandArgs &a, const T *V, const uint8_t *pi, int mode, int s0) {
        load_pack<C, VEC>(static_cast<const C *>(a.code) + s0, code);
        load_pack<T, VEC>(V + s0, vs);
        const int last = a.nstates - VEC;
#pragma unroll
        for (int d = 0; d < D - 1; d++) {
            int lo = s0 - a.stride[d], hi = s0 + a.stride[d];
            lo = lo < 0 ? 0 : lo;
            hi = hi > last ? last : hi;
            load_pack<T, VEC>(V + lo, rows[2 * d]);
            load_pack<T, VEC>(V + hi, rows[2 * d + 1]);
        }
        halo_m = V[s0 > 0 ? s0 - 1 : 0];
        halo_p = V[s0 + VEC < a.nstates ? s0 + VEC : a.nstates - 1];
#pragma unroll
        for (int k = 0; k < VEC; k++) r[k] = rew<TA>(a, s0 + k);
        if (mode == M_EVAL || mode == M_IMPROVE) {
#pragma unroll
            for (int k = 0; k < VEC; k++) act[k] = pi[s0 + k];
        }
    }

    // Returns the largest |V' - V| over the non-obstacle states.
    __device__ __forceinline__ TA finish(const BandArgs &a, T *W, uint8_t *pi, int mode, TA margin, int s0,
                                         unsigned &changed) const {
        constexpr unsigned OBST = 1u << (2 * D);
        constexpr unsigned TERM = 1u << (2 * D + 1);
        TA self[VEC];
#pragma unroll
        for (int k = 0; k < VEC; k++) self[k] = (TA)vs[k];
        TA nb[NB][VEC];
#pragma unroll
        for (int j = 0; j < 2 * (D - 1); j++)
#pragma unroll
            for (int k = 0; k < VEC; k++) nb[j][k] = ((code[k] >> j) & 1u) ? self[k] : (TA)rows[j][k];
        {
            const int jm = 2 * (D - 1), jp = jm + 1;
#pragma unroll
            for (int k = 0; k < VEC; k++) {
                const TA left = (k == 0) ? (TA)halo_m : self[k > 0 ? k - 1 : 0];
                const TA right = (k == VEC - 1) ? (TA)halo_p : self[k < VEC - 1 ? k + 1 : 0];
                nb[jm][k] = ((code[k] >> jm) & 1u) ? self[k] : left;
                nb[jp][k] = ((code[k] >> jp) & 1u) ? self[k] : right;
            }
        }
        const TA wm = (TA)a.w_move, wp = (TA)a.w_perp, wst = (TA)a.w_stay, g = (TA)a.gamma;
        TA out[VEC];
        TA res = 0;
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const int s = s0 + k;
            const unsigned c = code[k];
            const TA rk = r[k];
            TA v;
            if (c & OBST) {
                v = 0;
                if (pi && (mode == M_VI || mode == M_GREEDY)) pi[s] = 255;
            } else if (c & TERM) {
                v = rk;
                if (pi && (mode == M_VI || mode == M_GREEDY)) pi[s] = 255;
            } else {
                TA P[D], perp[D];
#pragma unroll
                for (int d = 0; d < D; d++) P[d] = nb[2 * d][k] + nb[2 * d + 1][k];
                TA acc = 0;
#pragma unroll
                for (int d = 0; d < D; d++) { perp[d] = acc; acc += P[d]; }
                acc = 0;
#pragma unroll
                for (int d = D - 1; d >= 0; d--) { perp[d] += acc; acc += P[d]; }
                const TA stay = wst * self[k];
                if (mode == M_EVAL) {
                    const int ak = act[k];
                    TA nbv = nb[0][k], pv = perp[0];
#pragma unroll
                    for (int j = 1; j < NB; j++)
                        if (ak == j) { nbv = nb[j][k]; pv = perp[j / 2]; }
                    v = rk + g * (wm * nbv + wp * pv + stay);
                } else {
                    TA best = rk + g * (wm * nb[0][k] + wp * perp[0] + stay);
                    int arg = 0;
                    TA qold = best;
                    const int old = (mode == M_IMPROVE) ? (int)act[k] : 0;
#pragma unroll
                    for (int j = 1; j < NB; j++) {
                        const TA q = rk + g * (wm * nb[j][k] + wp * perp[j / 2] + stay);
                        if (q > best) { best = q; arg = j; }
                        if (j == old) qold = q;
                    }
                    if (mode == M_IMPROVE) {
                        const TA thr = margin * ((TA)1 + (qold < 0 ? -qold : qold));
                        if (arg != old && best > qold + thr) { pi[s] = (uint8_t)arg; changed++; }
                        v = self[k];
                    } else {
                        if (pi) pi[s] = (uint8_t)arg;
                        v = best;
                    }
                }
            }
            out[k] = v;
            if (!(c & OBST) && (mode == M_VI || mode == M_EVAL)) {
                const TA dv = v > self[k] ? v - self[k] : self[k] - v;
                res = dv > res ? dv : res;
            }
        }
        if (W) {
            T o[VEC];
#pragma unroll
            for (int k = 0; k < VEC; k++) o[k] = (T)out[k];
            store_pack<T, VEC>(W + s0, o);
        }
        return res;
    }
};

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

__device__ __forceinline__ unsigned warp_sum(unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Block-wide max (result valid in thread 0). Needs blockDim a multiple of 32.
__device__ __forceinline__ double block_max(double v, double *sh) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        v = warp_max(v);
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0u;
        v = warp_sum(v);
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_add_release(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a co-resident (cooperative) grid that also counts
// how many blocks raised `flag` (thread 0's value) in the step it closes.
// Barrier number n uses counter bar[n % 2]: the low 32 bits count arrivals
// (n/2 + 1) * nblocks are expected once everyone has arrived, the high 32
// bits count raised flags. A block cannot reach barrier n+2 before every
// block has left barrier n+1, so the value read when barrier n completes
// holds exactly the arrivals up to barrier n; the flags of step n are its
// high part minus the high part seen at barrier n-2 (prev0 / prev1 for
// even / odd n, kept by thread 0).
// Every wait gives up after timeout_ns or when another block has recorded
// a status: returns -1 (CPMDP_ETIMEOUT stored in the status word).
// stall: testing aid, this block leaves without arriving.
__device__ __forceinline__ long long grid_sync_count(Ctrl *c, int n, unsigned nblocks, int flag,
                                                     unsigned long long timeout_ns,
                                                     unsigned long long &prev0, unsigned long long &prev1,
                                                     bool stall) {
    __shared__ long long result;
    __syncthreads();
    if (threadIdx.x == 0) {
        result = 0;
        if (stall) {
            if (nblocks == 1) atomicCAS(&c->status, 0, (int)CPMDP_ETIMEOUT);
            result = -1;
        } else {
            unsigned long long *ctr = &c->bar[n & 1];
            red_add_release(ctr, 1ull | ((unsigned long long)(flag != 0) << 32));
            const unsigned long long target = (unsigned long long)(n / 2 + 1) * nblocks;
            unsigned long long v = ld_acquire(ctr);
            if ((v & 0xFFFFFFFFull) < target) {
                const unsigned long long t0 = global_ns();
                unsigned spins = 0;
                do {
                    __nanosleep(32);
                    v = ld_acquire(ctr);
                    if ((++spins & 15u) == 0 && (v & 0xFFFFFFFFull) < target) {
                        if (*(volatile int *)&c->status != 0) { result = -1; break; }
                        if (global_ns() - t0 > timeout_ns) {
                            atomicCAS(&c->status, 0, (int)CPMDP_ETIMEOUT);
                            result = -1;
                            break;
                        }
                    }
                } while ((v & 0xFFFFFFFFull) < target);
            }
            if (result == 0) {
                const unsigned long long hi = v >> 32;
                const unsigned long long prev = (n & 1) ? prev1 : prev0;
                result = (long long)(hi - prev);
                if (n & 1) prev1 = hi;
                else prev0 = hi;
            }
        }
    }
    __syncthreads();
    return result;
}

struct SolveParams {
    int policy_iteration;
    int max_iter;
    int max_eval_iter;
    int max_rounds;
    double tol;
    double eval_tol;
    double margin;
    unsigned long long timeout_ns;
    int nactions;
    int inject_stall;
};

template <typename T, typename TA, int D, int VEC>
__device__ __forceinline__ TA sweep_all(const BandArgs &a, const T *V, T *W, uint8_t *pi, int mode,
                                        TA margin, unsigned &changed) {
    const int nitems = a.nstates / VEC;
    const int step = gridDim.x * blockDim.x;
    TA res = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nitems; i += 2 * step) {
        Segment<T, TA, D, VEC> s0, s1;
        const bool two = i + step < nitems;
        s0.load(a, V, pi, mode, i * VEC);
        if (two) s1.load(a, V, pi, mode, (i + step) * VEC);
        TA r = s0.finish(a, W, pi, mode, margin, i * VEC, changed);
        res = r > res ? r : res;
        if (two) {
            r = s1.finish(a, W, pi, mode, margin, (i + step) * VEC, changed);
            res = r > res ? r : res;
        }
    }
    return res;
}

// One backup sweep (any mode), non-persistent. res_out: atomic max of the
// residual (bits of a non-negative double); changed_out: atomic count.
template <typename T, typename TA, int D, int VEC>
__global__ void __launch_bounds__(256) sweep_kernel(BandArgs a, const T *__restrict__ V,
                                                    T *__restrict__ W, uint8_t *pi, int mode,
                                                    double margin, unsigned long long *res_out,
                                                    unsigned *changed_out) {
    __shared__ double shd[32];
    __shared__ unsigned shu[32];
    unsigned changed = 0;
    const TA r = sweep_all<T, TA, D, VEC>(a, V, W, pi, mode, (TA)margin, changed);
    if (res_out) {
        const double m = block_max((double)r, shd);
        if (threadIdx.x == 0 && m > 0.0) atomicMax(res_out, (unsigned long long)__double_as_longlong(m));
    }
    if (changed_out) {
        const unsigned c = block_sum(changed, shu);
        if (threadIdx.x == 0 && c) atomicAdd(changed_out, c);
    }
}

// Device-resident value iteration / policy iteration: one cooperative
// launch. Each sweep ends in a grid barrier whose arrival also reports
// whether the block's residual is still >= tol (VI, evaluation) or whether
// the block changed an action (improvement), so every block learns the
// stopping decision from the barrier itself. The residual value goes to
// res_slot[k % 3] by atomic max (slot k+1 is cleared by block 0 during
// sweep k, after every block has read slot k-2); it is read only for the
// trace and at the end.
template <typename T, int D, int VEC>
__global__ void __launch_bounds__(256) solve_kernel(BandArgs a, T *V, T *Wbuf, uint8_t *pi,
                                                    SolveParams sp, Ctrl *ctrl, double *trace) {
    typedef T TA;
    __shared__ double shd[32];
    __shared__ unsigned shu[32];
    const unsigned nb = gridDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    T *cur = V, *nxt = Wbuf;
    int ks = 0;              // residual-producing sweeps so far
    int total = 0;           // all sweeps
    int nbar = 0;            // grid barriers so far
    long long backups = 0;
    int converged = 0;
    unsigned dummy = 0;
    unsigned long long ph0 = 0ull, ph1 = 0ull;
    const bool stall = sp.inject_stall && blockIdx.x == 0;

    // block max of r; thread 0 posts it to the sweep's slot and returns
    // whether it is >= thr
    auto post_res = [&](TA r, double thr) -> int {
        const double m = block_max((double)r, shd);
        int flag = 0;
        if (threadIdx.x == 0) {
            if (m > 0.0) atomicMax(&ctrl->res_slot[ks % 3], (unsigned long long)__double_as_longlong(m));
            flag = !(m < thr);
        }
        if (lead) ctrl->res_slot[(ks + 1) % 3] = 0ull;
        return flag;
    };
    auto slot_value = [&](int k) {
        return __longlong_as_double((long long)*(volatile unsigned long long *)&ctrl->res_slot[k % 3]);
    };

    if (!sp.policy_iteration) {
        while (total < sp.max_iter) {
            const TA r = sweep_all<T, TA, D, VEC>(a, cur, nxt, nullptr, M_VI, (TA)0, dummy);
            const int flag = post_res(r, sp.tol);
            const long long open = grid_sync_count(ctrl, nbar++, nb, flag, sp.timeout_ns, ph0, ph1, stall);
            if (open < 0) return;
            if (trace && lead) trace[total] = slot_value(ks);
            ks++; total++;
            backups += (long long)a.nstates * sp.nactions;
            T *t = cur; cur = nxt; nxt = t;
            if (open == 0) { converged = 1; break; }
        }
    } else {
        // initial policy: greedy with respect to the input V
        sweep_all<T, TA, D, VEC>(a, cur, nullptr, pi, M_GREEDY, (TA)0, dummy);
        if (grid_sync_count(ctrl, nbar++, nb, 0, sp.timeout_ns, ph0, ph1, stall) < 0) return;
        total++;
        backups += (long long)a.nstates * sp.nactions;
        int round = 0, evals = 0;
        while (round < sp.max_rounds) {
            int e = 0, eval_ok = 0;
            while (e < sp.max_eval_iter) {
                const TA r = sweep_all<T, TA, D, VEC>(a, cur, nxt, pi, M_EVAL, (TA)0, dummy);
                const int flag = post_res(r, sp.eval_tol);
                const long long open = grid_sync_count(ctrl, nbar++, nb, flag, sp.timeout_ns, ph0, ph1, false);
                if (open < 0) return;
                ks++; e++; total++;
                backups += a.nstates;
                T *t = cur; cur = nxt; nxt = t;
                if (open == 0) { eval_ok = 1; break; }
            }
            evals += e;
            unsigned changed = 0;
            sweep_all<T, TA, D, VEC>(a, cur, nullptr, pi, M_IMPROVE, (TA)sp.margin, changed);
            const unsigned c = block_sum(changed, shu);
            if (threadIdx.x == 0 && c) atomicAdd(&ctrl->changed_total, c);
            const long long moved = grid_sync_count(ctrl, nbar++, nb, threadIdx.x == 0 && c > 0,
                                                    sp.timeout_ns, ph0, ph1, false);
            if (moved < 0) return;
            total++;
            round++;
            backups += (long long)a.nstates * sp.nactions;
            if (moved == 0) { converged = eval_ok; break; }
            if (!eval_ok) break;
        }
        if (lead) { ctrl->rounds = round; ctrl->eval_sweeps = evals; }
    }
    // the last iterate must end in V
    if (cur != V) {
        const int n = a.nstates;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) V[i] = cur[i];
    }
    if (lead) {
        ctrl->iterations = total;
        ctrl->converged = converged;
        ctrl->last_residual = ks > 0 ? slot_value(ks - 1) : 0.0;
        ctrl->backups = backups;
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
                               T *__restrict__ Q, int act) {
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
                                 T *__restrict__ W, uint8_t *pi, int nact) {
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
                                      const T *__restrict__ W, unsigned long long *res) {
    __shared__ double shd[32];
    double m = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        if (cell[s] != CPMDP_CELL_OBSTACLE) m = fmax(m, fabs((double)W[s] - (double)V[s]));
    m = block_max(m, shd);
    if (threadIdx.x == 0 && m > 0.0) atomicMax(res, (unsigned long long)__double_as_longlong(m));
}

// ---------------------------------------------------------------------------
// host side

static BandArgs make_args(const Factors &F) {
    BandArgs a;
    a.nstates = (int)F.nstates;
    a.nlast = (int)F.shape[F.ndim - 1];
    for (int d = 0; d < kMaxDim; d++) a.stride[d] = d < F.ndim ? (int)F.stride[d] : 0;
    a.w_move = F.w_move;
    a.w_perp = F.w_perp;
    a.w_stay = F.w_stay;
    a.gamma = F.gamma;
    a.code = F.d_code;
    a.R32 = F.d_R32;
    a.R64 = F.d_R64;
    return a;
}

static bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

// Widest segment length usable for this row length, element size and pointers.
static int pick_vec(const Factors &F, size_t elem, const void *p0, const void *p1) {
    const int64_t n = F.shape[F.ndim - 1];
    const int v = (int)(16 / elem);  // 4 floats or 2 doubles
    if (n % v == 0 && aligned16(p0) && aligned16(p1)) return v;
    return 1;
}

#define CPMDP_DISPATCH_D(D_, ...)                     \
    switch (D_) {                                     \
        case 1: { constexpr int DD = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int DD = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int DD = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int DD = 4; __VA_ARGS__; } break; \
        case 5: { constexpr int DD = 5; __VA_ARGS__; } break; \
        case 6: { constexpr int DD = 6; __VA_ARGS__; } break; \
        case 7: { constexpr int DD = 7; __VA_ARGS__; } break; \
        case 8: { constexpr int DD = 8; __VA_ARGS__; } break; \
        case 9: { constexpr int DD = 9; __VA_ARGS__; } break; \
        default: break;                               \
    }

template <typename T, typename TA, int D, int VEC>
static cudaError_t launch_sweep(const Factors &F, const T *V, T *W, uint8_t *pi, int mode, double margin,
                                unsigned long long *res, unsigned *chg, cudaStream_t st) {
    BandArgs a = make_args(F);
    const int nitems = (int)(F.nstates / VEC);
    int grid = (nitems + 255) / 256;
    const int cap = (F.num_sms > 0 ? F.num_sms : 148) * 16;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    sweep_kernel<T, TA, D, VEC><<<grid, 256, 0, st>>>(a, V, W, pi, mode, margin, res, chg);
    return cudaGetLastError();
}

template <typename T, typename TA>
static cudaError_t sweep_any(const Factors &F, const T *V, T *W, uint8_t *pi, int mode, double margin,
                             unsigned long long *res, unsigned *chg, cudaStream_t st) {
    const int vec = pick_vec(F, sizeof(T), V, W);
    cudaError_t e = cudaErrorInvalidValue;
    if (vec == 1) {
        CPMDP_DISPATCH_D(F.ndim, e = (launch_sweep<T, TA, DD, 1>(F, V, W, pi, mode, margin, res, chg, st)));
    } else {
        constexpr int V2 = (int)(16 / sizeof(T));
        CPMDP_DISPATCH_D(F.ndim, e = (launch_sweep<T, TA, DD, V2>(F, V, W, pi, mode, margin, res, chg, st)));
    }
    return e;
}

cpmdp_status banded_backup(const Factors &F, cpmdp_precision prec, const void *Vin, void *Vout,
                           uint8_t *pi, double *res, cudaStream_t st) {
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    if (rb) CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    cudaError_t e;
    if (prec == CPMDP_F64)
        e = sweep_any<double, double>(F, (const double *)Vin, (double *)Vout, pi, M_VI, 0.0, rb, nullptr, st);
    else
        e = sweep_any<float, float>(F, (const float *)Vin, (float *)Vout, pi, M_VI, 0.0, rb, nullptr, st);
    CPMDP_CUDA(e);
    return CPMDP_OK;
}

// FP64 sweep of a float value tensor: certified residual and FP64 argmax.
cpmdp_status banded_certify(const Factors &F, const float *V, uint8_t *pi, double *res, cudaStream_t st) {
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    CPMDP_CUDA((sweep_any<float, double>(F, V, (float *)nullptr, pi, M_VI, 0.0, rb, nullptr, st)));
    return CPMDP_OK;
}

template <typename T, int D, int VEC>
static cudaError_t launch_solve(const Factors &F, T *V, T *W, uint8_t *pi, const SolveParams &sp,
                                double *trace, cudaStream_t st) {
    BandArgs a = make_args(F);
    auto kern = solve_kernel<T, D, VEC>;
    static int occ = -1;  // per instantiation
    if (occ < 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 256, 0);
        if (e != cudaSuccess) return e;
        occ = o;
    }
    const int nitems = (int)(F.nstates / VEC);
    int grid = (nitems + 255) / 256;
    const int cap = occ * F.num_sms;
    if (cap < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    Ctrl *ctrl = F.d_ctrl;
    SolveParams spc = sp;
    void *args[] = {(void *)&a, (void *)&V, (void *)&W, (void *)&pi, (void *)&spc, (void *)&ctrl, (void *)&trace};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(256), args, 0, st);
}

cpmdp_status banded_solve(const Factors &F, cpmdp_precision prec, bool policy_iteration, void *V,
                          uint8_t *pi, const SolveOpts &o, cudaStream_t st) {
    SolveParams sp;
    sp.policy_iteration = policy_iteration ? 1 : 0;
    sp.max_iter = o.max_iter;
    sp.max_eval_iter = o.max_eval_iter;
    sp.max_rounds = o.max_rounds;
    sp.tol = o.tol;
    sp.eval_tol = o.eval_tol;
    sp.margin = prec == CPMDP_F64 ? 1e-12 : 1e-6;
    sp.timeout_ns = (unsigned long long)(o.timeout_s * 1e9);
    sp.nactions = F.nactions;
    sp.inject_stall = o.inject_stall;
    CPMDP_CUDA(cudaMemsetAsync(F.d_ctrl, 0, sizeof(Ctrl), st));
    cudaError_t e = cudaErrorInvalidValue;
    if (prec == CPMDP_F64) {
        double *Vd = (double *)V, *W = (double *)F.d_scratch;
        const int vec = pick_vec(F, sizeof(double), Vd, W);
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_solve<double, DD, 1>(F, Vd, W, pi, sp, o.trace, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_solve<double, DD, 2>(F, Vd, W, pi, sp, o.trace, st))); }
    } else {
        float *Vf = (float *)V, *W = (float *)F.d_scratch;
        const int vec = pick_vec(F, sizeof(float), Vf, W);
        if (vec == 1) { CPMDP_DISPATCH_D(F.ndim, e = (launch_solve<float, DD, 1>(F, Vf, W, pi, sp, o.trace, st))); }
        else { CPMDP_DISPATCH_D(F.ndim, e = (launch_solve<float, DD, 4>(F, Vf, W, pi, sp, o.trace, st))); }
    }
    CPMDP_CUDA(e);
    return CPMDP_OK;
}

// Plain baseline value iteration: per sweep |A| Q kernels, a max kernel, a
// residual kernel and a device-to-host copy of the residual checked on the
// host. Fills host_ctrl (iterations, converged, residual, backups).
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
    int k = 0, conv = 0;
    double res = INFINITY;
    while (k < o.max_iter) {
        CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(unsigned long long), st));
        for (int act = 0; act < F.nactions; act++) plain_q_kernel<T><<<grid, 256, 0, st>>>(a, cur, R, Q, act);
        plain_max_kernel<T><<<grid, 256, 0, st>>>(a, Q, R, nxt, nullptr, F.nactions);
        plain_residual_kernel<T><<<rgrid, 256, 0, st>>>(n, F.d_cell, cur, nxt, rb);
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
        for (int act = 0; act < F.nactions; act++) plain_q_kernel<T><<<grid, 256, 0, st>>>(a, V, R, Q, act);
        plain_max_kernel<T><<<grid, 256, 0, st>>>(a, Q, R, spare, pi, F.nactions);
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
