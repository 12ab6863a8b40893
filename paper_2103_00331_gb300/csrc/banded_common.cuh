// Device code shared by the banded (GridWorld) kernels.
//
// For a GridWorld every rank-1 CP term of an action is an outer product of
// identity factors and one shift factor (a unit move along one dimension,
// reflecting at the walls). E_a[V](s) therefore needs only the 2D face
// neighbours of s: with N_j the value reached by the unit move in direction
// j (V(s) itself when the move is blocked by a wall or an obstacle, the
// non-separable correction) and P_d = N_{2d} + N_{2d+1},
//     E_{(d,sigma)} = w_move N_{(d,sigma)} + w_perp sum_{d' != d} P_{d'} + w_stay V(s)
// (w_move = p, w_perp = (1-p)/(2(D-1)), w_stay = 1-p only for D = 1), and
// Eq. 1 gives Q_a = R(s) + gamma E_a, V'(s) = max_a Q_a. Work is
// O(|S| |C(s)| |A|) as in the paper's complexity section, with the pair
// sums shared by all actions.
//
// Layout: V, R, the per-state code and the policy are flat C-order arrays
// (Definition 2). A thread takes VEC consecutive states of one row of the
// last (contiguous) dimension: one 16-byte load per row neighbour, two
// scalar halo loads, the codes as one packed load.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

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
    float wf_move, wf_perp, wf_stay, wf_gamma;  // the same rounded to float, for the FP32 kernels
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

// Transition weights and gamma in the working precision (no conversion in
// the kernels: float <-> double conversions issue on GB300's narrow FP64 pipe).
template <typename TA>
__device__ __forceinline__ void weights(const BandArgs &a, TA &wm, TA &wp, TA &wst, TA &g);
template <>
__device__ __forceinline__ void weights<float>(const BandArgs &a, float &wm, float &wp, float &wst, float &g) {
    wm = a.wf_move; wp = a.wf_perp; wst = a.wf_stay; g = a.wf_gamma;
}
template <>
__device__ __forceinline__ void weights<double>(const BandArgs &a, double &wm, double &wp, double &wst, double &g) {
    wm = a.w_move; wp = a.w_perp; wst = a.w_stay; g = a.gamma;
}

// |a - b| with the sign bit cleared (never -0), so that residual maxima can
// be taken on bit patterns (block_max_bits).
__device__ __forceinline__ float abs_diff(float a, float b) { return fabsf(a - b); }
__device__ __forceinline__ double abs_diff(double a, double b) { return fabs(a - b); }

// Residual m (bits of a non-negative double, or a NaN) below tol > 0: the
// same order on the bits read as unsigned integers, with no FP64
// instruction; a NaN is never below tol, as in floating point.
__device__ __forceinline__ bool below_tol(unsigned long long mbits, double tol) {
    return mbits < (unsigned long long)__double_as_longlong(tol);
}

template <typename TA> __device__ __forceinline__ TA rew(const BandArgs &a, int s);
template <> __device__ __forceinline__ float rew<float>(const BandArgs &a, int s) { return a.R32[s]; }
template <> __device__ __forceinline__ double rew<double>(const BandArgs &a, int s) { return a.R64[s]; }

// perp[d] = sum over d' != d of the pair sums P_d' = N_{2d'} + N_{2d'+1}
// (prefix + suffix sums).
template <typename TA, int D>
__device__ __forceinline__ void perp_of(const TA (&nb)[2 * D], TA (&perp)[D]) {
    TA P[D];
#pragma unroll
    for (int d = 0; d < D; d++) P[d] = nb[2 * d] + nb[2 * d + 1];
    TA acc = 0;
#pragma unroll
    for (int d = 0; d < D; d++) { perp[d] = acc; acc += P[d]; }
    acc = 0;
#pragma unroll
    for (int d = D - 1; d >= 0; d--) { perp[d] += acc; acc += P[d]; }
}

// Larger of a and b: fmaxf for float (one instruction); for double the
// compare-select form (GB300's narrow FP64 pipe takes either as one op).
template <typename TA> __device__ __forceinline__ TA vmax(TA a, TA b) { return b > a ? b : a; }
template <> __device__ __forceinline__ float vmax<float>(float a, float b) { return fmaxf(a, b); }

// max over actions of E_a at one state, from its blocked-move-resolved
// neighbour values (value iteration without the argmax; see vi_state).
template <typename TA, int D>
__device__ __forceinline__ TA vi_best_e(TA self, const TA (&nb)[2 * D], TA wm, TA wp, TA wst) {
    TA perp[D];
    perp_of<TA, D>(nb, perp);
    const TA stay = (D == 1) ? wst * self : (TA)0;
    TA bestE = 0;
#pragma unroll
    for (int d = 0; d < D; d++) {
        const TA m = vmax<TA>(nb[2 * d], nb[2 * d + 1]);
        // D = 1: the slip stays in place with weight w_stay; D >= 2 has none
        const TA e = (D == 1) ? wm * m + wp * perp[d] + stay : wm * m + wp * perp[d];
        bestE = d == 0 ? e : vmax<TA>(bestE, e);
    }
    return bestE;
}

// Value-iteration backup of one state from its blocked-move-resolved
// neighbour values nb (Eq. 1). Because w_move, w_perp and gamma are >= 0 and
// rounding is monotone, max_sigma E_(d,sigma) is E at max(N_{d,-}, N_{d,+})
// and max_a fl(R + gamma E_a) = fl(R + gamma max_a E_a): the same value (and
// the same lowest-index argmax) as evaluating every action, with D instead
// of 2D expectation chains. Terminals keep R, obstacles 0. ARG = false
// leaves arg unset and takes both maxima with vmax (vi_best_e: the same
// values; only the sign of a zero maximum may differ from the compare-select
// form).
template <typename TA, int D, bool ARG = true>
__device__ __forceinline__ TA vi_state(TA self, const TA (&nb)[2 * D], unsigned c, TA r, TA wm, TA wp, TA wst, TA g,
                                       int &arg) {
    TA bestE = 0;
    if (ARG) {
        TA perp[D];
        perp_of<TA, D>(nb, perp);
        const TA stay = (D == 1) ? wst * self : (TA)0;
        arg = 0;
#pragma unroll
        for (int d = 0; d < D; d++) {
            const bool up = nb[2 * d + 1] > nb[2 * d];
            const TA m = up ? nb[2 * d + 1] : nb[2 * d];
            const TA e = (D == 1) ? wm * m + wp * perp[d] + stay : wm * m + wp * perp[d];
            if (d == 0 || e > bestE) { bestE = e; arg = 2 * d + (up ? 1 : 0); }
        }
    } else {
        bestE = vi_best_e<TA, D>(self, nb, wm, wp, wst);
    }
    TA v = r + g * bestE;
    if (c & (1u << (2 * D + 1))) v = r;
    if (c & (1u << (2 * D))) v = 0;
    return v;
}

// Policy-evaluation backup of one state for its fixed action `act` (Eq. 1
// with the action fixed). The action's neighbour and perpendicular sum are
// picked by a tree of selects on the action's bits for D <= 3 (depth 3
// instead of a chain of 2D - 1 selects; measured 3 % faster policy
// evaluation at 64^3), for larger D by a chain; for terminals and obstacles
// (act 255) the pick does not matter.
template <typename TA, int D>
__device__ __forceinline__ TA eval_state(TA self, const TA (&nb)[2 * D], unsigned c, TA r, int act, TA wm, TA wp,
                                         TA wst, TA g) {
    TA perp[D];
    perp_of<TA, D>(nb, perp);
    const TA stay = wst * self;
    const bool b0 = act & 1, b1 = (act >> 1) & 1, b2 = (act >> 2) & 1;
    TA nbv = nb[0], pv = perp[0];
    if (D > 3) {
#pragma unroll
        for (int j = 1; j < 2 * D; j++)
            if (act == j) { nbv = nb[j]; pv = perp[j / 2]; }
    } else if (D == 1) {
        nbv = b0 ? nb[1] : nb[0];
        pv = perp[0];
    } else if (D == 2) {
        const TA x01 = b0 ? nb[1] : nb[0], x23 = b0 ? nb[2 * D - 1] : nb[2 * D - 2];
        nbv = b1 ? x23 : x01;
        pv = b1 ? perp[D - 1] : perp[0];
    } else {
        const TA x01 = b0 ? nb[1] : nb[0], x23 = b0 ? nb[3 % (2 * D)] : nb[2 % (2 * D)];
        const TA x45 = b0 ? nb[5 % (2 * D)] : nb[4 % (2 * D)];
        const TA y = b1 ? x23 : x01;
        nbv = b2 ? x45 : y;
        const TA p01 = b1 ? perp[1 % D] : perp[0];
        pv = b2 ? perp[2 % D] : p01;
    }
    TA v = r + g * (wm * nbv + wp * pv + stay);
    if (c & (1u << (2 * D + 1))) v = r;
    if (c & (1u << (2 * D))) v = 0;
    return v;
}

// One row segment: states s0 .. s0+VEC-1 of a row of the last dimension.
// load() issues every global load of the segment at once: the neighbour
// addresses are clamped into [0, |S|) arithmetically instead of being chosen
// from the per-state code, so no load waits for another. A clamped address
// only differs from the true neighbour where that neighbour does not exist,
// and there the code marks the move as blocked and V(s) is used instead.
template <typename T, typename TA, int D, int VEC>
struct Segment {
    using C = typename CodeType<D>::type;
    static constexpr int NB = 2 * D;
    static constexpr unsigned OBST = 1u << (2 * D);
    static constexpr unsigned TERM = 1u << (2 * D + 1);
    C code[VEC];
    T vs[VEC];
    T rows[D > 1 ? 2 * (D - 1) : 1][VEC];
    T halo_m, halo_p;
    TA r[VEC];
    uint8_t act[VEC];

    template <int MODE>
    __device__ __forceinline__ void load(const BandArgs &a, const T *V, const uint8_t *pi, int s0) {
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
        if (MODE == M_EVAL || MODE == M_IMPROVE) {
#pragma unroll
            for (int k = 0; k < VEC; k++) act[k] = pi[s0 + k];
        }
    }

    // Neighbour values with the blocked moves replaced by V(s).
    __device__ __forceinline__ void neighbours(TA (&self)[VEC], TA (&nb)[NB][VEC]) const {
#pragma unroll
        for (int k = 0; k < VEC; k++) self[k] = (TA)vs[k];
#pragma unroll
        for (int j = 0; j < 2 * (D - 1); j++)
#pragma unroll
            for (int k = 0; k < VEC; k++) nb[j][k] = ((code[k] >> j) & 1u) ? self[k] : (TA)rows[j][k];
        const int jm = 2 * (D - 1), jp = jm + 1;
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const TA left = (k == 0) ? (TA)halo_m : self[k > 0 ? k - 1 : 0];
            const TA right = (k == VEC - 1) ? (TA)halo_p : self[k < VEC - 1 ? k + 1 : 0];
            nb[jm][k] = ((code[k] >> jm) & 1u) ? self[k] : left;
            nb[jp][k] = ((code[k] >> jp) & 1u) ? self[k] : right;
        }
    }

    // perp[d] = sum over d' != d of the pair sums (prefix + suffix sums).
    __device__ __forceinline__ static void perp_sums(const TA (&nb)[NB][VEC], int k, TA (&perp)[D]) {
        TA P[D];
#pragma unroll
        for (int d = 0; d < D; d++) P[d] = nb[2 * d][k] + nb[2 * d + 1][k];
        TA acc = 0;
#pragma unroll
        for (int d = 0; d < D; d++) { perp[d] = acc; acc += P[d]; }
        acc = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; d--) { perp[d] += acc; acc += P[d]; }
    }

    // Value-iteration backup of the segment (vi_state per state). Writes V'
    // to W (if not null) and the policy to pi (WITH_PI); returns the largest
    // |V' - V| over non-obstacle states.
    template <bool WITH_PI>
    __device__ __forceinline__ TA finish_vi(const BandArgs &a, T *W, uint8_t *pi, int s0) const {
        TA self[VEC], nb[NB][VEC];
        neighbours(self, nb);
        TA wm, wp, wst, g;
        weights<TA>(a, wm, wp, wst, g);
        TA out[VEC];
        TA res = 0;
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const unsigned c = code[k];
            TA nbk[NB];
#pragma unroll
            for (int j = 0; j < NB; j++) nbk[j] = nb[j][k];
            int arg;
            const TA v = vi_state<TA, D, WITH_PI>(self[k], nbk, c, r[k], wm, wp, wst, g, arg);
            out[k] = v;
            if (WITH_PI) pi[s0 + k] = (c & (OBST | TERM)) ? (uint8_t)255 : (uint8_t)arg;
            if (!(c & OBST)) {
                const TA dv = abs_diff(v, self[k]);
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

    // Policy-iteration sweeps: EVAL (V' = Q of the fixed action, returns the
    // residual), IMPROVE (switch to the argmax when it beats the current
    // action by more than margin (1 + |Q|), count switches; V' = Q of the
    // action kept or taken, the first evaluation step of the new policy,
    // and its residual) and GREEDY (policy = argmax, lowest index on ties).
    template <int MODE>
    __device__ __forceinline__ TA finish_pi(const BandArgs &a, T *W, uint8_t *pi, TA margin, int s0,
                                            unsigned &changed) const {
        TA self[VEC], nb[NB][VEC];
        neighbours(self, nb);
        TA wm, wp, wst, g;
        weights<TA>(a, wm, wp, wst, g);
        TA out[VEC];
        TA res = 0;
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const int s = s0 + k;
            const unsigned c = code[k];
            const TA rk = r[k];
            TA perp[D];
            perp_sums(nb, k, perp);
            const TA stay = wst * self[k];
            TA v = self[k];
            int na = (int)act[k];   // IMPROVE: the action after this sweep
            if (MODE == M_EVAL) {
                TA nbk[NB];
#pragma unroll
                for (int j = 0; j < NB; j++) nbk[j] = nb[j][k];
                v = eval_state<TA, D>(self[k], nbk, c, rk, (int)act[k], wm, wp, wst, g);
                if (!(c & OBST)) {
                    const TA dv = abs_diff(v, self[k]);
                    res = dv > res ? dv : res;
                }
            } else if (!(c & (OBST | TERM))) {
                TA best = rk + g * (wm * nb[0][k] + wp * perp[0] + stay);
                int arg = 0;
                TA qold = best;
                const int old = (MODE == M_IMPROVE) ? (int)act[k] : 0;
#pragma unroll
                for (int j = 1; j < NB; j++) {
                    const TA q = rk + g * (wm * nb[j][k] + wp * perp[j / 2] + stay);
                    if (q > best) { best = q; arg = j; }
                    if (j == old) qold = q;
                }
                if (MODE == M_IMPROVE) {
                    const TA thr = margin * ((TA)1 + (qold < 0 ? -qold : qold));
                    if (arg != old && best > qold + thr) { pi[s] = (uint8_t)arg; changed++; na = arg; }
                } else {
                    pi[s] = (uint8_t)arg;
                }
            } else if (MODE == M_GREEDY) {
                pi[s] = 255;
            }
            if (MODE == M_IMPROVE) {
                TA nbk[NB];
#pragma unroll
                for (int j = 0; j < NB; j++) nbk[j] = nb[j][k];
                v = eval_state<TA, D>(self[k], nbk, c, rk, na, wm, wp, wst, g);
                if (!(c & OBST)) {
                    const TA dv = abs_diff(v, self[k]);
                    res = dv > res ? dv : res;
                }
            }
            out[k] = v;
        }
        if (MODE == M_EVAL || MODE == M_IMPROVE) {
            T o[VEC];
#pragma unroll
            for (int k = 0; k < VEC; k++) o[k] = (T)out[k];
            store_pack<T, VEC>(W + s0, o);
        }
        return res;
    }
};

// All segments of one sweep, grid-stride, two segments in flight per thread.
// With a grid of co-resident blocks, the states being worked on at any time
// form one compact window, so the row neighbours one plane away are still in
// L2 when their own window comes.
template <typename T, typename TA, int D, int VEC, int MODE, bool WITH_PI>
__device__ __forceinline__ TA sweep_all(const BandArgs &a, const T *V, T *W, uint8_t *pi, TA margin,
                                        unsigned &changed) {
    const int nitems = a.nstates / VEC;
    const int step = gridDim.x * blockDim.x;
    TA res = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nitems; i += 2 * step) {
        Segment<T, TA, D, VEC> s0, s1;
        const bool two = i + step < nitems;
        s0.template load<MODE>(a, V, pi, i * VEC);
        if (two) s1.template load<MODE>(a, V, pi, (i + step) * VEC);
        TA r;
        if (MODE == M_VI) r = s0.template finish_vi<WITH_PI>(a, W, pi, i * VEC);
        else r = s0.template finish_pi<MODE>(a, W, pi, margin, i * VEC, changed);
        res = r > res ? r : res;
        if (two) {
            if (MODE == M_VI) r = s1.template finish_vi<WITH_PI>(a, W, pi, (i + step) * VEC);
            else r = s1.template finish_pi<MODE>(a, W, pi, margin, (i + step) * VEC, changed);
            res = r > res ? r : res;
        }
    }
    return res;
}

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

// Block-wide max (result valid in thread 0). blockDim must be a multiple of 32.
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

// Largest of the block's non-negative residuals, as the bits of a double
// (valid in thread 0; ready for an atomicMax on a residual slot). A
// non-negative IEEE-754 value orders like its bit pattern read as an
// unsigned integer (a NaN above +inf), so each warp step is one integer max
// reduction (redux.sync) and no FP64 instruction is issued: GB300's FP64
// pipe is narrow enough that a shuffle-and-fmax tree over doubles costs
// microseconds per sweep. sh: 32 words of shared memory.
__device__ __forceinline__ unsigned long long block_max_bits(float v, unsigned *sh) {
    unsigned u = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = u;
    __syncthreads();
    if (w == 0) {
        u = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0u;
        u = __reduce_max_sync(0xFFFFFFFFu, u);
    }
    __syncthreads();
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(u));
}

// The same for double residuals: the high words first, then the low words
// of the lanes holding the largest high word. sh: 64 words.
__device__ __forceinline__ unsigned long long block_max_bits(double v, unsigned *sh) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    unsigned hm = __reduce_max_sync(0xFFFFFFFFu, hi);
    unsigned lm = __reduce_max_sync(0xFFFFFFFFu, hi == hm ? lo : 0u);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[w] = hm; sh[32 + w] = lm; }
    __syncthreads();
    if (w == 0) {
        const bool in = l < (int)(blockDim.x >> 5);
        hi = in ? sh[l] : 0u;
        lo = in ? sh[32 + l] : 0u;
        hm = __reduce_max_sync(0xFFFFFFFFu, hi);
        lm = __reduce_max_sync(0xFFFFFFFFu, hi == hm ? lo : 0u);
    }
    __syncthreads();
    return ((unsigned long long)hm << 32) | lm;
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

// Whether a barrier counter v (arrivals in the low half, raised flags in
// the high half, one 64-bit sum) still misses arrivals of a barrier that is
// complete when the low half reaches a_lo (the low half of the arrival
// count); valid while at most 2^31 arrivals are missing.
__device__ __forceinline__ bool arrivals_short(unsigned long long v, unsigned a_lo) {
    return (int)((unsigned)v - a_lo) < 0;
}

// Grid-wide barrier of a co-resident (cooperative) grid that also counts
// how many blocks raised `flag` (thread 0's value) in the step it closes.
// Barrier number n uses counter bar[n % 2]: every arrival adds 1, and 2^32
// more when it raises its flag, so the counter is A + F * 2^32 with A =
// (n/2 + 1) * nblocks arrivals once everyone has arrived and F the flags
// raised on that counter so far. A block cannot reach barrier n+2 before
// every block has left barrier n+1, so the value read when barrier n
// completes holds exactly the arrivals up to barrier n; the flags of step n
// are (v - A) >> 32 minus the same count at barrier n-2 (prev0 / prev1 for
// even / odd n, kept by thread 0). Every wait gives up after timeout_ns or when another block has
// recorded a status: returns -1 (CPMDP_ETIMEOUT stored in the status word).
// stall: testing aid, this block leaves without arriving.
__device__ __forceinline__ long long grid_sync_count(Ctrl *c, int n, unsigned nblocks, int flag,
                                                     unsigned long long timeout_ns, unsigned long long &prev0,
                                                     unsigned long long &prev1, bool stall) {
    __shared__ long long result;
    __syncthreads();
    if (threadIdx.x == 0) {
        result = 0;
        if (stall) {
            if (nblocks == 1) atomicCAS(&c->status, 0, (int)CPMDP_ETIMEOUT);
            result = -1;
        } else if (nblocks == 1) {
            // a single block: the block barriers around this call already
            // order every thread's global accesses, so no arrival through L2
            // (small grids: the fence and round trip were most of a sweep)
            result = flag != 0 ? 1 : 0;
        } else {
            unsigned long long *ctr = &c->bar[n & 1];
            red_add_release(ctr, 1ull | ((unsigned long long)(flag != 0) << 32));
            // After this barrier completes, the counter holds A arrivals plus
            // F raised flags times 2^32 as one 64-bit sum (carries of the low
            // half included). While blocks still arrive, its low half lies in
            // [A - nblocks, A) modulo 2^32, so completion is tested on the
            // low halves' signed difference: no wrap, however many sweeps.
            const unsigned a_lo = (unsigned)(n / 2 + 1) * nblocks;   // low half of A
            unsigned long long v = ld_acquire(ctr);
            if (arrivals_short(v, a_lo)) {
                const unsigned long long t0 = global_ns();
                unsigned spins = 0;
                do {
                    __nanosleep(32);
                    v = ld_acquire(ctr);
                    if ((++spins & 15u) == 0 && arrivals_short(v, a_lo)) {
                        if (*(volatile int *)&c->status != 0) { result = -1; break; }
                        if (global_ns() - t0 > timeout_ns) {
                            atomicCAS(&c->status, 0, (int)CPMDP_ETIMEOUT);
                            result = -1;
                            break;
                        }
                    }
                } while (arrivals_short(v, a_lo));
            }
            if (result == 0) {
                // the low halves of v and A agree, so (v - A) >> 32 borrows nothing
                const unsigned long long F = (v >> 32) - (((unsigned long long)(n / 2 + 1) * nblocks) >> 32);
                const unsigned long long prev = (n & 1) ? prev1 : prev0;
                result = (long long)((F - prev) & 0xFFFFFFFFull);   // fewer than 2^32 blocks
                if (n & 1) prev1 = F;
                else prev0 = F;
            }
        }
    }
    __syncthreads();
    return result;
}

struct SolveParams {
    int max_iter;
    int max_eval_iter;
    int max_rounds;
    double tol;
    double eval_tol;
    double margin;
    unsigned long long timeout_ns;
    int nactions;
    int inject_stall;
    int partial_eval;   // policy iteration: evaluation sweep cap while the policy changes (0: none)
};

BandArgs make_band_args(const Factors &F);
int band_pick_vec(const Factors &F, size_t elem, const void *p0, const void *p1);

#define CPMDP_DISPATCH_D(D_, ...)                             \
    switch (D_) {                                             \
        case 1: { constexpr int DD = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int DD = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int DD = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int DD = 4; __VA_ARGS__; } break; \
        case 5: { constexpr int DD = 5; __VA_ARGS__; } break; \
        case 6: { constexpr int DD = 6; __VA_ARGS__; } break; \
        case 7: { constexpr int DD = 7; __VA_ARGS__; } break; \
        case 8: { constexpr int DD = 8; __VA_ARGS__; } break; \
        case 9: { constexpr int DD = 9; __VA_ARGS__; } break; \
        default: break;                                       \
    }

}  // namespace cpmdp
