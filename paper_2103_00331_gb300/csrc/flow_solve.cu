// Barrier-free persistent FP32 value iteration and policy iteration for
// GridWorld factors of 1 to 3 dimensions (background section: value
// iteration repeats the Eq. 1 backup until it converges; policy iteration
// alternates evaluation of a fixed policy with greedy improvement until no
// action changes).
//
// The grid-barrier solver (banded_solve.cu) ends every sweep with a
// grid-wide barrier. When the whole value tensor sits in L2 (64^3: 1 MB),
// that barrier takes about two thirds of a sweep. This solver has no
// barrier inside its sweep loop:
//
// * Each thread owns one segment of 4 consecutive states of a row of the
//   last dimension for the whole launch and keeps their values, rewards,
//   codes and actions in registers.
// * Values travel through kRing = 4 ring buffers of 64-bit words, each
//   holding (sweep tag << 32) | float bits. Sweep q reads buffer q mod 4 and
//   writes buffer (q + 1) mod 4. A thread waits (bounded) until every
//   neighbour word it needs carries the tag of sweep q; a 64-bit word is
//   written and read whole, so a matching tag also means a matching value.
//   Neighbours held by other lanes of the same warp (the left and right
//   neighbours, and rows less than 32 segments away) come by shuffle.
// * Each warp reports every sweep on an arrival counter (+1 in the low
//   half, +1 in the high half when its residual is still >= tol). Before it
//   stores sweep q, a warp checks that every warp has reported sweep
//   q - kLag (kLag = 3): nobody still reads the buffer it is about to
//   overwrite, and it learns whether sweep q - kLag met the stopping rule.
//   If it did, the warp returns the values of that sweep (its own words,
//   still in the ring) and kLag speculative sweeps are dropped. Values,
//   sweep counts and residuals are exactly those of the grid-barrier solver:
//   same Jacobi iterates, same per-state arithmetic (vi_state /
//   eval_state), same stopping sweep. Warps far apart on the grid drift up
//   to a couple of sweeps from each other, and the three-sweep slack keeps
//   that drift from stalling the check.
//
// Counters are cumulative per slot (arrival i uses slot i mod 8), spread
// over 8 counters of their own 128-byte lines to limit atomic contention.
// No warp can report arrival i + 8 before every warp has reported i + 5,
// which every warp checks before it stores sweep i + 8, and arrival i is
// checked at sweep i + 3: a check of arrival i sees exactly the arrivals i,
// i - 8, ... of its slot; flags are told apart with the count each lane saw
// at the slot's previous check.
// Every wait gives up after timeout_ns (CPMDP_ETIMEOUT in the status word)
// or when another warp has recorded a status.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "banded_common.cuh"
#include "flow.h"

namespace cpmdp {

namespace {

typedef unsigned long long u64;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kLag = 3;              // the stopping rule of sweep q is settled at sweep q + kLag
constexpr int kRing = kLag + 1;      // tagged value buffers
constexpr int kSlots = 8;            // arrival slots (arrival i uses slot i % kSlots; > 2 kLag + 1)
constexpr int kNC = 8;               // counters per slot (warp w adds to counter w % kNC)
constexpr int kLineWords = 16;       // 64-bit words per 128-byte line
constexpr int kMaxWarps = 14;        // warps per block at most (one block per SM, 448 threads)
constexpr int kMaxThreads = 32 * kMaxWarps;

__device__ __forceinline__ u64 ld_rlx(const u64 *p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ld_rlx2(const u64 *p, u64 &x, u64 &y) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_rlx2(u64 *p, u64 x, u64 y) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y) : "memory");
}
__device__ __forceinline__ void red_add_rlx(u64 *p, u64 v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u64 word(float v, unsigned tag) { return ((u64)tag << 32) | __float_as_uint(v); }
__device__ __forceinline__ float val(u64 w) { return __uint_as_float((unsigned)w); }
__device__ __forceinline__ bool has(u64 w, unsigned tag) { return (unsigned)(w >> 32) == tag; }

struct FlowArgs {
    BandArgs a;
    unsigned tol_bits;         // bits of the smallest float >= tol (value iteration) ...
    unsigned eval_tol_bits;    // ... and >= eval_tol (policy evaluation)
    u64 *buf[kRing];           // tagged value ring
    u64 *ctr;                  // kSlots x kNC arrival counters, kLineWords apart
    float *V;                  // caller's values: start in, result out
    uint8_t *pi;               // caller's policy (policy iteration)
    double *trace;             // optional per-sweep residual (value iteration)
    unsigned base;             // tag of sweep 0
    int nsegs;                 // |S| / 4
};

__device__ __forceinline__ u64 *ring(const FlowArgs &f, unsigned q) { return f.buf[q % (unsigned)kRing]; }

// Warp-uniform: true when this warp must stop waiting (another warp
// recorded a status, or this wait ran past timeout_ns: then it records
// CPMDP_ETIMEOUT). t0: start of the wait (lane 0's clock, 0 = not started).
__device__ __forceinline__ bool give_up(Ctrl *c, u64 &t0, u64 timeout_ns) {
    int stop = 0;
    if ((threadIdx.x & 31) == 0) {
        const u64 t = global_ns();
        if (t0 == 0) t0 = t;
        if (*(volatile int *)&c->status != 0) {
            stop = 1;
        } else if (t - t0 > timeout_ns) {
            atomicCAS(&c->status, 0, (int)CPMDP_ETIMEOUT);
            stop = 1;
        }
    }
    return __shfl_sync(FULL, stop, 0) != 0;
}

// Arrival bookkeeping of one warp.
struct Arrivals {
    u64 *ctr;
    unsigned *prevhi;   // shared, kSlots x kNC: high half seen at each slot's last check
    unsigned nw_lane;   // warps that add to counter `lane` (lanes < kNC)
    int gw;             // global warp index
    unsigned na = 0;    // arrivals made
    unsigned nchk = 0;  // arrivals checked (always in order)

    __device__ __forceinline__ void arrive(bool flag) {
        if ((threadIdx.x & 31) == 0)
            red_add_rlx(ctr + ((na % kSlots) * kNC + (unsigned)gw % kNC) * kLineWords,
                        1ull | ((u64)(flag ? 1u : 0u) << 32));
        na++;
    }
    __device__ __forceinline__ u64 peek(unsigned i) const {
        const int lane = threadIdx.x & 31;
        return lane < kNC ? ld_rlx(ctr + ((i % kSlots) * kNC + lane) * kLineWords) : 0ull;
    }
    // Warps that raised their flag at arrival i, or -1 if some warp has not
    // reported it yet (then nothing is recorded). After A arrivals with F
    // raised flags a counter holds A + F * 2^32 as a 64-bit integer, carries
    // from the low half included, so with A known from i the check needs
    // only the low halves and F = (v - A) >> 32.
    __device__ __forceinline__ int settle(u64 v, unsigned i) {
        const int lane = threadIdx.x & 31;
        const u64 A = ((u64)(i / kSlots) + 1ull) * nw_lane;
        const bool ok = lane >= kNC || (unsigned)v == (unsigned)A;
        if (!__all_sync(FULL, ok)) return -1;
        unsigned d = 0;
        if (lane < kNC) {
            unsigned *ph = prevhi + (i % kSlots) * kNC + lane;
            const unsigned F = (unsigned)((v - A) >> 32);
            d = F - *ph;
            *ph = F;
        }
        return (int)__reduce_add_sync(FULL, d);
    }
    // Check the next unchecked arrival, starting from a value read earlier
    // (pk) and waiting (bounded) if it is not complete yet. Returns the
    // number of raised flags, or -1 when the warp must stop.
    __device__ __forceinline__ int check(u64 pk, Ctrl *ctrl, u64 timeout_ns) {
        int r = settle(pk, nchk);
        u64 t0 = 0;
        unsigned spins = 0;
        while (r < 0) {
            if ((++spins & 15u) == 0 && give_up(ctrl, t0, timeout_ns)) return -1;
            __nanosleep(32);
            r = settle(peek(nchk), nchk);
        }
        nchk++;
        return r;
    }
    __device__ __forceinline__ int check_next(Ctrl *ctrl, u64 timeout_ns) { return check(peek(nchk), ctrl, timeout_ns); }
};

// One thread's segment: states s0 .. s0+3 of a row of the last dimension.
template <int D>
struct FlowSeg {
    static constexpr int NRR = 2 * (D - 1);          // row-neighbour directions (other dimensions)
    static constexpr int NR = NRR > 0 ? NRR : 1;
    static constexpr int HM = 2 * NRR, HP = 2 * NRR + 1;  // need bits of the left / right halo words
    static constexpr unsigned OBST = 1u << (2 * D), TERM = 1u << (2 * D + 1);

    int s0;
    bool valid;
    unsigned code;        // the 4 codes, state k in byte k
    unsigned inw;         // served by a shuffle in this warp: bits 2j, 2j+1 (row j), HM, HP
    unsigned need;        // needed from memory: bit 2j + h (row j, half h), HM, HP
    int own;              // first ring word of this segment (a lane without one: the last segment's)
    float R[4], cur[4];
    unsigned act;         // policy iteration: 4 actions, state k in byte k

    __device__ __forceinline__ void init(const FlowArgs &f, int seg, int lane) {
        const BandArgs &a = f.a;
        valid = seg < f.nsegs;
        s0 = seg * 4;
        code = 0;
        act = 0;
        inw = 0;
        int off[NR];
#pragma unroll
        for (int j = 0; j < NR; j++) {
            off[j] = 0;
            if (j < NRR) {
                const int st = a.stride[j / 2];
                const int so = st / 4;
                const bool up = (j & 1) != 0;
                off[j] = up ? st : -st;
                if (so < 32 && (up ? lane + so < 32 : lane >= so)) inw |= 3u << (2 * j);
            }
        }
        if (lane >= 1) inw |= 1u << HM;
        if (lane <= 30) inw |= 1u << HP;
#pragma unroll
        for (int k = 0; k < 4; k++) { R[k] = 0.f; cur[k] = 0.f; }
        // A lane without a segment reads the last segment's words, which
        // its owner (the last valid lane of this warp) writes every sweep.
        own = valid ? s0 : a.nstates - 4;
        need = 0;
        if (!valid) return;
        code = *reinterpret_cast<const unsigned *>(static_cast<const uint8_t *>(a.code) + s0);
        const float4 r = *reinterpret_cast<const float4 *>(a.R32 + s0);
        const float4 v = *reinterpret_cast<const float4 *>(f.V + s0);
        R[0] = r.x; R[1] = r.y; R[2] = r.z; R[3] = r.w;
        cur[0] = v.x; cur[1] = v.y; cur[2] = v.z; cur[3] = v.w;
        unsigned nd = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const unsigned c = (code >> (8 * k)) & 0xFFu;
            if (c & (OBST | TERM)) continue;
#pragma unroll
            for (int j = 0; j < NRR; j++)
                if (!((c >> j) & 1u)) nd |= 1u << (2 * j + (k >> 1));
            if (k == 0 && !((c >> NRR) & 1u)) nd |= 1u << HM;
            if (k == 3 && !((c >> (NRR + 1)) & 1u)) nd |= 1u << HP;
        }
        need = nd & ~inw;
    }

    // Ring word read for row j, half h: the neighbours' pair when it is
    // needed from memory, else this segment's own pair (already written).
    __device__ __forceinline__ int wo(const BandArgs &a, int j, int h) const {
        const int st = a.stride[j / 2];
        return own + 2 * h + (((need >> (2 * j + h)) & 1u) ? ((j & 1) ? st : -st) : 0);
    }
    __device__ __forceinline__ int wol() const { return own - (int)((need >> HM) & 1u); }
    __device__ __forceinline__ int wor() const { return own + (int)(((need >> HP) & 1u) << 2); }

    // This segment's own values of sequence q, read back from the ring: its
    // own words, written by this thread and still there while q is one of
    // the kRing - 1 latest sequences written.
    __device__ __forceinline__ void own_values(const FlowArgs &f, unsigned q, float (&v)[4]) const {
        if (!valid) return;
        const u64 *in = ring(f, q);
        u64 a, b, c, d;
        ld_rlx2(in + s0, a, b);
        ld_rlx2(in + s0 + 2, c, d);
        v[0] = val(a); v[1] = val(b); v[2] = val(c); v[3] = val(d);
    }

    __device__ __forceinline__ void publish(const FlowArgs &f, unsigned q, unsigned base, const float (&v)[4]) const {
        if (!valid) return;
        u64 *out = ring(f, q);
        const unsigned tg = base + q;
        st_rlx2(out + s0, word(v[0], tg), word(v[1], tg));
        st_rlx2(out + s0 + 2, word(v[2], tg), word(v[3], tg));
    }

    // Neighbour values of sweep q (tag base + q, buffer q mod 3) for the
    // values `self` (this segment's values of sweep q): rows[j][k] is the
    // value one move in direction j from state k, hl / hr the states just
    // left of state 0 and right of state 3 (for blocked moves: anything).
    // Every lane reads all its ring words at once (words it does not need
    // are its own, already written), checks all tags with one OR and
    // re-reads only on a mismatch. Returns false when the warp must stop
    // (status recorded).
    __device__ __forceinline__ bool gather(const FlowArgs &f, unsigned q, unsigned base, const float (&self)[4],
                                           float (&rows)[NR][4], float &hl, float &hr, Ctrl *ctrl,
                                           u64 timeout_ns) const {
        const unsigned tg = base + q;
        const u64 *in = ring(f, q);
        u64 w[NR][2][2];
        u64 wl, wr;
        // The neighbours' words of sweep q are usually stored just as this
        // warp finishes sweep q - 1; a read that reaches L2 before them costs
        // a second round trip. A short pause first lowers that share
        // (measured at 64^3 and 32^3: about 2 % and 4 % faster sweeps).
        __nanosleep(100);
#pragma unroll
        for (int j = 0; j < NRR; j++)
#pragma unroll
            for (int h = 0; h < 2; h++) ld_rlx2(in + wo(f.a, j, h), w[j][h][0], w[j][h][1]);
        wl = ld_rlx(in + wol());
        wr = ld_rlx(in + wor());
        // rows less than 32 segments away: the lanes holding them (the
        // stride is the same for every thread, so this branch is uniform)
        const int lane = threadIdx.x & 31;
        float sh[NR][4];
#pragma unroll
        for (int j = 0; j < NRR; j++) {
            const int so = f.a.stride[j / 2] >> 2;
            if (so < 32) {
                const int src = ((j & 1) ? lane + so : lane - so) & 31;
#pragma unroll
                for (int k = 0; k < 4; k++) sh[j][k] = __shfl_sync(FULL, self[k], src);
            }
        }
        const float sl = __shfl_up_sync(FULL, self[3], 1);
        const float sr = __shfl_down_sync(FULL, self[0], 1);
        unsigned bad = ((unsigned)(wl >> 32) ^ tg) | ((unsigned)(wr >> 32) ^ tg);
#pragma unroll
        for (int j = 0; j < NRR; j++)
#pragma unroll
            for (int h = 0; h < 2; h++) bad |= ((unsigned)(w[j][h][0] >> 32) ^ tg) | ((unsigned)(w[j][h][1] >> 32) ^ tg);
        if (__any_sync(FULL, bad != 0u)) {
            // slow path: re-read the words whose tag is not there yet
            u64 t0 = 0;
            unsigned spins = 0;
            for (;;) {
                unsigned pend = 0;
#pragma unroll
                for (int j = 0; j < NRR; j++)
#pragma unroll
                    for (int h = 0; h < 2; h++)
                        if (!has(w[j][h][0], tg) || !has(w[j][h][1], tg)) pend |= 1u << (2 * j + h);
                if (!has(wl, tg)) pend |= 1u << HM;
                if (!has(wr, tg)) pend |= 1u << HP;
                if (!__any_sync(FULL, pend != 0u)) break;
                if ((++spins & 15u) == 0 && give_up(ctrl, t0, timeout_ns)) return false;
#pragma unroll
                for (int j = 0; j < NRR; j++)
#pragma unroll
                    for (int h = 0; h < 2; h++)
                        if ((pend >> (2 * j + h)) & 1u) ld_rlx2(in + wo(f.a, j, h), w[j][h][0], w[j][h][1]);
                if ((pend >> HM) & 1u) wl = ld_rlx(in + wol());
                if ((pend >> HP) & 1u) wr = ld_rlx(in + wor());
            }
        }
#pragma unroll
        for (int j = 0; j < NRR; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float m = val(w[j][k >> 1][k & 1]);
                rows[j][k] = ((inw >> (2 * j)) & 1u) ? sh[j][k] : m;
            }
        if (NRR == 0) {
#pragma unroll
            for (int k = 0; k < 4; k++) rows[0][k] = 0.f;
        }
        hl = ((inw >> HM) & 1u) ? sl : val(wl);
        hr = ((inw >> HP) & 1u) ? sr : val(wr);
        return true;
    }

    // Neighbour values of state k with blocked moves replaced by V(s), in
    // the order of the codes' move bits (as Segment::neighbours).
    __device__ __forceinline__ void nbk(const float (&self)[4], const float (&rows)[NR][4], float hl, float hr, int k,
                                        float (&nb)[2 * D]) const {
        const unsigned c = (code >> (8 * k)) & 0xFFu;
#pragma unroll
        for (int j = 0; j < NRR; j++) nb[j] = ((c >> j) & 1u) ? self[k] : rows[j][k];
        const float left = (k == 0) ? hl : self[k > 0 ? k - 1 : 0];
        const float right = (k == 3) ? hr : self[k < 3 ? k + 1 : 0];
        nb[NRR] = ((c >> NRR) & 1u) ? self[k] : left;
        nb[NRR + 1] = ((c >> (NRR + 1)) & 1u) ? self[k] : right;
    }
};

// Whether the warp's largest residual r is still >= the tolerance whose
// float round-up has bits tb: for a float r >= 0, (double)r < tol exactly
// when r < the smallest float >= tol, and non-negative floats (a NaN above
// +inf) order like their bits, so no FP64 instruction is needed.
__device__ __forceinline__ bool warp_open(float r, unsigned tb) {
    return __reduce_max_sync(FULL, __float_as_uint(r)) >= tb;
}

__device__ __forceinline__ unsigned long long warp_res_bits(float r) {
    const unsigned u = __reduce_max_sync(FULL, __float_as_uint(r));
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(u));
}

// Greedy / improvement choice of one state (same expressions as
// Segment::finish_pi): returns the new action.
template <int D>
__device__ __forceinline__ int improve_state(const float (&nb)[2 * D], float self, unsigned c, float rk, int old,
                                             bool greedy, float margin, float wm, float wp, float wst, float g,
                                             unsigned &changed) {
    constexpr unsigned OBST = 1u << (2 * D), TERM = 1u << (2 * D + 1);
    if (c & (OBST | TERM)) return greedy ? 255 : old;
    float perp[D];
    perp_of<float, D>(nb, perp);
    const float stay = wst * self;
    float best = rk + g * (wm * nb[0] + wp * perp[0] + stay);
    int arg = 0;
    float qold = best;
#pragma unroll
    for (int j = 1; j < 2 * D; j++) {
        const float q = rk + g * (wm * nb[j] + wp * perp[j / 2] + stay);
        if (q > best) { best = q; arg = j; }
        if (j == old) qold = q;
    }
    if (greedy) return arg;
    const float thr = margin * (1.0f + (qold < 0 ? -qold : qold));
    if (arg != old && best > qold + thr) { changed++; return arg; }
    return old;
}

// Final bookkeeping: every warp adds its residual and arrives; the lead
// waits for all warps, then fills the control block.
__device__ __forceinline__ void flow_finish(Ctrl *ctrl, float rres, u64 timeout_ns, int NW, bool lead,
                                            int iterations, int converged, long long backups, int rounds,
                                            int evals, unsigned tags) {
    const u64 rb = warp_res_bits(rres);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        if (rb) atomicMax(&ctrl->res_slot[0], rb);
        red_add_release(&ctrl->bar[0], 1ull);
    }
    if (!lead) return;
    u64 t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire(&ctrl->bar[0]) < (u64)NW) {
        __nanosleep(64);
        if ((++spins & 15u) == 0) {
            if (*(volatile int *)&ctrl->status != 0) return;
            if (global_ns() - t0 > timeout_ns) { atomicCAS(&ctrl->status, 0, (int)CPMDP_ETIMEOUT); return; }
        }
    }
    ctrl->iterations = iterations;
    ctrl->converged = converged;
    ctrl->rounds = rounds;
    ctrl->eval_sweeps = evals;
    ctrl->backups = backups;
    ctrl->flow_tags = tags;
    ctrl->last_residual = __longlong_as_double((long long)*(volatile u64 *)&ctrl->res_slot[0]);
}

template <int D>
__global__ void __launch_bounds__(kMaxThreads, 1) flow_vi_kernel(FlowArgs f, SolveParams sp, Ctrl *ctrl) {
    __shared__ unsigned prevhi_all[kMaxWarps][kSlots * kNC];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int NW = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    Arrivals arv;
    arv.ctr = f.ctr;
    arv.prevhi = prevhi_all[wib];
    arv.nw_lane = (unsigned)(NW / kNC) + ((unsigned)lane < (unsigned)(NW % kNC) ? 1u : 0u);
    arv.gw = gw;
    for (int t = lane; t < kSlots * kNC; t += 32) arv.prevhi[t] = 0u;
    __syncwarp();
    if (sp.inject_stall && blockIdx.x == 0) {  // testing aid: this block never publishes
        if (gridDim.x == 1 && threadIdx.x == 0) atomicCAS(&ctrl->status, 0, (int)CPMDP_ETIMEOUT);
        return;
    }

    float wm, wp, wst, g;
    weights<float>(f.a, wm, wp, wst, g);
    FlowSeg<D> sg;
    sg.init(f, blockIdx.x * blockDim.x + threadIdx.x, lane);
    const unsigned base = f.base;
    sg.publish(f, 0, base, sg.cur);

    constexpr int NR = FlowSeg<D>::NR;
    constexpr unsigned OBST = FlowSeg<D>::OBST;
    const unsigned maxq = (unsigned)sp.max_iter;
    unsigned q = 0;
    float rh[kLag];                        // thread residuals of sweeps q-1, q-2, ...
#pragma unroll
    for (int i = 0; i < kLag; i++) rh[i] = 0.f;
    float res[4];
    float rres = 0.f;
    int iters = 0, conv = 0;
    for (;;) {
        const u64 pk = q >= kLag ? arv.peek(arv.nchk) : 0ull;
        float rows[NR][4], hl, hr;
        if (!sg.gather(f, q, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
        float nxt[4];
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float nb[2 * D];
            sg.nbk(sg.cur, rows, hl, hr, k, nb);
            const unsigned c = (sg.code >> (8 * k)) & 0xFFu;
            int arg;
            const float v = vi_state<float, D>(sg.cur[k], nb, c, sg.R[k], wm, wp, wst, g, arg);
            nxt[k] = v;
            if (!(c & OBST)) {
                const float dv = abs_diff(v, sg.cur[k]);
                r = dv > r ? dv : r;
            }
        }
        if (!sg.valid) r = 0.f;
        if (q >= kLag) {
            const int nf = arv.check(pk, ctrl, sp.timeout_ns);
            if (nf < 0) return;
            if (nf == 0) {  // sweep q - kLag met the stopping rule: its result is V_{q-kLag+1}
                sg.own_values(f, q - kLag + 1, res);
                rres = rh[kLag - 1];
                iters = (int)q - kLag + 1;
                conv = 1;
                break;
            }
        }
        sg.publish(f, q + 1, base, nxt);
        arv.arrive(warp_open(r, f.tol_bits));
        if (f.trace) {
            const u64 mb = warp_res_bits(r);
            if (lane == 0 && mb) atomicMax(reinterpret_cast<u64 *>(f.trace) + q, mb);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) sg.cur[k] = nxt[k];
#pragma unroll
        for (int i = kLag - 1; i > 0; i--) rh[i] = rh[i - 1];
        rh[0] = r;
        q++;
        if (q == maxq) {
            // the limit: settle the unchecked sweeps in order
#pragma unroll
            for (int k = 0; k < 4; k++) res[k] = sg.cur[k];
            rres = rh[0];
            iters = (int)q;
            while (arv.nchk < arv.na) {
                const unsigned sweep = arv.nchk;  // value iteration: arrival i is sweep i
                const int nf = arv.check_next(ctrl, sp.timeout_ns);
                if (nf < 0) return;
                if (nf == 0 && !conv) {
                    conv = 1;
                    iters = (int)sweep + 1;
                    if (sweep + 1 != q) sg.own_values(f, sweep + 1, res);
                    const unsigned back = q - 1 - sweep;   // 0 .. kLag-1
#pragma unroll
                    for (int i = 0; i < kLag; i++)
                        if ((unsigned)i == back) rres = rh[i];
                }
            }
            break;
        }
    }
    if (sg.valid) *reinterpret_cast<float4 *>(f.V + sg.s0) = make_float4(res[0], res[1], res[2], res[3]);
    if (!sg.valid) rres = 0.f;
    flow_finish(ctrl, rres, sp.timeout_ns, NW, gw == 0 && lane == 0, iters, conv,
                (long long)iters * f.a.nstates * sp.nactions, 0, 0, q + 2);
}

template <int D>
__global__ void __launch_bounds__(kMaxThreads, 1) flow_pi_kernel(FlowArgs f, SolveParams sp, Ctrl *ctrl) {
    __shared__ unsigned prevhi_all[kMaxWarps][kSlots * kNC];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int NW = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    Arrivals arv;
    arv.ctr = f.ctr;
    arv.prevhi = prevhi_all[wib];
    arv.nw_lane = (unsigned)(NW / kNC) + ((unsigned)lane < (unsigned)(NW % kNC) ? 1u : 0u);
    arv.gw = gw;
    for (int t = lane; t < kSlots * kNC; t += 32) arv.prevhi[t] = 0u;
    __syncwarp();
    if (sp.inject_stall && blockIdx.x == 0) {  // testing aid: this block never publishes
        if (gridDim.x == 1 && threadIdx.x == 0) atomicCAS(&ctrl->status, 0, (int)CPMDP_ETIMEOUT);
        return;
    }

    float wm, wp, wst, g;
    weights<float>(f.a, wm, wp, wst, g);
    const float margin = (float)sp.margin;
    FlowSeg<D> sg;
    sg.init(f, blockIdx.x * blockDim.x + threadIdx.x, lane);
    const unsigned base = f.base;
    constexpr int NR = FlowSeg<D>::NR;
    constexpr unsigned OBST = FlowSeg<D>::OBST;

    // initial policy: greedy with respect to the input V
    unsigned q = 0;
    sg.publish(f, 0, base, sg.cur);
    {
        float rows[NR][4], hl, hr;
        if (!sg.gather(f, 0, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
        unsigned dummy = 0, act = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float nb[2 * D];
            sg.nbk(sg.cur, rows, hl, hr, k, nb);
            const unsigned c = (sg.code >> (8 * k)) & 0xFFu;
            const int a = improve_state<D>(nb, sg.cur[k], c, sg.R[k], 0, true, margin, wm, wp, wst, g, dummy);
            act |= (unsigned)a << (8 * k);
        }
        sg.act = act;
    }
    int evals = 0, round = 0, conv = 0;
    float rres = 0.f;
    while (round < sp.max_rounds) {
        // evaluation of the current policy from V_q (tag base + q)
        const unsigned q0 = q;
        unsigned rq = q;
        int e = 0, eval_ok = 0;
        float rh[kLag];
#pragma unroll
        for (int i = 0; i < kLag; i++) rh[i] = 0.f;
        for (;;) {
            const bool chk = q - q0 >= (unsigned)kLag;
            const u64 pk = chk ? arv.peek(arv.nchk) : 0ull;
            float rows[NR][4], hl, hr;
            if (!sg.gather(f, q, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
            float nxt[4];
            float r = 0.f;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float nb[2 * D];
                sg.nbk(sg.cur, rows, hl, hr, k, nb);
                const unsigned c = (sg.code >> (8 * k)) & 0xFFu;
                const float v = eval_state<float, D>(sg.cur[k], nb, c, sg.R[k], (int)((sg.act >> (8 * k)) & 0xFFu),
                                                     wm, wp, wst, g);
                nxt[k] = v;
                if (!(c & OBST)) {
                    const float dv = abs_diff(v, sg.cur[k]);
                    r = dv > r ? dv : r;
                }
            }
            if (!sg.valid) r = 0.f;
            if (chk) {
                const int nf = arv.check(pk, ctrl, sp.timeout_ns);
                if (nf < 0) return;
                if (nf == 0) {  // sweep q - kLag met eval_tol: its result is V_{q-kLag+1}
                    sg.own_values(f, q - kLag + 1, sg.cur);
                    rres = rh[kLag - 1];
                    rq = q - kLag + 1;
                    eval_ok = 1;
                    break;
                }
            }
            sg.publish(f, q + 1, base, nxt);
            arv.arrive(warp_open(r, f.eval_tol_bits));
#pragma unroll
            for (int k = 0; k < 4; k++) sg.cur[k] = nxt[k];
#pragma unroll
            for (int i = kLag - 1; i > 0; i--) rh[i] = rh[i - 1];
            rh[0] = r;
            q++;
            e++;
            if (e == sp.max_eval_iter) {
                rres = rh[0];
                rq = q;
                // arrivals of this phase are its sweeps q0, q0 + 1, ... in order
                const unsigned na0 = arv.na - (unsigned)e;
                while (arv.nchk < arv.na) {
                    const unsigned sweep = q0 + (arv.nchk - na0);
                    const int nf = arv.check_next(ctrl, sp.timeout_ns);
                    if (nf < 0) return;
                    if (nf == 0 && !eval_ok) {
                        eval_ok = 1;
                        rq = sweep + 1;
                        if (rq != q) sg.own_values(f, rq, sg.cur);
                        const unsigned back = q - 1 - sweep;   // 0 .. kLag-1
#pragma unroll
                        for (int i2 = 0; i2 < kLag; i2++)
                            if ((unsigned)i2 == back) rres = rh[i2];
                    }
                }
                break;
            }
        }
        evals += (int)(rq - q0);
        // every earlier arrival is settled before the improvement's own
        while (arv.nchk < arv.na)
            if (arv.check_next(ctrl, sp.timeout_ns) < 0) return;
        const unsigned hq = q;  // highest tag sequence written so far
        // sg.cur now holds V_rq, the values of this evaluation
        // improvement on V_rq (tag base + rq, buffer rq mod 3)
        unsigned changed = 0;
        {
            float rows[NR][4], hl, hr;
            if (!sg.gather(f, rq, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
            unsigned act = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float nb[2 * D];
                sg.nbk(sg.cur, rows, hl, hr, k, nb);
                const unsigned c = (sg.code >> (8 * k)) & 0xFFu;
                const int old = (int)((sg.act >> (8 * k)) & 0xFFu);
                const int a = improve_state<D>(nb, sg.cur[k], c, sg.R[k], old, false, margin, wm, wp, wst, g,
                                               changed);
                act |= (unsigned)a << (8 * k);
            }
            if (sg.valid) sg.act = act;
            else changed = 0;
        }
        // the next evaluation starts from V_rq republished as sequence hq + 1
        q = hq + 1;
        sg.publish(f, q, base, sg.cur);
        const unsigned wc = __reduce_add_sync(FULL, changed);
        if (lane == 0 && wc) atomicAdd(&ctrl->changed_total, wc);
        arv.arrive(wc > 0);
        const int moved = arv.check_next(ctrl, sp.timeout_ns);
        if (moved < 0) return;
        round++;
        if (moved == 0) { conv = eval_ok; break; }
        if (!eval_ok) break;
    }
    if (sg.valid) {
        *reinterpret_cast<float4 *>(f.V + sg.s0) = make_float4(sg.cur[0], sg.cur[1], sg.cur[2], sg.cur[3]);
        *reinterpret_cast<unsigned *>(f.pi + sg.s0) = sg.act;
    } else {
        rres = 0.f;
    }
    // sweeps: greedy + evaluations + improvements; backups: |S||A| per greedy
    // or improvement sweep, |S| per evaluation sweep
    flow_finish(ctrl, rres, sp.timeout_ns, NW, gw == 0 && lane == 0, 1 + evals + round, conv,
                (long long)(1 + round) * f.a.nstates * sp.nactions + (long long)evals * f.a.nstates, round, evals,
                q + 2);
}

// Launch shape: one block per SM (as far as the warps go), every block with
// the same number of warps, one warp per 32 consecutive segments. Sweeps
// move at the pace of the busiest SM, so the warps are spread evenly.
static bool flow_shape(const Factors &F, int &block, int &grid) {
    const long long nwarps = (F.nstates / 4 + 31) / 32;
    const long long w = (nwarps + F.num_sms - 1) / F.num_sms;
    if (w < 1 || w > kMaxWarps) return false;
    block = 32 * (int)w;
    grid = (int)((nwarps + w - 1) / w);
    return true;
}

// Both kernels keep one block of up to kMaxThreads threads per SM resident.
template <int D>
static bool flow_resident() {
    static int ok = -1;
    if (ok < 0) {
        int a = 0, b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, flow_vi_kernel<D>, kMaxThreads, 0) != cudaSuccess) a = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, flow_pi_kernel<D>, kMaxThreads, 0) != cudaSuccess) b = 0;
        ok = (a >= 1 && b >= 1) ? 1 : 0;
    }
    return ok == 1;
}

template <int D>
static cudaError_t launch_flow(const Factors &F, bool pim, const FlowArgs &fa, const SolveParams &sp, Ctrl *ctrl,
                               cudaStream_t st) {
    int block = 0, grid = 0;
    if (!flow_shape(F, block, grid) || !flow_resident<D>()) return cudaErrorCooperativeLaunchTooLarge;
    FlowArgs f = fa;
    SolveParams spc = sp;
    void *args[] = {(void *)&f, (void *)&spc, (void *)&ctrl};
    const void *kern = pim ? (const void *)flow_pi_kernel<D> : (const void *)flow_vi_kernel<D>;
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(block), args, 0, st);
}

// Bits of the smallest non-negative float >= t (t > 0; +inf above the
// float range).
unsigned float_ceil_bits(double t) {
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    unsigned u;
    memcpy(&u, &f, sizeof u);
    return u;
}

}  // namespace

bool flow_eligible(const Factors &F, bool policy_iteration, const void *V, const uint8_t *pi,
                   const SolveOpts &o) {
    if (F.ndim < 1 || F.ndim > 3 || F.num_sms <= 0) return false;
    if (F.shape[F.ndim - 1] % 4 != 0 || F.nstates % 4 != 0 || F.nstates >= (1ll << 30)) return false;
    if (((uintptr_t)V & 15u) != 0) return false;
    if (policy_iteration && ((uintptr_t)pi & 3u) != 0) return false;
    int block = 0, grid = 0;
    if (!flow_shape(F, block, grid) || grid > F.num_sms) return false;
    bool res = false;
    switch (F.ndim) {
        case 1: res = flow_resident<1>(); break;
        case 2: res = flow_resident<2>(); break;
        default: res = flow_resident<3>(); break;
    }
    if (!res) return false;
    // tags (base <= 2^30, plus the sweeps of one launch) stay below 2^32 - 1
    const long long sweeps = policy_iteration
                                 ? (long long)o.max_rounds * ((long long)o.max_eval_iter + 2) + 2
                                 : (long long)o.max_iter + 2;
    return sweeps < (1ll << 31);
}

size_t flow_bytes(const Factors &F) {
    return (size_t)kSlots * kNC * kLineWords * sizeof(u64) + (size_t)kRing * F.nstates * sizeof(u64);
}

size_t flow_counter_bytes() { return (size_t)kSlots * kNC * kLineWords * sizeof(u64); }

cpmdp_status flow_solve(const Factors &F, bool policy_iteration, float *V, uint8_t *pi, const SolveParams &sp,
                        double *trace, cudaStream_t st) {
    FlowArgs fa;
    fa.a = make_band_args(F);
    char *base = static_cast<char *>(F.d_flow);
    fa.ctr = reinterpret_cast<u64 *>(base);
    u64 *bufs = reinterpret_cast<u64 *>(base + flow_counter_bytes());
    for (int i = 0; i < kRing; i++) fa.buf[i] = bufs + (size_t)i * F.nstates;
    fa.V = V;
    fa.pi = pi;
    fa.trace = policy_iteration ? nullptr : trace;
    fa.base = F.flow_base;
    fa.tol_bits = float_ceil_bits(sp.tol);
    fa.eval_tol_bits = float_ceil_bits(sp.eval_tol);
    fa.nsegs = (int)(F.nstates / 4);
    CPMDP_CUDA(cudaMemsetAsync(F.d_flow, 0, flow_counter_bytes(), st));
    if (fa.trace) CPMDP_CUDA(cudaMemsetAsync(fa.trace, 0, (size_t)sp.max_iter * sizeof(double), st));
    cudaError_t e;
    switch (F.ndim) {
        case 1: e = launch_flow<1>(F, policy_iteration, fa, sp, F.d_ctrl, st); break;
        case 2: e = launch_flow<2>(F, policy_iteration, fa, sp, F.d_ctrl, st); break;
        default: e = launch_flow<3>(F, policy_iteration, fa, sp, F.d_ctrl, st); break;
    }
    CPMDP_CUDA(e);
    return CPMDP_OK;
}

}  // namespace cpmdp
