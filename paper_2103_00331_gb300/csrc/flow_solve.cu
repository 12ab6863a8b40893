// Barrier-free persistent FP32 value iteration and policy iteration for
// GridWorld factors of 1 to 3 dimensions (background section: value
// iteration repeats the Eq. 1 backup until it converges; policy iteration
// alternates evaluation of a fixed policy with greedy improvement until no
// action changes; here in its modified form, whose improvement sweep also
// takes the new policy's first evaluation step).
//
// The grid-barrier solver (banded_solve.cu) ends every sweep with a
// grid-wide barrier. When the whole value tensor sits in L2 (64^3: 1 MB),
// that barrier takes about two thirds of a sweep. This solver has no
// barrier inside its sweep loop:
//
// * Each thread owns one segment of 4 consecutive states of a row of the
//   last dimension for the whole launch and keeps their values, rewards,
//   codes and actions in registers. Grids too large for that take columns
//   of 2 or 4 segments stacked along dimension 0 in one thread (their
//   dimension-0 neighbours inside the column come from registers): up to
//   about 620,000 states stay in one co-resident grid.
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
#include "flow_common.cuh"

namespace cpmdp {

namespace {

using namespace tw;

constexpr int kNC = 8;               // counters per slot (warp w adds to counter w % kNC)
constexpr int kLineWords = 16;       // 64-bit words per 128-byte line
constexpr int kMaxWarps = 14;        // warps per block at most (one block per SM, 448 threads)
// Warps per block at most for a column of ZS segments: 14 single segments
// fit 128 registers a thread (4 warps per scheduler); columns take more
// registers and fewer, fuller warps.
template <int ZS> struct ColWarps { static constexpr int value = ZS == 1 ? 14 : 8; };

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
    int slice;                 // segments per dimension-0 slice (all of them for one dimension)
    int nz;                    // dimension-0 slices (1 for one dimension)
    int ncols;                 // columns: slice * ceil(nz / ZS)
};

__device__ __forceinline__ u64 *ring(const FlowArgs &f, unsigned q) { return f.buf[q % (unsigned)kRing]; }

// Arrival bookkeeping of one warp.
struct Arrivals {
    u64 *ctr;
    unsigned *prevhi;   // shared, kSlots x kNC: high half seen at each slot's last check
    unsigned nw_lane;   // warps that add to counter `lane` (lanes < kNC)
    int gw;             // global warp index
    unsigned na = 0;    // arrivals made
    unsigned nchk = 0;  // arrivals checked (always in order)

    __device__ __forceinline__ void arrive(bool flag) { arrive_count(flag ? 1u : 0u); }
    // Arrive adding `count` to the arrival's flag total (the checks return
    // the sum over warps).
    __device__ __forceinline__ void arrive_count(unsigned count) {
        if ((threadIdx.x & 31) == 0)
            red_add_rlx(ctr + ((na % kSlots) * kNC + (unsigned)gw % kNC) * kLineWords, 1ull | ((u64)count << 32));
        na++;
    }
    __device__ __forceinline__ u64 peek(unsigned i) const {
        const int lane = threadIdx.x & 31;
        return lane < kNC ? ld_rlx(ctr + ((i % kSlots) * kNC + lane) * kLineWords) : 0ull;
    }
    // Warps that raised their flag at arrival i (the sum of their counts),
    // or -1 if some warp has not reported it yet (then nothing is recorded). After A arrivals with F
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

// One thread's column: ZS segments of 4 consecutive states of a row of the
// last dimension, at the same place of ZS consecutive slices of dimension 0
// (ZS = 1 for one-dimensional grids). Columns are numbered slice group by
// slice group, so consecutive lanes hold neighbouring segments of a slice;
// the dimension-0 neighbours inside a column are in this thread's registers.
template <int D, int ZS>
struct FlowCol {
    static constexpr int NRR = 2 * (D - 1);          // row-neighbour directions (other dimensions)
    static constexpr int NR = NRR > 0 ? NRR : 1;
    static constexpr int HM = 2 * NRR, HP = 2 * NRR + 1;  // bits of the left / right halo words
    static constexpr unsigned OBST = 1u << (2 * D), TERM = 1u << (2 * D + 1);

    int s0[ZS];
    bool valid[ZS];
    unsigned code[ZS];    // the 4 codes of segment i, state k in byte k
    unsigned inw[ZS];     // not from memory (shuffle, or a register inside the column):
                          // bits 2j, 2j+1 (row j), HM, HP
    unsigned need[ZS];    // needed from memory: bit 2j + h (row j, half h), HM, HP
    int own[ZS];          // first ring word of segment i (a lane without one: the last segment's)
    float R[ZS][4], cur[ZS][4];
    unsigned act[ZS];     // policy iteration: 4 actions, state k in byte k

    // Row j of segment i can come from memory: the other dimensions always,
    // dimension 0 only at the column's ends.
    static __device__ __forceinline__ constexpr bool memrow(int i, int j) {
        return j >= 2 || (j == 0 && i == 0) || (j == 1 && i == ZS - 1);
    }

    __device__ __forceinline__ void init(const FlowArgs &f, int col, int lane) {
        const BandArgs &a = f.a;
        const int P = f.slice;                    // segments per dimension-0 slice
        const int zc = col / P, ps = col - zc * P;
        const bool colok = col < f.ncols;
#pragma unroll
        for (int i = 0; i < ZS; i++) {
            const int z = zc * ZS + i;
            valid[i] = colok && z < f.nz;
            s0[i] = (D == 1) ? 4 * col : z * a.stride[0] + 4 * ps;
            code[i] = 0;
            act[i] = 0;
            need[i] = 0;
            own[i] = valid[i] ? s0[i] : a.nstates - 4;
            unsigned m = 0;
#pragma unroll
            for (int j = 0; j < NRR; j++) {
                const bool up = (j & 1) != 0;
                if (j < 2 && ((!up && i > 0) || (up && i < ZS - 1))) { m |= 3u << (2 * j); continue; }
                const int so = a.stride[j / 2] / 4;
                if (so < 32 && (up ? lane + so < 32 : lane >= so)) m |= 3u << (2 * j);
            }
            if (lane >= 1) m |= 1u << HM;
            if (lane <= 30) m |= 1u << HP;
            inw[i] = m;
#pragma unroll
            for (int k = 0; k < 4; k++) { R[i][k] = 0.f; cur[i][k] = 0.f; }
            if (!valid[i]) continue;
            code[i] = *reinterpret_cast<const unsigned *>(static_cast<const uint8_t *>(a.code) + s0[i]);
            const float4 r = *reinterpret_cast<const float4 *>(a.R32 + s0[i]);
            const float4 v = *reinterpret_cast<const float4 *>(f.V + s0[i]);
            R[i][0] = r.x; R[i][1] = r.y; R[i][2] = r.z; R[i][3] = r.w;
            cur[i][0] = v.x; cur[i][1] = v.y; cur[i][2] = v.z; cur[i][3] = v.w;
            unsigned nd = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned c = (code[i] >> (8 * k)) & 0xFFu;
                if (c & (OBST | TERM)) continue;
#pragma unroll
                for (int j = 0; j < NRR; j++)
                    if (!((c >> j) & 1u)) nd |= 1u << (2 * j + (k >> 1));
                if (k == 0 && !((c >> NRR) & 1u)) nd |= 1u << HM;
                if (k == 3 && !((c >> (NRR + 1)) & 1u)) nd |= 1u << HP;
            }
            need[i] = nd & ~m;
        }
    }

    // Ring word read for row j, half h of segment i: the neighbours' pair
    // when it is needed from memory, else the segment's own pair (already
    // written).
    __device__ __forceinline__ int wo(const BandArgs &a, int i, int j, int h) const {
        const int st = a.stride[j / 2];
        return own[i] + 2 * h + (((need[i] >> (2 * j + h)) & 1u) ? ((j & 1) ? st : -st) : 0);
    }
    __device__ __forceinline__ int wol(int i) const { return own[i] - (int)((need[i] >> HM) & 1u); }
    __device__ __forceinline__ int wor(int i) const { return own[i] + (int)(((need[i] >> HP) & 1u) << 2); }

    // Segment i's own values of sequence q, read back from the ring: its own
    // words, written by this thread and still there while q is one of the
    // kRing - 1 latest sequences written.
    __device__ __forceinline__ void own_values(const FlowArgs &f, unsigned q, int i, float (&v)[4]) const {
        if (!valid[i]) return;
        const u64 *in = ring(f, q);
        u64 a, b, c, d;
        ld_rlx2(in + s0[i], a, b);
        ld_rlx2(in + s0[i] + 2, c, d);
        v[0] = val(a); v[1] = val(b); v[2] = val(c); v[3] = val(d);
    }
    __device__ __forceinline__ void own_values_all(const FlowArgs &f, unsigned q, float (&v)[ZS][4]) const {
#pragma unroll
        for (int i = 0; i < ZS; i++) own_values(f, q, i, v[i]);
    }

    __device__ __forceinline__ void publish(const FlowArgs &f, unsigned q, unsigned base,
                                            const float (&v)[ZS][4]) const {
        u64 *out = ring(f, q);
        const unsigned tg = base + q;
#pragma unroll
        for (int i = 0; i < ZS; i++) {
            if (!valid[i]) continue;
            st_rlx2(out + s0[i], word(v[i][0], tg), word(v[i][1], tg));
            st_rlx2(out + s0[i] + 2, word(v[i][2], tg), word(v[i][3], tg));
        }
    }

    // Neighbour values of sweep q (tag base + q, buffer q mod kRing) for the
    // column's values `self` of sweep q: rows[i][j][k] is the value one move
    // in direction j from state k of segment i, hl[i] / hr[i] the states
    // just left of state 0 and right of state 3 (for blocked moves:
    // anything). Every lane issues the loads of all the ring words it needs
    // at once (a word it does not need is not read: it stands in with the
    // right tag and a value nothing uses), checks all tags with one OR and
    // re-reads only on a mismatch. Returns false when the warp must stop
    // (status recorded). Skipping the unneeded words (in-warp neighbours,
    // walls) took 64^3 sweeps from 1.90 to 1.72 us: the L2 requests count.
    __device__ __forceinline__ bool gather(const FlowArgs &f, unsigned q, unsigned base, const float (&self)[ZS][4],
                                           float (&rows)[ZS][NR][4], float (&hl)[ZS], float (&hr)[ZS], Ctrl *ctrl,
                                           u64 timeout_ns) const {
        const unsigned tg = base + q;
        const u64 *in = ring(f, q);
        u64 w[ZS][NR][2][2];
        u64 wl[ZS], wr[ZS];
        // The neighbours' words of sweep q are usually stored just as this
        // warp finishes sweep q - 1; a read that reaches L2 before them costs
        // a second round trip. A short pause first lowers that share
        // (measured at 64^3 and 32^3: about 2 % and 4 % faster sweeps).
        __nanosleep(100);
        const u64 dflt = (u64)tg << 32;
#pragma unroll
        for (int i = 0; i < ZS; i++) {
#pragma unroll
            for (int j = 0; j < NRR; j++)
                if (memrow(i, j))
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        w[i][j][h][0] = dflt; w[i][j][h][1] = dflt;
                        if ((need[i] >> (2 * j + h)) & 1u) ld_rlx2(in + wo(f.a, i, j, h), w[i][j][h][0], w[i][j][h][1]);
                    }
            wl[i] = dflt; wr[i] = dflt;
            if ((need[i] >> HM) & 1u) wl[i] = ld_rlx(in + wol(i));
            if ((need[i] >> HP) & 1u) wr[i] = ld_rlx(in + wor(i));
        }
        // neighbours held by other lanes (the stride is the same for every
        // thread, so these branches are uniform)
        const int lane = threadIdx.x & 31;
        float sh[ZS][NR][4];
#pragma unroll
        for (int i = 0; i < ZS; i++)
#pragma unroll
            for (int j = 0; j < NRR; j++) {
                if (!memrow(i, j)) continue;
                const int so = f.a.stride[j / 2] >> 2;
                if (so < 32) {
                    const int src = ((j & 1) ? lane + so : lane - so) & 31;
                    // dimension 0 across columns: the other end of the neighbouring column
                    const int si = j >= 2 ? i : ((j & 1) ? 0 : ZS - 1);
#pragma unroll
                    for (int k = 0; k < 4; k++) sh[i][j][k] = __shfl_sync(FULL, self[si][k], src);
                }
            }
        float sl[ZS], sr[ZS];
#pragma unroll
        for (int i = 0; i < ZS; i++) {
            sl[i] = __shfl_up_sync(FULL, self[i][3], 1);
            sr[i] = __shfl_down_sync(FULL, self[i][0], 1);
        }
        unsigned bad = 0;
#pragma unroll
        for (int i = 0; i < ZS; i++) {
            bad |= ((unsigned)(wl[i] >> 32) ^ tg) | ((unsigned)(wr[i] >> 32) ^ tg);
#pragma unroll
            for (int j = 0; j < NRR; j++)
                if (memrow(i, j))
#pragma unroll
                    for (int h = 0; h < 2; h++)
                        bad |= ((unsigned)(w[i][j][h][0] >> 32) ^ tg) | ((unsigned)(w[i][j][h][1] >> 32) ^ tg);
        }
        if (__any_sync(FULL, bad != 0u)) {
            // slow path: re-read the words whose tag is not there yet
            u64 t0 = 0;
            unsigned spins = 0;
            for (;;) {
                unsigned pend[ZS];
                unsigned any = 0;
#pragma unroll
                for (int i = 0; i < ZS; i++) {
                    pend[i] = 0;
#pragma unroll
                    for (int j = 0; j < NRR; j++)
                        if (memrow(i, j))
#pragma unroll
                            for (int h = 0; h < 2; h++)
                                if (!has(w[i][j][h][0], tg) || !has(w[i][j][h][1], tg)) pend[i] |= 1u << (2 * j + h);
                    if (!has(wl[i], tg)) pend[i] |= 1u << HM;
                    if (!has(wr[i], tg)) pend[i] |= 1u << HP;
                    any |= pend[i];
                }
                if (!__any_sync(FULL, any != 0u)) break;
                if ((++spins & 15u) == 0 && give_up(ctrl, t0, timeout_ns)) return false;
#pragma unroll
                for (int i = 0; i < ZS; i++) {
#pragma unroll
                    for (int j = 0; j < NRR; j++)
                        if (memrow(i, j))
#pragma unroll
                            for (int h = 0; h < 2; h++)
                                if ((pend[i] >> (2 * j + h)) & 1u)
                                    ld_rlx2(in + wo(f.a, i, j, h), w[i][j][h][0], w[i][j][h][1]);
                    if ((pend[i] >> HM) & 1u) wl[i] = ld_rlx(in + wol(i));
                    if ((pend[i] >> HP) & 1u) wr[i] = ld_rlx(in + wor(i));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < ZS; i++) {
#pragma unroll
            for (int j = 0; j < NRR; j++)
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (!memrow(i, j)) {
                        rows[i][j][k] = (j & 1) ? self[i < ZS - 1 ? i + 1 : i][k] : self[i > 0 ? i - 1 : 0][k];
                    } else {
                        const float m = val(w[i][j][k >> 1][k & 1]);
                        rows[i][j][k] = ((inw[i] >> (2 * j)) & 1u) ? sh[i][j][k] : m;
                    }
                }
            if (NRR == 0) {
#pragma unroll
                for (int k = 0; k < 4; k++) rows[i][0][k] = 0.f;
            }
            hl[i] = ((inw[i] >> HM) & 1u) ? sl[i] : val(wl[i]);
            hr[i] = ((inw[i] >> HP) & 1u) ? sr[i] : val(wr[i]);
        }
        return true;
    }

    // Neighbour values of state k of segment i with blocked moves replaced
    // by V(s), in the order of the codes' move bits (as Segment::neighbours).
    __device__ __forceinline__ void nbk(const float (&self)[ZS][4], const float (&rows)[ZS][NR][4],
                                        const float (&hl)[ZS], const float (&hr)[ZS], int i, int k,
                                        float (&nb)[2 * D]) const {
        const unsigned c = (code[i] >> (8 * k)) & 0xFFu;
#pragma unroll
        for (int j = 0; j < NRR; j++) nb[j] = ((c >> j) & 1u) ? self[i][k] : rows[i][j][k];
        const float left = (k == 0) ? hl[i] : self[i][k > 0 ? k - 1 : 0];
        const float right = (k == 3) ? hr[i] : self[i][k < 3 ? k + 1 : 0];
        nb[NRR] = ((c >> NRR) & 1u) ? self[i][k] : left;
        nb[NRR + 1] = ((c >> (NRR + 1)) & 1u) ? self[i][k] : right;
    }
};

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

// The decision after an improvement sweep of policy iteration, from its
// arrival (warps that changed an action in the low 16 bits, warps whose
// residual is >= eval_tol in the high 16) and whether the evaluation before
// it reached eval_tol (the same rules as the grid-barrier solver): 0 go on
// (after a stable policy whose evaluation was capped: evaluate to eval_tol
// from now on, full = true and the running phase's cap raised), 1 converged,
// 2 stop (the evaluation limit ran out).
__device__ __forceinline__ int pi_decide(int moved, int prev_ok, bool &full, int &cap, int max_eval) {
    const int nchg = moved & 0xFFFF, nopen = moved >> 16;
    if (nchg == 0) {
        if (nopen == 0) return 1;
        if (!prev_ok) {
            if (full) return 2;
            full = true;
            cap = max_eval;
        }
        return 0;
    }
    return (!prev_ok && full) ? 2 : 0;
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

template <int D, int ZS>
__global__ void __launch_bounds__(32 * ColWarps<ZS>::value, 1) flow_vi_kernel(FlowArgs f, SolveParams sp, Ctrl *ctrl) {
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
    typedef FlowCol<D, ZS> Col;
    Col sg;
    sg.init(f, blockIdx.x * blockDim.x + threadIdx.x, lane);
    const unsigned base = f.base;
    sg.publish(f, 0, base, sg.cur);

    constexpr int NR = Col::NR;
    constexpr unsigned OBST = Col::OBST;
    const unsigned maxq = (unsigned)sp.max_iter;
    unsigned q = 0;
    float rh[kLag];                        // thread residuals of sweeps q-1, q-2, ...
#pragma unroll
    for (int i = 0; i < kLag; i++) rh[i] = 0.f;
    float res[ZS][4];
    float rres = 0.f;
    int iters = 0, conv = 0;
    for (;;) {
        const u64 pk = q >= kLag ? arv.peek(arv.nchk) : 0ull;
        float rows[ZS][NR][4], hl[ZS], hr[ZS];
        if (!sg.gather(f, q, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
        float nxt[ZS][4];
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < ZS; i++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float nb[2 * D];
                sg.nbk(sg.cur, rows, hl, hr, i, k, nb);
                const unsigned c = (sg.code[i] >> (8 * k)) & 0xFFu;
                int arg;
                const float v = vi_state<float, D, false>(sg.cur[i][k], nb, c, sg.R[i][k], wm, wp, wst, g, arg);
                nxt[i][k] = v;
                if (sg.valid[i] && !(c & OBST)) {
                    const float dv = abs_diff(v, sg.cur[i][k]);
                    r = dv > r ? dv : r;
                }
            }
        if (q >= kLag) {
            const int nf = arv.check(pk, ctrl, sp.timeout_ns);
            if (nf < 0) return;
            if (nf == 0) {  // sweep q - kLag met the stopping rule: its result is V_{q-kLag+1}
                sg.own_values_all(f, q - kLag + 1, res);
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
        for (int i = 0; i < ZS; i++)
#pragma unroll
            for (int k = 0; k < 4; k++) sg.cur[i][k] = nxt[i][k];
#pragma unroll
        for (int i = kLag - 1; i > 0; i--) rh[i] = rh[i - 1];
        rh[0] = r;
        q++;
        if (q == maxq) {
            // the limit: settle the unchecked sweeps in order
#pragma unroll
            for (int i = 0; i < ZS; i++)
#pragma unroll
                for (int k = 0; k < 4; k++) res[i][k] = sg.cur[i][k];
            rres = rh[0];
            iters = (int)q;
            while (arv.nchk < arv.na) {
                const unsigned sweep = arv.nchk;  // value iteration: arrival i is sweep i
                const int nf = arv.check_next(ctrl, sp.timeout_ns);
                if (nf < 0) return;
                if (nf == 0 && !conv) {
                    conv = 1;
                    iters = (int)sweep + 1;
                    if (sweep + 1 != q) sg.own_values_all(f, sweep + 1, res);
                    const unsigned back = q - 1 - sweep;   // 0 .. kLag-1
#pragma unroll
                    for (int i = 0; i < kLag; i++)
                        if ((unsigned)i == back) rres = rh[i];
                }
            }
            break;
        }
    }
#pragma unroll
    for (int i = 0; i < ZS; i++)
        if (sg.valid[i])
            *reinterpret_cast<float4 *>(f.V + sg.s0[i]) = make_float4(res[i][0], res[i][1], res[i][2], res[i][3]);
    flow_finish(ctrl, rres, sp.timeout_ns, NW, gw == 0 && lane == 0, iters, conv,
                (long long)iters * f.a.nstates * sp.nactions, 0, 0, q + 2);
}

template <int D, int ZS>
__global__ void __launch_bounds__(32 * ColWarps<ZS>::value, 1) flow_pi_kernel(FlowArgs f, SolveParams sp, Ctrl *ctrl) {
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
    typedef FlowCol<D, ZS> Col;
    Col sg;
    sg.init(f, blockIdx.x * blockDim.x + threadIdx.x, lane);
    const unsigned base = f.base;
    constexpr int NR = Col::NR;
    constexpr unsigned OBST = Col::OBST;

    // initial policy: greedy with respect to the input V
    unsigned q = 0;
    sg.publish(f, 0, base, sg.cur);
    {
        float rows[ZS][NR][4], hl[ZS], hr[ZS];
        if (!sg.gather(f, 0, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
#pragma unroll
        for (int i = 0; i < ZS; i++) {
            unsigned dummy = 0, act = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float nb[2 * D];
                sg.nbk(sg.cur, rows, hl, hr, i, k, nb);
                const unsigned c = (sg.code[i] >> (8 * k)) & 0xFFu;
                const int a = improve_state<D>(nb, sg.cur[i][k], c, sg.R[i][k], 0, true, margin, wm, wp, wst, g,
                                               dummy);
                act |= (unsigned)a << (8 * k);
            }
            sg.act[i] = act;
        }
    }
    int evals = 0, round = 0, conv = 0, stop = 0;
    float rres = 0.f;
    // modified policy iteration, the same schedule as the grid-barrier
    // solver (so the same rounds and sweeps): while the policy changes, each
    // evaluation runs exactly partial_eval sweeps; once an improvement after
    // such a capped evaluation changes no action, evaluations run to
    // eval_tol. Every store of sequence x first checks the arrivals of the
    // sequences up to x - 3 (four rings: nobody still reads the ring it
    // overwrites). A capped evaluation needs no other check: its improvement
    // follows at once, on its last sweep, and the improvement's decision
    // (stop, evaluate to eval_tol, go on) is read when its arrival comes up
    // in that order, at the latest when the next evaluation reaches its cap;
    // a "stop" returns every warp to the improvement's values (its own ring
    // words, still intact) and drops what followed.
    bool full = sp.partial_eval <= 0;
    unsigned chk_out = 1;       // output sequence of the next unchecked arrival
    bool pend = false;          // an improvement's arrival not checked yet
    unsigned pend_seq = 0;      // its output sequence (V')
    float pend_r = 0.f;         // its residual
    int pend_ok = 0;            // whether the evaluation before it reached eval_tol
    while (round < sp.max_rounds) {
        int cap = full ? sp.max_eval_iter : min(sp.partial_eval, sp.max_eval_iter);
        // evaluation of the current policy from V_q (tag base + q)
        const unsigned q0 = q;
        unsigned rq = q;
        int e = 0, eval_ok = 0;
        float rh[kLag];
#pragma unroll
        for (int i = 0; i < kLag; i++) rh[i] = 0.f;
        for (;;) {
            // the check due before this iteration's store of q + 1: sequence q - 2
            const bool chk = chk_out + 2u <= q;
            const u64 pk = chk ? arv.peek(arv.nchk) : 0ull;
            float rows[ZS][NR][4], hl[ZS], hr[ZS];
            if (!sg.gather(f, q, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
            float nxt[ZS][4];
            float r = 0.f;
#pragma unroll
            for (int i = 0; i < ZS; i++)
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    float nb[2 * D];
                    sg.nbk(sg.cur, rows, hl, hr, i, k, nb);
                    const unsigned c = (sg.code[i] >> (8 * k)) & 0xFFu;
                    const float v = eval_state<float, D>(sg.cur[i][k], nb, c, sg.R[i][k],
                                                         (int)((sg.act[i] >> (8 * k)) & 0xFFu), wm, wp, wst, g);
                    nxt[i][k] = v;
                    if (sg.valid[i] && !(c & OBST)) {
                        const float dv = abs_diff(v, sg.cur[i][k]);
                        r = dv > r ? dv : r;
                    }
                }
            if (chk) {
                const int nf = arv.check(pk, ctrl, sp.timeout_ns);
                if (nf < 0) return;
                const unsigned s = chk_out++;
                if (pend && s == pend_seq) {   // the last improvement's decision
                    pend = false;
                    stop = pi_decide(nf, pend_ok, full, cap, sp.max_eval_iter);
                    if (stop) {
                        sg.own_values_all(f, pend_seq, sg.cur);
                        rres = pend_r;
                        break;
                    }
                } else if (full && s > q0 && nf == 0) {
                    // the sweep that produced V_s met eval_tol (s = q - 2): V_s ends the evaluation
                    sg.own_values_all(f, s, sg.cur);
                    rres = rh[kLag - 1];
                    rq = s;
                    eval_ok = 1;
                    break;
                }
                // otherwise an evaluation sweep of a capped phase: its check only orders the rings
            }
            sg.publish(f, q + 1, base, nxt);
            arv.arrive(warp_open(r, f.eval_tol_bits));
#pragma unroll
            for (int i = 0; i < ZS; i++)
#pragma unroll
                for (int k = 0; k < 4; k++) sg.cur[i][k] = nxt[i][k];
#pragma unroll
            for (int i = kLag - 1; i > 0; i--) rh[i] = rh[i - 1];
            rh[0] = r;
            q++;
            e++;
            if (e == cap && pend) {
                // the last improvement's decision is still out: take it now
                while (pend) {
                    const int nf = arv.check_next(ctrl, sp.timeout_ns);
                    if (nf < 0) return;
                    const unsigned s = chk_out++;
                    if (s == pend_seq) {
                        pend = false;
                        stop = pi_decide(nf, pend_ok, full, cap, sp.max_eval_iter);
                    }
                }
                if (stop) {
                    sg.own_values_all(f, pend_seq, sg.cur);
                    rres = pend_r;
                    break;
                }
                if (e < cap) continue;   // cap raised: this evaluation runs to eval_tol
            }
            if (e == cap) {
                rres = rh[0];
                rq = q;
                if (full) {
                    // an evaluation to eval_tol that reached max_eval_iter:
                    // whether one of its last sweeps met eval_tol after all
                    while (chk_out <= q) {
                        const int nf = arv.check_next(ctrl, sp.timeout_ns);
                        if (nf < 0) return;
                        const unsigned s = chk_out++;
                        if (s > q0 && nf == 0 && !eval_ok) {
                            eval_ok = 1;
                            rq = s;
                            if (rq != q) sg.own_values_all(f, rq, sg.cur);
                            const unsigned back = q - s;   // 0 .. kLag-1
#pragma unroll
                            for (int i2 = 0; i2 < kLag; i2++)
                                if ((unsigned)i2 == back) rres = rh[i2];
                        }
                    }
                }
                break;
            }
        }
        if (stop) break;   // the last improvement ended the solve
        evals += (int)(rq - q0);
        if (full) {
            // every earlier arrival is settled before the improvement (it
            // reads V_rq, possibly an older ring than the last one written)
            while (chk_out <= q) {
                if (arv.check_next(ctrl, sp.timeout_ns) < 0) return;
                chk_out++;
            }
        } else {
            // the checks due before the improvement's store of q + 1
            while (chk_out + 2u <= q) {
                if (arv.check_next(ctrl, sp.timeout_ns) < 0) return;
                chk_out++;
            }
        }
        const unsigned hq = q;  // highest tag sequence written so far
        // sg.cur now holds V_rq, the values of this evaluation
        // improvement on V_rq (tag base + rq, buffer rq mod kRing), and the
        // new policy's first evaluation step V' = Q of the action kept or
        // taken (modified policy iteration)
        unsigned changed = 0;
        float nxt[ZS][4];
        float r = 0.f;
        {
            float rows[ZS][NR][4], hl[ZS], hr[ZS];
            if (!sg.gather(f, rq, base, sg.cur, rows, hl, hr, ctrl, sp.timeout_ns)) return;
#pragma unroll
            for (int i = 0; i < ZS; i++) {
                unsigned act = 0, ch = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    float nb[2 * D];
                    sg.nbk(sg.cur, rows, hl, hr, i, k, nb);
                    const unsigned c = (sg.code[i] >> (8 * k)) & 0xFFu;
                    const int old = (int)((sg.act[i] >> (8 * k)) & 0xFFu);
                    const int a = improve_state<D>(nb, sg.cur[i][k], c, sg.R[i][k], old, false, margin, wm, wp, wst,
                                                   g, ch);
                    act |= (unsigned)a << (8 * k);
                    const float v = eval_state<float, D>(sg.cur[i][k], nb, c, sg.R[i][k], a, wm, wp, wst, g);
                    nxt[i][k] = v;
                    if (sg.valid[i] && !(c & OBST)) {
                        const float dv = abs_diff(v, sg.cur[i][k]);
                        r = dv > r ? dv : r;
                    }
                }
                if (sg.valid[i]) {
                    sg.act[i] = act;
                    changed += ch;
                }
            }
        }
        // the next evaluation starts from V' published as sequence hq + 1
        q = hq + 1;
        sg.publish(f, q, base, nxt);
#pragma unroll
        for (int i = 0; i < ZS; i++)
#pragma unroll
            for (int k = 0; k < 4; k++) sg.cur[i][k] = nxt[i][k];
        rres = r;
        const unsigned wc = __reduce_add_sync(FULL, changed);
        if (lane == 0 && wc) atomicAdd(&ctrl->changed_total, wc);
        // one arrival carries both counts: warps whose actions changed (low
        // 16 bits) and warps whose residual is at or above eval_tol (high 16)
        const bool wopen = warp_open(r, f.eval_tol_bits);
        arv.arrive_count((wc > 0 ? 1u : 0u) + (wopen ? 65536u : 0u));
        round++;
        if (rq == hq) {
            // the improvement read ring hq, which later stores overwrite only
            // from sequence hq + 4 on: its decision is read in order (or below,
            // after the last round)
            pend = true;
            pend_seq = q;
            pend_r = r;
            pend_ok = eval_ok;
        } else {
            // an evaluation to eval_tol that stopped early leaves the
            // improvement reading an older ring, one the next stores overwrite
            // sooner: every arrival before its own was settled above
            const int moved = arv.check_next(ctrl, sp.timeout_ns);
            if (moved < 0) return;
            chk_out++;
            int cap_unused = 0;
            stop = pi_decide(moved, eval_ok, full, cap_unused, sp.max_eval_iter);
            if (stop) break;
        }
    }
    while (pend) {   // the round limit came first: the last improvement's decision
        const int nf = arv.check_next(ctrl, sp.timeout_ns);
        if (nf < 0) return;
        const unsigned s = chk_out++;
        if (s == pend_seq) {
            pend = false;
            int cap_unused = 0;
            stop = pi_decide(nf, pend_ok, full, cap_unused, sp.max_eval_iter);
        }
    }
    conv = stop == 1;
#pragma unroll
    for (int i = 0; i < ZS; i++)
        if (sg.valid[i]) {
            *reinterpret_cast<float4 *>(f.V + sg.s0[i]) =
                make_float4(sg.cur[i][0], sg.cur[i][1], sg.cur[i][2], sg.cur[i][3]);
            *reinterpret_cast<unsigned *>(f.pi + sg.s0[i]) = sg.act[i];
        }
    // sweeps: greedy + evaluations + improvements; backups: |S||A| per greedy
    // or improvement sweep, |S| per evaluation sweep
    flow_finish(ctrl, rres, sp.timeout_ns, NW, gw == 0 && lane == 0, 1 + evals + round, conv,
                (long long)(1 + round) * f.a.nstates * sp.nactions + (long long)evals * f.a.nstates, round, evals,
                q + 2);
}

// Launch shape: one block per SM (as far as the warps go), every block with
// the same number of warps, one warp per 32 consecutive columns. Sweeps
// move at the pace of the busiest SM, so the warps are spread evenly.
struct FlowShape {
    int zs, block, grid, slice, nz, ncols;
};

template <int D, int ZS>
static bool shape_for(const Factors &F, FlowShape &s) {
    s.zs = ZS;
    s.slice = D == 1 ? (int)(F.nstates / 4) : (int)(F.stride[0] / 4);
    s.nz = D == 1 ? 1 : (int)F.shape[0];
    const long long ncols = (long long)s.slice * ((s.nz + ZS - 1) / ZS);
    const long long nwarps = (ncols + 31) / 32;
    const long long w = (nwarps + F.num_sms - 1) / F.num_sms;
    if (w < 1 || w > ColWarps<ZS>::value || ncols > (1ll << 30)) return false;
    s.ncols = (int)ncols;
    s.block = 32 * (int)w;
    s.grid = (int)((nwarps + w - 1) / w);
    if (s.grid > F.num_sms) return false;
    // both kernels keep one such block per SM resident
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, flow_vi_kernel<D, ZS>, s.block, 0) != cudaSuccess) a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, flow_pi_kernel<D, ZS>, s.block, 0) != cudaSuccess) b = 0;
    return a >= 1 && b >= 1;
}

#ifndef CPMDP_FLOW_ZS
#define CPMDP_FLOW_ZS 1
#endif

// Column height: the preferred one if the grid fits, else the next that does.
// Policy iteration on 3-D grids takes columns of two segments when single
// segments would fill more than three quarters of the co-resident warps:
// fewer warps then contend for issue (measured per evaluation sweep: 64^3
// 1.63 against 1.67 us; at 32^3 and 48^3 single segments are faster, and
// value iteration is faster with single segments at 64^3 too).
template <int D>
static bool flow_pick(const Factors &F, FlowShape &s, bool policy_iteration) {
    if (D == 1) return shape_for<D, 1>(F, s);
    if (policy_iteration && D == 3) {
        FlowShape s1;
        const long long full = (long long)F.num_sms * 32 * ColWarps<1>::value;
        if (shape_for<D, 1>(F, s1) && 4ll * s1.grid * s1.block > 3ll * full && shape_for<D, D == 1 ? 1 : 2>(F, s))
            return true;
    }
    const int order[3] = {CPMDP_FLOW_ZS, CPMDP_FLOW_ZS == 1 ? 2 : 1, CPMDP_FLOW_ZS == 4 ? 2 : 4};
    for (int zs : order) {
        if (zs == 1 && shape_for<D, 1>(F, s)) return true;
        if (zs == 2 && shape_for<D, D == 1 ? 1 : 2>(F, s)) return true;
        if (zs == 4 && shape_for<D, D == 1 ? 1 : 4>(F, s)) return true;
    }
    return false;
}

static bool flow_pick_any(const Factors &F, FlowShape &s, bool policy_iteration) {
    switch (F.ndim) {
        case 1: return flow_pick<1>(F, s, policy_iteration);
        case 2: return flow_pick<2>(F, s, policy_iteration);
        case 3: return flow_pick<3>(F, s, policy_iteration);
        default: return false;
    }
}

template <int D, int ZS>
static cudaError_t launch_zs(const FlowShape &s, bool pim, FlowArgs &f, SolveParams &spc, Ctrl *ctrl, cudaStream_t st) {
    void *args[] = {(void *)&f, (void *)&spc, (void *)&ctrl};
    const void *kern = pim ? (const void *)flow_pi_kernel<D, ZS> : (const void *)flow_vi_kernel<D, ZS>;
    return cudaLaunchCooperativeKernel(kern, dim3(s.grid), dim3(s.block), args, 0, st);
}

template <int D>
static cudaError_t launch_flow(const FlowShape &s, bool pim, const FlowArgs &fa, const SolveParams &sp, Ctrl *ctrl,
                               cudaStream_t st) {
    FlowArgs f = fa;
    SolveParams spc = sp;
    f.slice = s.slice;
    f.nz = s.nz;
    f.ncols = s.ncols;
    if (s.zs == 1 || D == 1) return launch_zs<D, 1>(s, pim, f, spc, ctrl, st);
    if (s.zs == 2) return launch_zs<D, D == 1 ? 1 : 2>(s, pim, f, spc, ctrl, st);
    return launch_zs<D, D == 1 ? 1 : 4>(s, pim, f, spc, ctrl, st);
}

}  // namespace

bool flow_eligible(const Factors &F, bool policy_iteration, const void *V, const uint8_t *pi,
                   const SolveOpts &o) {
    if (F.ndim < 1 || F.ndim > 3 || F.num_sms <= 0) return false;
    if (F.shape[F.ndim - 1] % 4 != 0 || F.nstates % 4 != 0 || F.nstates >= (1ll << 30)) return false;
    if (((uintptr_t)V & 15u) != 0) return false;
    if (policy_iteration && ((uintptr_t)pi & 3u) != 0) return false;
    FlowShape s;
    if (!flow_pick_any(F, s, policy_iteration)) return false;
    // tags (base <= 2^30, plus the sweeps of one launch) stay below 2^32 - 1
    const long long sweeps = policy_iteration
                                 ? (long long)o.max_rounds * ((long long)o.max_eval_iter + 2) + 2
                                 : (long long)o.max_iter + 2;
    return sweeps < (1ll << 31);
}

bool flow_shape_ok(const Factors &F) {
    if (F.ndim < 1 || F.ndim > 3 || F.num_sms <= 0) return false;
    if (F.shape[F.ndim - 1] % 4 != 0 || F.nstates % 4 != 0 || F.nstates >= (1ll << 30)) return false;
    FlowShape s;
    return flow_pick_any(F, s, false) || flow_pick_any(F, s, true);
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
    FlowShape shp;
    if (!flow_pick_any(F, shp, policy_iteration)) CPMDP_CUDA(cudaErrorCooperativeLaunchTooLarge);
    cudaError_t e;
    switch (F.ndim) {
        case 1: e = launch_flow<1>(shp, policy_iteration, fa, sp, F.d_ctrl, st); break;
        case 2: e = launch_flow<2>(shp, policy_iteration, fa, sp, F.d_ctrl, st); break;
        default: e = launch_flow<3>(shp, policy_iteration, fa, sp, F.d_ctrl, st); break;
    }
    CPMDP_CUDA(e);
    return CPMDP_OK;
}

}  // namespace cpmdp
