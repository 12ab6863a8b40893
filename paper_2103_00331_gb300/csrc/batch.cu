// Batched value iteration: thousands of independent, uneven GridWorld MDPs
// (each a tuple <S, A, P, R, gamma> of its own, background section) solved
// in one persistent launch.
//
// The instances are packed back to back (values, FP32 rewards, per-state
// move codes in the encoding of the single-instance path). The work is cut
// into warp tiles: a tile is up to 32 x spl segments of one instance, each
// segment 4 consecutive states (instances start 16-byte aligned and are
// padded to a multiple of 4 states; a segment of an instance whose rows are
// not a multiple of 4 long may span two rows). Every global sweep the
// warps of the cooperative grid take the tiles of instances that are still
// running; an instance stops on its own as soon as its residual falls below
// tol, so short and long solves share the launch. Per-instance residuals use
// three rotating slots (slot k+1 is cleared during sweep k by the block that
// owns the instance's first tile, after every block has read slot k-2); the
// grid stops after a sweep in which no block found a running instance.
//
// The tile size (segments per lane) and block size are chosen by a small
// autotuner (time a few sweeps of each candidate on the actual batch), and
// the solve is recorded once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "banded_common.cuh"
#include "batch_flow.h"
#include "batch_internal.h"

namespace cpmdp {

struct BatchArgs {
    const BatchTile *tiles;
    int ntiles;
    int ninst;
    const uint8_t *code;
    const float *R;
    float *V;
    float *W;
    unsigned long long *res;   // [3][ninst]
    int *done_at;              // per instance: sweeps done when it stopped (0 = running)
    double tol;
    int max_iter;
    int spl;                   // segments per lane of a tile (tile = 32 spl segments)
    unsigned long long timeout_ns;
    Ctrl *ctrl;
    int handoff_warps;         // > 0: stop once the running instances need at most this many warps
};

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of the 128-byte lines holding elements [lo, hi) of an array
// of `esize`-byte elements (every line start lies inside the array).
__device__ __forceinline__ void prefetch_span(const void *base, long long lo, long long hi, int esize) {
    const char *p = static_cast<const char *>(base);
    for (long long a = (lo * esize) & ~127ll; a < hi * esize; a += 128) prefetch_l2(p + a);
}

// Everything a tile's backups read: its states (plus the row halo) of V, R
// and the codes, and the rows one stride away in each leading dimension.
// Issued by the lane that found the tile running, for all running tiles of
// a round at once, so that the warp, working through them one by one, waits
// for HBM once per round instead of once per tile.
__device__ __forceinline__ void prefetch_tile(const BatchTile &T, const float *V, const float *R, const uint8_t *code) {
    const long long base = T.offset, end = T.offset + T.nstates;
    const long long a0 = base + 4ll * T.first_item;
    long long a1 = base + 4ll * (T.first_item + T.nitems);
    a1 = a1 < end ? a1 : end;
    const long long h0 = a0 > base ? a0 - 1 : a0, h1 = a1 < end ? a1 + 1 : a1;
    prefetch_span(V, h0, h1, 4);
    prefetch_span(R, a0, a1, 4);
    prefetch_span(code, a0, a1, 1);
    const int ndim = T.cls >> 1;
    if (ndim >= 2) {
        const long long st = T.stride0;
        if (a0 - st >= base) prefetch_span(V, a0 - st, a1 - st, 4);
        if (a1 + st <= end) prefetch_span(V, a0 + st, a1 + st, 4);
    }
    if (ndim >= 3) {
        const long long st = T.stride1;
        if (a0 - st >= base) prefetch_span(V, a0 - st, a1 - st, 4);
        if (a1 + st <= end) prefetch_span(V, a0 + st, a1 + st, 4);
    }
}

// Loads of a 4-state segment whose rows are not a multiple of 4 states
// long: the segment may end one row and start the next, and the neighbour
// rows one stride away are not 16-byte aligned. The segment's own values,
// rewards and codes are (instances start 16-byte aligned and are padded to
// a multiple of 4 states with obstacle codes, so the last segment stays
// inside the packed arrays); each neighbour is loaded on its own with its
// index clamped into [0, npad). A clamped index only differs from the true
// neighbour where that neighbour does not exist, and there the move is
// blocked in the code (a wall at the end of a row included), so the backup
// uses V(s) instead. Padding states are obstacles: value 0, no residual.
template <typename TA, int D>
__device__ __forceinline__ void load_rows_any(Segment<float, TA, D, 4> &sg, const BandArgs &a, const float *V,
                                              int s0, int npad) {
    load_pack<uint8_t, 4>(static_cast<const uint8_t *>(a.code) + s0, sg.code);
    load_pack<float, 4>(V + s0, sg.vs);
#pragma unroll
    for (int d = 0; d < D - 1; d++) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int lo = s0 + k - a.stride[d], hi = s0 + k + a.stride[d];
            sg.rows[2 * d][k] = V[lo < 0 ? 0 : lo];
            sg.rows[2 * d + 1][k] = V[hi >= npad ? npad - 1 : hi];
        }
    }
    sg.halo_m = V[s0 > 0 ? s0 - 1 : 0];
    sg.halo_p = V[s0 + 4 < npad ? s0 + 4 : npad - 1];
    if constexpr (std::is_same<TA, float>::value) {
        load_pack<float, 4>(a.R32 + s0, sg.r);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) sg.r[k] = a.R64[s0 + k];
    }
}

// One 4-state segment of a tile per lane (segment first + lane of the
// instance), D fixed at compile time; ROWS4: rows a multiple of 4 states
// long (16-byte neighbour-row loads), else load_rows_any. (Two or more
// segments per lane in flight were measured slower: with every shape class
// compiled into one kernel their register needs add up and spill.)
template <int D, bool ROWS4>
__device__ __forceinline__ float batch_tile(const BatchTile &T, const uint8_t *code, const float *R, const float *V,
                                            float *W, int first, int nitems, int lane) {
    constexpr int VEC = 4;
    BandArgs a;
    a.nstates = T.nstates;
    a.nlast = T.nlast;
#pragma unroll
    for (int d = 0; d < kMaxDim; d++) a.stride[d] = 0;
    if (D >= 2) a.stride[0] = T.stride0;
    if (D >= 3) a.stride[1] = T.stride1;
    a.wf_move = T.w_move;
    a.wf_perp = T.w_perp;
    a.wf_stay = T.w_stay;
    a.wf_gamma = T.gamma;
    a.code = code + T.offset;
    a.R32 = R + T.offset;
    a.R64 = nullptr;
    const float *Vi = V + T.offset;
    float *Wi = W + T.offset;
    if (lane >= nitems) return 0.f;
    Segment<float, float, D, VEC> sg;
    if (ROWS4) sg.template load<M_VI>(a, Vi, nullptr, (first + lane) * VEC);
    else load_rows_any<float, D>(sg, a, Vi, (first + lane) * VEC, (T.nstates + 3) & ~3);
    return sg.template finish_vi<false>(a, Wi, nullptr, (first + lane) * VEC);
}

// Broadcast lane src's tile record to the warp.
__device__ __forceinline__ BatchTile shfl_tile(const BatchTile &x, int src) {
    BatchTile y;
    y.offset = __shfl_sync(0xFFFFFFFFu, x.offset, src);
    y.inst = __shfl_sync(0xFFFFFFFFu, x.inst, src);
    y.first_item = __shfl_sync(0xFFFFFFFFu, x.first_item, src);
    y.nitems = __shfl_sync(0xFFFFFFFFu, x.nitems, src);
    y.nstates = __shfl_sync(0xFFFFFFFFu, x.nstates, src);
    y.cls = __shfl_sync(0xFFFFFFFFu, x.cls, src);
    y.nlast = __shfl_sync(0xFFFFFFFFu, x.nlast, src);
    y.stride0 = __shfl_sync(0xFFFFFFFFu, x.stride0, src);
    y.stride1 = __shfl_sync(0xFFFFFFFFu, x.stride1, src);
    y.w_move = __shfl_sync(0xFFFFFFFFu, x.w_move, src);
    y.w_perp = __shfl_sync(0xFFFFFFFFu, x.w_perp, src);
    y.w_stay = __shfl_sync(0xFFFFFFFFu, x.w_stay, src);
    y.gamma = __shfl_sync(0xFFFFFFFFu, x.gamma, src);
    return y;
}

// The running tiles of one shape class (D, ROWS4) among the warp's round:
// run marks the lanes whose tile runs.
template <int D, bool ROWS4>
__device__ __forceinline__ void batch_class(const BatchArgs &b, const BatchTile &T, bool run, const float *cur,
                                            float *nxt, int k, int lane) {
    unsigned m = __ballot_sync(0xFFFFFFFFu, run && T.cls == D * 2 + (ROWS4 ? 1 : 0));
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const BatchTile Tb = shfl_tile(T, src);
        // b.spl groups of 32 segments, one after another (their lines are
        // already on their way to L2)
        float r = 0.f;
        for (int u = 0; u < b.spl; u++)
            r = fmaxf(r, batch_tile<D, ROWS4>(Tb, b.code, b.R, cur, nxt, Tb.first_item + 32 * u, Tb.nitems - 32 * u,
                                              lane));
        // non-negative residuals: integer max of the bit patterns
        const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(r));
        if (lane == 0 && mx)
            atomicMax(&b.res[(size_t)(k % 3) * b.ninst + Tb.inst],
                      (unsigned long long)__double_as_longlong((double)__uint_as_float(mx)));
    }
}

// One persistent launch. Every global sweep k, each warp takes the tiles
// t = w + j NW (w its global warp index, NW the number of warps, j = 0, 1,
// ...; consecutive tiles of an instance land on different warps), 32 at a
// time: lane l classifies tile w + (j0 + l) NW itself (its instance stopped
// earlier, stops now, or runs) and, if it runs, loads the instance record,
// so one round of loads serves 32 tiles. A lane remembers in a register
// which of its tiles belong to stopped instances (an instance never
// restarts within a solve) and loads nothing for them again. The warp then
// works through the running tiles of the round, each lane taking spl
// segments one after another, and reduces the tile's residual
// with one integer max (redux) and one atomicMax on the instance's slot.
// Warps never wait for one another inside a sweep; the block meets the grid
// barrier at the end, reporting whether any of its warps found a running
// tile.
__global__ void __launch_bounds__(512, 1) batch_vi_kernel(BatchArgs b) {
    __shared__ int s_worked;
    __shared__ unsigned long long s_need;
    const int tid = threadIdx.x, lane = tid & 31;
    const int wpb = blockDim.x >> 5;
    const long long nw = (long long)gridDim.x * wpb;
    const long long gw = (long long)blockIdx.x * wpb + (tid >> 5);
    const unsigned nb = gridDim.x;
    unsigned long long ph0 = 0ull, ph1 = 0ull;
    unsigned stopped = 0u;   // bit r: this lane's tile of round r belongs to a stopped instance
    int k = 0;
    bool handoff = false;
    for (; k <= b.max_iter; k++) {
        const float *cur = (k & 1) ? b.W : b.V;
        float *nxt = (k & 1) ? b.V : b.W;
        if (tid == 0) {
            s_worked = 0;
            s_need = 0ull;
            // slot k+1 was last read after the barrier of sweep k-2, which
            // every block has passed
            if (blockIdx.x == 0) b.ctrl->need_slot[(k + 1) % 3] = 0ull;
        }
        __syncthreads();
        bool worked = false;
        int round = 0;
        for (long long j0 = 0; gw + j0 * nw < b.ntiles; j0 += 32, round++) {
            const long long tl = gw + (j0 + lane) * nw;
            const bool known = round < 32 && ((stopped >> round) & 1u);
            if (__all_sync(0xFFFFFFFFu, known || tl >= b.ntiles)) continue;
            bool run = false;
            BatchTile T;
            T.inst = 0;
            T.cls = 0;
            if (tl < b.ntiles && !known) {
                T = b.tiles[tl];
                int st = 1;
                if (b.done_at[T.inst] != 0) {
                    st = 0;
                } else if (k > 0) {
                    const unsigned long long rb =
                        *(volatile unsigned long long *)&b.res[(size_t)((k - 1) % 3) * b.ninst + T.inst];
                    if (below_tol(rb, b.tol)) st = 2;
                }
                if (st == 1 && k == b.max_iter) st = 3;   // limit reached: stop without a sweep
                // every lane that sees the stop writes the same value
                if (st >= 2) b.done_at[T.inst] = st == 2 ? k : -k;
                run = st == 1;
                if (!run && round < 32) stopped |= 1u << round;
                if (run) {
                    if (T.first_item == 0) {
                        b.res[(size_t)((k + 1) % 3) * b.ninst + T.inst] = 0ull;
                        // warps this instance would take in the barrier-free tail
                        if (b.handoff_warps > 0)
                            atomicAdd(&s_need, (unsigned long long)(((T.nstates + 3) / 4 + 31) / 32));
                    }
                    prefetch_tile(T, cur, b.R, b.code);
                }
            }
            const unsigned act = __ballot_sync(0xFFFFFFFFu, run);
            worked |= act != 0u;
            if (!act) continue;
            // the running tiles, one instance shape class (D, rows of 4) at a
            // time: each class is its own loop
            batch_class<1, true>(b, T, run, cur, nxt, k, lane);
            batch_class<1, false>(b, T, run, cur, nxt, k, lane);
            batch_class<2, true>(b, T, run, cur, nxt, k, lane);
            batch_class<2, false>(b, T, run, cur, nxt, k, lane);
            batch_class<3, true>(b, T, run, cur, nxt, k, lane);
            batch_class<3, false>(b, T, run, cur, nxt, k, lane);
        }
        if (worked && lane == 0) s_worked = 1;
        __syncthreads();
        if (tid == 0 && s_need) atomicAdd(&b.ctrl->need_slot[k % 3], s_need);
        const long long busy = grid_sync_count(b.ctrl, k, nb, tid == 0 ? s_worked : 0, b.timeout_ns, ph0, ph1, false);
        if (busy < 0) return;
        if (busy == 0) break;
        // the instances that ran sweep k fit the barrier-free tail: stop here
        // (every block reads the same complete count after the barrier)
        if (b.handoff_warps > 0 &&
            *(volatile unsigned long long *)&b.ctrl->need_slot[k % 3] <= (unsigned long long)b.handoff_warps) {
            handoff = true;
            k++;
            break;
        }
    }
    // results: an instance stopped at sweep count n has its values in V if n
    // is even, in W if n is odd
    for (int t = blockIdx.x; t < b.ntiles; t += nb) {
        const BatchTile T = b.tiles[t];
        const int n = b.done_at[T.inst];
        const int sweeps = n < 0 ? -n : n;
        if (!(sweeps & 1)) continue;
        const int s0 = 4 * T.first_item, s1 = min(4 * (T.first_item + T.nitems), T.nstates);
        for (int s = s0 + tid; s < s1; s += blockDim.x) b.V[T.offset + s] = b.W[T.offset + s];
    }
    if (blockIdx.x == 0 && tid == 0) {
        b.ctrl->iterations = k;
        if (handoff) {
            b.ctrl->handoff_sweeps = k;
            b.ctrl->handoff = 1;
        }
    }
}

// One FP64 backup of every instance of the packed values (Eq. 1 in double
// arithmetic on the float iterate, FP64 rewards and weights): per instance
// the certified residual max |T(V) - V| over its non-obstacle states, and
// the FP64 argmax policy (lowest action on exact ties; 255 on obstacles and
// terminals). One warp per tile, lane l taking segments l, l + 32, ... of
// the tile; the padding states between instances are neither read as
// states nor written.
struct BatchCertArgs {
    const BatchTile *tiles;
    int ntiles;
    const uint8_t *code;
    const double *R64;
    const double *instw;       // per instance: w_move, w_perp, w_stay, gamma
    const float *V;
    uint8_t *pi;               // packed policy (nullable)
    unsigned long long *cert;  // per instance: bits of the certified residual
};

template <int D, bool ROWS4>
__device__ __forceinline__ double certify_segment(const BatchCertArgs &c, const BatchTile &T, int item) {
    BandArgs a;
    a.nstates = T.nstates;
    a.nlast = T.nlast;
#pragma unroll
    for (int d = 0; d < kMaxDim; d++) a.stride[d] = 0;
    if (D >= 2) a.stride[0] = T.stride0;
    if (D >= 3) a.stride[1] = T.stride1;
    const double *w = c.instw + 4 * (size_t)T.inst;
    a.w_move = w[0];
    a.w_perp = w[1];
    a.w_stay = w[2];
    a.gamma = w[3];
    a.code = c.code + T.offset;
    a.R32 = nullptr;
    a.R64 = c.R64 + T.offset;
    const float *Vi = c.V + T.offset;
    const int s0 = item * 4;
    Segment<float, double, D, 4> sg;
    if (ROWS4) sg.template load<M_VI>(a, Vi, nullptr, s0);
    else load_rows_any<double, D>(sg, a, Vi, s0, (T.nstates + 3) & ~3);
    double self[4], nb[2 * D][4];
    sg.neighbours(self, nb);
    double wm, wp, wst, g;
    weights<double>(a, wm, wp, wst, g);
    constexpr unsigned OBST = 1u << (2 * D), TERM = 1u << (2 * D + 1);
    double res = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (s0 + k >= T.nstates) break;
        const unsigned code = sg.code[k];
        double nbk[2 * D];
#pragma unroll
        for (int j = 0; j < 2 * D; j++) nbk[j] = nb[j][k];
        int arg;
        const double v = vi_state<double, D>(self[k], nbk, code, sg.r[k], wm, wp, wst, g, arg);
        if (c.pi) c.pi[T.offset + s0 + k] = (code & (OBST | TERM)) ? (uint8_t)255 : (uint8_t)arg;
        if (!(code & OBST)) res = fmax(res, fabs(v - self[k]));
    }
    return res;
}

__global__ void __launch_bounds__(256) batch_certify_kernel(BatchCertArgs c) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < c.ntiles; t += nw) {
        const BatchTile T = c.tiles[t];
        double r = 0.0;
        for (int i = lane; i < T.nitems; i += 32) {
            const int item = T.first_item + i;
            double x = 0.0;
            switch (T.cls) {
                case 2: x = certify_segment<1, false>(c, T, item); break;
                case 3: x = certify_segment<1, true>(c, T, item); break;
                case 4: x = certify_segment<2, false>(c, T, item); break;
                case 5: x = certify_segment<2, true>(c, T, item); break;
                case 6: x = certify_segment<3, false>(c, T, item); break;
                default: x = certify_segment<3, true>(c, T, item); break;
            }
            r = fmax(r, x);
        }
        // non-negative doubles order like their bit patterns
        const unsigned long long b = (unsigned long long)__double_as_longlong(r);
        unsigned long long m = b;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
            m = y > m ? y : m;
        }
        if (lane == 0 && m) atomicMax(&c.cert[T.inst], m);
    }
}

}  // namespace cpmdp

// ---------------------------------------------------------------------------
// host side

namespace cpmdp {

static void free_batch_device(cpmdp_batch &B) {
    void *ptrs[] = {B.d_inst, B.d_tiles, B.d_code, B.d_R, B.d_W, B.d_res, B.d_done, B.d_ctrl,
                    B.d_ring, B.d_p2ctr, B.d_p2tab, B.d_p2hdr, B.d_p2epoch, B.d_p2res,
                    B.d_R64, B.d_instw, B.d_cert, B.d_Rp, B.d_Gp, B.d_codep, B.d_rparts, B.d_rmulti,
                    B.d_rsolo, B.d_rhdr};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (B.graph) cudaGraphExecDestroy(B.graph);
    B.graph = nullptr;
}

static std::vector<BatchTile> make_tiles(const std::vector<BatchInst> &inst, int tile_items,
                                         std::vector<int> *first_tile) {
    std::vector<BatchTile> tiles;
    first_tile->assign(inst.size(), 0);
    for (size_t i = 0; i < inst.size(); i++) {
        const BatchInst &I = inst[i];
        const int nitems = (I.nstates + I.vec - 1) / I.vec;
        (*first_tile)[i] = (int)tiles.size();
        for (int f = 0; f < nitems; f += tile_items) {
            BatchTile T;
            memset(&T, 0, sizeof(T));
            T.offset = I.offset;
            T.inst = (int)i;
            T.first_item = f;
            T.nitems = std::min(tile_items, nitems - f);
            T.nstates = I.nstates;
            T.cls = I.ndim * 2 + I.rows4;
            T.nlast = I.nlast;
            T.stride0 = I.ndim >= 2 ? I.stride[0] : 0;
            T.stride1 = I.ndim >= 3 ? I.stride[1] : 0;
            T.w_move = I.w_move;
            T.w_perp = I.w_perp;
            T.w_stay = I.w_stay;
            T.gamma = I.gamma;
            tiles.push_back(T);
        }
    }
    return tiles;
}

// Autotuner result cache: (number of instances, total states / 64K) -> (block, segments per lane)
static std::mutex g_tune_mutex;
static std::map<std::pair<int, long long>, std::pair<int, int>> g_tune_cache;

static cudaError_t launch_batch(const cpmdp_batch &B, int block, const BatchArgs &args, cudaStream_t st, int *grid_out) {
    static int occ[3] = {0, 0, 0};
    const int bi = block == 128 ? 0 : (block == 256 ? 1 : 2);
    if (occ[bi] <= 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, batch_vi_kernel, block, 0);
        if (e != cudaSuccess) return e;
        occ[bi] = o > 0 ? o : 1;
    }
    // all co-resident blocks, but no more warps than tiles
    int grid = occ[bi] * B.num_sms;
    const int wpb = block / 32;
    if ((long long)grid * wpb > B.ntiles) grid = (B.ntiles + wpb - 1) / wpb;
    if (grid < 1) grid = 1;
    *grid_out = grid;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_vi_kernel, args);
}

// Tail phase buffers: allocated once per batch; without them (or past the
// tag range of the tail, 65,534 sweeps) the batched kernel runs to the end.
static void prepare_tail(cpmdp_batch &B) {
    if (B.flow_tried) return;
    B.flow_tried = true;
    const int cap = batch_flow_capacity_warps(B.num_sms);
    if (cap <= 0) return;
    bool ok = cudaMalloc(&B.d_ring, sizeof(unsigned long long) * batch_flow_ring_words(B.total_states)) == cudaSuccess &&
              cudaMalloc(&B.d_p2ctr, sizeof(unsigned long long) * batch_flow_counter_words(B.ninst)) == cudaSuccess &&
              cudaMalloc(&B.d_p2tab, sizeof(int2) * (size_t)cap) == cudaSuccess &&
              cudaMalloc(&B.d_p2hdr, sizeof(int) * 4) == cudaSuccess &&
              cudaMalloc(&B.d_p2epoch, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&B.d_p2res, sizeof(unsigned long long) * B.ninst) == cudaSuccess;
    ok = ok && cudaMemset(B.d_ring, 0xFF, sizeof(unsigned long long) * batch_flow_ring_words(B.total_states)) == cudaSuccess &&
         cudaMemset(B.d_p2epoch, 0, sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(B.d_p2hdr, 0, sizeof(int) * 4) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        void *ptrs[] = {B.d_ring, B.d_p2ctr, B.d_p2tab, B.d_p2hdr, B.d_p2epoch, B.d_p2res};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        B.d_ring = nullptr; B.d_p2ctr = nullptr; B.d_p2tab = nullptr;
        B.d_p2hdr = nullptr; B.d_p2epoch = nullptr; B.d_p2res = nullptr;
        return;
    }
    B.flow_cap_warps = cap;
}

static bool tail_enabled(const cpmdp_batch &B, int max_iter) { return B.flow_cap_warps > 0 && max_iter < 65534; }

static cudaError_t enqueue_batch(const cpmdp_batch &B, float *V, double tol, int max_iter, double timeout_s,
                                 int block, int spl, cudaStream_t st, int *grid_out, bool tail) {
    cudaError_t e;
    tail = tail && tail_enabled(B, max_iter);
    if ((e = cudaMemsetAsync(B.d_ctrl, 0, sizeof(Ctrl), st)) != cudaSuccess) return e;
    if (tail) {
        if ((e = cudaMemsetAsync(B.d_p2ctr, 0, sizeof(unsigned long long) * batch_flow_counter_words(B.ninst), st)) !=
            cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(B.d_p2res, 0, sizeof(unsigned long long) * B.ninst, st)) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(B.d_res, 0, sizeof(unsigned long long) * 3 * B.ninst, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(B.d_done, 0, sizeof(int) * B.ninst, st)) != cudaSuccess) return e;
    BatchArgs a;
    a.tiles = B.d_tiles;
    a.ntiles = B.ntiles;
    a.ninst = B.ninst;
    a.code = B.d_code;
    a.R = B.d_R;
    a.V = V;
    a.W = B.d_W;
    a.res = B.d_res;
    a.done_at = B.d_done;
    a.tol = tol;
    a.max_iter = max_iter;
    a.spl = spl;
    a.timeout_ns = (unsigned long long)(timeout_s * 1e9);
    a.ctrl = B.d_ctrl;
    a.handoff_warps = tail ? B.flow_cap_warps : 0;
    if ((e = launch_batch(B, block, a, st, grid_out)) != cudaSuccess) return e;
    if (!tail) return cudaSuccess;
    BatchFlowBuffers fb;
    fb.ring = B.d_ring;
    fb.ctr = B.d_p2ctr;
    fb.tab = B.d_p2tab;
    fb.hdr = B.d_p2hdr;
    fb.epoch = B.d_p2epoch;
    fb.p2res = B.d_p2res;
    return batch_flow_enqueue(fb, B.d_inst, B.ninst, B.d_code, B.d_R, V, B.d_W, B.d_done, B.d_res, B.d_ctrl,
                              B.total_states, B.num_sms, tol, max_iter, timeout_s, st);
}

static cpmdp_status upload_tiles(cpmdp_batch &B, int tile_items) {
    std::vector<int> first;
    std::vector<BatchTile> tiles = make_tiles(B.inst, tile_items, &first);
    for (int i = 0; i < B.ninst; i++) B.inst[(size_t)i].first_tile = first[(size_t)i];
    if (B.d_tiles) cudaFree(B.d_tiles);
    B.d_tiles = nullptr;
    CPMDP_CUDA(cudaMalloc(&B.d_tiles, tiles.size() * sizeof(BatchTile)));
    CPMDP_CUDA(cudaMemcpy(B.d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice));
    CPMDP_CUDA(cudaMemcpy(B.d_inst, B.inst.data(), B.inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
    B.ntiles = (int)tiles.size();
    B.tile_items = tile_items;
    B.tiles_host = tiles;
    return CPMDP_OK;
}

// Time 8 global sweeps for each (block, segments per lane) candidate
// on the batch itself (values from zero, scratch output), keep the fastest.
static cpmdp_status autotune(cpmdp_batch &B, cudaStream_t st) {
    const std::pair<int, long long> key(B.ninst, B.total_states >> 16);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            B.block = it->second.first;
            B.spl = it->second.second;
            return upload_tiles(B, 32 * B.spl);
        }
    }
    // (block size, segments per lane of a warp tile)
    const int cand[][2] = {{128, 1}, {128, 2}, {128, 4}, {256, 1}, {256, 4}, {512, 1}};
    const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
    // the candidates run on a temporary value tensor (the caller's V is the start)
    float *V = nullptr;
    CPMDP_CUDA(cudaMalloc(&V, sizeof(float) * B.total_states));
    struct FreeV { float *p; ~FreeV() { cudaFree(p); } } free_v{V};
    float best_ms = 1e30f;
    int best = 1;
    cudaEvent_t e0, e1;
    CPMDP_CUDA(cudaEventCreate(&e0));
    CPMDP_CUDA(cudaEventCreate(&e1));
    for (int c = 0; c < ncand; c++) {
        cpmdp_status s = upload_tiles(B, 32 * cand[c][1]);
        if (s != CPMDP_OK) return s;
        float ms_sum = 0.f;
        for (int rep = 0; rep < 3; rep++) {
            CPMDP_CUDA(cudaMemsetAsync(V, 0, sizeof(float) * B.total_states, st));
            CPMDP_CUDA(cudaEventRecord(e0, st));
            int grid = 0;
            CPMDP_CUDA(enqueue_batch(B, V, 0.0, 8, 2.0, cand[c][0], cand[c][1], st, &grid, false));
            CPMDP_CUDA(cudaEventRecord(e1, st));
            CPMDP_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_sum += ms;
        }
        if (ms_sum < best_ms) { best_ms = ms_sum; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B.block = cand[best][0];
    B.spl = cand[best][1];
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = std::make_pair(B.block, B.spl);
    }
    return upload_tiles(B, 32 * B.spl);
}

}  // namespace cpmdp

using namespace cpmdp;

extern "C" {

cpmdp_status cpmdp_batch_build(const cpmdp_problem *problems, int32_t count, int device, cpmdp_batch **out) {
    if (!out || !problems || count < 1) { set_error("batch: problems, count >= 1 and out are required"); return CPMDP_EINVAL; }
    *out = nullptr;
    if (device < 0) { set_error("batch: a CUDA device is required"); return CPMDP_EINVAL; }
    cpmdp_batch *B = new (std::nothrow) cpmdp_batch();
    if (!B) { set_error("host allocation failed"); return CPMDP_ENOMEM; }
    B->device = device;
    B->ninst = count;
    std::vector<uint8_t> codes;
    std::vector<float> rew;
    std::vector<double> rew64, instw;
    long long off = 0;
    for (int i = 0; i < count; i++) {
        const cpmdp_problem &p = problems[i];
        if (p.kind != CPMDP_GRIDWORLD || p.ndim < 1 || p.ndim > 3) {
            set_error("batch instance %d: GridWorld with 1 to 3 dimensions required", i);
            delete B;
            return CPMDP_EINVAL;
        }
        // reuse the single-instance validation and factor construction
        cpmdp_factors *f = nullptr;
        cpmdp_status st = cpmdp_build_factors(&p, -1, &f);
        if (st != CPMDP_OK) {
            char msg[400];
            snprintf(msg, sizeof(msg), "batch instance %d: %s", i, cpmdp_last_error());
            set_error("%s", msg);
            delete B;
            return st;
        }
        const Factors &F = f->f;
        BatchInst I;
        memset(&I, 0, sizeof(I));
        I.offset = off;
        I.nstates = (int)F.nstates;
        I.ndim = F.ndim;
        I.nlast = (int)F.shape[F.ndim - 1];
        for (int d = 0; d < F.ndim; d++) {
            I.stride[d] = (int)F.stride[d];
            I.shape[d] = (int)F.shape[d];
        }
        // segments of 4 states for every instance (instances start 16-byte
        // aligned and are padded to a multiple of 4 states); rows whose length
        // is a multiple of 4 also take 16-byte loads of the neighbour rows
        I.vec = 4;
        I.rows4 = I.nlast % 4 == 0 ? 1 : 0;
        I.w_move = (float)F.w_move;
        I.w_perp = (float)F.w_perp;
        I.w_stay = (float)F.w_stay;
        I.gamma = (float)F.gamma;
        instw.push_back(F.w_move);
        instw.push_back(F.w_perp);
        instw.push_back(F.w_stay);
        instw.push_back(F.gamma);
        B->inst.push_back(I);
        B->inst_actions.push_back(F.nactions);
        B->offsets.push_back(off);
        for (int64_t s = 0; s < F.nstates; s++) {
            codes.push_back((uint8_t)F.code[(size_t)s]);
            rew.push_back((float)F.reward[(size_t)s]);
            rew64.push_back(F.reward[(size_t)s]);
        }
        // pad each instance to a multiple of 4 states so every instance starts 16-byte aligned
        off += F.nstates;
        while (off % 4) { codes.push_back(0xFF); rew.push_back(0.f); rew64.push_back(0.0); off++; }
        cpmdp_free_factors(f);
    }
    B->offsets.push_back(off);
    B->total_states = off;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) { set_error("cannot select CUDA device %d", device); delete B; return CPMDP_ECUDA; }
    auto fail = [&](cudaError_t e, const char *w) {
        cuda_fail(e, w);
        free_batch_device(*B);
        delete B;
        if (prev >= 0) cudaSetDevice(prev);
        return CPMDP_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return fail(e, "attr");
    if ((e = cudaMalloc(&B->d_code, (size_t)off)) != cudaSuccess) return fail(e, "cudaMalloc code");
    if ((e = cudaMalloc(&B->d_R, (size_t)off * sizeof(float))) != cudaSuccess) return fail(e, "cudaMalloc R");
    if ((e = cudaMalloc(&B->d_W, (size_t)off * sizeof(float))) != cudaSuccess) return fail(e, "cudaMalloc W");
    if ((e = cudaMalloc(&B->d_res, sizeof(unsigned long long) * 3 * count)) != cudaSuccess) return fail(e, "cudaMalloc res");
    if ((e = cudaMalloc(&B->d_done, sizeof(int) * count)) != cudaSuccess) return fail(e, "cudaMalloc done");
    if ((e = cudaMalloc(&B->d_ctrl, sizeof(Ctrl))) != cudaSuccess) return fail(e, "cudaMalloc ctrl");
    if ((e = cudaMalloc(&B->d_inst, sizeof(BatchInst) * count)) != cudaSuccess) return fail(e, "cudaMalloc inst");
    if ((e = cudaMemcpy(B->d_code, codes.data(), (size_t)off, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "copy code");
    if ((e = cudaMemcpy(B->d_R, rew.data(), (size_t)off * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "copy R");
    // FP64 rewards and weights of the certifying sweep (cpmdp_batch_certify)
    if ((e = cudaMalloc(&B->d_R64, (size_t)off * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc R64");
    if ((e = cudaMalloc(&B->d_instw, sizeof(double) * 4 * count)) != cudaSuccess) return fail(e, "cudaMalloc instw");
    if ((e = cudaMalloc(&B->d_cert, sizeof(unsigned long long) * count)) != cudaSuccess) return fail(e, "cudaMalloc cert");
    if ((e = cudaMemcpy(B->d_R64, rew64.data(), (size_t)off * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "copy R64");
    if ((e = cudaMemcpy(B->d_instw, instw.data(), sizeof(double) * 4 * count, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "copy instw");
    B->block = 256;
    B->spl = 1;
    if (upload_tiles(*B, 32) != CPMDP_OK) { free_batch_device(*B); delete B; if (prev >= 0) cudaSetDevice(prev); return CPMDP_ECUDA; }
    if (prev >= 0) cudaSetDevice(prev);
    *out = B;
    return CPMDP_OK;
}

void cpmdp_batch_free(cpmdp_batch *B) {
    if (!B) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(B->device);
    free_batch_device(*B);
    if (prev >= 0) cudaSetDevice(prev);
    delete B;
}

cpmdp_status cpmdp_batch_info(const cpmdp_batch *B, int32_t *count, int64_t *total_states, int64_t *offsets) {
    if (!B) { set_error("batch is NULL"); return CPMDP_EINVAL; }
    if (count) *count = B->ninst;
    if (total_states) *total_states = B->total_states;
    if (offsets) memcpy(offsets, B->offsets.data(), sizeof(int64_t) * B->offsets.size());
    return CPMDP_OK;
}

cpmdp_status cpmdp_batch_value_iteration(cpmdp_batch *B, float *V, const cpmdp_solve_opts *opts,
                                         int32_t *iterations_out, double *residual_out, cpmdp_result *info,
                                         void *stream) {
    if (!B || !V) { set_error("batch and V are required"); return CPMDP_EINVAL; }
    if (((uintptr_t)V & 15u) != 0) { set_error("V must be 16-byte aligned"); return CPMDP_EINVAL; }
    SolveOpts o = resolve_opts(opts, CPMDP_F32);
    if (!(o.tol > 0) || o.max_iter < 1 || !(o.timeout_s > 0)) { set_error("invalid solve options"); return CPMDP_EINVAL; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(B->device) != cudaSuccess) { set_error("cannot select CUDA device %d", B->device); return CPMDP_ECUDA; }
    struct Restore { int p; ~Restore() { if (p >= 0) cudaSetDevice(p); } } restore{prev};
    cudaStream_t st = (cudaStream_t)stream;
    // fused = 1: every instance resident in shared memory when all fit (one
    // CTA, or a cluster of CTAs, per instance); otherwise, and for fused = 4,
    // the batched kernel with the barrier-free tail; fused = 2: the batched
    // kernel to the end
    bool resident = false;
    if (o.fused == 1) {
        cpmdp_status s = batch_resident_prepare(*B);
        if (s != CPMDP_OK) return s;
        resident = B->res_ok;
    }
    if (resident) {
        if (!B->res_planned || B->res_planned_for != B->res_est) {
            cpmdp_status s = batch_resident_plan(*B, o.tol, o.max_iter);
            if (s != CPMDP_OK) return s;
        }
    } else {
        if (!B->tuned) {
            // first solve: pick block and tile sizes on this batch
            cpmdp_status s = autotune(*B, st);
            if (s != CPMDP_OK) return s;
            B->tuned = true;
        }
        prepare_tail(*B);
    }
    // record the solve (state resets + the launches) into a CUDA graph once
    // per (V, stream, options) and replay it; if recording is refused,
    // launch directly
    const bool tail = !resident && o.fused != 2;
    const int kind = resident ? 2 : (tail ? 1 : 0);
    auto enqueue = [&](cudaStream_t s2, int *grid) -> cudaError_t {
        if (resident) {
            *grid = B->res_grid;
            return batch_resident_enqueue(*B, V, o.tol, o.max_iter, s2);
        }
        return enqueue_batch(*B, V, o.tol, o.max_iter, o.timeout_s, B->block, B->spl, s2, grid, tail);
    };
    const bool same = B->graph && B->graph_V == (void *)V && B->graph_stream == st && B->graph_tol == o.tol &&
                      B->graph_max_iter == o.max_iter && B->graph_timeout == o.timeout_s &&
                      B->graph_kind == kind;
    if (!same && !B->graph_failed) {
        if (B->graph) { cudaGraphExecDestroy(B->graph); B->graph = nullptr; }
        cudaStream_t cap;
        CPMDP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int grid = 0;
        if (e == cudaSuccess) e = enqueue(cap, &grid);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e == cudaSuccess && e2 == cudaSuccess && g) e = cudaGraphInstantiate(&B->graph, g, 0);
        else if (e == cudaSuccess) e = e2;
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            B->graph_failed = true;
            B->graph = nullptr;
        } else {
            B->grid = grid;
            B->graph_V = V;
            B->graph_stream = st;
            B->graph_tol = o.tol;
            B->graph_max_iter = o.max_iter;
            B->graph_timeout = o.timeout_s;
            B->graph_kind = kind;
        }
    }
    cudaEvent_t e0, e1;
    CPMDP_CUDA(cudaEventCreate(&e0));
    CPMDP_CUDA(cudaEventCreate(&e1));
    CPMDP_CUDA(cudaEventRecord(e0, st));
    if (B->graph && !B->graph_failed) {
        CPMDP_CUDA(cudaGraphLaunch(B->graph, st));
    } else {
        int grid = 0;
        CPMDP_CUDA(enqueue(st, &grid));
    }
    CPMDP_CUDA(cudaEventRecord(e1, st));
    Ctrl hc;
    std::vector<int> done((size_t)B->ninst);
    std::vector<unsigned long long> res((size_t)3 * B->ninst);
    std::vector<unsigned long long> p2res;
    CPMDP_CUDA(cudaMemcpyAsync(&hc, B->d_ctrl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    if (tail && tail_enabled(*B, o.max_iter)) {
        p2res.resize((size_t)B->ninst);
        CPMDP_CUDA(cudaMemcpyAsync(p2res.data(), B->d_p2res, sizeof(unsigned long long) * B->ninst,
                                   cudaMemcpyDeviceToHost, st));
    }
    CPMDP_CUDA(cudaMemcpyAsync(done.data(), B->d_done, sizeof(int) * B->ninst, cudaMemcpyDeviceToHost, st));
    CPMDP_CUDA(cudaMemcpyAsync(res.data(), B->d_res, sizeof(unsigned long long) * 3 * B->ninst, cudaMemcpyDeviceToHost, st));
    CPMDP_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (hc.status != 0) {
        set_error("a device-side wait exceeded %.3g s; results are undefined", o.timeout_s);
        return (cpmdp_status)hc.status;
    }
    int not_conv = 0;
    long long backups = 0;
    double worst = 0.0;
    for (int i = 0; i < B->ninst; i++) {
        const int n = done[(size_t)i];
        const int sweeps = n < 0 ? -n : n;
        if (n <= 0) not_conv++;
        double r = 0.0;
        // the last sweep ran in the barrier-free tail, or in the batched kernel
        if (hc.handoff && sweeps > hc.handoff_sweeps && !p2res.empty()) memcpy(&r, &p2res[(size_t)i], sizeof(double));
        else if (sweeps > 0) memcpy(&r, &res[(size_t)((sweeps - 1) % 3) * B->ninst + i], sizeof(double));
        if (iterations_out) iterations_out[i] = sweeps;
        if (resident) B->res_est[(size_t)i] = sweeps;
        if (residual_out) residual_out[i] = r;
        worst = r > worst ? r : worst;
        backups += (long long)sweeps * B->inst[(size_t)i].nstates * B->inst_actions[(size_t)i];
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = not_conv ? CPMDP_ENOCONV : CPMDP_OK;
        info->iterations = hc.iterations;
        info->rounds = (B->graph && !B->graph_failed) ? 1 : 0;   // 1 when replayed from a CUDA graph
        info->residual = worst;
        info->certified_residual = -1.0;
        info->error_bound = -1.0;
        info->backups = backups;
        info->elapsed_ms = ms;
        info->solver = resident ? CPMDP_SOLVER_BATCH_RESIDENT : CPMDP_SOLVER_BATCH;
        info->tail_from = hc.handoff ? hc.handoff_sweeps : 0;
    }
    if (not_conv) {
        set_error("%d instance(s) reached max_iter before tol", not_conv);
        return CPMDP_ENOCONV;
    }
    return CPMDP_OK;
}

cpmdp_status cpmdp_batch_certify(const cpmdp_batch *B, const float *V, uint8_t *policy_out, double *certified_out,
                                 void *stream) {
    if (!B || !V) { set_error("batch and V are required"); return CPMDP_EINVAL; }
    if (((uintptr_t)V & 15u) != 0) { set_error("V must be 16-byte aligned"); return CPMDP_EINVAL; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(B->device) != cudaSuccess) { set_error("cannot select CUDA device %d", B->device); return CPMDP_ECUDA; }
    struct Restore { int p; ~Restore() { if (p >= 0) cudaSetDevice(p); } } restore{prev};
    cudaStream_t st = (cudaStream_t)stream;
    CPMDP_CUDA(cudaMemsetAsync(B->d_cert, 0, sizeof(unsigned long long) * B->ninst, st));
    BatchCertArgs c;
    c.tiles = B->d_tiles;
    c.ntiles = B->ntiles;
    c.code = B->d_code;
    c.R64 = B->d_R64;
    c.instw = B->d_instw;
    c.V = V;
    c.pi = policy_out;
    c.cert = B->d_cert;
    const int grid = B->num_sms * 8;
    batch_certify_kernel<<<grid, 256, 0, st>>>(c);
    CPMDP_CUDA(cudaGetLastError());
    if (certified_out) {
        std::vector<unsigned long long> bits((size_t)B->ninst);
        CPMDP_CUDA(cudaMemcpyAsync(bits.data(), B->d_cert, sizeof(unsigned long long) * B->ninst,
                                   cudaMemcpyDeviceToHost, st));
        CPMDP_CUDA(cudaStreamSynchronize(st));
        memcpy(certified_out, bits.data(), sizeof(double) * B->ninst);
    } else {
        CPMDP_CUDA(cudaStreamSynchronize(st));
    }
    return CPMDP_OK;
}

}  // extern "C"
