// The tail of a batched value-iteration solve, without a grid barrier.
//
// The batched kernel (batch.cu) ends every sweep in a grid barrier. Late in
// a solve few instances still run (4096 instances: after sweep 399 of 1826
// fewer than 272k states), and each sweep then costs the barrier and one
// load round trip while moving a few states. Once the instances still
// running fit one co-resident grid at one warp per 32 segments of 4 states,
// the batched kernel stops and this phase takes over:
//
// * batch_flow_setup (one block) applies the stopping decisions the
//   batched kernel left pending, and lays the running instances' segments
//   out over warps (warp table: instance, first segment).
// * batch_flow_kernel runs every instance on its own, as the barrier-free
//   solver does for one grid (flow_solve.cu): values in registers, the
//   neighbours' values through four rings of sweep-tagged 64-bit words over
//   the packed layout, per-instance arrival counters, the stopping rule
//   settled three sweeps late, the result read back from the ring. An
//   instance's warps stop when it stops; no warp waits for another
//   instance. Row neighbours are read one state at a time, so rows of any
//   length work (a 4-state segment may span two rows, as in the batched
//   kernel).
//
// The per-state arithmetic is vi_state with the batch's float weights, as
// in the batched kernel, so sweep counts and values are the same as if the
// batched kernel had run to the end.
#include <cuda_runtime.h>
#include <stdint.h>

#include "banded_common.cuh"
#include "batch_flow.h"
#include "batch_internal.h"
#include "flow_common.cuh"

namespace cpmdp {

using namespace tw;

namespace {

constexpr int kWarpsPerBlock = kBatchFlowWarpsPerBlock;

struct P2Args {
    const BatchInst *inst;
    const uint8_t *code;
    const float *R;
    float *V;                  // caller's packed values: start (even phase-1 sweeps) and result
    const float *W;            // the batched kernel's second buffer (odd phase-1 sweeps)
    u64 *ring[kRing];          // tagged words over the packed layout
    u64 *ctr;                  // [ninst][kSlots] arrival counters (count | flags << 32)
    const int2 *tab;           // per warp: instance, first segment
    const int *hdr;            // [0] warps in use, [1] epoch, [2] phase-1 sweeps
    int *done_at;              // per instance: sweeps done (negative: max_iter reached)
    u64 *p2res;                // per instance: bits of the last sweep's residual
    unsigned tol_bits;
    int max_iter;
    u64 timeout_ns;
    Ctrl *ctrl;
};

template <int D>
__device__ void run_instance(const P2Args &a, const BatchInst &I, int inst, int first_seg, unsigned *prevhi) {
    constexpr int NRR = 2 * (D - 1);
    constexpr int NR = NRR > 0 ? NRR : 1;
    constexpr unsigned OBST = 1u << (2 * D), TERM = 1u << (2 * D + 1);
    const int lane = threadIdx.x & 31;
    const int nseg = (I.nstates + 3) / 4;
    const unsigned nw = (unsigned)((nseg + 31) / 32);
    const int seg = first_seg + lane;
    const bool valid = seg < nseg;
    const int s0 = 4 * seg;
    const long long g0 = I.offset + s0;
    const int k1 = a.hdr[2];
    const unsigned epoch = (unsigned)a.hdr[1];
    const unsigned jmax = (unsigned)(a.max_iter - k1);
    const float wm = I.w_move, wp = I.w_perp, wst = I.w_stay, g = I.gamma;
    int stride[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) stride[j] = j < NRR ? I.stride[j / 2] : 0;

    unsigned code = 0;
    float R[4] = {0.f, 0.f, 0.f, 0.f}, cur[4] = {0.f, 0.f, 0.f, 0.f};
    unsigned need = 0;   // bit 4 jr + k: row neighbour jr of state k; bits 4 NRR, 4 NRR + 1: halos
    constexpr int HM = 4 * NRR, HP = 4 * NRR + 1;
    if (valid) {
        code = *reinterpret_cast<const unsigned *>(a.code + g0);
        const float4 r = *reinterpret_cast<const float4 *>(a.R + g0);
        const float4 v = *reinterpret_cast<const float4 *>(((k1 & 1) ? a.W : a.V) + g0);
        R[0] = r.x; R[1] = r.y; R[2] = r.z; R[3] = r.w;
        cur[0] = v.x; cur[1] = v.y; cur[2] = v.z; cur[3] = v.w;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const unsigned c = (code >> (8 * k)) & 0xFFu;
            if (c & (OBST | TERM)) continue;
#pragma unroll
            for (int jr = 0; jr < NRR; jr++)
                if (!((c >> jr) & 1u)) need |= 1u << (4 * jr + k);
            if (k == 0 && !((c >> NRR) & 1u) && lane == 0) need |= 1u << HM;
            if (k == 3 && !((c >> (NRR + 1)) & 1u) && lane == 31) need |= 1u << HP;
        }
    }
    auto tag_of = [&](unsigned j) -> unsigned { return (epoch << 16) | j; };
    auto publish = [&](unsigned j, const float (&v)[4]) {
        if (!valid) return;
        u64 *out = a.ring[j % (unsigned)kRing] + g0;
        const unsigned tg = tag_of(j);
        st_rlx2(out, word(v[0], tg), word(v[1], tg));
        st_rlx2(out + 2, word(v[2], tg), word(v[3], tg));
    };
    auto own_values = [&](unsigned j, float (&v)[4]) {
        if (!valid) return;
        const u64 *in = a.ring[j % (unsigned)kRing] + g0;
        u64 x, y, z, w;
        ld_rlx2(in, x, y);
        ld_rlx2(in + 2, z, w);
        v[0] = val(x); v[1] = val(y); v[2] = val(z); v[3] = val(w);
    };
    // arrival counter of this instance's slot for sweep i
    u64 *ictr = a.ctr + (size_t)inst * kSlots;
    unsigned na = 0, nchk = 0;
    auto settle = [&](u64 v, unsigned i) -> int {
        // lane 0 holds the counter; the others follow its decision
        int r = -1;
        if (lane == 0) {
            const u64 A = ((u64)(i / kSlots) + 1ull) * nw;
            if ((unsigned)v == (unsigned)A) {
                const unsigned F = (unsigned)((v - A) >> 32);
                r = (int)(F - prevhi[i % kSlots]);
                prevhi[i % kSlots] = F;
            }
        }
        return __shfl_sync(FULL, r, 0);
    };
    auto peek = [&](unsigned i) -> u64 { return lane == 0 ? ld_rlx(ictr + i % kSlots) : 0ull; };
    auto check = [&](u64 pk) -> int {
        int r = settle(pk, nchk);
        u64 t0 = 0;
        unsigned spins = 0;
        while (r < 0) {
            if ((++spins & 15u) == 0 && give_up(a.ctrl, t0, a.timeout_ns)) return -2;
            __nanosleep(32);
            r = settle(peek(nchk), nchk);
        }
        nchk++;
        return r;
    };

    publish(0, cur);
    float rh[kLag];
#pragma unroll
    for (int i = 0; i < kLag; i++) rh[i] = 0.f;
    float res[4];
    float rres = 0.f;
    int sweeps = 0;     // sweeps of this phase whose result is returned
    bool conv = false;
    unsigned j = 0;
    for (;;) {
        const u64 pk = j >= (unsigned)kLag ? peek(nchk) : 0ull;
        // neighbour words of sweep j
        const unsigned tg = tag_of(j);
        const u64 *in = a.ring[j % (unsigned)kRing];
        u64 w[NR][4];
        u64 wl = 0, wr = 0;
#pragma unroll
        for (int jr = 0; jr < NR; jr++)
#pragma unroll
            for (int k = 0; k < 4; k++) w[jr][k] = 0;
        __nanosleep(100);
        unsigned pend = need;
        u64 t0 = 0;
        unsigned spins = 0;
        for (;;) {
#pragma unroll
            for (int jr = 0; jr < NRR; jr++)
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if ((pend >> (4 * jr + k)) & 1u)
                        w[jr][k] = ld_rlx(in + g0 + k + ((jr & 1) ? stride[jr] : -stride[jr]));
            if ((pend >> HM) & 1u) wl = ld_rlx(in + g0 - 1);
            if ((pend >> HP) & 1u) wr = ld_rlx(in + g0 + 4);
            unsigned still = 0;
#pragma unroll
            for (int jr = 0; jr < NRR; jr++)
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (((pend >> (4 * jr + k)) & 1u) && !has(w[jr][k], tg)) still |= 1u << (4 * jr + k);
            if (((pend >> HM) & 1u) && !has(wl, tg)) still |= 1u << HM;
            if (((pend >> HP) & 1u) && !has(wr, tg)) still |= 1u << HP;
            pend = still;
            if (!__any_sync(FULL, pend != 0u)) break;
            if ((++spins & 15u) == 0 && give_up(a.ctrl, t0, a.timeout_ns)) return;
        }
        const float sl = __shfl_up_sync(FULL, cur[3], 1);
        const float sr = __shfl_down_sync(FULL, cur[0], 1);
        const float hl = lane == 0 ? val(wl) : sl;
        const float hr = lane == 31 ? val(wr) : sr;
        // backups (neighbours of blocked moves replaced by V(s), as Segment::neighbours)
        float nxt[4];
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const unsigned c = (code >> (8 * k)) & 0xFFu;
            float nb[2 * D];
#pragma unroll
            for (int jr = 0; jr < NRR; jr++) nb[jr] = ((c >> jr) & 1u) ? cur[k] : val(w[jr][k]);
            const float left = (k == 0) ? hl : cur[k > 0 ? k - 1 : 0];
            const float right = (k == 3) ? hr : cur[k < 3 ? k + 1 : 0];
            nb[NRR] = ((c >> NRR) & 1u) ? cur[k] : left;
            nb[NRR + 1] = ((c >> (NRR + 1)) & 1u) ? cur[k] : right;
            int arg;
            const float v = vi_state<float, D, false>(cur[k], nb, c, R[k], wm, wp, wst, g, arg);
            nxt[k] = v;
            if (valid && !(c & OBST)) {
                const float dv = abs_diff(v, cur[k]);
                r = dv > r ? dv : r;
            }
        }
        if (j >= (unsigned)kLag) {
            const int nf = check(pk);
            if (nf == -2) return;
            if (nf == 0) {   // sweep j - kLag met tol: its result is V_{j-kLag+1}
#pragma unroll
                for (int k = 0; k < 4; k++) res[k] = cur[k];
                own_values(j - kLag + 1, res);
                rres = rh[kLag - 1];
                sweeps = (int)j - kLag + 1;
                conv = true;
                break;
            }
        }
        publish(j + 1, nxt);
        const bool open = warp_open(r, a.tol_bits);
        if (lane == 0) red_add_rlx(ictr + na % kSlots, 1ull | ((u64)(open ? 1u : 0u) << 32));
        na++;
#pragma unroll
        for (int k = 0; k < 4; k++) cur[k] = nxt[k];
#pragma unroll
        for (int i = kLag - 1; i > 0; i--) rh[i] = rh[i - 1];
        rh[0] = r;
        j++;
        if (j == jmax) {
            // max_iter: settle the unchecked sweeps in order
#pragma unroll
            for (int k = 0; k < 4; k++) res[k] = cur[k];
            rres = rh[0];
            sweeps = (int)j;
            while (nchk < na) {
                const unsigned sweep = nchk;   // arrival i is sweep i of this phase
                const int nf = check(peek(nchk));
                if (nf == -2) return;
                if (nf == 0 && !conv) {
                    conv = true;
                    sweeps = (int)sweep + 1;
                    if (sweep + 1 != j) own_values(sweep + 1, res);
                    const unsigned back = j - 1 - sweep;
#pragma unroll
                    for (int i = 0; i < kLag; i++)
                        if ((unsigned)i == back) rres = rh[i];
                }
            }
            break;
        }
    }
    if (valid) *reinterpret_cast<float4 *>(a.V + g0) = make_float4(res[0], res[1], res[2], res[3]);
    const unsigned long long rb = warp_res_bits(valid ? rres : 0.f);
    if (lane == 0) {
        const int total = k1 + sweeps;
        a.done_at[inst] = conv ? total : -total;
        if (rb) atomicMax(a.p2res + inst, rb);
        atomicMax(&a.ctrl->iterations, total);
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock, 1) batch_flow_kernel(P2Args a) {
    __shared__ unsigned prevhi_all[kWarpsPerBlock][kSlots];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kWarpsPerBlock + wib;
    if (gw >= a.hdr[0]) return;
    if (lane < kSlots) prevhi_all[wib][lane] = 0u;
    __syncwarp();
    const int2 t = a.tab[gw];
    const BatchInst I = a.inst[t.x];
    switch (I.ndim) {
        case 1: run_instance<1>(a, I, t.x, t.y, prevhi_all[wib]); break;
        case 2: run_instance<2>(a, I, t.x, t.y, prevhi_all[wib]); break;
        default: run_instance<3>(a, I, t.x, t.y, prevhi_all[wib]); break;
    }
}

// One block of 1024 threads. Runs only after a hand-off (ctrl->handoff):
// instances whose last residual is below tol, or that reached max_iter,
// stop here as the batched kernel would have stopped them; the others get
// ceil(segments / 32) warps each, laid out in instance order.
__global__ void __launch_bounds__(1024) batch_flow_setup(const BatchInst *inst, int ninst, int *done_at,
                                                         const u64 *res, Ctrl *ctrl, int2 *tab, int *hdr,
                                                         unsigned *epoch, double tol, int max_iter, int cap_warps,
                                                         float *V, const float *W) {
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    if (!*(volatile int *)&ctrl->handoff) {
        if (tid == 0) { hdr[0] = 0; hdr[3] = 0; }
        return;
    }
    const int k1 = ctrl->handoff_sweeps;
    const int chunk = (ninst + 1023) / 1024;
    const int i0 = tid * chunk, i1 = min(ninst, i0 + chunk);
    int sum = 0;
    for (int i = i0; i < i1; i++) {
        if (done_at[i] != 0) continue;
        const u64 rb = res[(size_t)((k1 - 1) % 3) * ninst + i];
        if (below_tol(rb, tol)) { done_at[i] = k1; continue; }
        if (k1 >= max_iter) { done_at[i] = -k1; continue; }
        sum += ((inst[i].nstates + 3) / 4 + 31) / 32;
    }
    part[tid] = sum;
    __syncthreads();
    // exclusive prefix sum over the 1024 partial counts
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    const int total = part[1023];
    int base = part[tid] - sum;
    if (total > cap_warps) {   // cannot happen: the batched kernel hands off only when they fit
        if (tid == 0) { atomicCAS(&ctrl->status, 0, (int)CPMDP_EINVAL); hdr[0] = 0; }
        return;
    }
    for (int i = i0; i < i1; i++) {
        if (done_at[i] != 0) continue;
        const int nw = ((inst[i].nstates + 3) / 4 + 31) / 32;
        for (int w = 0; w < nw; w++) tab[base + w] = make_int2(i, 32 * w);
        base += nw;
    }
    // instances stopped here after an odd number of sweeps: their values
    // are in W (the batched kernel copies those it stopped itself)
    if (k1 & 1) {
        for (int i = 0; i < ninst; i++) {
            const int n = done_at[i];
            if (n != k1 && n != -k1) continue;
            const long long o = inst[i].offset;
            for (int t = tid; t < inst[i].nstates; t += blockDim.x) V[o + t] = W[o + t];
        }
    }
    if (tid == 0) {
        unsigned e = *epoch;
        hdr[3] = e >= 0xFFFEu ? 1 : 0;   // tags would wrap: clear the rings first
        if (e >= 0xFFFEu) e = 0;
        *epoch = e + 1;
        hdr[0] = total;
        hdr[1] = (int)e;
        hdr[2] = k1;
    }
}

// Clears the rings to the unused tag 0xFFFFFFFF when the epoch wrapped.
__global__ void batch_flow_clear(u64 *ring, long long nwords, const int *hdr) {
    if (!*(volatile const int *)&hdr[3]) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (long long)gridDim.x * blockDim.x)
        ring[i] = ~0ull;
}

}  // namespace

int batch_flow_capacity_warps(int num_sms) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, batch_flow_kernel, 32 * kWarpsPerBlock, 0) != cudaSuccess ||
        o < 1)
        return 0;
    return num_sms * kWarpsPerBlock;
}

size_t batch_flow_ring_words(long long total_states) { return (size_t)kRing * (size_t)total_states; }
size_t batch_flow_counter_words(int ninst) { return (size_t)ninst * kSlots; }

cudaError_t batch_flow_enqueue(const BatchFlowBuffers &b, const BatchInst *inst, int ninst, const uint8_t *code,
                               const float *R, float *V, const float *W, int *done_at, const unsigned long long *res,
                               Ctrl *ctrl, long long total_states, int num_sms, double tol, int max_iter,
                               double timeout_s, cudaStream_t st) {
    cudaError_t e;
    const int cap = num_sms * kWarpsPerBlock;
    batch_flow_setup<<<1, 1024, 0, st>>>(inst, ninst, done_at, res, ctrl, b.tab, b.hdr, b.epoch, tol, max_iter, cap,
                                         V, W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batch_flow_clear<<<num_sms * 4, 256, 0, st>>>(b.ring, (long long)batch_flow_ring_words(total_states), b.hdr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    P2Args a;
    a.inst = inst;
    a.code = code;
    a.R = R;
    a.V = V;
    a.W = W;
    for (int i = 0; i < kRing; i++) a.ring[i] = b.ring + (size_t)i * total_states;
    a.ctr = b.ctr;
    a.tab = b.tab;
    a.hdr = b.hdr;
    a.done_at = done_at;
    a.p2res = b.p2res;
    a.tol_bits = float_ceil_bits(tol);
    a.max_iter = max_iter;
    a.timeout_ns = (u64)(timeout_s * 1e9);
    a.ctrl = ctrl;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(num_sms);
    cfg.blockDim = dim3(32 * kWarpsPerBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_flow_kernel, a);
}

}  // namespace cpmdp
