// One fused backup sweep of a large 3-D GridWorld (Eq. 1 for every state:
// expectation over the CP terms, + R, x gamma, max over actions, residual)
// that reads each value from DRAM about once.
//
// The grid-stride sweep (banded.cu) reads the two z-neighbour rows of a
// segment from wherever they are; once the value tensor is larger than L2
// (512^3 floats: 512 MB), part of those reads come from DRAM a second time
// (traffic 1.26 x the algorithmic bytes). Here a block owns a tile of
// 8 rows x 128 states of the (y, x) plane and marches along z through a
// chunk of planes. A thread keeps its 4-state segment of planes z-1, z and
// z+1 in registers (the z-neighbours), fetches plane z+2 one step ahead,
// takes the x-neighbours from the adjacent lanes by shuffle and the
// y-neighbour rows (written to L1 by the adjacent warps of the block, or to
// L2 by the adjacent tile) a step ahead too. Rewards and codes stream in
// one step ahead. DRAM then sees V, R, the codes and V' about once, plus
// two planes per chunk.
//
// The per-state arithmetic is vi_state, as in every other banded kernel,
// so the result equals the grid-stride sweep's bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "banded_common.cuh"
#include "march.h"

namespace cpmdp {

namespace {

constexpr int kTileX = 128;   // states of a row per tile (32 lanes x 4)
constexpr int kTileY = 8;     // rows per tile (one warp each)
constexpr int kChunk = 32;    // planes per block

struct MarchArgs {
    BandArgs a;
    int nz, ny, nx;
    int xtiles, ytiles;
};

__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ unsigned ldc4(const void *code, size_t s) {
    return __ldg(reinterpret_cast<const unsigned *>(static_cast<const uint8_t *>(code) + s));
}
__device__ __forceinline__ float comp(const float4 &v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }

// Rewards of a segment in the working precision.
template <typename TA> struct Rew4;
template <> struct Rew4<float> {
    float r[4];
    __device__ __forceinline__ void load(const BandArgs &a, size_t s) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(a.R32 + s));
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    }
};
template <> struct Rew4<double> {
    double r[4];
    __device__ __forceinline__ void load(const BandArgs &a, size_t s) {
        const double2 u = __ldg(reinterpret_cast<const double2 *>(a.R64 + s));
        const double2 v = __ldg(reinterpret_cast<const double2 *>(a.R64 + s + 2));
        r[0] = u.x; r[1] = u.y; r[2] = v.x; r[3] = v.y;
    }
};

template <typename TA, bool WITH_PI>
__global__ void __launch_bounds__(256) march_kernel(MarchArgs m, const float *__restrict__ V, float *__restrict__ W,
                                                    uint8_t *__restrict__ pi, unsigned long long *res_out,
                                                    const int *stop) {
    __shared__ unsigned shm[64];
    if (stop && *(volatile const int *)stop) return;   // value iteration: a sweep after the stopping one
    constexpr int D = 3;
    constexpr unsigned OBST = 1u << (2 * D), TERM = 1u << (2 * D + 1);
    const BandArgs &a = m.a;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    int b = blockIdx.x;
    const int xt = b % m.xtiles;
    b /= m.xtiles;
    const int yt = b % m.ytiles;
    const int zc = b / m.ytiles;
    const int x0 = xt * kTileX + lane * 4;
    const int y = yt * kTileY + wy;
    const int z0 = zc * kChunk;
    const int z1 = min(m.nz, z0 + kChunk);
    const bool act = x0 < m.nx && y < m.ny;
    const size_t plane = (size_t)m.ny * m.nx;
    const size_t row = (size_t)y * m.nx + x0;
    const bool has_ym = y > 0, has_yp = y + 1 < m.ny;
    // lanes 0 and 31 take their halo from memory (the other lanes' halo is
    // the adjacent lane's; past the row end the move is blocked and unused)
    const bool right_mem = act && x0 + 4 < m.nx && (lane == 31);
    const bool left_mem = act && x0 > 0 && lane == 0;

    TA wm, wp, wst, g;
    weights<TA>(a, wm, wp, wst, g);

    float4 vm = make_float4(0.f, 0.f, 0.f, 0.f), vc = vm, vp = vm, vpp = vm, ym = vm, yp = vm, ymn = vm, ypn = vm;
    unsigned cc = 0, cn = 0;
    Rew4<TA> rc, rn;
#pragma unroll
    for (int k = 0; k < 4; k++) rc.r[k] = rn.r[k] = 0;
    if (act) {
        const size_t s = (size_t)z0 * plane + row;
        vc = ld4(V + s);
        vm = z0 > 0 ? ld4(V + s - plane) : vc;
        vp = z0 + 1 < m.nz ? ld4(V + s + plane) : vc;
        ym = has_ym ? ld4(V + s - m.nx) : vc;
        yp = has_yp ? ld4(V + s + m.nx) : vc;
        cc = ldc4(a.code, s);
        rc.load(a, s);
    }
    TA res = 0;
    for (int z = z0; z < z1; z++) {
        const size_t s = (size_t)z * plane + row;
        const bool next = z + 1 < z1;
        // one step ahead: plane z+2 (the next step's upper neighbour), the
        // next plane's y-neighbour rows and codes
        if (act && next) {
            if (z + 2 < m.nz) vpp = ld4(V + s + 2 * plane);
            ymn = has_ym ? ld4(V + s + plane - m.nx) : vp;
            ypn = has_yp ? ld4(V + s + plane + m.nx) : vp;
            cn = ldc4(a.code, s + plane);
            rn.load(a, s + plane);
        }
        float hl = __shfl_up_sync(0xFFFFFFFFu, vc.w, 1);
        float hr = __shfl_down_sync(0xFFFFFFFFu, vc.x, 1);
        if (left_mem) hl = __ldg(V + s - 1);
        if (right_mem) hr = __ldg(V + s + 4);
        if (act) {
            TA out[4];
            unsigned pol = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned c = (cc >> (8 * k)) & 0xFFu;
                const TA self = (TA)comp(vc, k);
                TA nb[2 * D];
                nb[0] = (c & 1u) ? self : (TA)comp(vm, k);
                nb[1] = (c & 2u) ? self : (TA)comp(vp, k);
                nb[2] = (c & 4u) ? self : (TA)comp(ym, k);
                nb[3] = (c & 8u) ? self : (TA)comp(yp, k);
                const TA left = (k == 0) ? (TA)hl : (TA)comp(vc, k > 0 ? k - 1 : 0);
                const TA right = (k == 3) ? (TA)hr : (TA)comp(vc, k < 3 ? k + 1 : 0);
                nb[4] = (c & 16u) ? self : left;
                nb[5] = (c & 32u) ? self : right;
                int arg;
                const TA v = vi_state<TA, D, WITH_PI>(self, nb, c, rc.r[k], wm, wp, wst, g, arg);
                out[k] = v;
                pol |= ((c & (OBST | TERM)) ? 255u : (unsigned)arg) << (8 * k);
                if (!(c & OBST)) {
                    const TA dv = abs_diff(v, self);
                    res = dv > res ? dv : res;
                }
            }
            if (WITH_PI) *reinterpret_cast<unsigned *>(pi + s) = pol;
            if (W)
                *reinterpret_cast<float4 *>(W + s) =
                    make_float4((float)out[0], (float)out[1], (float)out[2], (float)out[3]);
        }
        vm = vc;
        vc = vp;
        vp = vpp;
        ym = ymn;
        yp = ypn;
        cc = cn;
        rc = rn;
    }
    if (res_out) {
        const unsigned long long mb = block_max_bits(res, shm);
        if (threadIdx.x == 0 && mb) atomicMax(res_out, mb);
    }
}

static MarchArgs march_args(const Factors &F) {
    MarchArgs m;
    m.a = make_band_args(F);
    m.nz = (int)F.shape[0];
    m.ny = (int)F.shape[1];
    m.nx = (int)F.shape[2];
    m.xtiles = (m.nx + kTileX - 1) / kTileX;
    m.ytiles = (m.ny + kTileY - 1) / kTileY;
    return m;
}

// Stopping rule of the graph-driven value iteration: one thread reads the
// sweep's residual, clears its slot, counts the sweep (and its backups),
// writes the trace entry and raises stop once the residual is below tol or
// max_iter sweeps are done; later sweeps of the graph then return at once.
__global__ void march_check_kernel(Ctrl *c, double tol, int max_iter, long long backups_per_sweep, double *trace) {
    if (c->plain_stop) return;
    double r;
    memcpy(&r, &c->res_slot[0], sizeof(r));
    c->res_slot[0] = 0ull;
    if (trace) trace[c->iterations] = r;
    c->iterations += 1;
    c->backups += backups_per_sweep;
    c->last_residual = r;
    if (r < tol) {
        c->converged = 1;
        c->plain_stop = 1;
    } else if (c->iterations >= max_iter) {
        c->plain_stop = 1;
    }
}

template <typename TA, bool WITH_PI>
cudaError_t launch_march(const Factors &F, const float *V, float *W, uint8_t *pi, unsigned long long *res,
                         cudaStream_t st) {
    MarchArgs m;
    m.a = make_band_args(F);
    m.nz = (int)F.shape[0];
    m.ny = (int)F.shape[1];
    m.nx = (int)F.shape[2];
    m.xtiles = (m.nx + kTileX - 1) / kTileX;
    m.ytiles = (m.ny + kTileY - 1) / kTileY;
    const long long blocks = (long long)m.xtiles * m.ytiles * ((m.nz + kChunk - 1) / kChunk);
    if (blocks < 1 || blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    march_kernel<TA, WITH_PI><<<(unsigned)blocks, 256, 0, st>>>(m, V, W, pi, res, nullptr);
    return cudaGetLastError();
}

constexpr int kMarchChunkSweeps = 16;   // sweeps per recorded graph (even: it starts and ends in V)

}  // namespace

bool march_eligible(const Factors &F, const void *V, const void *W, const void *pi) {
    // 3-D, rows a multiple of 4 states, aligned buffers, and large enough
    // that the sweep is bound by DRAM rather than by L2 or its launch
    return F.ndim == 3 && F.shape[2] % 4 == 0 && F.nstates >= kMarchMinStates && F.shape[1] * F.shape[2] < (1ll << 31) &&
           ((uintptr_t)V & 15u) == 0 && ((uintptr_t)W & 15u) == 0 && ((uintptr_t)pi & 3u) == 0;
}

// FP32 value iteration of a large 3-D grid: kMarchChunkSweeps sweeps of
// march_kernel (V -> scratch -> V ...), each followed by march_check_kernel,
// recorded once into a CUDA graph (per V, tol, max_iter, trace) and replayed
// until the device raised stop; the host reads the control block once per
// graph. The result is in V after an even number of sweeps, in the scratch
// buffer (copied to V) after an odd number. Same per-state arithmetic and
// stopping sweep as the grid-barrier solver.
cudaError_t march_solve(const Factors &F, float *V, double tol, int max_iter, double *trace, cudaStream_t st) {
    Factors &M = const_cast<Factors &>(F);
    float *W = (float *)F.d_scratch;
    const MarchArgs m = march_args(F);
    const long long blocks = (long long)m.xtiles * m.ytiles * ((m.nz + kChunk - 1) / kChunk);
    if (blocks < 1 || blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    const int *stop = &F.d_ctrl->plain_stop;
    const long long bps = (long long)F.nstates * F.nactions;
    const bool same = M.march_graph && M.march_graph_V == (void *)V && M.march_graph_tol == tol &&
                      M.march_graph_max_iter == max_iter && M.march_graph_trace == (void *)trace;
    cudaError_t e = cudaSuccess;
    if (!same) {
        if (M.march_graph) { cudaGraphExecDestroy(M.march_graph); M.march_graph = nullptr; }
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < kMarchChunkSweeps && e == cudaSuccess; k++) {
            const float *cur = (k & 1) ? W : V;
            float *nxt = (k & 1) ? V : W;
            march_kernel<float, false><<<(unsigned)blocks, 256, 0, cap>>>(m, cur, nxt, nullptr, rb, stop);
            march_check_kernel<<<1, 1, 0, cap>>>(F.d_ctrl, tol, max_iter, bps, trace);
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&M.march_graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) { M.march_graph = nullptr; return e; }
        M.march_graph_V = (void *)V;
        M.march_graph_tol = tol;
        M.march_graph_max_iter = max_iter;
        M.march_graph_trace = (void *)trace;
    }
    // the control block was cleared by the caller
    if (trace && (e = cudaMemsetAsync(trace, 0, (size_t)max_iter * sizeof(double), st)) != cudaSuccess) return e;
    Ctrl h;
    for (;;) {
        if ((e = cudaGraphLaunch(M.march_graph, st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&h, F.d_ctrl, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (h.plain_stop) break;
    }
    if (h.iterations & 1) return cudaMemcpyAsync(V, W, sizeof(float) * F.nstates, cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
}

cudaError_t march_sweep(const Factors &F, const float *V, float *W, uint8_t *pi, unsigned long long *res, bool fp64,
                        cudaStream_t st) {
    if (fp64) {
        return pi ? launch_march<double, true>(F, V, W, pi, res, st) : launch_march<double, false>(F, V, W, pi, res, st);
    }
    return pi ? launch_march<float, true>(F, V, W, pi, res, st) : launch_march<float, false>(F, V, W, pi, res, st);
}

}  // namespace cpmdp
