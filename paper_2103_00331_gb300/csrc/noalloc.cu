// Value iteration for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running inside a
// memory pool or arena that owns every device byte of the process, plugin
// hosts and real-time loops that forbid allocation after start-up, or
// callers whose allocator is not reachable from the thread that solves.
// cpmdp_value_iteration_static serves them: it runs the fused FP32 GridWorld
// value iteration with all of its scratch (the second value buffer, the
// per-state move codes and the barrier / residual words) in one file-scope
// device array of fixed size, so the call itself allocates nothing. The
// caller passes the inputs and the value buffer in its own device memory.
//
// The array is kStaticScratchBytes (about 10 MiB) and exists on every GPU
// that loads this part of the library, until the process exits. Every call
// on a device uses the same array: calls that overlap on the GPU (other
// streams, other host threads) race and must be serialised by the caller.
// Each call clears the words that must start at zero before its kernels run.
//
// Host code never touches the array by name: on the first call on each
// device (with that device current) the library looks up the array's
// device address with cudaGetSymbolAddress and passes that address to the
// kernels. That first call also loads this module on the device, so make it
// before any stream capture.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.h"

namespace cpmdp {
namespace noalloc {

constexpr int kMaxStates = 1 << 21;                 // 2,097,152 states (e.g. 128^3)
constexpr size_t kCtrlBytes = 256;
constexpr size_t kStaticScratchBytes = kCtrlBytes + (size_t)kMaxStates * (1 + sizeof(float));
constexpr int kMaxDevices = 64;
constexpr int kBlock = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticCtrl {
    unsigned long long bar[2];
    unsigned long long res_slot[3];
    int status;
    int iterations;
    int converged;
    int pad;
};
static_assert(sizeof(StaticCtrl) <= kCtrlBytes, "control words exceed their reserved bytes");

struct StaticArgs {
    int ndim;
    int nstates;
    int shape[3];
    int stride[3];
    float w_move, w_perp, w_stay, gamma;
    double tol;
    int max_iter;
    unsigned long long timeout_ns;
};

// Per-state move codes, same encoding as the library's GridWorld factors:
// bit 2d + (sigma > 0) = unit move blocked by a wall or an obstacle, bit 2D
// = obstacle, bit 2D + 1 = terminal.
__global__ void static_codes_kernel(StaticArgs a, const uint8_t *__restrict__ cell, unsigned char *scratch) {
    uint8_t *code = scratch + kCtrlBytes;
    const int D = a.ndim;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nstates; s += gridDim.x * blockDim.x) {
        const uint8_t k = cell ? cell[s] : (uint8_t)CPMDP_CELL_FREE;
        const unsigned all = (1u << (2 * D)) - 1u;
        if (k > CPMDP_CELL_TERMINAL) {   // not a cell code: the solve is refused
            atomicCAS(&reinterpret_cast<StaticCtrl *>(scratch)->status, 0, (int)CPMDP_EINVAL);
            code[s] = (uint8_t)(all | (1u << (2 * D)));
            continue;
        }
        if (k == CPMDP_CELL_OBSTACLE) { code[s] = (uint8_t)(all | (1u << (2 * D))); continue; }
        if (k == CPMDP_CELL_TERMINAL) { code[s] = (uint8_t)(all | (1u << (2 * D + 1))); continue; }
        unsigned c = 0;
        int rem = s;
        for (int d = 0; d < D; d++) {
            const int x = rem / a.stride[d];
            rem -= x * a.stride[d];
            if (x == 0 || (cell && cell[s - a.stride[d]] == CPMDP_CELL_OBSTACLE)) c |= 1u << (2 * d);
            if (x == a.shape[d] - 1 || (cell && cell[s + a.stride[d]] == CPMDP_CELL_OBSTACLE)) c |= 1u << (2 * d + 1);
        }
        code[s] = (uint8_t)c;
    }
}

__device__ __forceinline__ unsigned long long static_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Counting grid barrier (bounded wait); returns the number of blocks that
// raised `flag`, or -1 when a wait ran out or another block gave up.
__device__ __forceinline__ long long static_grid_sync(StaticCtrl *c, int n, unsigned nblocks, int flag,
                                                      unsigned long long timeout_ns, unsigned long long &p0,
                                                      unsigned long long &p1) {
    __shared__ long long result;
    __syncthreads();
    if (threadIdx.x == 0) {
        result = 0;
        unsigned long long *ctr = &c->bar[n & 1];
        const unsigned long long add = 1ull | ((unsigned long long)(flag != 0) << 32);
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(ctr), "l"(add) : "memory");
        // complete at A arrivals; the counter is then A + F * 2^32 (F raised
        // flags so far on it, carries of the low half included), and while
        // blocks still arrive its low half trails A's by at most nblocks, so
        // the test on the low halves' signed difference never wraps
        const unsigned long long A = (unsigned long long)(n / 2 + 1) * nblocks;
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        const unsigned long long t0 = static_ns();
        unsigned spins = 0;
        while ((int)((unsigned)v - (unsigned)A) < 0) {
            __nanosleep(32);
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
            if ((++spins & 15u) == 0 && (int)((unsigned)v - (unsigned)A) < 0) {
                if (*(volatile int *)&c->status != 0) { result = -1; break; }
                if (static_ns() - t0 > timeout_ns) {
                    atomicCAS(&c->status, 0, (int)CPMDP_ETIMEOUT);
                    result = -1;
                    break;
                }
            }
        }
        if (result == 0) {
            const unsigned long long F = (v - A) >> 32;
            result = (long long)(F - ((n & 1) ? p1 : p0));
            if (n & 1) p1 = F;
            else p0 = F;
        }
    }
    __syncthreads();
    return result;
}

// Persistent value iteration over the codes in the static scratch; V holds
// the start on entry and the last iterate on exit.
__global__ void __launch_bounds__(kBlock) static_vi_kernel(StaticArgs a, const float *__restrict__ R, float *V,
                                                           unsigned char *scratch) {
    StaticCtrl *c = reinterpret_cast<StaticCtrl *>(scratch);
    const uint8_t *code = scratch + kCtrlBytes;
    float *W = reinterpret_cast<float *>(scratch + kCtrlBytes + kMaxStates);
    __shared__ unsigned shm[kBlock / 32];
    // the codes kernel (earlier on the stream) refused a cell code: every
    // block sees the same word and leaves before the first barrier
    if (*(volatile int *)&c->status != 0) return;
    const int D = a.ndim;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    float *cur = V, *nxt = W;
    unsigned long long p0 = 0, p1 = 0;
    int k = 0, converged = 0;
    while (k < a.max_iter) {
        float m = 0.f;
        for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nstates; s += gridDim.x * blockDim.x) {
            const unsigned cs = code[s];
            const float self = cur[s];
            float v;
            if (cs & (1u << (2 * D))) {
                v = 0.f;
            } else if (cs & (1u << (2 * D + 1))) {
                v = R[s];
            } else {
                float nb[6], P[3];
                for (int d = 0; d < 3; d++) {
                    if (d < D) {
                        nb[2 * d] = ((cs >> (2 * d)) & 1u) ? self : cur[s - a.stride[d]];
                        nb[2 * d + 1] = ((cs >> (2 * d + 1)) & 1u) ? self : cur[s + a.stride[d]];
                        P[d] = nb[2 * d] + nb[2 * d + 1];
                    } else {
                        nb[2 * d] = nb[2 * d + 1] = 0.f;
                        P[d] = 0.f;
                    }
                }
                float best = -INFINITY;
                for (int j = 0; j < 2 * D; j++) {
                    const int d = j / 2;
                    float perp = 0.f;
                    for (int e = 0; e < D; e++)
                        if (e != d) perp += P[e];
                    const float q = R[s] + a.gamma * (a.w_move * nb[j] + a.w_perp * perp + a.w_stay * self);
                    best = q > best ? q : best;
                }
                v = best;
            }
            nxt[s] = v;
            if (!(cs & (1u << (2 * D)))) m = fmaxf(m, fabsf(v - self));
        }
        // block max of the residual: non-negative floats order like their
        // bit patterns read as unsigned integers, so the warp step is one
        // integer max reduction (no FP64 instruction)
        unsigned um = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(m));
        if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = um;
        __syncthreads();
        int flag = 0;
        if (threadIdx.x == 0) {
            for (int w = 1; w < kBlock / 32; w++) um = um > shm[w] ? um : shm[w];
            const double dm = (double)__uint_as_float(um);
            if (um) atomicMax(&c->res_slot[k % 3], (unsigned long long)__double_as_longlong(dm));
            flag = !(dm < a.tol);
        }
        if (lead) c->res_slot[(k + 1) % 3] = 0ull;
        const long long open = static_grid_sync(c, k, gridDim.x, flag, a.timeout_ns, p0, p1);
        if (open < 0) return;
        k++;
        float *t = cur; cur = nxt; nxt = t;
        if (open == 0) { converged = 1; break; }
    }
    if (cur != V)
        for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nstates; s += gridDim.x * blockDim.x) V[s] = cur[s];
    if (lead) {
        c->iterations = k;
        c->converged = converged;
    }
}

static std::mutex g_setup_mutex;
static void *g_scratch_addr[kMaxDevices];

// Device address of the static scratch on the current device (looked up
// once per device).
static cpmdp_status scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return CPMDP_OK;
}

}  // namespace noalloc
}  // namespace cpmdp

using namespace cpmdp;
using namespace cpmdp::noalloc;

extern "C" cpmdp_status cpmdp_value_iteration_static(int32_t ndim, const int64_t *shape, double p_success,
                                                     double gamma, const uint8_t *cell, const float *reward,
                                                     float *V, double tol, int32_t max_iter,
                                                     int32_t *iterations_out, double *residual_out,
                                                     void *stream) {
    if (ndim < 1 || ndim > 3 || !shape) { set_error("static value iteration takes 1 <= ndim <= 3"); return CPMDP_EINVAL; }
    long long S = 1;
    for (int d = 0; d < ndim; d++) {
        if (shape[d] < 1) { set_error("shape[%d] = %lld < 1", d, (long long)shape[d]); return CPMDP_EINVAL; }
        S *= shape[d];
        if (S > kMaxStates) {
            set_error("static value iteration holds at most %d states; this grid has more", kMaxStates);
            return CPMDP_EINVAL;
        }
    }
    if (!reward || !V) { set_error("reward and V must be device pointers"); return CPMDP_EINVAL; }
    if (!(p_success >= 0.0 && p_success <= 1.0)) { set_error("p_success %g outside [0, 1]", p_success); return CPMDP_EINVAL; }
    if (!(gamma >= 0.0 && gamma <= 1.0)) { set_error("gamma %g outside [0, 1]", gamma); return CPMDP_EINVAL; }
    if (!(tol > 0.0) || max_iter < 1) { set_error("tol > 0 and max_iter >= 1 required"); return CPMDP_EINVAL; }
    int dev = 0;
    CPMDP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal %d not supported", dev); return CPMDP_EINVAL; }
    unsigned char *scratch = nullptr;
    cpmdp_status st = scratch_address(dev, &scratch);
    if (st != CPMDP_OK) return st;

    StaticArgs a;
    memset(&a, 0, sizeof(a));
    a.ndim = ndim;
    a.nstates = (int)S;
    int stride = 1;
    for (int d = ndim - 1; d >= 0; d--) {
        a.shape[d] = (int)shape[d];
        a.stride[d] = stride;
        stride *= (int)shape[d];
    }
    a.w_move = (float)p_success;
    a.w_perp = ndim >= 2 ? (float)((1.0 - p_success) / (2.0 * (ndim - 1))) : 0.f;
    a.w_stay = ndim == 1 ? (float)(1.0 - p_success) : 0.f;
    a.gamma = (float)gamma;
    a.tol = tol;
    a.max_iter = max_iter;
    a.timeout_ns = 2000000000ull;

    cudaStream_t s = (cudaStream_t)stream;
    CPMDP_CUDA(cudaMemsetAsync(scratch, 0, kCtrlBytes, s));
    int nsm = 0, occ = 0;
    CPMDP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CPMDP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, static_vi_kernel, kBlock, 0));
    int grid = (int)((S + kBlock - 1) / kBlock);
    if (grid > occ * nsm) grid = occ * nsm;
    if (grid < 1) grid = 1;
    static_codes_kernel<<<grid, kBlock, 0, s>>>(a, cell, scratch);
    CPMDP_CUDA(cudaGetLastError());
    void *args[] = {(void *)&a, (void *)&reward, (void *)&V, (void *)&scratch};
    CPMDP_CUDA(cudaLaunchCooperativeKernel((const void *)static_vi_kernel, dim3(grid), dim3(kBlock), args, 0, s));
    StaticCtrl h;
    CPMDP_CUDA(cudaMemcpyAsync(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s));
    CPMDP_CUDA(cudaStreamSynchronize(s));
    if (h.status == CPMDP_EINVAL) {
        set_error("cell codes must be 0 (free), 1 (obstacle) or 2 (terminal); V is unchanged");
        return CPMDP_EINVAL;
    }
    if (h.status != 0) {
        set_error("a device-side wait exceeded 2 s; V is undefined");
        return (cpmdp_status)h.status;
    }
    const int last = h.iterations > 0 ? (h.iterations - 1) % 3 : 0;
    double res = 0.0;
    memcpy(&res, &h.res_slot[last], sizeof(res));
    if (iterations_out) *iterations_out = h.iterations;
    if (residual_out) *residual_out = res;
    if (!h.converged) {
        set_error("not converged: %d sweeps, residual %.3g", h.iterations, res);
        return CPMDP_ENOCONV;
    }
    return CPMDP_OK;
}
