// C ABI entry points of libcpmdp: problem validation, CP factor
// construction (host), device upload, and dispatch to the solvers.
#include <cuda_runtime.h>
#include <stddef.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>

#include "internal.h"
#include "flow.h"

namespace cpmdp {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

cpmdp_status cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return CPMDP_ECUDA;
}

// Makes F.device current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

SolveOpts resolve_opts(const cpmdp_solve_opts *o, cpmdp_precision prec) {
    cpmdp_solve_opts d;
    cpmdp_default_opts(&d);
    if (!o) o = &d;
    SolveOpts r;
    r.tol = o->tol;
    r.max_iter = o->max_iter;
    r.certify = o->certify;
    r.fused = o->fused;
    r.eval_tol = o->eval_tol > 0 ? o->eval_tol : (prec == CPMDP_F64 ? 1e-10 : o->tol);
    r.max_eval_iter = o->max_eval_iter;
    r.max_rounds = o->max_rounds;
    r.timeout_s = o->timeout_s;
    r.trace = o->trace;
    r.partial_eval = o->partial_eval;
    r.inject_stall = o->inject_stall;
    return r;
}

// One stream-ordered memory pool per device for the factors' allocation:
// memory freed by one factors object is reused by the next build without a
// cudaMalloc, and a free does not synchronise the device (the pool keeps
// what it holds: release threshold at its maximum). Created on first use.
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[64];

static cudaError_t arena_pool(int device, cudaMemPool_t *out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[device]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) { cudaMemPoolDestroy(pool); return e; }
        g_pools[device] = pool;
    }
    *out = g_pools[device];
    return cudaSuccess;
}

static void free_device(Factors &F) {
    // the arena holds d_code, d_R32, d_R64, d_cell, d_scratch, d_ctrl and,
    // for shapes the barrier-free solver takes, d_flow
    void *ptrs[] = {F.d_arena, F.d_q, F.d_U32, F.d_U64, F.d_Ubf, F.d_lam32, F.d_lam64, F.d_dense_work,
                    F.d_Vd, F.d_RB, F.d_T, F.d_EB, F.d_Vbase, F.d_tc_err, F.flow_in_arena ? nullptr : F.d_flow,
                    F.d_pi_work, F.d_dense_loop};
    for (void *p : ptrs)
        if (p && p != F.d_arena) cudaFree(p);
    // the arena came from the pool: returned in stream order (every call on
    // this object has synchronised with its stream before returning)
    if (F.d_arena) cudaFreeAsync(F.d_arena, 0);
    if (F.plain_graph) cudaGraphExecDestroy(F.plain_graph);
    F.plain_graph = nullptr;
    if (F.march_graph) cudaGraphExecDestroy(F.march_graph);
    F.march_graph = nullptr;
    if (F.dense_graph) cudaGraphExecDestroy(F.dense_graph);
    F.dense_graph = nullptr;
    if (F.dense_pi_graph) cudaGraphExecDestroy(F.dense_pi_graph);
    F.dense_pi_graph = nullptr;
    if (F.simt_graph) cudaGraphExecDestroy(F.simt_graph);
    F.simt_graph = nullptr;
    F.d_dense_loop = nullptr;
    F.d_arena = nullptr;
    F.d_code = nullptr; F.d_R32 = nullptr; F.d_R64 = nullptr; F.d_cell = nullptr;
    F.d_scratch = nullptr; F.d_q = nullptr; F.d_ctrl = nullptr; F.d_U32 = nullptr;
    F.d_U64 = nullptr; F.d_Ubf = nullptr; F.d_lam32 = nullptr; F.d_lam64 = nullptr;
    F.d_dense_work = nullptr; F.d_Vd = nullptr; F.d_RB = nullptr; F.d_T = nullptr;
    F.d_EB = nullptr; F.d_Vbase = nullptr; F.d_tc_err = nullptr; F.d_pi_work = nullptr;
    F.d_flow = nullptr; F.flow_in_arena = false;
}

// Build the banded GridWorld factors: the slip weights of the rank-1 terms
// and, per state, the code of blocked moves (walls: the shift factor's
// reflecting rows; obstacles: the non-separable correction).
static void build_gridworld(Factors &F) {
    const int D = F.ndim;
    F.rank = D == 1 ? 2 : 2 * D - 1;
    F.w_move = F.p;
    F.w_perp = D >= 2 ? (1.0 - F.p) / (2.0 * (D - 1)) : 0.0;
    F.w_stay = D == 1 ? 1.0 - F.p : 0.0;
    F.code_bytes = code_bytes_for(D);
    // factors on a device get their codes from codes_kernel (upload); the
    // host keeps its own copy only for host-only factors
    if (F.device >= 0) return;
    const int64_t S = F.nstates;
    F.code.assign((size_t)S, 0u);
    const uint32_t all_dirs = (uint32_t)((1ull << (2 * D)) - 1);
    // locals: stores through the code array may not alias the byte reads of
    // the cells in the compiler's eyes, so nothing is reloaded per state
    const uint8_t *cell = F.cell.data();
    uint32_t *code = F.code.data();
    int64_t shape[CPMDP_MAX_DIM], stride[CPMDP_MAX_DIM];
    for (int d = 0; d < D; d++) { shape[d] = F.shape[d]; stride[d] = F.stride[d]; }
    const int64_t n = shape[D - 1];          // rows of the last dimension
    // coordinates of the row kept by an odometer (no divisions)
    int64_t x[CPMDP_MAX_DIM] = {0};
    for (int64_t row = 0; row < S; row += n) {
        // blocked moves of the leading dimensions are the same test for every
        // state of the row, against the neighbouring rows' cells
        for (int64_t i = 0; i < n; i++) {
            const int64_t s = row + i;
            const uint8_t k = cell[s];
            uint32_t c;
            if (k == CPMDP_CELL_OBSTACLE) {
                c = all_dirs | (1u << (2 * D));
            } else if (k == CPMDP_CELL_TERMINAL) {
                c = all_dirs | (1u << (2 * D + 1));
            } else {
                c = 0;
                // branch-free: at a wall the cell read is the state's own
                for (int d = 0; d < D - 1; d++) {
                    const bool lo = x[d] == 0, hi = x[d] == shape[d] - 1;
                    c |= (uint32_t)(lo | (cell[lo ? s : s - stride[d]] == CPMDP_CELL_OBSTACLE)) << (2 * d);
                    c |= (uint32_t)(hi | (cell[hi ? s : s + stride[d]] == CPMDP_CELL_OBSTACLE)) << (2 * d + 1);
                }
                const bool lo = i == 0, hi = i == n - 1;
                c |= (uint32_t)(lo | (cell[lo ? s : s - 1] == CPMDP_CELL_OBSTACLE)) << (2 * (D - 1));
                c |= (uint32_t)(hi | (cell[hi ? s : s + 1] == CPMDP_CELL_OBSTACLE)) << (2 * (D - 1) + 1);
            }
            code[s] = c;
        }
        for (int d = D - 2; d >= 0; d--) {
            if (++x[d] < shape[d]) break;
            x[d] = 0;
        }
    }
}

// per_state: also check every reward and cell code on the host (device
// GridWorld builds check them on the device instead, in the kernels that
// convert the rewards and derive the move codes).
static cpmdp_status validate(const cpmdp_problem *p, bool per_state) {
    if (!p) { set_error("problem is NULL"); return CPMDP_EINVAL; }
    if (p->ndim < 1 || p->ndim > CPMDP_MAX_DIM) { set_error("ndim %d outside [1, %d]", p->ndim, CPMDP_MAX_DIM); return CPMDP_EINVAL; }
    double S = 1;
    for (int d = 0; d < p->ndim; d++) {
        if (p->shape[d] < 1) { set_error("shape[%d] = %lld < 1", d, (long long)p->shape[d]); return CPMDP_EINVAL; }
        S *= (double)p->shape[d];
    }
    if (S >= 2147483648.0) { set_error("|S| = %.0f exceeds 2^31 - 1", S); return CPMDP_EINVAL; }
    if (!(p->gamma >= 0.0 && p->gamma <= 1.0)) { set_error("gamma %g outside [0, 1]", p->gamma); return CPMDP_EINVAL; }
    if (!p->reward) { set_error("reward is NULL"); return CPMDP_EINVAL; }
    if (per_state) {
        // a double is not finite exactly when its exponent bits are all ones:
        // one branch-free integer pass, then a search only when it failed
        const uint64_t *bits = reinterpret_cast<const uint64_t *>(p->reward);
        uint64_t bad = 0;
        for (int64_t s = 0; s < (int64_t)S; s++) bad |= ((bits[s] >> 52) & 0x7FFu) == 0x7FFu;
        if (bad)
            for (int64_t s = 0; s < (int64_t)S; s++)
                if (!isfinite(p->reward[s])) { set_error("reward[%lld] is not finite", (long long)s); return CPMDP_EINVAL; }
    }
    if (p->kind == CPMDP_GRIDWORLD) {
        if (p->nactions != 2 * p->ndim) { set_error("GridWorld needs nactions = 2*ndim = %d (got %d)", 2 * p->ndim, p->nactions); return CPMDP_EINVAL; }
        if (!(p->p_success >= 0.0 && p->p_success <= 1.0)) { set_error("p_success %g outside [0, 1]", p->p_success); return CPMDP_EINVAL; }
        if (p->cell && per_state) {
            uint8_t top = 0;
            for (int64_t s = 0; s < (int64_t)S; s++) top = p->cell[s] > top ? p->cell[s] : top;
            if (top > CPMDP_CELL_TERMINAL)
                for (int64_t s = 0; s < (int64_t)S; s++)
                    if (p->cell[s] > CPMDP_CELL_TERMINAL) { set_error("cell[%lld] = %d is not 0, 1 or 2", (long long)s, p->cell[s]); return CPMDP_EINVAL; }
        }
    } else if (p->kind == CPMDP_DENSE_CP) {
        if (p->nactions < 1 || p->nactions > 64) { set_error("dense nactions %d outside [1, 64]", p->nactions); return CPMDP_EINVAL; }
        if (p->rank < 1 || p->rank > 64) { set_error("dense rank %d outside [1, 64]", p->rank); return CPMDP_EINVAL; }
        if (!p->factors || !p->lambda) { set_error("dense factors or lambda is NULL"); return CPMDP_EINVAL; }
        if (p->cell) { set_error("dense models take no cell codes"); return CPMDP_EINVAL; }
        for (int d = 0; d < p->ndim; d++)
            if (p->shape[d] > 4096) { set_error("dense mode size %lld > 4096", (long long)p->shape[d]); return CPMDP_EINVAL; }
    } else {
        set_error("unknown kind %d", p->kind);
        return CPMDP_EINVAL;
    }
    return CPMDP_OK;
}

// Code of blocked moves of one state (the same rule as build_gridworld), for
// host queries on factors whose codes live on the device only.
static const uint8_t *host_cells(const Factors &F) {
    if ((int64_t)F.cell.size() != F.nstates) {
        F.cell.resize((size_t)F.nstates);
        DeviceGuard g(F.device);
        if (cudaMemcpy(F.cell.data(), F.d_cell, (size_t)F.nstates, cudaMemcpyDeviceToHost) != cudaSuccess) {
            (void)cudaGetLastError();
            F.cell.clear();
            return nullptr;
        }
    }
    return F.cell.data();
}

static uint32_t code_of(const Factors &F, int64_t s) {
    const int D = F.ndim;
    const uint32_t all_dirs = (uint32_t)((1ull << (2 * D)) - 1);
    const uint8_t k = F.cell[(size_t)s];
    if (k == CPMDP_CELL_OBSTACLE) return all_dirs | (1u << (2 * D));
    if (k == CPMDP_CELL_TERMINAL) return all_dirs | (1u << (2 * D + 1));
    uint32_t c = 0;
    int64_t rem = s;
    for (int d = 0; d < D; d++) {
        const int64_t x = rem / F.stride[d];
        rem -= x * F.stride[d];
        if (x == 0 || F.cell[(size_t)(s - F.stride[d])] == CPMDP_CELL_OBSTACLE) c |= 1u << (2 * d);
        if (x == F.shape[d] - 1 || F.cell[(size_t)(s + F.stride[d])] == CPMDP_CELL_OBSTACLE) c |= 1u << (2 * d + 1);
    }
    return c;
}

struct CodeGeom {
    int ndim;
    int shape[kMaxDim], stride[kMaxDim];
};

// Per-state codes of blocked moves from the cell kinds (device copy of the
// rule in build_gridworld), stored in `cb` bytes per state. |S| < 2^31 is
// validated, so 32-bit coordinates suffice (64-bit division is emulated).
// bad (nullable): set to 1 + the index of a cell code other than 0, 1, 2.
__global__ void codes_kernel(const uint8_t *__restrict__ cell, CodeGeom g, int S, int cb, uint8_t *__restrict__ out,
                             unsigned long long *bad) {
    const int D = g.ndim;
    const uint32_t all_dirs = (uint32_t)((1ull << (2 * D)) - 1);
    // the loop index is 64-bit so the stride step cannot overflow near |S| = 2^31
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)i;
        const uint8_t k = cell[s];
        if (bad && k > CPMDP_CELL_TERMINAL) atomicCAS(bad, 0ull, (unsigned long long)s + 1ull);
        uint32_t c;
        if (k == CPMDP_CELL_OBSTACLE) {
            c = all_dirs | (1u << (2 * D));
        } else if (k == CPMDP_CELL_TERMINAL) {
            c = all_dirs | (1u << (2 * D + 1));
        } else {
            c = 0;
            int rem = s;
            for (int d = 0; d < D; d++) {
                const int x = rem / g.stride[d];
                rem -= x * g.stride[d];
                if (x == 0 || cell[s - g.stride[d]] == CPMDP_CELL_OBSTACLE) c |= 1u << (2 * d);
                if (x == g.shape[d] - 1 || cell[s + g.stride[d]] == CPMDP_CELL_OBSTACLE) c |= 1u << (2 * d + 1);
            }
        }
        if (cb == 1) out[s] = (uint8_t)c;
        else if (cb == 2) reinterpret_cast<uint16_t *>(out)[s] = (uint16_t)c;
        else reinterpret_cast<uint32_t *>(out)[s] = c;
    }
}

// bad (nullable): set to 1 + the index of a value that is not finite (all
// exponent bits set; an integer test, no FP64 instruction).
__global__ void to_f32_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t n,
                              unsigned long long *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = a[i];
        if (bad && ((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF) atomicCAS(bad, 0ull, (unsigned long long)i + 1ull);
        b[i] = (float)x;
    }
}

// reward: the caller's rewards (device GridWorld builds keep no host copy),
// or F.reward; cell: the caller's cell kinds (NULL: all free) or F.cell.
// The copies and kernels go to the legacy default stream in order; device
// GridWorld builds check every reward (finite) and cell code (0, 1, 2) in
// the conversion and code kernels, and the one synchronising read of the
// build reads those checks.
static cpmdp_status upload(Factors &F, const double *reward, const uint8_t *cell) {
    DeviceGuard g(F.device);
    if (!g.ok) { set_error("cannot select CUDA device %d", F.device); return CPMDP_ECUDA; }
    CPMDP_CUDA(cudaDeviceGetAttribute(&F.num_sms, cudaDevAttrMultiProcessorCount, F.device));
    const size_t S = (size_t)F.nstates;
    const int blocks = (int)std::min<int64_t>((F.nstates + 255) / 256, (int64_t)F.num_sms * 16);
    // one allocation for the per-state arrays, the scratch and the control
    // block, each part 256-byte aligned
    const size_t cb = F.kind == CPMDP_GRIDWORLD ? (size_t)F.code_bytes : 0;
    auto up = [](size_t n) { return (n + 255) & ~(size_t)255; };
    F.scratch_bytes = S * sizeof(double);
    const size_t o_R64 = 0, o_scratch = o_R64 + up(S * sizeof(double)), o_R32 = o_scratch + up(F.scratch_bytes);
    const size_t o_cell = o_R32 + up(S * sizeof(float)), o_ctrl = o_cell + up(S), o_code = o_ctrl + up(sizeof(Ctrl));
    // the barrier-free solver's counters and rings, for shapes it can take
    // (one allocation and one free per factors object instead of two)
    const bool flow = F.kind == CPMDP_GRIDWORLD && flow_shape_ok(F);
    const size_t o_flow = o_code + up(S * cb);
    const size_t total = o_flow + (flow ? up(flow_bytes(F)) : 0);
    cudaMemPool_t pool;
    CPMDP_CUDA(arena_pool(F.device, &pool));
    CPMDP_CUDA(cudaMallocFromPoolAsync(&F.d_arena, total, pool, 0));
    char *arena = static_cast<char *>(F.d_arena);
    F.d_R64 = reinterpret_cast<double *>(arena + o_R64);
    F.d_scratch = arena + o_scratch;
    F.d_R32 = reinterpret_cast<float *>(arena + o_R32);
    F.d_cell = reinterpret_cast<uint8_t *>(arena + o_cell);
    F.d_ctrl = reinterpret_cast<Ctrl *>(arena + o_ctrl);
    F.d_code = cb ? arena + o_code : nullptr;
    if (flow) {
        F.d_flow = arena + o_flow;
        F.flow_in_arena = true;
        F.flow_base = 0;
        CPMDP_CUDA(cudaMemsetAsync(static_cast<char *>(F.d_flow) + flow_counter_bytes(), 0xFF,
                                   flow_bytes(F) - flow_counter_bytes(), 0));
    }
    const bool check = F.kind == CPMDP_GRIDWORLD;
    CPMDP_CUDA(cudaMemsetAsync(F.d_ctrl, 0, sizeof(Ctrl), 0));
    CPMDP_CUDA(cudaMemcpyAsync(F.d_R64, reward, S * sizeof(double), cudaMemcpyHostToDevice, 0));
    to_f32_kernel<<<blocks, 256>>>(F.d_R64, F.d_R32, F.nstates, check ? &F.d_ctrl->bad_reward : nullptr);
    CPMDP_CUDA(cudaGetLastError());
    if (cell) CPMDP_CUDA(cudaMemcpyAsync(F.d_cell, cell, S, cudaMemcpyHostToDevice, 0));
    else CPMDP_CUDA(cudaMemsetAsync(F.d_cell, CPMDP_CELL_FREE, S, 0));
    if (F.kind == CPMDP_GRIDWORLD) {
        CodeGeom geo{};
        geo.ndim = F.ndim;
        for (int d = 0; d < F.ndim; d++) { geo.shape[d] = (int)F.shape[d]; geo.stride[d] = (int)F.stride[d]; }
        codes_kernel<<<blocks, 256>>>(F.d_cell, geo, (int)F.nstates, (int)cb, static_cast<uint8_t *>(F.d_code),
                                      &F.d_ctrl->bad_cell);
        CPMDP_CUDA(cudaGetLastError());
    } else {
        cpmdp_status st = dense_prepare(F);
        if (st != CPMDP_OK) return st;
    }
    // building is synchronous: this read waits for the codes and FP32
    // rewards and returns the device-side checks
    unsigned long long bad[2] = {0ull, 0ull};
    static_assert(offsetof(Ctrl, bad_cell) == offsetof(Ctrl, bad_reward) + sizeof(unsigned long long),
                  "bad_reward and bad_cell are adjacent");
    CPMDP_CUDA(cudaMemcpy(bad, &F.d_ctrl->bad_reward, sizeof(bad), cudaMemcpyDeviceToHost));
    if (bad[0]) { set_error("reward[%lld] is not finite", (long long)(bad[0] - 1)); return CPMDP_EINVAL; }
    if (bad[1]) {
        const long long b = (long long)(bad[1] - 1);
        set_error("cell[%lld] = %d is not 0, 1 or 2", b, cell ? (int)cell[b] : -1);
        return CPMDP_EINVAL;
    }
    return CPMDP_OK;
}

}  // namespace cpmdp

using namespace cpmdp;

extern "C" {

void cpmdp_default_opts(cpmdp_solve_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->max_iter = 1000;
    o->certify = 1;
    o->fused = 1;
    o->eval_tol = 0.0;
    o->max_eval_iter = 100000;
    o->max_rounds = 1000;
    o->timeout_s = 2.0;
    o->trace = nullptr;
    o->partial_eval = -1;
}

const char *cpmdp_last_error(void) { return g_err; }

const char *cpmdp_version(void) { return "cpmdp-gb300 0.1 (sm_103a)"; }

cpmdp_status cpmdp_build_factors(const cpmdp_problem *p, int device, cpmdp_factors **out) {
    g_err[0] = 0;
    if (!out) { set_error("out is NULL"); return CPMDP_EINVAL; }
    *out = nullptr;
    // device GridWorld builds check the rewards and cell codes on the device
    const bool device_gw = device >= 0 && p && p->kind == CPMDP_GRIDWORLD;
    cpmdp_status st = validate(p, !device_gw);
    if (st != CPMDP_OK) return st;
    cpmdp_factors *h = new (std::nothrow) cpmdp_factors();
    if (!h) { set_error("host allocation failed"); return CPMDP_ENOMEM; }
    Factors &F = h->f;
    try {
        F.device = device;
        F.kind = p->kind;
        F.ndim = p->ndim;
        int64_t S = 1;
        for (int d = p->ndim - 1; d >= 0; d--) { F.stride[d] = S; S *= p->shape[d]; }
        for (int d = 0; d < p->ndim; d++) F.shape[d] = p->shape[d];
        F.nstates = S;
        F.nactions = p->nactions;
        F.p = p->p_success;
        F.gamma = p->gamma;
        // device GridWorld builds upload the caller's rewards directly; host-only
        // factors (batches) and dense models keep a host copy
        if (device < 0 || p->kind != CPMDP_GRIDWORLD) F.reward.assign(p->reward, p->reward + S);
        // device GridWorld builds upload the caller's cell kinds directly (a
        // host copy is made on the first host query that needs one)
        if (!device_gw) {
            if (p->cell) F.cell.assign(p->cell, p->cell + S);
            else F.cell.assign((size_t)S, (uint8_t)CPMDP_CELL_FREE);
        }
        if (F.kind == CPMDP_GRIDWORLD) {
            build_gridworld(F);
        } else {
            F.rank = p->rank;
            int64_t off = 0;
            for (int a = 0; a < F.nactions; a++)
                for (int r = 0; r < F.rank; r++)
                    for (int d = 0; d < F.ndim; d++) { F.factor_off.push_back(off); off += F.shape[d] * F.shape[d]; }
            F.dense_factors.assign(p->factors, p->factors + off);
            F.lambda.assign(p->lambda, p->lambda + (size_t)F.nactions * F.rank);
            for (int64_t i = 0; i < off; i++)
                if (!(F.dense_factors[(size_t)i] >= 0.0) || !isfinite(F.dense_factors[(size_t)i])) {
                    set_error("factor entry %lld is negative or not finite", (long long)i);
                    delete h;
                    return CPMDP_EINVAL;
                }
            for (int a = 0; a < F.nactions; a++) {
                double ls = 0;
                for (int r = 0; r < F.rank; r++) {
                    const double l = F.lambda[(size_t)a * F.rank + r];
                    if (!(l >= 0.0) || !isfinite(l)) { set_error("lambda[%d][%d] invalid", a, r); delete h; return CPMDP_EINVAL; }
                    ls += l;
                    for (int d = 0; d < F.ndim; d++) {
                        const int64_t n = F.shape[d];
                        const double *U = &F.dense_factors[(size_t)F.factor_off[((size_t)a * F.rank + r) * F.ndim + d]];
                        for (int64_t i = 0; i < n; i++) {
                            double rs = 0;
                            for (int64_t j = 0; j < n; j++) rs += U[i * n + j];
                            if (fabs(rs - 1.0) > 1e-9) {
                                set_error("factor (a=%d, r=%d, d=%d) row %lld sums to %.12g, not 1", a, r, d, (long long)i, rs);
                                delete h;
                                return CPMDP_EINVAL;
                            }
                        }
                    }
                }
                if (fabs(ls - 1.0) > 1e-9) { set_error("lambda of action %d sums to %.12g, not 1", a, ls); delete h; return CPMDP_EINVAL; }
            }
        }
    } catch (const std::bad_alloc &) {
        delete h;
        set_error("host allocation failed");
        return CPMDP_ENOMEM;
    }
    if (device >= 0) {
        st = upload(F, F.reward.empty() ? p->reward : F.reward.data(), device_gw ? p->cell : F.cell.data());
        if (st != CPMDP_OK) {
            DeviceGuard g(device);
            free_device(F);
            delete h;
            return st;
        }
    }
    *out = h;
    return CPMDP_OK;
}

void cpmdp_free_factors(cpmdp_factors *h) {
    if (!h) return;
    if (h->f.device >= 0) {
        DeviceGuard g(h->f.device);
        free_device(h->f);
    }
    delete h;
}

cpmdp_status cpmdp_factors_info(const cpmdp_factors *h, int64_t *nstates, int32_t *nactions,
                                int32_t *rank, int32_t *ndim) {
    if (!h) { set_error("factors is NULL"); return CPMDP_EINVAL; }
    if (nstates) *nstates = h->f.nstates;
    if (nactions) *nactions = h->f.nactions;
    if (rank) *rank = h->f.rank;
    if (ndim) *ndim = h->f.ndim;
    return CPMDP_OK;
}

cpmdp_status cpmdp_components(const cpmdp_factors *h, int64_t s, int32_t a, int64_t *next, double *prob,
                              int32_t cap, int32_t *count) {
    if (!h || !count) { set_error("factors or count is NULL"); return CPMDP_EINVAL; }
    const Factors &F = h->f;
    if (F.kind != CPMDP_GRIDWORLD) { set_error("components are listed for GridWorld models only"); return CPMDP_EINVAL; }
    if (s < 0 || s >= F.nstates || a < 0 || a >= F.nactions) { set_error("state or action out of range"); return CPMDP_EINVAL; }
    if (cap > 0 && (!next || !prob)) { set_error("next/prob NULL with cap > 0"); return CPMDP_EINVAL; }
    *count = 0;
    const uint8_t *cells = host_cells(F);
    if (!cells) { set_error("cannot read the cell kinds back from the device"); return CPMDP_ECUDA; }
    if (cells[(size_t)s] != CPMDP_CELL_FREE) return CPMDP_OK;
    const int D = F.ndim;
    const uint32_t code = F.code.empty() ? code_of(F, s) : F.code[(size_t)s];
    std::map<int64_t, double> acc;
    auto move = [&](int d, int sg, double w) {
        const int j = 2 * d + sg;
        const int64_t t = ((code >> j) & 1u) ? s : s + (sg ? F.stride[d] : -F.stride[d]);
        acc[t] += w;
    };
    const int d0 = a / 2, s0 = a & 1;
    move(d0, s0, F.w_move);
    if (D == 1) acc[s] += F.w_stay;
    else
        for (int d = 0; d < D; d++)
            if (d != d0) { move(d, 0, F.w_perp); move(d, 1, F.w_perp); }
    int n = 0;
    for (const auto &kv : acc) {
        if (kv.second <= 0.0) continue;
        if (n < cap) { next[n] = kv.first; prob[n] = kv.second; }
        n++;
    }
    *count = n;
    return CPMDP_OK;
}

static cpmdp_status check_solver_args(const cpmdp_factors *h, cpmdp_precision prec, const void *V) {
    if (!h) { set_error("factors is NULL"); return CPMDP_EINVAL; }
    if (h->f.device < 0) { set_error("factors were built host-only (device -1)"); return CPMDP_EINVAL; }
    if (!V) { set_error("value buffer is NULL"); return CPMDP_EINVAL; }
    if (prec != CPMDP_F32 && prec != CPMDP_F64 && prec != CPMDP_BF16X3) { set_error("unknown precision %d", (int)prec); return CPMDP_EINVAL; }
    if (prec == CPMDP_BF16X3 && h->f.kind != CPMDP_DENSE_CP) { set_error("BF16X3 applies to dense CP models only"); return CPMDP_EINVAL; }
    return CPMDP_OK;
}

cpmdp_status cpmdp_bellman_backup(const cpmdp_factors *h, cpmdp_precision prec, const void *Vin, void *Vout,
                                  uint8_t *pi, double *res, void *stream) {
    g_err[0] = 0;
    cpmdp_status st = check_solver_args(h, prec, Vin);
    if (st != CPMDP_OK) return st;
    if (!Vout) { set_error("V_out is NULL"); return CPMDP_EINVAL; }
    if (Vin == Vout) { set_error("V_in and V_out must not alias"); return CPMDP_EINVAL; }
    DeviceGuard g(h->f.device);
    if (!g.ok) { set_error("cannot select CUDA device %d", h->f.device); return CPMDP_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    if (h->f.kind == CPMDP_GRIDWORLD) return banded_backup(h->f, prec, Vin, Vout, pi, res, s);
    return dense_backup(h->f, prec, Vin, Vout, pi, res, s);
}

static cpmdp_status run_solver(const cpmdp_factors *h, cpmdp_precision prec, bool pi_mode, void *V,
                               uint8_t *pi, const cpmdp_solve_opts *opts, cpmdp_result *info, void *stream) {
    g_err[0] = 0;
    cpmdp_status st = check_solver_args(h, prec, V);
    if (st != CPMDP_OK) return st;
    if (pi_mode && !pi) { set_error("policy iteration needs a policy buffer"); return CPMDP_EINVAL; }
    const Factors &F = h->f;
    SolveOpts o = resolve_opts(opts, prec);
    // the evaluation cap that measured fastest: an improvement costs one
    // sweep on GridWorld models, two sweeps and a compare on dense ones
    if (o.partial_eval == -1) o.partial_eval = F.kind == CPMDP_DENSE_CP ? 4 : 2;
    if (!(o.tol > 0) || o.max_iter < 1 || o.max_eval_iter < 1 || o.max_rounds < 1 || !(o.timeout_s > 0) ||
        o.partial_eval < 0) {
        set_error("invalid solve options (tol > 0, max_iter >= 1, timeout_s > 0, partial_eval >= -1 required)");
        return CPMDP_EINVAL;
    }
    if (o.fused < 0 || o.fused > 3) { set_error("fused must be 0, 1, 2 or 3"); return CPMDP_EINVAL; }
    const bool plain = o.fused == 0 || o.fused == 3;
    if (pi_mode && plain) { set_error("the plain baseline implements value iteration only"); return CPMDP_EINVAL; }
    DeviceGuard g(F.device);
    if (!g.ok) { set_error("cannot select CUDA device %d", F.device); return CPMDP_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CPMDP_CUDA(cudaEventCreate(&e0));
    CPMDP_CUDA(cudaEventCreate(&e1));
    CPMDP_CUDA(cudaEventRecord(e0, s));
    Ctrl hc;
    memset(&hc, 0, sizeof(hc));
    bool have_ctrl = false;
    if (F.kind == CPMDP_GRIDWORLD) {
        if (!plain) {
            st = banded_solve(F, prec, pi_mode, V, pi, o, s);
        } else {
            if (!F.d_q) {
                Factors &Fm = const_cast<Factors &>(F);
                Fm.q_bytes = (size_t)F.nactions * F.nstates * sizeof(double);
                CPMDP_CUDA(cudaMalloc(&Fm.d_q, Fm.q_bytes));
            }
            st = banded_plain_vi(F, prec, V, pi, o, &hc, s);
            have_ctrl = true;
        }
    } else {
        st = dense_solve(F, prec, pi_mode, V, pi, o, &hc, s);
        have_ctrl = true;
    }
    if (st != CPMDP_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
    // certifying FP64 sweep (banded F32 / F64 fused path)
    double *cert = (double *)((char *)F.d_ctrl + offsetof(Ctrl, certify_residual));
    const bool do_cert = o.certify && F.kind == CPMDP_GRIDWORLD;
    // the dense BF16X3 solver runs its own FP64 certifying sweep
    const bool dense_cert = o.certify && F.kind == CPMDP_DENSE_CP && prec == CPMDP_BF16X3;
    if (do_cert) {
        if (prec == CPMDP_F64) {
            // one FP64 backup into scratch: residual + policy of the returned V
            uint8_t *pout = pi_mode ? nullptr : pi;
            st = banded_backup(F, CPMDP_F64, V, F.d_scratch, pout, cert, s);
        } else {
            st = banded_certify(F, (const float *)V, pi_mode ? nullptr : pi, cert, s);
        }
        if (st != CPMDP_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
    } else if (!pi_mode && pi && F.kind == CPMDP_GRIDWORLD && !plain) {
        st = banded_backup(F, prec, V, F.d_scratch, pi, nullptr, s);
        if (st != CPMDP_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
    }
    CPMDP_CUDA(cudaEventRecord(e1, s));
    Ctrl dc;
    CPMDP_CUDA(cudaMemcpyAsync(&dc, F.d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CPMDP_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int solver = F.kind != CPMDP_GRIDWORLD ? CPMDP_SOLVER_DENSE
                       : plain ? CPMDP_SOLVER_PLAIN
                       : F.flow_pending ? CPMDP_SOLVER_BARRIER_FREE
                       : F.march_pending ? CPMDP_SOLVER_MARCH_GRAPH : CPMDP_SOLVER_GRID_BARRIER;
    if (F.kind == CPMDP_GRIDWORLD && !plain) {
        st = banded_solve_finished(F, dc, s);
        if (st != CPMDP_OK) return st;
    }
    if (!have_ctrl) {
        hc = dc;
    } else {
        hc.certify_residual = dc.certify_residual;
    }
    if (dense_cert) hc.certify_residual = dc.certify_residual;
    if (dc.status != 0 && !have_ctrl) {
        set_error("a device-side wait exceeded %.3g s; results are undefined", o.timeout_s);
        if (info) { memset(info, 0, sizeof(*info)); info->status = dc.status; info->solver = solver; }
        return (cpmdp_status)dc.status;
    }
    cpmdp_result r;
    memset(&r, 0, sizeof(r));
    r.iterations = hc.iterations;
    r.rounds = hc.rounds;
    r.eval_sweeps = hc.eval_sweeps;
    r.residual = hc.last_residual;
    const bool have_cert = do_cert || dense_cert;
    r.certified_residual = have_cert ? hc.certify_residual : -1.0;
    r.error_bound = (have_cert && F.gamma < 1.0) ? hc.certify_residual / (1.0 - F.gamma) : -1.0;
    r.backups = hc.backups;
    r.elapsed_ms = ms;
    r.solver = solver;
    r.status = hc.converged ? CPMDP_OK : CPMDP_ENOCONV;
    if (info) *info = r;
    if (!hc.converged) {
        set_error("not converged: %d sweeps, residual %.3g", hc.iterations, hc.last_residual);
        return CPMDP_ENOCONV;
    }
    return CPMDP_OK;
}

cpmdp_status cpmdp_value_iteration(const cpmdp_factors *h, cpmdp_precision prec, void *V, uint8_t *pi,
                                   const cpmdp_solve_opts *opts, cpmdp_result *info, void *stream) {
    return run_solver(h, prec, false, V, pi, opts, info, stream);
}

cpmdp_status cpmdp_policy_iteration(const cpmdp_factors *h, cpmdp_precision prec, void *V, uint8_t *pi,
                                    const cpmdp_solve_opts *opts, cpmdp_result *info, void *stream) {
    return run_solver(h, prec, true, V, pi, opts, info, stream);
}

}  // extern "C"
