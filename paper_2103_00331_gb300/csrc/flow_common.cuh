// Sweep-tagged value words, arrival counters and bounded waits shared by
// the barrier-free solvers (flow_solve.cu for one GridWorld, batch_flow.cu
// for the tail of a batch).
//
// A word holds (tag << 32) | float bits and is written and read whole (one
// relaxed 64-bit access at GPU scope), so a reader that sees the tag it
// expects also sees the value written with it.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "banded_common.cuh"

namespace cpmdp {
namespace tw {

typedef unsigned long long u64;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kLag = 3;              // the stopping rule of sweep q is settled at sweep q + kLag
constexpr int kRing = kLag + 1;      // tagged value buffers
constexpr int kSlots = 8;            // arrival slots (arrival i uses slot i % kSlots; > 2 kLag + 1)

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

// Bits of the smallest non-negative float >= t (t > 0; +inf above the
// float range).
inline unsigned float_ceil_bits(double t) {
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    unsigned u;
    memcpy(&u, &f, sizeof u);
    return u;
}

}  // namespace tw
}  // namespace cpmdp
