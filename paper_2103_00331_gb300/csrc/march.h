// Plane-marching fused backup sweep of large 3-D GridWorlds (banded_march.cu).
#pragma once

#include "internal.h"

namespace cpmdp {

// From this many states on the value tensor and its companions outgrow L2
// and the marching sweep, which reads them from DRAM about once, is used.
constexpr long long kMarchMinStates = 1ll << 23;

// 3-D float values with rows a multiple of 4 states, at least
// kMarchMinStates states, V and W 16-byte aligned (W may be null), policy
// 4-byte aligned (may be null).
bool march_eligible(const Factors &F, const void *V, const void *W, const void *pi);
// One backup sweep of V into W (may be null) with the policy (may be null)
// and the residual atomically maxed into *res (bits of a non-negative
// double, may be null): FP32 arithmetic, or FP64 when fp64 is set.
cudaError_t march_sweep(const Factors &F, const float *V, float *W, uint8_t *pi, unsigned long long *res, bool fp64,
                        cudaStream_t st);
// FP32 value iteration (V in place, the factors' scratch as the second
// buffer) by recorded graphs of marching sweeps with the stopping rule taken
// on the device; fills the control block (iterations, converged, residual,
// backups). The control block must be cleared before the call.
cudaError_t march_solve(const Factors &F, float *V, double tol, int max_iter, double *trace, cudaStream_t st);

}  // namespace cpmdp
