// Barrier-free persistent FP32 GridWorld solver (flow_solve.cu).
#pragma once

#include "internal.h"

namespace cpmdp {

struct SolveParams;

// True when the barrier-free solver can run this solve: 1 to 3 dimensions,
// rows a multiple of 4 states, V 16-byte aligned (policy 4-byte aligned),
// and one thread per 4 states fits in one co-resident grid.
bool flow_eligible(const Factors &F, bool policy_iteration, const void *V, const uint8_t *pi, const SolveOpts &o);
// Device bytes the solver needs beside the factors' own buffers: arrival
// counters and four rings of |S| tagged 64-bit words.
size_t flow_bytes(const Factors &F);
// True when the shape alone lets the barrier-free solver run value or
// policy iteration (the build then reserves its buffers with the factors).
bool flow_shape_ok(const Factors &F);
size_t flow_counter_bytes();
// One cooperative launch on `st` (F.d_flow allocated, tags above F.flow_base
// never written before). Fills the control block like banded_solve.
cpmdp_status flow_solve(const Factors &F, bool policy_iteration, float *V, uint8_t *pi, const SolveParams &sp,
                        double *trace, cudaStream_t st);

}  // namespace cpmdp
