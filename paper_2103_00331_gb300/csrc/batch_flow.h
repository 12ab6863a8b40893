// Barrier-free tail of a batched value-iteration solve (batch_flow.cu).
#pragma once

#include <cuda_runtime.h>

#include "batch_internal.h"

namespace cpmdp {

constexpr int kBatchFlowWarpsPerBlock = 14;   // one block of 448 threads per SM

// Device buffers of the tail phase (owned by the batch).
struct BatchFlowBuffers {
    unsigned long long *ring = nullptr;   // 4 x total_states tagged words
    unsigned long long *ctr = nullptr;    // ninst x 8 arrival counters
    int2 *tab = nullptr;                  // warp table (capacity entries)
    int *hdr = nullptr;                   // [0] warps, [1] epoch, [2] phase-1 sweeps, [3] clear flag
    unsigned *epoch = nullptr;            // tag epoch, kept across solves
    unsigned long long *p2res = nullptr;  // ninst residual bits
};

// Warps the tail phase keeps resident (0 if its kernel cannot run).
int batch_flow_capacity_warps(int num_sms);
size_t batch_flow_ring_words(long long total_states);
size_t batch_flow_counter_words(int ninst);
// Enqueue the tail phase after the batched kernel: set-up, ring clearing
// when the tag epoch wraps, and the cooperative launch. Does nothing on the
// device when the batched kernel did not hand off.
cudaError_t batch_flow_enqueue(const BatchFlowBuffers &b, const BatchInst *inst, int ninst, const uint8_t *code,
                               const float *R, float *V, const float *W, int *done_at, const unsigned long long *res,
                               Ctrl *ctrl, long long total_states, int num_sms, double tol, int max_iter,
                               double timeout_s, cudaStream_t st);

}  // namespace cpmdp
