// Internal layout of a packed batch of GridWorld instances (batch.cu),
// shared with the warm-start kernels (warmstart.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace cpmdp {

struct BatchInst {
    long long offset;      // first state in the packed arrays
    int nstates;
    int ndim;              // 1..3
    int nlast;
    int stride[3];
    int shape[3];
    int vec;               // states per segment (4)
    int rows4;             // 1: rows a multiple of 4 states long
    int first_tile;
    float w_move, w_perp, w_stay, gamma;
};

// One warp tile: up to 32 x spl 4-state segments of one instance, with the
// instance fields the backups need (one 64-byte record, no second lookup).
struct alignas(16) BatchTile {
    long long offset;      // instance's first state in the packed arrays
    int inst;
    int first_item;        // first segment of the tile
    int nitems;            // segments in the tile
    int nstates;           // instance states
    int cls;               // ndim * 2 + rows4
    int nlast;
    int stride0, stride1;  // strides of the leading dimensions (0 if absent)
    float w_move, w_perp, w_stay, gamma;
};

}  // namespace cpmdp

struct cpmdp_batch {
    int device = -1;
    int ninst = 0;
    long long total_states = 0;
    std::vector<cpmdp::BatchInst> inst;
    std::vector<int> inst_actions;
    std::vector<int64_t> offsets;
    cpmdp::BatchInst *d_inst = nullptr;
    cpmdp::BatchTile *d_tiles = nullptr;
    int ntiles = 0;
    int tile_items = 0;
    int block = 0;
    int spl = 1;           // segments per lane of a warp tile
    uint8_t *d_code = nullptr;
    float *d_R = nullptr;
    float *d_W = nullptr;
    unsigned long long *d_res = nullptr;
    int *d_done = nullptr;
    cpmdp::Ctrl *d_ctrl = nullptr;
    bool graph_failed = false;
    bool tuned = false;
    int num_sms = 0;
    int grid = 0;
    // CUDA graph of one solve, recorded for (V pointer, stream, options)
    cudaGraphExec_t graph = nullptr;
    void *graph_V = nullptr;
    cudaStream_t graph_stream = nullptr;
    double graph_tol = 0;
    int graph_max_iter = 0;
    double graph_timeout = 0;
    int graph_tail = 0;
    std::vector<cpmdp::BatchTile> tiles_host;
    // barrier-free tail (batch_flow.cu), allocated on the first solve
    bool flow_tried = false;
    int flow_cap_warps = 0;                // 0: the tail stays on the batched kernel
    unsigned long long *d_ring = nullptr;
    unsigned long long *d_p2ctr = nullptr;
    int2 *d_p2tab = nullptr;
    int *d_p2hdr = nullptr;
    unsigned *d_p2epoch = nullptr;
    unsigned long long *d_p2res = nullptr;
    // FP64 certifying sweep (cpmdp_batch_certify)
    double *d_R64 = nullptr;
    double *d_instw = nullptr;
    unsigned long long *d_cert = nullptr;
};

