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

// Shared-memory-resident batched solve (batch_resident.cu): one part of an
// instance held by one CTA, slices [z0, z0 + nsl) of its leading dimension
// (3-D: y-x planes, 2-D: rows, 1-D: the one row), rows padded to nxp states.
struct ResPart {
    long long goff;        // packed index of the part's first state
    long long poff;        // index of the part's first state in the padded reward / code copies
    int inst;
    int D, nx, nxp, ny, P; // dimensions; row, padded row, rows per slice, padded states per slice
    int nsl;               // slices held
    int base;              // shared-memory state offset (a multiple of 128)
    int nchunks;           // 128-state chunks
    int has_prev, has_next;  // the adjacent slice lives in the CTA of rank - 1 / rank + 1
    int prev_off;          // state offset of that CTA's last slice (rank - 1)
    unsigned prev_addr, next_addr;  // shared::cluster addresses (set in the kernel)
    float wm, wp, wst, g;
    int bidx;              // cluster bundles: index of the part's instance in the bundle
    int nbinst;            //   instances in the bundle (each over consecutive ranks)
    int lead;              //   rank of the instance's first part (records its result)
};

struct ResArgs {
    const ResPart *parts;
    const int2 *multi;     // cluster bundles: (first part, parts), part r on cluster rank r
    const int2 *solo;      // solo bundles: (first part, parts), all in one CTA
    const int *hdr;        // [0] cluster bundles, [1] solo bundles
    int *ctr;              // [0], [1]: queue counters, zeroed before each launch
    const float *Rp;       // padded FP32 rewards (0 on obstacles)
    const float *Gp;       // padded multipliers of max_a E_a: gamma on free states, else 0
    const uint8_t *codep;  // padded move codes (padding: obstacle)
    float *V;              // packed values, start in / result out
    int *done_at;          // per instance: sweeps done (negative: stopped at max_iter)
    unsigned long long *res;  // [3][ninst]: residual of the last sweep (bits of a double) at (sweeps - 1) % 3
    int ninst;
    unsigned tol_bits;     // bits of the largest float below tol
    int max_iter;
    Ctrl *ctrl;            // iterations = most sweeps of any instance
};

}  // namespace cpmdp

struct cpmdp_batch;
namespace cpmdp {
cpmdp_status batch_resident_prepare(cpmdp_batch &B);
cpmdp_status batch_resident_plan(cpmdp_batch &B, double tol, int max_iter);
cudaError_t batch_resident_enqueue(const cpmdp_batch &B, float *V, double tol, int max_iter, cudaStream_t st);
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
    // shared-memory-resident solve (batch_resident.cu), set up on the first solve
    bool res_tried = false;
    bool res_ok = false;
    int res_C = 1;                         // CTAs per cluster
    int res_grid = 0;                      // CTAs launched (co-resident clusters x res_C)
    float *d_Rp = nullptr;
    float *d_Gp = nullptr;
    uint8_t *d_codep = nullptr;
    cpmdp::ResPart *d_rparts = nullptr;
    int2 *d_rmulti = nullptr;
    int2 *d_rsolo = nullptr;
    int *d_rhdr = nullptr;
    std::vector<long long> res_pad;        // per instance: offset in the padded copies
    std::vector<int> res_est;              // per instance: sweeps of the last solve (0: unknown)
    std::vector<int> res_planned_for;      // res_est the current bundles were made for
    bool res_planned = false;
    int res_nmulti = 0, res_nsolo = 0;
    int graph_kind = -1;                   // recorded graph: 0 batched, 1 batched + tail, 2 resident
};

