// Internal declarations of libcpmdp (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cpmdp.h"

namespace cpmdp {

constexpr int kMaxDim = CPMDP_MAX_DIM;

// Per-state code of the banded GridWorld factors. Bit j (j = 2d + (sigma>0),
// j < 2D) is set when the unit move in direction j is blocked: it would
// leave the grid (the shift factor's reflecting row) or enter an obstacle
// (the non-separable correction). Bit 2D marks an obstacle, bit 2D+1 a
// terminal state. 8 bits hold D <= 3, 16 bits D <= 7, 32 bits D <= 9.
inline int code_bytes_for(int D) { return D <= 3 ? 1 : (D <= 7 ? 2 : 4); }

// Device control block of the persistent solvers (zeroed before a launch).
struct Ctrl {
    unsigned long long bar[2];     // grid barrier counters (arrivals | flags << 32)
    int status;                    // 0 ok, CPMDP_ETIMEOUT, ...
    int iterations;                // sweeps done
    int rounds;                    // PI improvement rounds
    int eval_sweeps;               // PI evaluation sweeps
    int converged;                 // 1 when the stopping rule was met
    unsigned int changed_total;    // PI: actions changed over all rounds
    unsigned long long res_slot[3];  // residual of sweep k in slot k % 3 (bits of a double)
    unsigned int changed_slot[3];  // dense PI: changed actions of the current round
    double last_residual;          // residual of the last sweep
    double certify_residual;       // FP64 certifying sweep
    long long backups;             // state-action backups done
    unsigned int flow_tags;        // barrier-free solver: tag sequences used by the launch
    unsigned long long need_slot[3];  // batch: warps the instances running sweep k would need, slot k % 3
    int handoff;                   // batch: 1 when the batched kernel stopped for the barrier-free tail
    int handoff_sweeps;            // batch: sweeps done before the hand-off
    int plain_stop;                // plain baseline, device-checked variant: stop every later kernel
    unsigned long long bad_reward; // factor build: 1 + index of a reward that is not finite (0: none)
    unsigned long long bad_cell;   // factor build: 1 + index of a cell code other than 0, 1, 2 (0: none)
};

struct Factors {
    int device = -1;
    int kind = CPMDP_GRIDWORLD;
    int ndim = 0;
    int64_t shape[kMaxDim] = {0};
    int64_t stride[kMaxDim] = {0};   // element strides, C order
    int64_t nstates = 0;
    int nactions = 0;
    int rank = 0;
    double p = 1.0;
    double gamma = 0.9;
    // GridWorld slip weights: intended move, each perpendicular move, stay (D = 1 only)
    double w_move = 1.0, w_perp = 0.0, w_stay = 0.0;
    int code_bytes = 1;

    // host copies
    // host copy of the cell kinds: host-only factors keep one from the build;
    // device GridWorld factors fill it from the device on the first host
    // query that needs it (cpmdp_components)
    mutable std::vector<uint8_t> cell;
    std::vector<double> reward;
    std::vector<uint32_t> code;        // banded code per state (host, widened)
    std::vector<double> dense_factors; // [a][r][d] blocks
    std::vector<double> lambda;        // [a][r]
    std::vector<int64_t> factor_off;   // offset of block (a, r, d) in dense_factors

    // device copies (rewards, cells, scratch, control block and codes share
    // one allocation, d_arena; free only that)
    void *d_arena = nullptr;
    void *d_code = nullptr;
    float *d_R32 = nullptr;
    double *d_R64 = nullptr;
    uint8_t *d_cell = nullptr;
    void *d_scratch = nullptr;         // |S| doubles: ping-pong value buffer
    size_t scratch_bytes = 0;
    void *d_q = nullptr;               // plain baseline: |A| x |S| Q values (lazily allocated)
    size_t q_bytes = 0;
    cudaGraphExec_t plain_graph = nullptr;   // plain baseline, fused = 3: one recorded chunk of sweeps
    void *plain_graph_V = nullptr;
    double plain_graph_tol = 0;
    int plain_graph_max_iter = 0;
    int plain_graph_prec = -1;
    cudaGraphExec_t march_graph = nullptr;   // large 3-D value iteration: one recorded chunk of marching sweeps
    void *march_graph_V = nullptr;
    void *march_graph_trace = nullptr;
    double march_graph_tol = 0;
    int march_graph_max_iter = 0;
    bool march_pending = false;              // the last solve ran march_solve
    Ctrl *d_ctrl = nullptr;
    int num_sms = 0;

    // dense CP device data
    float *d_U32 = nullptr;            // factors as float
    double *d_U64 = nullptr;           // factors as double
    void *d_Ubf = nullptr;             // bf16 hi/lo split of the factors (tensor-core path)
    float *d_lam32 = nullptr;
    double *d_lam64 = nullptr;
    void *d_dense_work = nullptr;      // dense chain intermediates
    size_t dense_work_bytes = 0;
    double *d_Vd = nullptr;            // dense FP64 certify: the float values as doubles
    // dense tensor-core path (64^4), allocated on first BF16X3 use
    float *d_RB = nullptr;             // rewards in the pass-B layout
    void *d_T = nullptr;               // per-chain intermediates (bf16 hi/lo pairs)
    float *d_EB = nullptr;             // base expectation per action, pass-B layout
    float *d_Vbase = nullptr;          // base value tensor of the defect correction
    void *d_pi_work = nullptr;         // BF16X3 policy iteration: Q of the current action, best Q, argmax
    void *d_dense_loop = nullptr;      // BF16X3 value iteration: the device-side loop control block
    cudaGraphExec_t dense_graph = nullptr;   // BF16X3 value iteration, recorded once per (V, pi, options)
    void *dense_graph_V = nullptr;
    void *dense_graph_pi = nullptr;
    void *dense_graph_trace = nullptr;
    double dense_graph_tol = 0;
    int dense_graph_max_iter = 0;
    int dense_graph_certify = -1;
    cudaGraphExec_t dense_pi_graph = nullptr;   // BF16X3 policy iteration, recorded once per (V, pi, options)
    void *dense_pi_graph_V = nullptr;
    void *dense_pi_graph_pi = nullptr;
    double dense_pi_graph_eval_tol = 0;
    int dense_pi_graph_rounds = 0;
    int dense_pi_graph_eval_iter = 0;
    int dense_pi_graph_partial = -1;
    cudaGraphExec_t simt_graph = nullptr;       // FP32 / FP64 dense VI or PI, recorded once per (buffers, options)
    void *simt_graph_V = nullptr;
    void *simt_graph_pi = nullptr;
    void *simt_graph_trace = nullptr;
    int simt_graph_pim = -1;
    int simt_graph_prec = -1;
    double simt_graph_tol = 0;
    double simt_graph_eval_tol = 0;
    int simt_graph_max_iter = 0;
    int simt_graph_rounds = 0;
    int simt_graph_eval_iter = 0;
    int simt_graph_partial = -1;
    int *d_tc_err = nullptr;           // error word of the tensor-core kernels
    // barrier-free FP32 solver (flow_solve.cu), allocated on first use
    void *d_flow = nullptr;            // arrival counters + four rings of |S| tagged words
    bool flow_in_arena = false;        // d_flow is part of d_arena (set up by the build)
    unsigned flow_base = 0;            // first tag not written to the rings yet
    bool flow_pending = false;         // a launch whose tags are not accounted for yet
};

// Thread-local error message.
void set_error(const char *fmt, ...);
cpmdp_status cuda_fail(cudaError_t e, const char *what);

#define CPMDP_CUDA(call)                                              \
    do {                                                              \
        cudaError_t e__ = (call);                                     \
        if (e__ != cudaSuccess) return ::cpmdp::cuda_fail(e__, #call); \
    } while (0)

struct SolveOpts {
    double tol;
    int max_iter;
    int certify;
    int fused;
    double eval_tol;
    int max_eval_iter;
    int max_rounds;
    double timeout_s;
    double *trace;
    int partial_eval;
    int inject_stall;
};
SolveOpts resolve_opts(const cpmdp_solve_opts *o, cpmdp_precision prec);

// banded.cu
cpmdp_status banded_backup(const Factors &F, cpmdp_precision prec, const void *Vin, void *Vout,
                           uint8_t *pi, double *res, cudaStream_t st);
cpmdp_status banded_certify(const Factors &F, const float *V, uint8_t *pi, double *res,
                            cudaStream_t st);
cpmdp_status banded_solve(const Factors &F, cpmdp_precision prec, bool policy_iteration, void *V,
                          uint8_t *pi, const SolveOpts &o, cudaStream_t st);
// After the control block of a fused GridWorld solve was read back: account
// for the barrier-free solver's tags (or clear its rings after a failure).
cpmdp_status banded_solve_finished(const Factors &F, const Ctrl &dc, cudaStream_t st);
cpmdp_status banded_plain_vi(const Factors &F, cpmdp_precision prec, void *V, uint8_t *pi,
                             const SolveOpts &o, Ctrl *host_ctrl, cudaStream_t st);

// dense.cu
cpmdp_status dense_backup(const Factors &F, cpmdp_precision prec, const void *Vin, void *Vout,
                          uint8_t *pi, double *res, cudaStream_t st);
cpmdp_status dense_solve(const Factors &F, cpmdp_precision prec, bool policy_iteration, void *V,
                         uint8_t *pi, const SolveOpts &o, Ctrl *host_ctrl, cudaStream_t st);
cpmdp_status dense_prepare(Factors &F);
// dense_tc.cu
bool dense_tc_supported(const Factors &F);
cpmdp_status dense_tc_backup(const Factors &F, const float *Vin, float *Vout, uint8_t *pi, double *res,
                             cudaStream_t st);
cpmdp_status dense_tc_solve(const Factors &F, float *V, uint8_t *pi, const SolveOpts &o, Ctrl *hc, cudaStream_t st);
cpmdp_status dense_tc_policy_iteration(const Factors &F, float *V, uint8_t *pi, const SolveOpts &o, Ctrl *hc,
                                       cudaStream_t st);


// ---------------------------------------------------------------------------
// Graph-driven dense loops (dense_tc.cu, dense.cu): device control block of
// policy iteration, its control kernels, and graph-building helpers.
constexpr size_t kLoopCtlBytes = 256;   // size of the device control block buffer (d_dense_loop)

// Policy-iteration state kept on the device between the graph's kernels.
struct DensePiCtl {
    int e;              // evaluation sweeps of this round
    int cap;            // their limit this round
    int ok;             // this round's evaluation reached eval_tol
    int full;           // evaluations run to eval_tol (no cap)
    int last_rebase;    // evaluation sweep of the last base refresh this round
    int rebases;
    int total;          // sweeps (greedy, evaluation, improvement)
    int rounds;
    int evals;          // evaluation sweeps of all rounds
    int conv;
    int stop;
    int which;          // buffer of the current iterate: 0 = V, 1 = scratch
    double res;         // last evaluation residual
    double hist[8];     // this round's evaluation residuals (sweep j at j mod 8)
};

__global__ void pi_init_kernel(DensePiCtl *c, const int *err, int max_rounds, cudaGraphConditionalHandle h_round);
__global__ void pi_round_start_kernel(DensePiCtl *c, int partial_eval, int max_eval_iter,
                                      cudaGraphConditionalHandle h_eval);
__global__ void pi_eval_ctl_kernel(DensePiCtl *c, unsigned long long *res_slot, const int *err, double eval_tol,
                                   int step, int can_rebase, cudaGraphConditionalHandle h_eval,
                                   cudaGraphConditionalHandle h_rebase, cudaGraphConditionalHandle h_second);
__global__ void pi_after_eval_kernel(const DensePiCtl *c, cudaGraphConditionalHandle h_odd);
__global__ void pi_round_end_kernel(DensePiCtl *c, const unsigned *changed, const int *err, int max_rounds,
                                    cudaGraphConditionalHandle h_round);
// Nodes of g that no other node depends on.
cudaError_t graph_leaves(cudaGraph_t g, std::vector<cudaGraphNode_t> &out);
// Add a conditional node (IF or WHILE) after `deps` in g; returns its body.
cudaError_t add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, cudaGraphNode_t *node, cudaGraph_t *body);

}  // namespace cpmdp

struct cpmdp_factors {
    cpmdp::Factors f;
};
