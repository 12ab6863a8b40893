/*
 * cpmdp.h -- C ABI of the GB300 CP-MDP library (libcpmdp.so).
 *
 * CP-MDP (Kuinchtner, Sales and Meneguzzi, AAAI 2021) solves a Markov
 * decision process <S, A, P, R, gamma> (background section, "Markov Decision
 * Process") whose states are the tuples of an n-dimensional grid
 * (Definitions 1 and 2) and whose transition model P is held as CANDECOMP-
 * PARAFAC components: per action, a sum of rank-1 terms, each an outer
 * product of small per-dimension factor matrices (background section,
 * "Tensor Decomposition", Fig. 1; Definition 3). The library computes the
 * Bellman backup of Eq. 1,
 *     V'(s) = R(s) + gamma * max_a sum_{s'} P(s'|s,a) V(s'),
 * without ever expanding P to an |S| x |S| matrix, and runs value iteration
 * and policy iteration (background section) entirely on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - States are flat indices in C order over (N_1, ..., N_D): the last
 *   dimension varies fastest (Definition 2). Every per-state array (cell
 *   codes, rewards, values, policies) uses this layout, densely packed.
 * - GridWorld actions (scenario section: two actions per axis, |A| = 2D):
 *   action a = 2*d + (sigma > 0) moves by sigma = -1 or +1 along dimension
 *   d (d = 0 is the slowest dimension). In 2-D: N, S on the first axis and
 *   W, E on the second.
 * - Slip model: the intended move happens with probability p_success; the
 *   remaining mass is split evenly over the 2(D-1) perpendicular unit
 *   moves (for D = 1 the agent stays put instead). A move that leaves the
 *   grid or enters an obstacle leaves the agent in place.
 * - Cell codes: 0 free, 1 obstacle (never entered, not a state: value 0,
 *   policy 255), 2 terminal (the interaction ends: V(t) = R(t), policy 255).
 * - Values are float (CPMDP_F32, CPMDP_BF16X3) or double (CPMDP_F64), in
 *   caller-owned DEVICE memory. Policies are uint8 action indices in
 *   caller-owned device memory, 255 where no action applies.
 * - Device buffers passed in must be at least 16-byte aligned for the
 *   vectorised kernels (PyTorch allocations are); other alignments are
 *   accepted and take a scalar path.
 * - Every call that takes a stream enqueues its kernels on that stream
 *   (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *   Calls that fill a cpmdp_result synchronise with the stream before they
 *   return. Two calls that use the same cpmdp_factors object must not run
 *   concurrently: the object owns the scratch buffers of the solvers.
 * - No call throws or aborts. Each returns a cpmdp_status; on failure
 *   cpmdp_last_error() gives a message (per host thread).
 */
#ifndef CPMDP_H
#define CPMDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPMDP_MAX_DIM 9

typedef enum {
    CPMDP_OK = 0,
    CPMDP_EINVAL = 1,    /* invalid argument: nothing was enqueued */
    CPMDP_ENOMEM = 2,    /* host or device allocation failed */
    CPMDP_ECUDA = 3,     /* a CUDA runtime call failed (message has details) */
    CPMDP_ENOCONV = 4,   /* max_iter sweeps done without reaching tol; outputs hold the last iterate */
    CPMDP_ETIMEOUT = 5   /* a device-side wait gave up after timeout_s; outputs undefined */
} cpmdp_status;

typedef enum {
    CPMDP_F32 = 0,       /* float values, float arithmetic */
    CPMDP_F64 = 1,       /* double values, double arithmetic */
    CPMDP_BF16X3 = 2     /* dense CP only: float values, mode products as three bf16 tensor-core products */
} cpmdp_precision;

typedef enum {
    CPMDP_GRIDWORLD = 0, /* banded factors from the slip model above */
    CPMDP_DENSE_CP = 1   /* general dense rank-R factors */
} cpmdp_kind;

enum { CPMDP_CELL_FREE = 0, CPMDP_CELL_OBSTACLE = 1, CPMDP_CELL_TERMINAL = 2 };

/* Which solver ran (cpmdp_result.solver). */
typedef enum {
    CPMDP_SOLVER_PLAIN = 0,         /* plain unfused baseline (fused = 0) */
    CPMDP_SOLVER_GRID_BARRIER = 1,  /* fused GridWorld solver, one grid barrier per sweep */
    CPMDP_SOLVER_BARRIER_FREE = 2,  /* fused FP32 GridWorld solver without a barrier in its sweep loop */
    CPMDP_SOLVER_DENSE = 3,         /* dense CP solver */
    CPMDP_SOLVER_BATCH = 4,         /* batched value iteration */
    CPMDP_SOLVER_MARCH_GRAPH = 5,   /* FP32 value iteration of a 3-D grid of 2^23+ states: plane-marching
                                       sweeps replayed from a CUDA graph, stopping rule taken on the device */
    CPMDP_SOLVER_BATCH_RESIDENT = 6 /* batched value iteration with every instance held in the shared memory
                                       of one CTA or of one thread-block cluster for its whole solve */
} cpmdp_solver;

/*
 * The MDP tuple <S, A, P, R, gamma> (background section).
 *   ndim, shape[0..ndim-1]  S = N_1 x ... x N_D (Definitions 1-2), each N_d >= 1,
 *                           1 <= ndim <= CPMDP_MAX_DIM, |S| < 2^31.
 *   nactions                GridWorld: must equal 2*ndim. Dense: 1..64.
 *   kind                    cpmdp_kind.
 *   p_success               GridWorld: probability of the intended move, in [0, 1].
 *   cell                    host, |S| codes (see above); NULL = all free. Dense: must be NULL.
 *   reward                  host, |S| state rewards R(s) (finite).
 *   rank                    dense: R >= 1 terms per action (GridWorld: ignored).
 *   factors                 dense, host: U[a][r][d] as N_d x N_d row-major blocks,
 *                           packed in the order a, r, d; U[a][r][d][i][j] is the
 *                           factor of moving coordinate d from i to j. Rows must be
 *                           non-negative; P_a is row-stochastic when every row sums
 *                           to 1 and lambda[a][.] sums to 1 (checked to 1e-9).
 *   lambda                  dense, host: [A][R] rank weights.
 *   gamma                   discount in [0, 1]; gamma == 1 needs terminals reachable
 *                           (value iteration then stops only through tol or max_iter).
 * The library copies everything it needs; the caller may free these
 * buffers after cpmdp_build_factors returns.
 */
typedef struct {
    int32_t ndim;
    int64_t shape[CPMDP_MAX_DIM];
    int32_t nactions;
    int32_t kind;
    double p_success;
    const uint8_t *cell;
    const double *reward;
    int32_t rank;
    const double *factors;
    const double *lambda;
    double gamma;
} cpmdp_problem;

/* Opaque, library-owned transition model plus its device copies and solver scratch. */
typedef struct cpmdp_factors cpmdp_factors;

typedef struct {
    double tol;              /* stop when max |V' - V| over non-obstacle states < tol (default 1e-6) */
    int32_t max_iter;        /* sweep limit (default 1000, the paper's maxIter) */
    int32_t certify;         /* 1 (default): after F32 solves, one FP64 sweep of the result gives the
                                certified residual and the policy (FP64 argmax) */
    int32_t fused;           /* 1 (default): fused device-resident solver; GridWorlds one block covers
                                (at most 256 segments of the vector width) run in a single block with
                                the values in shared memory (same values and sweep counts as the
                                grid-barrier solver); FP32 GridWorld solves of
                                1 to 3 dimensions whose rows are a multiple of 4 states and that fit
                                one co-resident grid at one thread per column of 1, 2 or 4 segments of
                                4 states run barrier-free (sweeps synchronised through sweep-tagged
                                values, the stopping rule checked three sweeps late; same values and
                                sweep counts); FP32 value iteration of 3-D grids of 2^23 states or
                                more runs plane-marching sweeps from a replayed CUDA graph with the
                                stopping rule on the device (same values and sweep counts); the rest
                                with a grid barrier per sweep; 2: always the grid-barrier solver; 0: the
                                plain unfused FP32/FP64 baseline (one kernel per action, separate max
                                and residual kernels, residual checked on the host every sweep); 3: the
                                same plain kernels with the stopping rule taken on the device (a
                                one-thread check kernel after each sweep raises a flag on which every
                                later kernel returns at once), 32 sweeps recorded once into a CUDA
                                graph that is replayed until the flag is up (the host reads it once
                                per 32 sweeps); 0 and 3 run value iteration only. Batches
                                (cpmdp_batch_value_iteration): 1 shared-memory-resident solver,
                                4 batched kernel with the barrier-free tail, 2 batched kernel only */
    double eval_tol;         /* policy iteration: evaluation stops below this residual
                                (default: tol for F32, 1e-10 for F64) */
    int32_t max_eval_iter;   /* policy iteration: evaluation sweep limit per round (default 100000) */
    int32_t max_rounds;      /* policy iteration: improvement round limit (default 1000) */
    double timeout_s;        /* limit of every device-side wait (default 2 s) */
    double *trace;           /* optional device buffer of max_iter doubles: residual of each sweep
                                (value iteration, fused path only; the barrier-free solver zeroes it
                                first and also fills the entries of its two dropped sweeps) */
    int32_t partial_eval;    /* policy iteration (default -1: 2 on GridWorld models, 4 on dense ones,
                                the caps measured fastest; other values below -1 are EINVAL):
                                while the policy keeps changing, each
                                round's evaluation runs exactly this many sweeps (modified policy
                                iteration); once an improvement changes no action after such a
                                capped evaluation, every later round evaluates to eval_tol. The
                                solve stops when an improvement changes no action and its own
                                values are within eval_tol of its input. 0: every round evaluates
                                to eval_tol. Dense models take the same caps with an improvement
                                that writes no values: they stop after an evaluation to eval_tol
                                whose improvement changes no action */
    int32_t inject_stall;    /* testing aid (default 0): 1 makes one block of the fused GridWorld
                                solver leave at once (without arriving at its first grid barrier, or,
                                barrier-free, without publishing its values), so the other blocks'
                                bounded waits run out after timeout_s and the call returns
                                CPMDP_ETIMEOUT; the device stays usable */
} cpmdp_solve_opts;

typedef struct {
    int32_t status;              /* cpmdp_status of the solve */
    int32_t iterations;          /* sweeps: VI backups, or PI evaluation + improvement sweeps */
    int32_t rounds;              /* policy iteration improvement rounds (0 for VI) */
    int32_t eval_sweeps;         /* policy iteration evaluation sweeps (0 for VI); BF16X3 value
                                    iteration: the FP64 certifying sweeps it took */
    double residual;             /* last max |V' - V| in working precision */
    double certified_residual;   /* FP64 max |T(V) - V| of the returned V (-1 if not computed) */
    double error_bound;          /* certified_residual / (1 - gamma): bound on max |V - V*| (-1 if n/a) */
    int64_t backups;             /* state-action backups done: |S|*|A| per VI sweep, |S| per evaluation sweep */
    double elapsed_ms;           /* device time of the solve, CUDA events on the stream */
    int32_t solver;              /* cpmdp_solver: which solver ran */
    int32_t tail_from;           /* batches: launch-wide sweep after which the running instances went on
                                    barrier-free, each at its own pace (0: the batched kernel ran to the end) */
} cpmdp_result;

/* Fill *opts with the defaults listed above. */
void cpmdp_default_opts(cpmdp_solve_opts *opts);

/*
 * Validate the problem and build its CP factors (background section, Fig. 1;
 * Definition 3): GridWorld -> per action the 2D-1 rank-1 terms (intended
 * move, perpendicular slips; 2 terms for D = 1) with banded shift/identity
 * factors, plus the obstacle and terminal correction, encoded per state;
 * dense -> the given factors. Copies rewards, codes and factors to device
 * `device` and allocates the solvers' scratch there (about 8 bytes per
 * state; dense adds 2 value tensors). device = -1 builds a host-only object
 * usable by cpmdp_factors_info and cpmdp_components only.
 * On success *out owns everything; release it with cpmdp_free_factors.
 * Errors: EINVAL (problem invalid), ENOMEM, ECUDA.
 */
cpmdp_status cpmdp_build_factors(const cpmdp_problem *problem, int device, cpmdp_factors **out);

/* Release a factors object and its device memory (NULL is ignored). */
void cpmdp_free_factors(cpmdp_factors *factors);

/* Sizes of a built model. Any output pointer may be NULL. */
cpmdp_status cpmdp_factors_info(const cpmdp_factors *factors, int64_t *nstates, int32_t *nactions,
                                int32_t *rank, int32_t *ndim);

/*
 * Definition 3, for one (state, action): the successor states s' with
 * P(s'|s,a) > 0 and their probabilities, expanded on the host from the
 * factors (successors in increasing index order, duplicates merged).
 * Writes up to `cap` entries to next[] / prob[] and the full count to
 * *count. Obstacle and terminal states have no components (count 0).
 * GridWorld only (dense models: EINVAL). Host memory only.
 */
cpmdp_status cpmdp_components(const cpmdp_factors *factors, int64_t state, int32_t action,
                              int64_t *next, double *prob, int32_t cap, int32_t *count);

/*
 * One Bellman backup, Eq. 1, fused: E_a[V] for every action from the CP
 * factors, + R, x gamma, max/argmax over actions, and the infinity-norm
 * residual.
 *   V_in, V_out     device, |S| values (float or double per precision); may not alias.
 *   policy_out      device, |S| uint8 argmax (lowest action on exact ties), or NULL.
 *   residual_out    device, one double: max |V_out - V_in| over non-obstacle states, or NULL.
 * Asynchronous on `stream`. Errors: EINVAL, ECUDA.
 */
cpmdp_status cpmdp_bellman_backup(const cpmdp_factors *factors, cpmdp_precision precision,
                                  const void *V_in, void *V_out, uint8_t *policy_out,
                                  double *residual_out, void *stream);

/*
 * Value iteration (background section): from V (device, in: warm start or
 * zeros, out: the last iterate), repeat the fused backup until the residual
 * falls below opts->tol or opts->max_iter sweeps; the loop, its residual
 * test and the buffer swaps stay on the device (one persistent launch).
 * policy_out (device, |S|, may be NULL) receives the greedy policy of the
 * returned V (FP64 argmax when certify is on). opts may be NULL (defaults);
 * info may be NULL. Synchronises with `stream` before returning.
 * BF16X3 (dense models) with certify on: the working FP32 residual of float
 * iterates cannot resolve differences below a few units in the last place
 * of the largest |V|, so once it is below tol the solve runs
 * ceil(ln 2 / ln(1/gamma)) more sweeps and then an FP64 backup; it repeats
 * that until the FP64 residual max |T(V) - V| is below tol, so the returned
 * V meets the stopping rule in FP64 (info->eval_sweeps = FP64 sweeps taken).
 * Errors: EINVAL, ECUDA, ENOCONV (max_iter reached), ETIMEOUT.
 */
cpmdp_status cpmdp_value_iteration(const cpmdp_factors *factors, cpmdp_precision precision,
                                   void *V, uint8_t *policy_out, const cpmdp_solve_opts *opts,
                                   cpmdp_result *info, void *stream);

/*
 * Policy iteration (background section): start from the greedy policy of
 * the input V (device, in/out), then alternate evaluation of the fixed
 * policy (backup sweeps without the max, until opts->eval_tol or the
 * partial_eval cap) and greedy improvement (an action changes only when
 * another beats it by more than 1e-6 (F32) or 1e-12 (F64) times 1 + |Q|).
 * GridWorld models: the improvement sweep also writes the new policy's
 * first evaluation step (Q of the action kept or taken, as in modified
 * policy iteration), and the solve stops when it changes no action and
 * moves no value by eval_tol or more. V receives the value of the final
 * policy, policy (device, |S|, not NULL) the final policy. Synchronises
 * with `stream` before returning.
 * BF16X3 (dense models, 64^4): evaluation sweeps are the tensor-core backup
 * with each state's own action (defect correction against an FP32 base, as
 * in value iteration); an improvement takes an evaluation-mode sweep, a max
 * sweep and the keep-margin compare; with certify on, one FP64 backup of the
 * result gives the certified residual max |T(V) - V| (policy unchanged).
 * Errors: EINVAL, ECUDA, ENOCONV (round or evaluation limit), ETIMEOUT.
 */
cpmdp_status cpmdp_policy_iteration(const cpmdp_factors *factors, cpmdp_precision precision,
                                    void *V, uint8_t *policy, const cpmdp_solve_opts *opts,
                                    cpmdp_result *info, void *stream);

/*
 * Value iteration that allocates nothing (the paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * running under an arena or pool that owns all device memory of the process,
 * or loops that forbid allocation after start-up).
 *   ndim, shape      1 <= ndim <= 3, |S| = prod(shape) <= 2,097,152 states; larger
 *                    grids are rejected with CPMDP_EINVAL.
 *   p_success, gamma the GridWorld slip model and discount as in cpmdp_problem.
 *   cell             device, |S| cell codes (0 free, 1 obstacle, 2 terminal), or NULL.
 *   reward           device, |S| float state rewards.
 *   V                device, |S| floats: start values in, last iterate out.
 *   tol, max_iter    stopping rule of cpmdp_value_iteration (FP32 arithmetic).
 *   iterations_out, residual_out  host, may be NULL: sweeps done, last residual.
 * All scratch (second value buffer, move codes, barrier words: about 10 MiB)
 * is one static device array that every GPU loading this library keeps until
 * the process exits. All calls share it: calls that overlap on the GPU race,
 * so serialise them. The first call on each device looks up the array's
 * address and loads its module; make it before any stream capture. Device
 * waits give up after 2 s (CPMDP_ETIMEOUT). Synchronises with `stream`.
 */
cpmdp_status cpmdp_value_iteration_static(int32_t ndim, const int64_t *shape, double p_success,
                                          double gamma, const uint8_t *cell, const float *reward,
                                          float *V, double tol, int32_t max_iter,
                                          int32_t *iterations_out, double *residual_out, void *stream);

/*
 * Batched value iteration: many independent GridWorld MDPs (each its own
 * tuple <S, A, P, R, gamma>, 1 to 3 dimensions) solved by one persistent
 * launch in which every instance stops on its own residual.
 */
typedef struct cpmdp_batch cpmdp_batch;

/*
 * Build a batch from `count` GridWorld problems (validated and factored as
 * by cpmdp_build_factors) on CUDA device `device`. Instance i's states
 * occupy [offsets[i], offsets[i] + |S_i|) of the packed value array; each
 * instance starts on a multiple of 4 states (padding between instances is
 * never read or written). Errors: EINVAL (an instance is invalid: the
 * message names it), ENOMEM, ECUDA.
 */
cpmdp_status cpmdp_batch_build(const cpmdp_problem *problems, int32_t count, int device, cpmdp_batch **out);

/* Release a batch (NULL is ignored). */
void cpmdp_batch_free(cpmdp_batch *batch);

/* count, total packed states, and offsets[count + 1] (host; any may be NULL). */
cpmdp_status cpmdp_batch_info(const cpmdp_batch *batch, int32_t *count, int64_t *total_states, int64_t *offsets);

/*
 * FP32 value iteration of every instance of the batch (fused backup of
 * cpmdp_value_iteration, per-instance stopping at opts->tol or
 * opts->max_iter). V: device, packed values (start in, result out), 16-byte
 * aligned. iterations_out / residual_out: host arrays of `count` (may be
 * NULL): sweeps and last residual per instance. info (may be NULL):
 * iterations = most sweeps of any instance, backups = sum over instances,
 * elapsed_ms, rounds = 1 when the solve was replayed from a CUDA graph,
 * solver = CPMDP_SOLVER_BATCH_RESIDENT or CPMDP_SOLVER_BATCH.
 * opts->fused selects the solver (same sweeps, values and residuals, bit for
 * bit, whichever runs):
 *   1 (default) every instance held in shared memory for its whole solve,
 *     one persistent launch of 1024-thread CTAs (up to 27,648 states per
 *     CTA): small instances packed several to a CTA, larger ones cut into
 *     slices over the CTAs of a thread-block cluster (2, 4 or 8, the
 *     smallest that every instance fits) that read the slices next to their
 *     part through distributed shared memory. The work is scheduled from
 *     the previous solve's sweep counts of each instance (the first solve of
 *     a batch from a gamma-based guess). Batches with an instance that does
 *     not fit eight CTAs run as with fused = 4.
 *   4 one cooperative persistent launch over all instances (one grid barrier
 *     per sweep); once the instances still running fit one co-resident grid
 *     (one warp per 128 states) they continue without the grid barrier, each
 *     instance at its own pace (info->tail_from tells when). The first call
 *     tunes block and tile sizes on the batch (a few sweeps on a temporary
 *     buffer).
 *   2 as 4, without the barrier-free tail.
 * Each solve is recorded once into a CUDA graph, replayed by later calls
 * with the same V, stream and options. Synchronises with `stream`.
 * Errors: EINVAL, ECUDA, ENOCONV (some instance hit max_iter), ETIMEOUT
 * (fused = 2 / 4: a device-side wait ran out; the resident solver waits only
 * at hardware CTA and cluster barriers).
 */
cpmdp_status cpmdp_batch_value_iteration(cpmdp_batch *batch, float *V, const cpmdp_solve_opts *opts,
                                         int32_t *iterations_out, double *residual_out, cpmdp_result *info,
                                         void *stream);

/*
 * One FP64 backup (Eq. 1 in double arithmetic, FP64 rewards and weights) of
 * every instance of a packed float value array V (device, 16-byte aligned),
 * for instance the result of cpmdp_batch_value_iteration: the greedy policy
 * of the returned values (background section: value iteration ends with
 * the greedy policy) and per instance the certified residual
 * max |T(V) - V| over its non-obstacle states, which bounds the distance
 * to V* by certified / (1 - gamma_i).
 *   policy_out     device, packed like V (uint8, FP64 argmax, lowest action
 *                  on exact ties, 255 on obstacles and terminals), or NULL;
 *                  the padding between instances is not written.
 *   certified_out  host array of `count` doubles, or NULL.
 * Synchronises with `stream`. Errors: EINVAL, ECUDA.
 */
cpmdp_status cpmdp_batch_certify(const cpmdp_batch *batch, const float *V, uint8_t *policy_out,
                                 double *certified_out, void *stream);

/*
 * Learned warm start (no counterpart in the paper's method; it only changes
 * where value iteration starts). A fully convolutional 3-D network works on
 * a grid coarsened by 4 in every dimension. Activations are channels-last
 * bf16 arrays [n][z][y][x][64] (as uint16), weights per layer FP32
 * W[27][64][64] (tap, out, in; tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) for
 * offsets dilation * (dz, dy, dx)), "same" zero padding. All device memory
 * caller-owned; all calls asynchronous on `stream`; errors EINVAL / ECUDA.
 *
 * cpmdp_ws_features: coarse features of batch instances first..first+count-1
 *   (3-D, one shape): per 4x4x4 cell the mean reward of its
 *   non-obstacle states, its obstacle fraction, its largest terminal reward
 *   (0 if none), -log(1 - gamma) / 5; channels 4..63 zero.
 * cpmdp_ws_coarse_vi: value iteration of a coarsened copy of every instance
 *   (the same Eq. 1 backup on the coarse grid; one CTA per instance, in
 *   shared memory, at most 8192 coarse cells): a coarse cell is an obstacle
 *   when at least half of its states are, else a terminal of value max R(t)
 *   when it holds terminals, else free with reward (mean fine reward of its
 *   free states) x (1 + gamma + gamma^2 + gamma^3); discount gamma^4, the
 *   instance's slip model. Jacobi sweeps from zero until max |dV| < tol or
 *   max_sweeps. Writes coarse_v (float [count][cells]) and, when feat is not
 *   NULL, its bf16 copy into feature channel 4.
 * cpmdp_ws_targets: per coarse cell the mean of V over its non-obstacle
 *   states minus base (float [count][cells], NULL = 0), and a mask (1 if the
 *   cell has any non-obstacle state).
 * cpmdp_ws_upsample: V (packed batch layout) = coarse + base (base NULL = 0)
 *   at the cell centres, interpolated trilinearly to every free state
 *   (clamped to the outermost centres); R(t) on terminals, 0 on obstacles.
 * cpmdp_ws_fine_loss_grad: the loss of a coarse estimate on the full grid.
 *   With Vh = the upsampling of pred + base (as cpmdp_ws_upsample) and
 *   n = count * states per instance: r(s) = Vh(s) - V_target(s) on free
 *   states, 0 on terminals and obstacles (written to resid, float
 *   [count][states per instance], caller-owned scratch); *loss += sum r^2 / n
 *   (loss device float, or NULL); dy channel 0 (bf16 [count][cells][64]) =
 *   dloss/dpred = 2/n times the transpose of the interpolation applied to r,
 *   channels 1..63 zero. V_target is in the packed batch layout.
 */
cpmdp_status cpmdp_ws_features(const cpmdp_batch *batch, int32_t first, int32_t count, uint16_t *feat, void *stream);
cpmdp_status cpmdp_ws_coarse_vi(const cpmdp_batch *batch, int32_t first, int32_t count, float tol, int32_t max_sweeps,
                                float *coarse_v, uint16_t *feat, void *stream);
cpmdp_status cpmdp_ws_targets(const cpmdp_batch *batch, const float *V, int32_t first, int32_t count, const float *base,
                              float *target, float *mask, void *stream);
cpmdp_status cpmdp_ws_upsample(const cpmdp_batch *batch, const float *coarse, const float *base, int32_t first,
                               int32_t count, float *V, void *stream);
cpmdp_status cpmdp_ws_fine_loss_grad(const cpmdp_batch *batch, const float *V_target, int32_t first, int32_t count,
                                     const float *pred, const float *base, float *resid, uint16_t *dy, float *loss,
                                     void *stream);
/* y = conv(x, W) + b (ReLU if relu); wf = the forward weight tiles written by cpmdp_ws_cast_weights;
 * y0 (nullable) gets channel 0 in FP32. Runs on the tcgen05 tensor cores (bf16 operands, FP32
 * accumulation in TMEM): persistent CTAs, tiles of 128 voxels x 64 channels, 27 taps x K = 64,
 * inputs brought in by tensor copies (zero fill outside the grid). x and y 16-byte aligned; x is read
 * through a tensor map, so the call fails with ECUDA where the driver offers none. Errors: EINVAL
 * (dimensions, null pointers), ECUDA; a tensor-core wait that runs out is reported by
 * cpmdp_ws_sync. */
cpmdp_status cpmdp_conv3d_forward(const uint16_t *x, const uint16_t *wf, const float *bias, uint16_t *y, float *y0,
                                  int32_t n, int32_t z, int32_t y_, int32_t x_, int32_t dilation, int32_t relu,
                                  void *stream);
/* dx = conv^T(dy, W) times (act_in > 0) when act_in is given; wb = the data-gradient weight tiles
 * written by cpmdp_ws_cast_weights. Tensor cores, as the forward call. */
cpmdp_status cpmdp_conv3d_backward_data(const uint16_t *dy, const uint16_t *wb, const uint16_t *act_in, uint16_t *dx,
                                        int32_t n, int32_t z, int32_t y_, int32_t x_, int32_t dilation, void *stream);
/* dw += dL/dW (FP32 [27][64][64]), db += dL/db (FP32 [64], nullable). */
cpmdp_status cpmdp_conv3d_backward_weight(const uint16_t *x, const uint16_t *dy, float *dw, float *db, int32_t n,
                                          int32_t z, int32_t y_, int32_t x_, int32_t dilation, void *stream);
/* Mean over nvox cells of mask (pred - target)^2: dy channel 0 = its gradient, other channels 0; *loss += value. */
cpmdp_status cpmdp_ws_loss_grad(const float *pred, const float *target, const float *mask, int32_t nvox, uint16_t *dy,
                                float *loss, void *stream);
/* One Adam step (bias-corrected, step >= 1) on n FP32 parameters. */
cpmdp_status cpmdp_adam_step(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                             float beta2, float eps, int32_t step, void *stream);
/* FP32 W[layers][27][64][64] -> bf16 weight tiles, per layer and tap 64 x 64 bf16 (8 KB) in the
 * tensor cores' shared-memory layout (128-byte rows, 16-byte chunk c of row r stored at chunk
 * c ^ (r % 8)): wf row = out, column = in (forward); wb row = in, column = out (data gradient).
 * wf and wb each hold layers * 27 * 4096 bf16. */
cpmdp_status cpmdp_ws_cast_weights(const float *w, uint16_t *wf, uint16_t *wb, int32_t layers, void *stream);
/* Waits for the work queued on `stream`; ETIMEOUT if a bounded tensor-core wait in a convolution
 * ran out since the last call (the error is cleared; outputs of that call are not valid). */
cpmdp_status cpmdp_ws_sync(void *stream);

/* Message of the last failed call on this host thread ("" if none). */
const char *cpmdp_last_error(void);

/* Library version string. */
const char *cpmdp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CPMDP_H */
