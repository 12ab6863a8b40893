// Batched value iteration with every instance resident in shared memory.
//
// Each GridWorld of a batch (its own tuple <S, A, P, R, gamma>, background
// section) is held, for its whole solve, in the shared memory of one CTA or
// of the CTAs of one thread-block cluster: its value tensor is double
// buffered there (Jacobi sweeps of Eq. 1 read one buffer and write the
// other), so a sweep touches global memory only for the rewards and codes
// (a padded copy, L2-resident while the instance runs) and the values never
// leave the chip between the first load and the final store.
//
// Layout in shared memory: rows of the last dimension padded to a multiple
// of 4 states (nxp), slices of the leading dimension (3-D: y-x planes; 2-D:
// rows; 1-D: the one row) stored one after another, parts rounded up to
// chunks of 128 states (one warp's 32 four-state segments). A CTA holds up
// to kResCap states.
//
//  * A solo bundle is a set of whole instances packed into one CTA; they
//    sweep in lockstep (one __syncthreads per sweep), each stopping on its
//    own residual (its chunks are skipped from then on).
//  * A cluster bundle is one instance cut into C parts of consecutive
//    slices, one per CTA of a cluster of C (or two instances of C / 2 parts
//    each); the slices adjacent to a part are read from the neighbouring
//    CTA's buffer through distributed shared memory, each CTA's residual of
//    a sweep goes to its instance's slot in every CTA of the cluster, and
//    the cluster barrier (hardware, release / acquire) separates the sweeps.
//
// The backup of a 4-state segment resolves blocked moves with
// Segment::neighbours and takes max_a E_a with vi_best_e, the arithmetic of
// the batched kernel's value iteration; terminals and obstacles take a
// per-state multiplier of max_a E_a (0 on them) instead of selects. Values,
// sweep counts and residuals equal the batched kernel's, bit for bit.
// Stopping: an instance stops after the first sweep
// whose residual is below tol (or after max_iter sweeps); per instance the
// residual of sweep q goes to slot q % 3 (slot q + 1 is cleared during
// sweep q, after every reader of its previous use passed the barrier of
// sweep q - 1), and a stopped instance's slots are never written again, so
// it reads as stopped from then on.
//
// The launch is persistent: clusters take cluster bundles from a queue
// (atomic counter), then every CTA takes solo bundles from a second queue.
// Nothing waits on another cluster; the only waits are the hardware CTA and
// cluster barriers, which every thread of every CTA of a cluster reaches
// the same number of times (every decision that ends a loop is taken from
// values all of them read after the same barrier).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "banded_common.cuh"
#include "batch_internal.h"

namespace cpmdp {

constexpr int kResChunk = 128;                       // states of one warp's 32 segments
constexpr int kResChunks = 216;                      // chunks per CTA
constexpr int kResCap = kResChunk * kResChunks;      // 27,648 states per CTA (a 48^3 instance in 4 CTAs)
constexpr int kResMaxParts = 64;                     // instances of one solo bundle
constexpr int kResThreads = 1024;
constexpr int kResWarps = kResThreads / 32;

struct ResShared {
    ResPart part[kResMaxParts];
    unsigned slot[kResMaxParts][3];   // residual bits of sweep q in slot q % 3 (cluster: slot[b] of instance b)
    int done[kResMaxParts];           // sweeps done (negative: stopped at max_iter)
    unsigned lmax[2];                 // cluster bundles: this CTA's residual of the sweep, by parity
    int job;
    uint8_t chunk_part[kResChunks];
};
constexpr size_t kResSmem = sizeof(float) * 2 * kResCap + sizeof(ResShared);

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned cluster_map(unsigned addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void ld_cluster4(unsigned addr, float (&v)[4]) {
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(addr)
                 : "memory");
}

__device__ __forceinline__ unsigned ld_cluster_u32(unsigned addr) {
    unsigned v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void red_cluster_max(unsigned addr, unsigned v) {
    asm volatile("red.shared::cluster.max.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Float residual bits below tol: the host passes the bits of the largest
// float f with (double) f < tol, so the test is one unsigned compare (a NaN
// is never below).
__device__ __forceinline__ bool res_below(unsigned bits, unsigned tol_bits) { return bits <= tol_bits; }

// What a segment's backup needs of its part, in registers (loaded once per
// part, not once per segment: the stores of the sweep go to shared memory,
// which the compiler cannot tell apart from the part table).
struct SegGeo {
    long long poff;
    int base, P, nslp, nxp;
    unsigned prev_addr, next_addr;   // 0: the instance ends there (a wall)
    float wm, wp, wst, g;
    __device__ __forceinline__ void load(const ResPart &pt) {
        poff = pt.poff;
        base = pt.base;
        P = pt.P;
        nslp = pt.nsl * pt.P;
        nxp = pt.nxp;
        prev_addr = pt.has_prev ? pt.prev_addr : 0u;
        next_addr = pt.has_next ? pt.next_addr : 0u;
        wm = pt.wm;
        wp = pt.wp;
        wst = pt.wst;
        g = pt.g;
    }
};

// Backup of the segment of part pt at shared-memory state o (4 states,
// 16-byte aligned), from buffer cur into nxt. Returns the segment's
// residual. Terminals and obstacles need no select: the padded copies hold,
// per state, R (0 on obstacles) and the multiplier of the expectation (gamma,
// 0 on terminals, obstacles and padding), so V' = R + g_s max_a E_a is R on
// a terminal and 0 on an obstacle; obstacle values are loaded as 0, so an
// obstacle's |V' - V| is 0 (no state reads an obstacle's value: a move into
// one is blocked). Free states get vi_state's arithmetic exactly.
template <int D>
__device__ __forceinline__ float res_segment(const SegGeo &pt, const float *cur, float *nxt, unsigned bufoff,
                                             const ResArgs &a, int o) {
    const int rel = o - pt.base;
    const int nslp = pt.nslp;
    Segment<float, float, D, 4> sg;
    float gs[4];
    if (rel < nslp) {
        load_pack<uint8_t, 4>(a.codep + pt.poff + rel, sg.code);
        load_pack<float, 4>(a.Rp + pt.poff + rel, sg.r);
        load_pack<float, 4>(a.Gp + pt.poff + rel, gs);
    } else {
        // padding up to the part's last chunk: every move blocked, value 0
#pragma unroll
        for (int k = 0; k < 4; k++) { sg.code[k] = 0xFF; sg.r[k] = 0.f; gs[k] = 0.f; }
    }
    load_pack<float, 4>(cur + o, sg.vs);
    sg.halo_m = cur[o > 0 ? o - 1 : 0];
    sg.halo_p = cur[o + 4 < kResCap ? o + 4 : kResCap - 1];
    if (D >= 2) {
        // leading dimension: the slice before / after, from the neighbouring
        // CTA's buffer at the part's first / last slice (a wall where the
        // instance ends: the code blocks the move, any value will do)
        const int P = pt.P;
        if (rel < P) {
            if (pt.prev_addr) ld_cluster4(pt.prev_addr + bufoff + 4u * (unsigned)rel, sg.rows[0]);
            else load_pack<float, 4>(cur + o, sg.rows[0]);
        } else {
            load_pack<float, 4>(cur + o - P, sg.rows[0]);
        }
        const int lastrel = rel - nslp + P;
        if (lastrel >= 0) {
            if (pt.next_addr) ld_cluster4(pt.next_addr + bufoff + 4u * (unsigned)lastrel, sg.rows[1]);
            else load_pack<float, 4>(cur + o, sg.rows[1]);
        } else {
            load_pack<float, 4>(cur + o + P, sg.rows[1]);
        }
    }
    if (D >= 3) {
        // rows of the same slice: clamped into the buffer (outside the slice
        // only where the move is blocked)
        const int m = o - pt.nxp, p = o + pt.nxp;
        load_pack<float, 4>(cur + (m < 0 ? 0 : m), sg.rows[2]);
        load_pack<float, 4>(cur + (p > kResCap - 4 ? kResCap - 4 : p), sg.rows[3]);
    }
    float self[4], nb[2 * D][4];
    sg.neighbours(self, nb);
    float out[4], res = 0.f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float nbk[2 * D];
#pragma unroll
        for (int j = 0; j < 2 * D; j++) nbk[j] = nb[j][k];
        const float v = sg.r[k] + gs[k] * vi_best_e<float, D>(self[k], nbk, pt.wm, pt.wp, pt.wst);
        out[k] = v;
        res = fmaxf(res, fabsf(v - self[k]));
    }
    store_pack<float, 4>(nxt + o, out);
    return res;
}

__device__ __forceinline__ float res_chunk(int D, const SegGeo &pt, const float *cur, float *nxt, unsigned bufoff,
                                           const ResArgs &a, int o) {
    switch (D) {
    case 1: return res_segment<1>(pt, cur, nxt, bufoff, a, o);
    case 2: return res_segment<2>(pt, cur, nxt, bufoff, a, o);
    default: return res_segment<3>(pt, cur, nxt, bufoff, a, o);
    }
}

// Global packed index of the part's state at padded offset rel, or -1 for
// padding (the packed layout has no row padding).
__device__ __forceinline__ long long res_global(const ResPart &pt, int rel) {
    if (rel >= pt.nsl * pt.P) return -1;
    const int zl = rel / pt.P, rem = rel - zl * pt.P;
    const int y = rem / pt.nxp, x = rem - y * pt.nxp;
    if (x >= pt.nx) return -1;
    return pt.goff + ((long long)zl * pt.ny + y) * pt.nx + x;
}

// The part's values into buffer 0: padding and obstacles as 0 (an
// obstacle's value is never read and its result is 0).
__device__ __forceinline__ void res_load(const ResPart &pt, float *buf0, const float *V, const uint8_t *codep) {
    const int n = pt.nchunks * kResChunk;
    const unsigned obst = 1u << (2 * pt.D);
    for (int rel = threadIdx.x; rel < n; rel += blockDim.x) {
        const long long g = res_global(pt, rel);
        buf0[pt.base + rel] = g >= 0 && !(codep[pt.poff + rel] & obst) ? V[g] : 0.f;
    }
}

__device__ __forceinline__ void res_store(const ResPart &pt, const float *src, float *V) {
    const int n = pt.nsl * pt.P;
    for (int rel = threadIdx.x; rel < n; rel += blockDim.x) {
        const long long g = res_global(pt, rel);
        if (g >= 0) V[g] = src[pt.base + rel];
    }
}

__device__ __forceinline__ void res_record(const ResArgs &a, int inst, int done, unsigned bits, int q) {
    a.done_at[inst] = done;
    a.res[(size_t)(q % 3) * a.ninst + inst] =
        (unsigned long long)__double_as_longlong((double)__uint_as_float(bits));
    atomicMax(&a.ctrl->iterations, done < 0 ? -done : done);
}

// Solo bundles: one CTA, up to kResMaxParts whole instances in lockstep.
__device__ void res_solo(const ResArgs &a, ResShared &S, float *buf) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) S.job = atomicAdd(&a.ctr[1], 1);
        __syncthreads();
        const int job = S.job;
        if (job >= a.hdr[1]) break;
        const int2 bd = a.solo[job];
        const int np = bd.y;
        if (tid < np) {
            S.part[tid] = a.parts[bd.x + tid];
            S.slot[tid][0] = S.slot[tid][1] = S.slot[tid][2] = 0u;
            S.done[tid] = 0;
        }
        __syncthreads();
        int nch = 0;
        if (tid < np) {
            const ResPart &pt = S.part[tid];
            for (int c = 0; c < pt.nchunks; c++) S.chunk_part[pt.base / kResChunk + c] = (uint8_t)tid;
        }
        {
            const ResPart &lastp = S.part[np - 1];
            nch = lastp.base / kResChunk + lastp.nchunks;
        }
        for (int p = 0; p < np; p++) res_load(S.part[p], buf, a.V, a.codep);
        __syncthreads();
        for (int q = 0;; q++) {
            if (tid < np) S.slot[tid][(q + 1) % 3] = 0u;
            const float *cur = buf + (q & 1) * kResCap;
            float *nxt = buf + ((q + 1) & 1) * kResCap;
            bool worked = false;
            int gp = -1, gD = 3;
            SegGeo geo;
            for (int c = warp; c < nch; c += kResWarps) {
                const int p = S.chunk_part[c];
                if (q > 0 && (q >= a.max_iter || res_below(S.slot[p][(q - 1) % 3], a.tol_bits))) continue;
                if (p != gp) {
                    geo.load(S.part[p]);
                    gD = S.part[p].D;
                    gp = p;
                }
                const float r = res_chunk(gD, geo, cur, nxt, 0u, a, c * kResChunk + 4 * lane);
                const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(r));
                if (lane == 0) atomicMax(&S.slot[p][q % 3], mx);
                worked = true;
            }
            const int any = __syncthreads_or(worked ? 1 : 0);
            if (tid < np && S.done[tid] == 0) {
                const unsigned v = S.slot[tid][q % 3];
                int d = 0;
                if (res_below(v, a.tol_bits)) d = q + 1;
                else if (q + 1 >= a.max_iter) d = -(q + 1);
                if (d != 0) {
                    S.done[tid] = d;
                    res_record(a, S.part[tid].inst, d, v, q);
                }
            }
            if (!any) break;
        }
        __syncthreads();
        for (int p = 0; p < np; p++) {
            const int d = S.done[p] < 0 ? -S.done[p] : S.done[p];
            res_store(S.part[p], buf + (d & 1) * kResCap, a.V);
        }
        __syncthreads();
    }
}

// Cluster bundles: one instance over the C CTAs of the cluster, or two
// instances over C / 2 consecutive ranks each (part r on rank r). Every CTA
// sends its residual of a sweep to its instance's slot in every CTA of the
// cluster (C remote max reductions), so after the cluster barrier each CTA
// reads every instance's residual from its own shared memory: an instance
// stops on its own (its CTAs keep the barriers until the bundle ends, and
// its slots, no longer written, read as below tol from then on), and the
// bundle ends when none runs.
__device__ void res_cluster(const ResArgs &a, ResShared &S, float *buf, int C) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned rank = cluster_ctarank();
    const unsigned job_addr0 = cluster_map(smem_addr(&S.job), 0);
    for (;;) {
        if (rank == 0 && tid == 0) S.job = atomicAdd(&a.ctr[0], 1);
        cluster_sync_all();
        const int job = (int)ld_cluster_u32(job_addr0);
        if (job >= a.hdr[0]) {
            // nobody reads rank 0's shared memory after this barrier
            cluster_sync_all();
            break;
        }
        const int2 bd = a.multi[job];
        const bool have = (int)rank < bd.y;
        if (tid < 8) S.slot[tid][0] = S.slot[tid][1] = S.slot[tid][2] = 0u;
        if (tid == 0) {
            S.lmax[0] = S.lmax[1] = 0u;
            if (have) {
                ResPart pt = a.parts[bd.x + rank];
                const unsigned b0 = smem_addr(buf);
                pt.prev_addr = pt.has_prev ? cluster_map(b0 + 4u * (unsigned)pt.prev_off, rank - 1) : 0u;
                pt.next_addr = pt.has_next ? cluster_map(b0, rank + 1) : 0u;
                S.part[0] = pt;
            }
        }
        __syncthreads();
        if (have) res_load(S.part[0], buf, a.V, a.codep);
        SegGeo geo;
        geo.load(S.part[0]);
        const int D = S.part[0].D, inst = S.part[0].inst;
        const int bidx = have ? S.part[0].bidx : 0, nb = have ? S.part[0].nbinst : 1;
        const bool lead = have && (int)rank == S.part[0].lead;
        // lane t < C of warp 0 sends to rank t's slot of this CTA's instance
        const unsigned slot_remote =
            tid < C ? cluster_map(smem_addr(&S.slot[bidx][0]), (unsigned)tid) : 0u;
        cluster_sync_all();
        const int nch = have ? S.part[0].nchunks : 0;
        int sweeps = 0;
        bool running = have;
        for (int q = 0;; q++) {
            if (q > 0) {
                // every instance's residual of sweep q - 1, complete in this
                // CTA's own slots (every CTA reads the same values)
                bool any = false;
                for (int b = 0; b < nb; b++) {
                    const unsigned v = S.slot[b][(q - 1) % 3];
                    const bool stop = res_below(v, a.tol_bits) || q >= a.max_iter;
                    any |= !stop;
                    if (b == bidx && stop && running) {
                        running = false;
                        sweeps = q;
                        if (lead && tid == 0) res_record(a, inst, res_below(v, a.tol_bits) ? q : -q, v, q - 1);
                    }
                }
                if (!any) break;
            }
            if (tid < nb) S.slot[tid][(q + 1) % 3] = 0u;
            if (tid == 0) S.lmax[(q + 1) & 1] = 0u;
            const float *cur = buf + (q & 1) * kResCap;
            float *nxt = buf + ((q + 1) & 1) * kResCap;
            const unsigned bufoff = (unsigned)((q & 1) * kResCap * 4);
            if (running) {
                for (int c = warp; c < nch; c += kResWarps) {
                    const float r = res_chunk(D, geo, cur, nxt, bufoff, a, c * kResChunk + 4 * lane);
                    const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(r));
                    if (lane == 0) atomicMax(&S.lmax[q & 1], mx);
                }
            }
            __syncthreads();
            if (tid < C && running) red_cluster_max(slot_remote + 4u * (unsigned)(q % 3), S.lmax[q & 1]);
            cluster_sync_all();
        }
        if (have) res_store(S.part[0], buf + (sweeps & 1) * kResCap, a.V);
        // every CTA reads only its own slots now, and rank 0's job word was
        // read before the bundle's sweeps
        __syncthreads();
    }
}

template <bool CLUSTER>
__global__ void __launch_bounds__(kResThreads, 1) resident_vi_kernel(ResArgs a) {
    extern __shared__ __align__(16) float res_smem[];
    float *buf = res_smem;
    ResShared &S = *reinterpret_cast<ResShared *>(res_smem + 2 * kResCap);
    if (CLUSTER) {
        unsigned nrank;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(nrank));
        res_cluster(a, S, buf, (int)nrank);
    }
    res_solo(a, S, buf);
}

// Padded copies of the rewards, the expectation multipliers and the codes:
// instance i at pad_off[i], its leading slices one after another, rows
// padded to nxp with obstacle codes. Multiplier: gamma on free states, 0 on
// terminals, obstacles and padding; reward 0 on obstacles and padding.
__global__ void res_pad_kernel(const BatchInst *inst, const long long *pad_off, const float *R, const uint8_t *code,
                               float *Rp, float *Gp, uint8_t *codep) {
    const BatchInst I = inst[blockIdx.x];
    const int nx = I.shape[I.ndim - 1], nxp = (nx + 3) & ~3;
    const int ny = I.ndim == 3 ? I.shape[1] : 1;
    const int L = I.ndim == 1 ? 1 : I.shape[0];
    const int P = ny * nxp;
    const unsigned obst = 1u << (2 * I.ndim), term = 1u << (2 * I.ndim + 1);
    const long long n = (long long)L * P, base = pad_off[blockIdx.x];
    for (long long idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int zl = (int)(idx / P), rem = (int)(idx - (long long)zl * P);
        const int y = rem / nxp, x = rem - y * nxp;
        if (x < nx) {
            const long long g = I.offset + ((long long)zl * ny + y) * nx + x;
            const unsigned c = code[g];
            Rp[base + idx] = (c & obst) ? 0.f : R[g];
            Gp[base + idx] = (c & (obst | term)) ? 0.f : I.gamma;
            codep[base + idx] = (uint8_t)c;
        } else {
            Rp[base + idx] = 0.f;
            Gp[base + idx] = 0.f;
            codep[base + idx] = 0xFF;
        }
    }
}

// ---------------------------------------------------------------------------
// host side

namespace {

struct InstGeo {
    int nx, nxp, ny, L, P;   // row, padded row, rows per slice, slices, padded states per slice
    int kmin;                // CTAs needed (0: does not fit a cluster of 8)
};

InstGeo geometry(const BatchInst &I) {
    InstGeo g;
    g.nx = I.shape[I.ndim - 1];
    g.nxp = (g.nx + 3) & ~3;
    g.ny = I.ndim == 3 ? I.shape[1] : 1;
    g.L = I.ndim == 1 ? 1 : I.shape[0];
    g.P = g.ny * g.nxp;
    g.kmin = 0;
    if (g.P <= kResCap) {
        const int per = kResCap / g.P;                 // slices per CTA
        const int k = (g.L + per - 1) / per;
        if (k <= 8 && (k == 1 || g.L >= k)) g.kmin = k;
    }
    return g;
}

int chunks_of(long long states) { return (int)((states + kResChunk - 1) / kResChunk); }

// Per-sweep time of a CTA working through n chunks (units of one round of
// the 32 warps; the barrier and decisions cost about one round).
double sweep_cost(int n, bool cluster) { return (cluster ? 1.5 : 1.0) + (double)((n + kResWarps - 1) / kResWarps); }

}  // namespace

// Capability, cluster size and padded copies; called once per batch.
cpmdp_status batch_resident_prepare(cpmdp_batch &B) {
    if (B.res_tried) return CPMDP_OK;
    B.res_tried = true;
    int kmax = 1;
    std::vector<long long> pad((size_t)B.ninst);
    long long off = 0;
    for (int i = 0; i < B.ninst; i++) {
        const InstGeo g = geometry(B.inst[(size_t)i]);
        if (g.kmin == 0) return CPMDP_OK;            // an instance does not fit: the batched kernel
        kmax = std::max(kmax, g.kmin);
        pad[(size_t)i] = off;
        off += ((long long)g.L * g.P + 3) & ~3ll;
    }
    int C = 1;
    while (C < kmax) C *= 2;
    int dev_smem = 0;
    CPMDP_CUDA(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, B.device));
    if ((size_t)dev_smem < kResSmem) return CPMDP_OK;
    const void *fn = C > 1 ? (const void *)resident_vi_kernel<true> : (const void *)resident_vi_kernel<false>;
    CPMDP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResSmem));
    int nclusters = 0;
    {
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(C * 8);
        cfg.blockDim = dim3(kResThreads);
        cfg.dynamicSmemBytes = kResSmem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = C > 1 ? cudaOccupancyMaxActiveClusters(&nclusters, resident_vi_kernel<true>, &cfg)
                              : cudaOccupancyMaxActiveClusters(&nclusters, resident_vi_kernel<false>, &cfg);
        if (e != cudaSuccess || nclusters < 1) { (void)cudaGetLastError(); return CPMDP_OK; }
    }
    const size_t nparts_max = (size_t)B.ninst * C;
    CPMDP_CUDA(cudaMalloc(&B.d_Rp, sizeof(float) * (size_t)off));
    CPMDP_CUDA(cudaMalloc(&B.d_Gp, sizeof(float) * (size_t)off));
    CPMDP_CUDA(cudaMalloc(&B.d_codep, (size_t)off));
    CPMDP_CUDA(cudaMalloc(&B.d_rparts, sizeof(ResPart) * nparts_max));
    CPMDP_CUDA(cudaMalloc(&B.d_rmulti, sizeof(int2) * (size_t)B.ninst));
    CPMDP_CUDA(cudaMalloc(&B.d_rsolo, sizeof(int2) * (size_t)B.ninst));
    CPMDP_CUDA(cudaMalloc(&B.d_rhdr, sizeof(int) * 4));
    long long *d_pad = nullptr;
    CPMDP_CUDA(cudaMalloc(&d_pad, sizeof(long long) * (size_t)B.ninst));
    struct FreePad { long long *p; ~FreePad() { cudaFree(p); } } free_pad{d_pad};
    CPMDP_CUDA(cudaMemcpy(d_pad, pad.data(), sizeof(long long) * (size_t)B.ninst, cudaMemcpyHostToDevice));
    res_pad_kernel<<<B.ninst, 256>>>(B.d_inst, d_pad, B.d_R, B.d_code, B.d_Rp, B.d_Gp, B.d_codep);
    CPMDP_CUDA(cudaGetLastError());
    CPMDP_CUDA(cudaDeviceSynchronize());
    B.res_pad = pad;
    B.res_C = C;
    B.res_grid = nclusters * C;
    B.res_est.assign((size_t)B.ninst, 0);
    B.res_ok = true;
    return CPMDP_OK;
}

// Bundles from the expected sweep counts (the previous solve's, or a
// gamma-based guess before the first): instances whose solo solve would
// set the length of the whole launch are cut over a cluster; the others are
// packed, most sweeps first, into CTAs as long as the bundle's time stays
// under about a third of the launch's average load per CTA.
cpmdp_status batch_resident_plan(cpmdp_batch &B, double tol, int max_iter) {
    const int n = B.ninst, C = B.res_C;
    std::vector<double> est((size_t)n);
    for (int i = 0; i < n; i++) {
        int e = B.res_est[(size_t)i];
        if (e <= 0) {
            const double gm = B.inst[(size_t)i].gamma;
            double k = gm > 0.0 && gm < 1.0 ? std::log(tol * (1.0 - gm)) / std::log(gm) : (double)max_iter;
            e = (int)std::min<double>(std::max(k, 1.0), (double)max_iter);
        }
        est[(size_t)i] = std::min(e, max_iter);
    }
    std::vector<InstGeo> geo((size_t)n);
    std::vector<int> split((size_t)n, 0);
    double work = 0.0, crit = 0.0;
    for (int i = 0; i < n; i++) {
        geo[(size_t)i] = geometry(B.inst[(size_t)i]);
        const InstGeo &g = geo[(size_t)i];
        split[(size_t)i] = g.kmin > 1 ? 1 : 0;
    }
    // split long solo solves while one would exceed the average load
    for (int pass = 0; pass < 2; pass++) {
        work = 0.0;
        crit = 0.0;
        for (int i = 0; i < n; i++) {
            const InstGeo &g = geo[(size_t)i];
            double t;
            if (split[(size_t)i]) {
                const int per = (g.L + C - 1) / C;
                t = est[(size_t)i] * sweep_cost(chunks_of((long long)per * g.P), true);
                work += t * C;
            } else {
                t = est[(size_t)i] * sweep_cost(chunks_of((long long)g.L * g.P), false);
                work += est[(size_t)i] * (double)chunks_of((long long)g.L * g.P) / kResWarps;
            }
            crit = std::max(crit, t);
        }
        const double avg = work / std::max(1, B.res_grid);
        if (C < 2) break;
        for (int i = 0; i < n; i++) {
            const InstGeo &g = geo[(size_t)i];
            if (split[(size_t)i] || g.L < C) continue;
            const double t = est[(size_t)i] * sweep_cost(chunks_of((long long)g.L * g.P), false);
            if (t > avg) split[(size_t)i] = 1;
        }
    }
    // solo bundles run after the cluster bundles: keeping each one well
    // under the launch's average load lets the last ones even out the end
    const double target = std::max(crit, 0.35 * work / std::max(1, B.res_grid));
    std::vector<int> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return est[(size_t)x] > est[(size_t)y]; });
    std::vector<ResPart> parts;
    std::vector<int2> multi, solo;
    auto make_part = [&](int i, int z0, int nsl, int base) {
        const BatchInst &I = B.inst[(size_t)i];
        const InstGeo &g = geo[(size_t)i];
        ResPart p;
        memset(&p, 0, sizeof(p));
        p.goff = I.offset + (long long)z0 * g.ny * g.nx;
        p.poff = B.res_pad[(size_t)i] + (long long)z0 * g.P;
        p.inst = i;
        p.D = I.ndim;
        p.nx = g.nx;
        p.nxp = g.nxp;
        p.ny = g.ny;
        p.P = g.P;
        p.nsl = nsl;
        p.base = base;
        p.nchunks = chunks_of((long long)nsl * g.P);
        p.wm = I.w_move;
        p.wp = I.w_perp;
        p.wst = I.w_stay;
        p.g = I.gamma;
        return p;
    };
    // cluster bundles, longest first: an instance that needs at most C / 2
    // CTAs for its size goes with another such instance of similar sweep
    // count, C / 2 ranks each (half the barriers per instance); the others,
    // and the solo-sized instances cut for the length of the launch, take
    // all C ranks
    auto cluster_parts = [&](int i, int r0, int k, int bidx, int nb) {
        const InstGeo &g = geo[(size_t)i];
        int z0 = 0;
        std::vector<int> nsl((size_t)k);
        for (int r = 0; r < k; r++) nsl[(size_t)r] = g.L / k + (r < g.L % k ? 1 : 0);
        for (int r = 0; r < k; r++) {
            ResPart p = make_part(i, z0, nsl[(size_t)r], 0);
            p.has_prev = r > 0 ? 1 : 0;
            p.has_next = r + 1 < k ? 1 : 0;
            p.prev_off = r > 0 ? (nsl[(size_t)r - 1] - 1) * g.P : 0;
            p.bidx = bidx;
            p.nbinst = nb;
            p.lead = r0;
            parts.push_back(p);
            z0 += nsl[(size_t)r];
        }
    };
    std::vector<int> halves;
    std::vector<std::pair<double, std::pair<int, int>>> mlist;   // (time, (instance, partner or -1))
    for (int i : order) {
        if (!split[(size_t)i]) continue;
        const InstGeo &g = geo[(size_t)i];
        if (C >= 4 && g.kmin >= 2 && 2 * g.kmin <= C) {
            halves.push_back(i);
        } else {
            const int per = (g.L + C - 1) / C;
            mlist.push_back({est[(size_t)i] * sweep_cost(chunks_of((long long)per * g.P), true), {i, -1}});
        }
    }
    for (size_t h = 0; h < halves.size(); h += 2) {
        const int i = halves[h];
        const InstGeo &g = geo[(size_t)i];
        if (h + 1 < halves.size()) {
            const int j2 = halves[h + 1];
            const InstGeo &g2 = geo[(size_t)j2];
            const int per = std::max((g.L + C / 2 - 1) / (C / 2) * g.P, (g2.L + C / 2 - 1) / (C / 2) * g2.P);
            mlist.push_back({est[(size_t)i] * sweep_cost(chunks_of(per), true), {i, j2}});
        } else {
            const int per = (g.L + C - 1) / C;
            mlist.push_back({est[(size_t)i] * sweep_cost(chunks_of((long long)per * g.P), true), {i, -1}});
        }
    }
    std::stable_sort(mlist.begin(), mlist.end(),
                     [](const std::pair<double, std::pair<int, int>> &x, const std::pair<double, std::pair<int, int>> &y) {
                         return x.first > y.first;
                     });
    for (const auto &m : mlist) {
        const int first = (int)parts.size();
        if (m.second.second < 0) {
            cluster_parts(m.second.first, 0, C, 0, 1);
        } else {
            cluster_parts(m.second.first, 0, C / 2, 0, 2);
            cluster_parts(m.second.second, C / 2, C / 2, 1, 2);
        }
        multi.push_back(make_int2(first, C));
    }
    // solo bundles: most sweeps first, packed while the bundle's time stays
    // under the target (a bundle's instances stop one by one, so its time is
    // about the sum of their work plus the longest one's barriers)
    std::vector<std::pair<double, int2>> slist;
    size_t oi = 0;
    std::vector<int> solo_order;
    for (int i : order)
        if (!split[(size_t)i]) solo_order.push_back(i);
    while (oi < solo_order.size()) {
        const int first = (int)parts.size();
        int chunks = 0, np = 0;
        double t_bar = 0.0, t_work = 0.0;
        while (oi < solo_order.size() && np < kResMaxParts) {
            const int i = solo_order[oi];
            const InstGeo &g = geo[(size_t)i];
            const int ch = chunks_of((long long)g.L * g.P);
            if (chunks + ch > kResChunks) break;
            const double tb = std::max(t_bar, est[(size_t)i]);
            const double tw = t_work + est[(size_t)i] * (double)ch / kResWarps;
            if (np > 0 && tb + tw > target) break;
            parts.push_back(make_part(i, 0, g.L, chunks * kResChunk));
            chunks += ch;
            np++;
            t_bar = tb;
            t_work = tw;
            oi++;
        }
        slist.push_back({t_bar + t_work, make_int2(first, np)});
    }
    std::stable_sort(slist.begin(), slist.end(), [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) {
        return x.first > y.first;
    });
    for (const auto &s : slist) solo.push_back(s.second);
    const int hdr[4] = {(int)multi.size(), (int)solo.size(), 0, 0};
    CPMDP_CUDA(cudaMemcpy(B.d_rparts, parts.data(), sizeof(ResPart) * parts.size(), cudaMemcpyHostToDevice));
    if (!multi.empty())
        CPMDP_CUDA(cudaMemcpy(B.d_rmulti, multi.data(), sizeof(int2) * multi.size(), cudaMemcpyHostToDevice));
    if (!solo.empty())
        CPMDP_CUDA(cudaMemcpy(B.d_rsolo, solo.data(), sizeof(int2) * solo.size(), cudaMemcpyHostToDevice));
    CPMDP_CUDA(cudaMemcpy(B.d_rhdr, hdr, sizeof(hdr), cudaMemcpyHostToDevice));
    B.res_planned_for = B.res_est;
    B.res_planned = true;
    B.res_nmulti = (int)multi.size();
    B.res_nsolo = (int)solo.size();
    return CPMDP_OK;
}

unsigned res_tol_bits(double tol) {
    float f = (float)tol;
    if ((double)f >= tol) f = std::nextafter(f, 0.0f);
    if (!(f >= 0.0f)) f = 0.0f;
    unsigned b;
    memcpy(&b, &f, sizeof(b));
    return b;
}

cudaError_t batch_resident_enqueue(const cpmdp_batch &B, float *V, double tol, int max_iter, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(B.d_ctrl, 0, sizeof(Ctrl), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(B.d_done, 0, sizeof(int) * B.ninst, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(B.d_rhdr + 2, 0, sizeof(int) * 2, st)) != cudaSuccess) return e;
    ResArgs a;
    a.parts = B.d_rparts;
    a.multi = B.d_rmulti;
    a.solo = B.d_rsolo;
    a.hdr = B.d_rhdr;
    a.ctr = B.d_rhdr + 2;
    a.Rp = B.d_Rp;
    a.Gp = B.d_Gp;
    a.codep = B.d_codep;
    a.V = V;
    a.done_at = B.d_done;
    a.res = B.d_res;
    a.ninst = B.ninst;
    a.tol_bits = res_tol_bits(tol);
    a.max_iter = max_iter;
    a.ctrl = B.d_ctrl;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(B.res_grid);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = kResSmem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = B.res_C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return B.res_C > 1 ? cudaLaunchKernelEx(&cfg, resident_vi_kernel<true>, a)
                       : cudaLaunchKernelEx(&cfg, resident_vi_kernel<false>, a);
}

}  // namespace cpmdp
