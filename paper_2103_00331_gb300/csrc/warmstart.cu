// Learned warm start for value iteration: value iteration of a coarsened
// copy of each GridWorld (cells of 4 x 4 x 4 states) gives a coarse value
// per cell, and a fully convolutional 3-D network maps the cell features
// (mean reward of the non-obstacle states, obstacle fraction, largest
// terminal reward, -log(1 - gamma) / 5, the coarse value) to a correction of
// it; value iteration then starts from the corrected coarse values upsampled
// to the full grid. The solver is unchanged: a poor estimate only costs
// sweeps.
//
// Kernels (BF16 storage, FP32 accumulation, channels-last activations with
// 64 channels, "same" dilated 3 x 3 x 3 convolutions, tap t = (dz+1) * 9 +
// (dy+1) * 3 + (dx+1)):
//   conv_tma_kernel  y[v, n] = sum_t sum_k x[v + s d off(t), k] B_t[n, k] (+ b, ReLU, mask)
//                    on the tcgen05 tensor cores, operands by tensor copy:
//                    forward (s = +1, B_t[co, ci] = W[t, co, ci]) and data
//                    gradient (s = -1, B_t[ci, co] = W[t, co, ci], times the
//                    ReLU mask of the layer input)
//   conv_dw_kernel   dW[t, co, ci] = sum_v dy[v, co] x[v + d off(t), ci] (SIMT)
//   plus features / targets / upsampling from a packed batch, the coarse
//   value iteration, the cell-level and full-grid loss gradients, Adam and
//   the FP32 -> BF16 weight casts.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "batch_internal.h"
#include "tc_common.cuh"

namespace cpmdp {

constexpr int kC = 64;        // channels of every activation
constexpr int kF = 4;         // coarsening factor per dimension

struct Dims {
    int n, z, y, x;           // instances and coarse grid
    __host__ __device__ int nvox() const { return n * z * y * x; }
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

constexpr int kCvBTile = 64 * 128;                   // one tap's weights: 64 channels x 64 bf16
constexpr long long kCvWaitCycles = 2000000000LL;    // about 1 s at 2 GHz

__device__ int g_conv_err = 0;

// Element offset of (row r, k) in a 64-wide bf16 tile with 128-byte rows
// and the 128-byte swizzle (16-byte chunk k / 8 of row r at chunk
// (k / 8) ^ (r % 8)).
__host__ __device__ __forceinline__ int sw_elem(int r, int k) { return r * 64 + ((((k >> 3) ^ (r & 7)) & 7) << 3) + (k & 7); }

// ---------------------------------------------------------------------------
// convolution (forward and data gradient): tiled tensor copies feed the
// tcgen05 tensor cores
//
// The same implicit GEMM. The output is cut into tiles of 128 voxels, a box
// of bx x by x bz voxels of one instance (tile row r = voxel
// (r / (bx by), (r / bx) % by, r % bx) of the box). A persistent CTA works
// through batches of 4 tiles whose accumulators (128 x 64 FP32 each) sit side
// by side in TMEM, twice over, so that the epilogue of one batch runs under
// the MMAs of the next. For each of the 9 tap groups (oz, ox) of a batch, the
// group's three weight tiles (oy = -1, 0, 1; pre-swizzled by the weight cast)
// arrive by bulk copy once for the 4 tiles, and each tile's input arrives by
// tensor copy of its box shifted by s d (oz, ., ox) (channels-last rows of
// 128 bytes, 128-byte swizzle: the K-major operand layout). In "tall" mode
// (one-plane tiles, bx a multiple of 8) one box of by + 2 d rows of y serves
// the group's three taps, which read it from row (s d oy + d) bx on (whole
// 1024-byte swizzle atoms); otherwise three boxes of the tile's own shape,
// one per oy, are copied. Voxels outside the grid arrive as zeros: the
// "same" padding. Roles: warp 4 issues the copies, one thread of warp 5 the
// MMAs (12 per tile and group: 3 taps x 4 K-steps of 16), warps 0-3 read the
// accumulators (thread = tile row = TMEM lane), apply bias and ReLU, or the
// ReLU mask of the layer input, and write bf16 rows (and FP32 channel 0).
// Every wait is bounded; one that runs out records an error (read by
// cpmdp_ws_sync) and stops every role, each after the copies and MMAs it
// issued have completed.

constexpr int kTmTiles = 4;                          // tiles (accumulators) per batch
constexpr uint32_t kTmCols = 2 * kTmTiles * 64;      // TMEM columns: two accumulator sets
constexpr int kTmThreads = 192;
constexpr int kTmBStage = 3 * kCvBTile;              // weight tiles of one tap group
constexpr int kTmBStages = 2;                        // weight ring
constexpr int kTmAMax = 3 * 128 * 128;               // largest input stage (three 128-row boxes)
constexpr int kTmMaxStages = 12;
constexpr int kTmSmemMax = 227 * 1024;

struct ConvGeo {
    int n, z, y, x;            // instances and grid
    int bx, by, bz;            // tile box
    int tx, ty, tz;            // tiles per dimension
    int tiles;
    int tall;                  // one (by + 2 dil)-row box per tap group
    int stage_bytes, stages;   // input ring
    int dil, sign, relu;
};

struct TmShared {
    uint64_t afull[kTmMaxStages], aempty[kTmMaxStages];
    uint64_t bfull[kTmBStages], bempty[kTmBStages], accf[2], acce[2];
    uint32_t tslot;
    int abort;
};

__device__ __forceinline__ bool tm_wait(uint64_t *bar, uint32_t phase, volatile int *abort) {
    const long long t0 = clock64();
    while (!tc::mbar_try(bar, phase)) {
        if (*abort) return false;
        if (clock64() - t0 > kCvWaitCycles) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tile_origin(const ConvGeo &g, int tile, int &nn, int &x0, int &y0, int &z0) {
    int r = tile;
    const int ix = r % g.tx; r /= g.tx;
    const int iy = r % g.ty; r /= g.ty;
    const int iz = r % g.tz;
    nn = r / g.tz;
    x0 = ix * g.bx;
    y0 = iy * g.by;
    z0 = iz * g.bz;
}

__global__ void __launch_bounds__(kTmThreads, 1) conv_tma_kernel(const __grid_constant__ CUtensorMap tmx,
                                                                const uint8_t *__restrict__ wimg,
                                                                const float *__restrict__ bias,
                                                                const __nv_bfloat16 *__restrict__ mask_act,
                                                                __nv_bfloat16 *__restrict__ y,
                                                                float *__restrict__ y0, ConvGeo g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = sm;
    uint8_t *sA = sm + kTmBStages * kTmBStage;
    TmShared &S = *reinterpret_cast<TmShared *>(sA + (size_t)g.stages * g.stage_bytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < g.stages; i++) {
            tc::mbar_init(&S.afull[i], 1);
            tc::mbar_init(&S.aempty[i], 1);
        }
        for (int i = 0; i < kTmBStages; i++) {
            tc::mbar_init(&S.bfull[i], 1);
            tc::mbar_init(&S.bempty[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&S.accf[i], 1);
            tc::mbar_init(&S.acce[i], 128);
        }
        S.abort = 0;
    }
    if (warp == 5) tc::tmem_alloc(&S.tslot, kTmCols);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tslot;
    volatile int *abort = &S.abort;
    const int nbatch = (g.tiles + kTmTiles - 1) / kTmTiles;
    const int d = g.dil, sg = g.sign;

    if (warp == 4) {
        if (lane == 0) {
            // producer: weight tiles per tap group, input boxes per tile and group
            int alast[kTmMaxStages], blast[kTmBStages];
            for (int i = 0; i < kTmMaxStages; i++) alast[i] = -1;
            for (int i = 0; i < kTmBStages; i++) blast[i] = -1;
            uint32_t acount = 0, gcount = 0;
            bool ok = true;
            for (int b = blockIdx.x; ok && b < nbatch; b += gridDim.x) {
                for (int grp = 0; ok && grp < 9; grp++) {
                    const int oz = grp / 3 - 1, ox = grp % 3 - 1;
                    const int bs = (int)(gcount % kTmBStages);
                    const uint32_t bph = (gcount / kTmBStages) & 1;
                    if (gcount >= kTmBStages && !tm_wait(&S.bempty[bs], bph ^ 1u, abort)) { ok = false; break; }
                    tc::mbar_expect_tx(&S.bfull[bs], kTmBStage);
                    for (int oy = 0; oy < 3; oy++) {
                        const int t = (oz + 1) * 9 + oy * 3 + (ox + 1);
                        tc::bulk_g2s(tc::smem_u32(sB + bs * kTmBStage + oy * kCvBTile), wimg + (size_t)t * kCvBTile,
                                     kCvBTile, &S.bfull[bs]);
                    }
                    blast[bs] = (int)bph;
                    gcount++;
                    for (int j = 0; j < kTmTiles; j++) {
                        const int tile = b * kTmTiles + j;
                        if (tile >= g.tiles) break;
                        int nn, x0, y0t, z0;
                        tile_origin(g, tile, nn, x0, y0t, z0);
                        const int as = (int)(acount % (uint32_t)g.stages);
                        const uint32_t ph = (acount / (uint32_t)g.stages) & 1;
                        if (acount >= (uint32_t)g.stages && !tm_wait(&S.aempty[as], ph ^ 1u, abort)) { ok = false; break; }
                        const uint32_t dst = tc::smem_u32(sA + (size_t)as * g.stage_bytes);
                        const int xs = x0 + sg * d * ox, zs = z0 + sg * d * oz;
                        if (g.tall) {
                            tc::mbar_expect_tx(&S.afull[as], (uint32_t)((g.by + 2 * d) * g.bx * 128));
                            tc::tma_load_5d(dst, &tmx, 0, xs, y0t - d, zs, nn, &S.afull[as]);
                        } else {
                            tc::mbar_expect_tx(&S.afull[as], 3u * 128u * 128u);
                            for (int oy = 0; oy < 3; oy++)
                                tc::tma_load_5d(dst + oy * 16384u, &tmx, 0, xs, y0t + sg * d * (oy - 1), zs, nn,
                                                &S.afull[as]);
                        }
                        alast[as] = (int)ph;
                        acount++;
                    }
                }
            }
            // every copy this thread issued lands before the CTA's shared memory goes
            for (int i = 0; i < g.stages; i++)
                if (alast[i] >= 0) tc::mbar_wait(&S.afull[i], (uint32_t)alast[i], kCvWaitCycles);
            for (int i = 0; i < kTmBStages; i++)
                if (blast[i] >= 0) tc::mbar_wait(&S.bfull[i], (uint32_t)blast[i], kCvWaitCycles);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer
            uint32_t acount = 0, gcount = 0, bcount = 0;
            uint64_t *lastbar = nullptr;
            uint32_t lastph = 0;
            bool ok = true;
            for (int b = blockIdx.x; ok && b < nbatch; b += gridDim.x, bcount++) {
                const int buf = bcount & 1;
                if (bcount >= 2 && !tm_wait(&S.acce[buf], ((bcount >> 1) - 1) & 1, abort)) { ok = false; break; }
                tc::fence_after();
                const uint32_t dacc = tmem + (uint32_t)buf * (kTmCols / 2);
                for (int grp = 0; ok && grp < 9; grp++) {
                    const int bs = (int)(gcount % kTmBStages);
                    const uint32_t bph = (gcount / kTmBStages) & 1;
                    if (!tm_wait(&S.bfull[bs], bph, abort)) { ok = false; break; }
                    tc::fence_after();
                    const uint32_t bb = tc::smem_u32(sB + bs * kTmBStage);
                    for (int j = 0; j < kTmTiles; j++) {
                        if (b * kTmTiles + j >= g.tiles) break;
                        const int as = (int)(acount % (uint32_t)g.stages);
                        const uint32_t ph = (acount / (uint32_t)g.stages) & 1;
                        if (!tm_wait(&S.afull[as], ph, abort)) { ok = false; break; }
                        tc::fence_after();
                        const uint32_t ab = tc::smem_u32(sA + (size_t)as * g.stage_bytes);
                        for (int oy = 0; oy < 3; oy++) {
                            const uint32_t aoff = g.tall ? (uint32_t)((sg * d * (oy - 1) + d) * g.bx * 128)
                                                         : (uint32_t)(oy * 16384);
#pragma unroll
                            for (int ks = 0; ks < 4; ks++)
                                tc::mma(dacc + (uint32_t)j * 64u, tc::sdesc(ab + aoff + ks * 32),
                                        tc::sdesc(bb + oy * kCvBTile + ks * 32), tc::kIdescM128N64,
                                        (grp > 0 || oy > 0 || ks > 0) ? 1u : 0u);
                        }
                        tc::commit(&S.aempty[as]);
                        lastbar = &S.aempty[as];
                        lastph = ph;
                        acount++;
                    }
                    if (!ok) break;
                    tc::commit(&S.bempty[bs]);
                    lastbar = &S.bempty[bs];
                    lastph = bph;
                    gcount++;
                }
                if (!ok) break;
                tc::commit(&S.accf[buf]);
                lastbar = &S.accf[buf];
                lastph = (bcount >> 1) & 1;
            }
            // the MMAs complete in order: the last commit covers them all
            if (lastbar) tc::mbar_wait(lastbar, lastph, kCvWaitCycles);
        }
    } else {
        // epilogue: warps 0-3, thread = tile row = TMEM lane
        const int r = tid;
        const int xl = r % g.bx, yl = (r / g.bx) % g.by, zl = r / (g.bx * g.by);
        uint32_t bcount = 0;
        for (int b = blockIdx.x; b < nbatch; b += gridDim.x, bcount++) {
            const int buf = bcount & 1;
            const bool okw = tm_wait(&S.accf[buf], (bcount >> 1) & 1, abort);
            if (!__all_sync(0xFFFFFFFFu, okw)) break;
            tc::fence_after();
            for (int j = 0; j < kTmTiles; j++) {
                const int tile = b * kTmTiles + j;
                if (tile >= g.tiles) break;
                int nn, x0, y0t, z0;
                tile_origin(g, tile, nn, x0, y0t, z0);
                float acc[64];
                tc::tmem_ld64(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)buf * (kTmCols / 2) + (uint32_t)j * 64u,
                              acc);
                const int gx = x0 + xl, gy = y0t + yl, gz = z0 + zl;
                if (gx < g.x && gy < g.y && gz < g.z) {
                    const size_t v = ((size_t)(nn * g.z + gz) * g.y + gy) * g.x + gx;
#pragma unroll
                    for (int c = 0; c < 64; c++) acc[c] += bias ? bias[c] : 0.f;
                    if (mask_act) {
                        const uint4 *mrow = reinterpret_cast<const uint4 *>(mask_act + v * kC);
#pragma unroll
                        for (int q = 0; q < 8; q++) {
                            const uint4 m = mrow[q];
                            const uint32_t w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                            for (int h = 0; h < 8; h++) {
                                const uint16_t bits = (uint16_t)(w[h >> 1] >> (16 * (h & 1)));
                                if (!(bf(__ushort_as_bfloat16(bits)) > 0.f)) acc[8 * q + h] = 0.f;
                            }
                        }
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(y + v * kC);
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        uint32_t w[4];
#pragma unroll
                        for (int h = 0; h < 4; h++) {
                            float a0 = acc[8 * q + 2 * h], a1 = acc[8 * q + 2 * h + 1];
                            if (g.relu) { a0 = fmaxf(a0, 0.f); a1 = fmaxf(a1, 0.f); }
                            if (q == 0 && h == 0 && y0) y0[v] = a0;
                            w[h] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a0)) |
                                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a1)) << 16);
                        }
                        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            }
            tc::fence_before();
            tc::mbar_arrive(&S.acce[buf]);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0 && S.abort) atomicExch(&g_conv_err, 1);
    if (warp == 5) tc::tmem_dealloc(tmem, kTmCols);
}

// dW[t, co, ci] += sum over a chunk of voxels of dy[v, co] x[v + d off(t), ci]
__global__ void __launch_bounds__(256) conv_dw_kernel(const __nv_bfloat16 *__restrict__ x,
                                                      const __nv_bfloat16 *__restrict__ dy, float *__restrict__ dw,
                                                      Dims dm, int dil, int chunk) {
    __shared__ float sD[32][65];   // [voxel][co]
    __shared__ float sX[32][65];   // [voxel][ci]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int t = blockIdx.y;
    const int oz = dil * (t / 9 - 1), oy = dil * ((t / 3) % 3 - 1), ox = dil * (t % 3 - 1);
    const int nvox = dm.nvox();
    const int vbeg = blockIdx.x * chunk, vend = min(vbeg + chunk, nvox);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
    for (int vb = vbeg; vb < vend; vb += 32) {
        for (int e = tid; e < 32 * 64; e += 256) {
            const int vv = e >> 6, c = e & 63;
            const int v = vb + vv;
            float dv = 0.f, xv = 0.f;
            if (v < vend) {
                dv = bf(dy[(size_t)v * kC + c]);
                int r = v;
                const int xx = r % dm.x; r /= dm.x;
                const int yy = r % dm.y; r /= dm.y;
                const int zz = r % dm.z; const int nn = r / dm.z;
                const int z2 = zz + oz, y2 = yy + oy, x2 = xx + ox;
                if (z2 >= 0 && z2 < dm.z && y2 >= 0 && y2 < dm.y && x2 >= 0 && x2 < dm.x)
                    xv = bf(x[((size_t)((nn * dm.z + z2) * dm.y + y2) * dm.x + x2) * kC + c]);
            }
            sD[vv][c] = dv;
            sX[vv][c] = xv;
        }
        __syncthreads();
#pragma unroll 8
        for (int vv = 0; vv < 32; vv++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = sD[vv][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = sX[vv][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            atomicAdd(&dw[(size_t)t * kC * kC + (ty + 16 * i) * kC + tx + 16 * j], acc[i][j]);
}

// db[c] += sum_v dy[v, c]
__global__ void conv_db_kernel(const __nv_bfloat16 *__restrict__ dy, float *__restrict__ db, int nvox) {
    const int c = threadIdx.x & 63, lane_group = threadIdx.x >> 6;   // 4 groups of 64 threads
    float s = 0.f;
    for (int v = blockIdx.x * 4 + lane_group; v < nvox; v += gridDim.x * 4) s += bf(dy[(size_t)v * kC + c]);
    atomicAdd(&db[c], s);
}

// dy[v, 0] = 2 (pred - target) mask / nvox, other channels 0; loss += sum mask (pred - target)^2 / nvox
__global__ void loss_grad_kernel(const float *__restrict__ pred, const float *__restrict__ target,
                                 const float *__restrict__ mask, __nv_bfloat16 *__restrict__ dy, float *loss, int nvox) {
    __shared__ float sh[8];
    float l = 0.f;
    const float inv = 1.f / (float)nvox;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += gridDim.x * blockDim.x) {
        const float d = (pred[v] - target[v]) * mask[v];
        l += d * d * inv;
        dy[(size_t)v * kC] = __float2bfloat16_rn(2.f * d * inv);
#pragma unroll 4
        for (int c = 1; c < kC; c++) dy[(size_t)v * kC + c] = __float2bfloat16_rn(0.f);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
        if (loss) atomicAdd(loss, s);
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// W [t][co][ci] (FP32) -> per tap the B tiles of the tensor-core convolution
// (64 rows x 64 bf16, 128-byte swizzle): wf row co, column ci (forward) and
// wb row ci, column co (data gradient).
__global__ void cast_weights_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf,
                                    __nv_bfloat16 *__restrict__ wb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / (kC * kC), r = i % (kC * kC);
        const int co = (int)(r / kC), ci = (int)(r % kC);
        const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
        wf[t * kC * kC + sw_elem(co, ci)] = h;
        wb[t * kC * kC + sw_elem(ci, co)] = h;
    }
}

// ---------------------------------------------------------------------------
// batch <-> coarse grids (instances first .. first + count - 1, equal shapes)

__device__ __forceinline__ void coarse_of(const BatchInst &I, int cell, int &cz, int &cy, int &cx, int &zc, int &yc,
                                          int &xc) {
    zc = (I.shape[0] + kF - 1) / kF;
    yc = (I.shape[1] + kF - 1) / kF;
    xc = (I.shape[2] + kF - 1) / kF;
    cx = cell % xc;
    cy = (cell / xc) % yc;
    cz = cell / (xc * yc);
}

// One thread per coarse cell; rows of the cell whose x extent is a full
// aligned group of 4 (every row of an instance with x side a multiple of
// 4) are read as one 16-byte reward load and one 4-byte code load, so
// neighbouring cells' threads read neighbouring bytes.
__global__ void features_kernel(const BatchInst *__restrict__ inst, const uint8_t *__restrict__ code,
                                const float *__restrict__ R, int first, int count, int cells,
                                __nv_bfloat16 *__restrict__ feat) {
    const long long total = (long long)count * cells;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / cells), cell = (int)(g % cells);
        const BatchInst I = inst[first + i];
        int cz, cy, cx, zc, yc, xc;
        coarse_of(I, cell, cz, cy, cx, zc, yc, xc);
        const unsigned ob = 1u << (2 * I.ndim), tb = 1u << (2 * I.ndim + 1);
        float rsum = 0.f, tmax = 0.f;
        int live = 0, obst = 0, n = 0, any_t = 0;
        const int x0 = cx * kF, x1 = min(x0 + kF, I.shape[2]);
        const bool vec = x1 - x0 == kF && I.shape[2] % 4 == 0 && I.offset % 4 == 0;
        for (int z = cz * kF; z < min((cz + 1) * kF, I.shape[0]); z++)
            for (int y = cy * kF; y < min((cy + 1) * kF, I.shape[1]); y++) {
                const long long row = I.offset + (long long)z * I.stride[0] + y * I.stride[1];
                float r4[kF];
                unsigned c4[kF];
                if (vec) {
                    const float4 rv = *reinterpret_cast<const float4 *>(R + row + x0);
                    const unsigned cw = *reinterpret_cast<const unsigned *>(code + row + x0);
                    r4[0] = rv.x; r4[1] = rv.y; r4[2] = rv.z; r4[3] = rv.w;
#pragma unroll
                    for (int k = 0; k < kF; k++) c4[k] = (cw >> (8 * k)) & 0xFFu;
                } else {
#pragma unroll
                    for (int k = 0; k < kF; k++) {
                        const bool in = x0 + k < x1;
                        r4[k] = in ? R[row + x0 + k] : 0.f;
                        c4[k] = in ? code[row + x0 + k] : 0xFFFFFFFFu;   // marks "outside the grid"
                    }
                }
#pragma unroll
                for (int k = 0; k < kF; k++) {
                    const unsigned c = c4[k];
                    if (c == 0xFFFFFFFFu) continue;
                    n++;
                    if (c & ob) { obst++; continue; }
                    live++;
                    rsum += r4[k];
                    if (c & tb) { tmax = any_t ? fmaxf(tmax, r4[k]) : r4[k]; any_t = 1; }
                }
            }
        __nv_bfloat16 *f = feat + g * kC;
        f[0] = __float2bfloat16_rn(live ? rsum / live : 0.f);
        f[1] = __float2bfloat16_rn((float)obst / (float)n);
        f[2] = __float2bfloat16_rn(any_t ? tmax : 0.f);
        f[3] = __float2bfloat16_rn(-logf(1.f - I.gamma) / 5.f);
        uint4 *f16 = reinterpret_cast<uint4 *>(f);
        // channels 4..63: zero (channel 4 is the coarse value, written later)
        uint2 *f2 = reinterpret_cast<uint2 *>(f);
        f2[1] = make_uint2(0u, 0u);
#pragma unroll
        for (int j = 1; j < 8; j++) f16[j] = make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void targets_kernel(const BatchInst *__restrict__ inst, const uint8_t *__restrict__ code,
                               const float *__restrict__ V, int first, int count, int cells,
                               const float *__restrict__ base, float *__restrict__ target, float *__restrict__ mask) {
    const long long total = (long long)count * cells;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / cells), cell = (int)(g % cells);
        const BatchInst I = inst[first + i];
        int cz, cy, cx, zc, yc, xc;
        coarse_of(I, cell, cz, cy, cx, zc, yc, xc);
        const unsigned ob = 1u << (2 * I.ndim);
        float s = 0.f;
        int live = 0;
        for (int z = cz * kF; z < min((cz + 1) * kF, I.shape[0]); z++)
            for (int y = cy * kF; y < min((cy + 1) * kF, I.shape[1]); y++)
                for (int x = cx * kF; x < min((cx + 1) * kF, I.shape[2]); x++) {
                    const long long st = I.offset + (long long)z * I.stride[0] + y * I.stride[1] + x;
                    if (code[st] & ob) continue;
                    live++;
                    s += V[st];
                }
        target[g] = (live ? s / live : 0.f) - (base ? base[g] : 0.f);
        mask[g] = live ? 1.f : 0.f;
    }
}

// Trilinear interpolation of a coarse array (plus base, if given) at fine
// state s of instance I: the coarse values sit at the cell centres, a fine
// coordinate x at (x + 0.5) / 4 - 0.5 in cell units, clamped to the
// outermost centres.
struct Interp {
    int lo[3], hi[3];
    float t[3];
    int yc, xc;
    __device__ void at(const BatchInst &I, int s) {
        const int z = s / I.stride[0], y = (s / I.stride[1]) % I.shape[1], x = s % I.shape[2];
        const int nc[3] = {(I.shape[0] + kF - 1) / kF, (I.shape[1] + kF - 1) / kF, (I.shape[2] + kF - 1) / kF};
        const int pos[3] = {z, y, x};
        yc = nc[1];
        xc = nc[2];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            float u = ((float)pos[d] + 0.5f) / (float)kF - 0.5f;
            u = fminf(fmaxf(u, 0.f), (float)(nc[d] - 1));
            lo[d] = (int)floorf(u);
            hi[d] = min(lo[d] + 1, nc[d] - 1);
            t[d] = u - (float)lo[d];
        }
    }
    __device__ float value(const float *cv, const float *bv) const {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int cz = (k & 4) ? hi[0] : lo[0], cy = (k & 2) ? hi[1] : lo[1], cx = (k & 1) ? hi[2] : lo[2];
            const float w = ((k & 4) ? t[0] : 1.f - t[0]) * ((k & 2) ? t[1] : 1.f - t[1]) * ((k & 1) ? t[2] : 1.f - t[2]);
            const int cell = (cz * yc + cy) * xc + cx;
            v += w * (cv[cell] + (bv ? bv[cell] : 0.f));
        }
        return v;
    }
};

// Weight of coarse index c in the interpolation at fine coordinate p of a
// dimension with nc cells (both corners may be c where the clamp folds them).
__device__ __forceinline__ float interp_weight(int p, int c, int nc) {
    float u = ((float)p + 0.5f) / (float)kF - 0.5f;
    u = fminf(fmaxf(u, 0.f), (float)(nc - 1));
    const int lo = (int)floorf(u), hi = min(lo + 1, nc - 1);
    const float t = u - (float)lo;
    return (lo == c ? 1.f - t : 0.f) + (hi == c ? t : 0.f);
}

// Coarse estimate (plus base) upsampled to every fine state: free states
// take the interpolation, terminals R(t), obstacles 0. One thread per group
// of 4 consecutive states of a row: the z and y weights are set once per
// row, and rows whose length is a multiple of 4 (16-byte aligned, as every
// instance starts on a multiple of 4 states) are written with one 16-byte
// store.
__device__ __forceinline__ void axis_weights(int p, int nc, int &lo, int &hi, float &t) {
    float u = ((float)p + 0.5f) / (float)kF - 0.5f;
    u = fminf(fmaxf(u, 0.f), (float)(nc - 1));
    lo = (int)floorf(u);
    hi = min(lo + 1, nc - 1);
    t = u - (float)lo;
}

__global__ void upsample_kernel(const BatchInst *__restrict__ inst, const uint8_t *__restrict__ code,
                                const float *__restrict__ R, int first, int count, int cells,
                                const float *__restrict__ coarse, const float *__restrict__ base,
                                float *__restrict__ V) {
    const BatchInst I0 = inst[first];
    const int Z = I0.shape[0], Y = I0.shape[1], X = I0.shape[2];
    const int nq = (X + 3) / 4;
    const int zc = (Z + kF - 1) / kF, yc = (Y + kF - 1) / kF, xc = (X + kF - 1) / kF;
    const long long total = (long long)count * Z * Y * nq;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(g % nq);
        const long long row = g / nq;
        const int y = (int)(row % Y);
        const long long zr = row / Y;
        const int z = (int)(zr % Z), i = (int)(zr / Z);
        const BatchInst I = inst[first + i];
        const unsigned ob = 1u << (2 * I.ndim), tb = 1u << (2 * I.ndim + 1);
        int zlo, zhi, ylo, yhi;
        float tz, ty;
        axis_weights(z, zc, zlo, zhi, tz);
        axis_weights(y, yc, ylo, yhi, ty);
        const float *cv = coarse + (long long)i * cells;
        const float *bv = base ? base + (long long)i * cells : nullptr;
        const long long s0 = I.offset + (long long)z * I.stride[0] + (long long)y * I.stride[1];
        float out[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int x = 4 * q + k;
            out[k] = 0.f;
            if (x >= X) continue;
            const unsigned c = code[s0 + x];
            if (c & ob) continue;
            if (c & tb) { out[k] = R[s0 + x]; continue; }
            int xlo, xhi;
            float tx;
            axis_weights(x, xc, xlo, xhi, tx);
            float v = 0.f;
#pragma unroll
            for (int m = 0; m < 8; m++) {
                const int cz = (m & 4) ? zhi : zlo, cy = (m & 2) ? yhi : ylo, cx = (m & 1) ? xhi : xlo;
                const float w = ((m & 4) ? tz : 1.f - tz) * ((m & 2) ? ty : 1.f - ty) * ((m & 1) ? tx : 1.f - tx);
                const int cell = (cz * yc + cy) * xc + cx;
                v += w * (cv[cell] + (bv ? bv[cell] : 0.f));
            }
            out[k] = v;
        }
        if (X % 4 == 0) {
            *reinterpret_cast<float4 *>(V + s0 + 4 * q) = make_float4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (4 * q + k < X) V[s0 + 4 * q + k] = out[k];
        }
    }
}

// Fine-level loss of a coarse estimate: with Vh = upsample(base + pred),
// r(s) = Vh(s) - Vt(s) on the free states (0 on terminals and obstacles,
// where the upsampling is exact); loss += sum r^2 * inv.
__global__ void fine_resid_kernel(const BatchInst *__restrict__ inst, const uint8_t *__restrict__ code, int first,
                                  int count, int cells, const float *__restrict__ pred,
                                  const float *__restrict__ base, const float *__restrict__ Vt,
                                  float *__restrict__ r, float inv, float *loss) {
    __shared__ float sh[8];
    const BatchInst I0 = inst[first];
    const long long per = I0.nstates;
    const long long total = (long long)count * per;
    float l = 0.f;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / per);
        const int s = (int)(g % per);
        const BatchInst I = inst[first + i];
        const unsigned c = code[I.offset + s];
        float d = 0.f;
        if (!(c & (3u << (2 * I.ndim)))) {
            Interp ip;
            ip.at(I, s);
            d = ip.value(pred + (long long)i * cells, base ? base + (long long)i * cells : nullptr) - Vt[I.offset + s];
        }
        r[g] = d;
        l += d * d * inv;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float sum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) sum += sh[w];
        if (loss) atomicAdd(loss, sum);
    }
}

// Gradient of that loss with respect to the coarse estimate: the transpose
// of the interpolation, dL/dpred(c) = 2 inv sum_s w(s, c) r(s) over the fine
// states whose interpolation reads cell c (coordinates 4c - 2 .. 4c + 5 in
// each dimension); written into channel 0 of dy, the other channels 0.
__global__ void fine_grad_kernel(const BatchInst *__restrict__ inst, int first, int count, int cells,
                                 const float *__restrict__ r, float inv, __nv_bfloat16 *__restrict__ dy) {
    const long long total = (long long)count * cells;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / cells), cell = (int)(g % cells);
        const BatchInst I = inst[first + i];
        int cz, cy, cx, zc, yc, xc;
        coarse_of(I, cell, cz, cy, cx, zc, yc, xc);
        const float *ri = r + (long long)i * I.nstates;
        float acc = 0.f;
        for (int z = max(0, kF * cz - 2); z <= min(I.shape[0] - 1, kF * cz + 5); z++) {
            const float wz = interp_weight(z, cz, zc);
            if (wz == 0.f) continue;
            for (int y = max(0, kF * cy - 2); y <= min(I.shape[1] - 1, kF * cy + 5); y++) {
                const float wzy = wz * interp_weight(y, cy, yc);
                if (wzy == 0.f) continue;
                for (int x = max(0, kF * cx - 2); x <= min(I.shape[2] - 1, kF * cx + 5); x++)
                    acc += wzy * interp_weight(x, cx, xc) * ri[z * I.stride[0] + y * I.stride[1] + x];
            }
        }
        __nv_bfloat16 *d = dy + g * kC;
        d[0] = __float2bfloat16_rn(2.f * inv * acc);
        for (int ch = 1; ch < kC; ch++) d[ch] = __float2bfloat16_rn(0.f);
    }
}

// Value iteration of a coarsened copy of each instance, one CTA per
// instance, entirely in shared memory (the input feature that gives the
// network a view of the whole grid). Coarse cell = 4 x 4 x 4 fine states:
// an obstacle when at least half of its states are obstacles, else a
// terminal of value max R(t) when it holds terminals, else a free cell whose
// reward per coarse step is the mean fine reward of its free states times
// 1 + gamma + gamma^2 + gamma^3 (four fine steps); discount gamma^4, the
// instance's slip model, walls and obstacle cells block moves. Jacobi sweeps
// from zero until max |dV| < tol or max_sweeps.
constexpr int kCoarseThreads = 512;
constexpr int kMaxCoarseCells = 8192;

__global__ void __launch_bounds__(kCoarseThreads) coarse_vi_kernel(const BatchInst *__restrict__ inst,
                                                                   const uint8_t *__restrict__ code,
                                                                   const float *__restrict__ R, int first, int cells,
                                                                   float tol, int max_sweeps,
                                                                   float *__restrict__ coarse_v,
                                                                   __nv_bfloat16 *__restrict__ feat) {
    extern __shared__ uint8_t smem_raw[];
    float *va = reinterpret_cast<float *>(smem_raw);                 // V (even sweeps)
    float *vb = va + cells;                                          // V (odd sweeps)
    float *rsum = vb + cells;                                        // coarse reward
    uint8_t *kind = reinterpret_cast<uint8_t *>(rsum + cells);      // bits 0-5 blocked moves, 6 obstacle, 7 terminal
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const BatchInst I = inst[first + i];
    const int zc = (I.shape[0] + kF - 1) / kF, yc = (I.shape[1] + kF - 1) / kF, xc = (I.shape[2] + kF - 1) / kF;
    const unsigned ob = 1u << (2 * I.ndim), tb = 1u << (2 * I.ndim + 1);
    const float g = I.gamma;
    const float gc = g * g * g * g, steps = 1.f + g + g * g + g * g * g;
    // per cell, over its rows of up to 4 fine states (one 16-byte reward load
    // and one 4-byte code load where the row is a full aligned group of 4)
    for (int c = tid; c < cells; c += kCoarseThreads) {
        const int cz = c / (yc * xc), cy = (c / xc) % yc, cx = c % xc;
        const int x0 = cx * kF, x1 = min(x0 + kF, I.shape[2]);
        const bool vec = x1 - x0 == kF && I.shape[2] % 4 == 0 && I.offset % 4 == 0;
        int n = 0, n_obst = 0, n_free = 0, any_t = 0;
        float rs = 0.f, tmax = 0.f;
        for (int z = cz * kF; z < min((cz + 1) * kF, I.shape[0]); z++)
            for (int y = cy * kF; y < min((cy + 1) * kF, I.shape[1]); y++) {
                const long long row = I.offset + (long long)z * I.stride[0] + (long long)y * I.stride[1];
                float r4[kF];
                unsigned c4[kF];
                if (vec) {
                    const float4 rv = *reinterpret_cast<const float4 *>(R + row + x0);
                    const unsigned cw = *reinterpret_cast<const unsigned *>(code + row + x0);
                    r4[0] = rv.x; r4[1] = rv.y; r4[2] = rv.z; r4[3] = rv.w;
#pragma unroll
                    for (int k = 0; k < kF; k++) c4[k] = (cw >> (8 * k)) & 0xFFu;
                } else {
#pragma unroll
                    for (int k = 0; k < kF; k++) {
                        const bool in = x0 + k < x1;
                        r4[k] = in ? R[row + x0 + k] : 0.f;
                        c4[k] = in ? code[row + x0 + k] : 0xFFFFFFFFu;   // outside the grid
                    }
                }
#pragma unroll
                for (int k = 0; k < kF; k++) {
                    const unsigned cs = c4[k];
                    if (cs == 0xFFFFFFFFu) continue;
                    n++;
                    if (cs & ob) { n_obst++; continue; }
                    if (cs & tb) { tmax = any_t ? fmaxf(tmax, r4[k]) : r4[k]; any_t = 1; continue; }
                    n_free++;
                    rs += r4[k];
                }
            }
        uint8_t k = 0;
        float r = 0.f;
        if (2 * n_obst >= n) k = 0x40;
        else if (any_t) { k = 0x80; r = tmax; }
        else r = n_free ? rs / (float)n_free * steps : 0.f;
        kind[c] = k;
        rsum[c] = r;
    }
    __syncthreads();
    for (int c = tid; c < cells; c += kCoarseThreads) {
        const int cz = c / (yc * xc), cy = (c / xc) % yc, cx = c % xc;
        uint8_t k = kind[c];
        const int nbr[6] = {cz > 0 ? c - yc * xc : -1, cz < zc - 1 ? c + yc * xc : -1, cy > 0 ? c - xc : -1,
                            cy < yc - 1 ? c + xc : -1, cx > 0 ? c - 1 : -1, cx < xc - 1 ? c + 1 : -1};
#pragma unroll
        for (int j = 0; j < 6; j++)
            if (nbr[j] < 0 || (kind[nbr[j]] & 0x40)) k |= (uint8_t)(1u << j);
        kind[c] = k;
        const float v0 = (k & 0x80) ? rsum[c] : 0.f;
        va[c] = v0;
        vb[c] = v0;
    }
    __syncthreads();
    const float wm = I.w_move, wp = I.w_perp, wst = I.w_stay;
    float *src = va, *dst = vb;
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        int open = 0;
        for (int c = tid; c < cells; c += kCoarseThreads) {
            const uint8_t k = kind[c];
            if (k & 0xC0) continue;   // obstacles (0) and terminals (their value) never change
            const float self = src[c];
            float nb[6];
            const int step[3] = {yc * xc, xc, 1};
#pragma unroll
            for (int d = 0; d < 3; d++) {
                nb[2 * d] = ((k >> (2 * d)) & 1u) ? self : src[c - step[d]];
                nb[2 * d + 1] = ((k >> (2 * d + 1)) & 1u) ? self : src[c + step[d]];
            }
            const float P0 = nb[0] + nb[1], P1 = nb[2] + nb[3], P2 = nb[4] + nb[5];
            const float perp[3] = {P1 + P2, P0 + P2, P0 + P1};
            float best = -INFINITY;
#pragma unroll
            for (int j = 0; j < 6; j++) best = fmaxf(best, wm * nb[j] + wp * perp[j / 2] + wst * self);
            const float v = rsum[c] + gc * best;
            dst[c] = v;
            open |= fabsf(v - self) >= tol;
        }
        float *t = src; src = dst; dst = t;
        if (!__syncthreads_or(open)) break;
    }
    for (int c = tid; c < cells; c += kCoarseThreads) {
        const uint8_t k = kind[c];
        const float v = (k & 0x40) ? 0.f : src[c];
        coarse_v[(long long)i * cells + c] = v;
        if (feat) feat[((long long)i * cells + c) * kC + 4] = __float2bfloat16_rn(v);
    }
}

static int grid_for(long long n, int per_block) {
    long long g = (n + per_block - 1) / per_block;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)(g < 1 ? 1 : g);
}

// Shape check shared by the batch <-> coarse calls: instances first..first+count-1
// must be 3-D and of one shape (each is addressed through its own offset in
// the packed layout); returns the coarse cell count.
static cpmdp_status batch_range(const cpmdp_batch *B, int first, int count, int *cells) {
    if (!B || count < 1 || first < 0 || first + count > B->ninst) { set_error("instance range outside the batch"); return CPMDP_EINVAL; }
    const BatchInst &I0 = B->inst[(size_t)first];
    if (I0.ndim != 3) { set_error("the warm start takes 3-D instances"); return CPMDP_EINVAL; }
    for (int i = first; i < first + count; i++) {
        const BatchInst &I = B->inst[(size_t)i];
        if (I.ndim != 3 || I.shape[0] != I0.shape[0] || I.shape[1] != I0.shape[1] || I.shape[2] != I0.shape[2]) {
            set_error("instances %d..%d must share one shape", first, first + count - 1);
            return CPMDP_EINVAL;
        }
    }
    *cells = ((I0.shape[0] + kF - 1) / kF) * ((I0.shape[1] + kF - 1) / kF) * ((I0.shape[2] + kF - 1) / kF);
    return CPMDP_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

static int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Tile shape, input ring and tensor map of one convolution launch.
static cudaError_t launch_conv(const __nv_bfloat16 *x, const uint8_t *wimg, const float *bias,
                               const __nv_bfloat16 *mask_act, __nv_bfloat16 *y, float *y0, Dims dm, int dil, int sign,
                               int relu, cudaStream_t st) {
    ConvGeo g;
    g.n = dm.n; g.z = dm.z; g.y = dm.y; g.x = dm.x;
    g.bx = std::min(16, std::max(8, pow2_at_least(dm.x)));
    g.by = std::min(128 / g.bx, pow2_at_least(dm.y));
    g.bz = 128 / (g.bx * g.by);
    g.tx = (dm.x + g.bx - 1) / g.bx;
    g.ty = (dm.y + g.by - 1) / g.by;
    g.tz = (dm.z + g.bz - 1) / g.bz;
    const long long tiles = (long long)g.tx * g.ty * g.tz * dm.n;
    if (tiles > (1LL << 30)) return cudaErrorInvalidValue;
    g.tiles = (int)tiles;
    const int tall_rows = (g.by + 2 * dil) * g.bx;
    g.tall = g.bz == 1 && g.bx % 8 == 0 && g.by + 2 * dil <= 256 && tall_rows * 128 <= kTmAMax;
    g.stage_bytes = g.tall ? ((tall_rows * 128 + 1023) & ~1023) : kTmAMax;
    g.stages = std::min(kTmMaxStages,
                        (kTmSmemMax - 1024 - kTmBStages * kTmBStage - (int)sizeof(TmShared)) / g.stage_bytes);
    g.dil = dil;
    g.sign = sign;
    g.relu = relu;
    const size_t smem = 1024 + (size_t)kTmBStages * kTmBStage + (size_t)g.stages * g.stage_bytes + sizeof(TmShared);

    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t gdim[5] = {(cuuint64_t)kC, (cuuint64_t)dm.x, (cuuint64_t)dm.y, (cuuint64_t)dm.z, (cuuint64_t)dm.n};
    const cuuint64_t gstride[4] = {(cuuint64_t)kC * 2, (cuuint64_t)kC * 2 * dm.x, (cuuint64_t)kC * 2 * dm.x * dm.y,
                                   (cuuint64_t)kC * 2 * dm.x * dm.y * dm.z};
    const cuuint32_t box[5] = {(cuuint32_t)kC, (cuuint32_t)g.bx, (cuuint32_t)(g.tall ? g.by + 2 * dil : g.by),
                               (cuuint32_t)g.bz, 1u};
    const cuuint32_t estride[5] = {1u, 1u, 1u, 1u, 1u};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(x), gdim, gstride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(conv_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmSmemMax)) !=
        cudaSuccess)
        return e;
    const int nbatch = (g.tiles + kTmTiles - 1) / kTmTiles;
    const int grid = std::max(1, std::min(nbatch, sms));
    conv_tma_kernel<<<grid, kTmThreads, smem, st>>>(map, wimg, bias, mask_act, y, y0, g);
    return cudaGetLastError();
}

static cpmdp_status dims_ok(int n, int z, int y, int x, int dil) {
    if (n < 1 || z < 1 || y < 1 || x < 1 || dil < 1 || (long long)n * z * y * x > (1LL << 31) - 64) {
        set_error("invalid convolution dimensions");
        return CPMDP_EINVAL;
    }
    return CPMDP_OK;
}

}  // namespace cpmdp

using namespace cpmdp;

extern "C" {

cpmdp_status cpmdp_ws_features(const cpmdp_batch *B, int32_t first, int32_t count, uint16_t *feat, void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    const long long n = (long long)count * cells;
    features_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, B->d_R, first, count,
                                                                        cells, (__nv_bfloat16 *)feat);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_targets(const cpmdp_batch *B, const float *V, int32_t first, int32_t count, const float *base,
                              float *target, float *mask, void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    const long long n = (long long)count * cells;
    targets_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, V, first, count, cells,
                                                                       base, target, mask);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_upsample(const cpmdp_batch *B, const float *coarse, const float *base, int32_t first,
                               int32_t count, float *V, void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    const BatchInst &I0 = B->inst[(size_t)first];
    const long long n = (long long)count * I0.shape[0] * I0.shape[1] * ((I0.shape[2] + 3) / 4);
    upsample_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, B->d_R, first, count,
                                                                        cells, coarse, base, V);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_fine_loss_grad(const cpmdp_batch *B, const float *V_target, int32_t first, int32_t count,
                                     const float *pred, const float *base, float *resid, uint16_t *dy, float *loss,
                                     void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    if (!V_target || !pred || !resid || !dy) { set_error("V_target, pred, resid and dy are required"); return CPMDP_EINVAL; }
    const long long n = (long long)count * B->inst[(size_t)first].nstates;
    const float inv = (float)(1.0 / (double)n);
    fine_resid_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, first, count, cells,
                                                                          pred, base, V_target, resid, inv, loss);
    CPMDP_CUDA(cudaGetLastError());
    const long long nc = (long long)count * cells;
    fine_grad_kernel<<<grid_for(nc, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, first, count, cells, resid, inv,
                                                                          (__nv_bfloat16 *)dy);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_coarse_vi(const cpmdp_batch *B, int32_t first, int32_t count, float tol, int32_t max_sweeps,
                                float *coarse_v, uint16_t *feat, void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    if (cells > kMaxCoarseCells) {
        set_error("coarse value iteration holds at most %d coarse cells per instance", kMaxCoarseCells);
        return CPMDP_EINVAL;
    }
    if (!coarse_v || !(tol > 0.f) || max_sweeps < 1) { set_error("coarse_v, tol > 0 and max_sweeps >= 1 required"); return CPMDP_EINVAL; }
    const size_t smem = (size_t)cells * 13;
    CPMDP_CUDA(cudaFuncSetAttribute(coarse_vi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    coarse_vi_kernel<<<count, kCoarseThreads, smem, (cudaStream_t)stream>>>(B->d_inst, B->d_code, B->d_R, first, cells,
                                                                          tol, max_sweeps, coarse_v,
                                                                          (__nv_bfloat16 *)feat);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_conv3d_forward(const uint16_t *x, const uint16_t *wf, const float *bias, uint16_t *y, float *y0,
                                  int32_t n, int32_t z, int32_t yy, int32_t xx, int32_t dilation, int32_t relu,
                                  void *stream) {
    cpmdp_status s = dims_ok(n, z, yy, xx, dilation);
    if (s != CPMDP_OK) return s;
    if (!x || !wf || !y) { set_error("x, w and y are required"); return CPMDP_EINVAL; }
    Dims dm{n, z, yy, xx};
    CPMDP_CUDA(launch_conv((const __nv_bfloat16 *)x, (const uint8_t *)wf, bias, nullptr, (__nv_bfloat16 *)y, y0, dm,
                           dilation, 1, relu, (cudaStream_t)stream));
    return CPMDP_OK;
}

cpmdp_status cpmdp_conv3d_backward_data(const uint16_t *dy, const uint16_t *wb, const uint16_t *act_in, uint16_t *dx,
                                        int32_t n, int32_t z, int32_t yy, int32_t xx, int32_t dilation, void *stream) {
    cpmdp_status s = dims_ok(n, z, yy, xx, dilation);
    if (s != CPMDP_OK) return s;
    if (!dy || !wb || !dx) { set_error("dy, w and dx are required"); return CPMDP_EINVAL; }
    Dims dm{n, z, yy, xx};
    CPMDP_CUDA(launch_conv((const __nv_bfloat16 *)dy, (const uint8_t *)wb, nullptr, (const __nv_bfloat16 *)act_in,
                           (__nv_bfloat16 *)dx, nullptr, dm, dilation, -1, 0, (cudaStream_t)stream));
    return CPMDP_OK;
}

cpmdp_status cpmdp_conv3d_backward_weight(const uint16_t *x, const uint16_t *dy, float *dw, float *db, int32_t n,
                                          int32_t z, int32_t yy, int32_t xx, int32_t dilation, void *stream) {
    cpmdp_status s = dims_ok(n, z, yy, xx, dilation);
    if (s != CPMDP_OK) return s;
    if (!x || !dy || !dw) { set_error("x, dy and dw are required"); return CPMDP_EINVAL; }
    Dims dm{n, z, yy, xx};
    const int chunk = 512;
    dim3 grid((dm.nvox() + chunk - 1) / chunk, 27);
    conv_dw_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)dy, dw, dm,
                                                          dilation, chunk);
    CPMDP_CUDA(cudaGetLastError());
    if (db) {
        conv_db_kernel<<<grid_for(dm.nvox(), 64), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)dy, db,
                                                                                    dm.nvox());
        CPMDP_CUDA(cudaGetLastError());
    }
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_loss_grad(const float *pred, const float *target, const float *mask, int32_t nvox, uint16_t *dy,
                                float *loss, void *stream) {
    if (nvox < 1 || !pred || !target || !mask || !dy) { set_error("invalid loss arguments"); return CPMDP_EINVAL; }
    loss_grad_kernel<<<grid_for(nvox, 256), 256, 0, (cudaStream_t)stream>>>(pred, target, mask, (__nv_bfloat16 *)dy,
                                                                            loss, nvox);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_adam_step(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                             float beta2, float eps, int32_t step, void *stream) {
    if (n < 1 || !p || !g || !m || !v || step < 1) { set_error("invalid Adam arguments"); return CPMDP_EINVAL; }
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_cast_weights(const float *w, uint16_t *wf, uint16_t *wb, int32_t layers, void *stream) {
    if (layers < 1 || !w || !wf || !wb) { set_error("invalid weight-cast arguments"); return CPMDP_EINVAL; }
    const long long n = (long long)layers * 27 * kC * kC;
    cast_weights_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(w, (__nv_bfloat16 *)wf,
                                                                            (__nv_bfloat16 *)wb, n);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_sync(void *stream) {
    CPMDP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int e = 0;
    CPMDP_CUDA(cudaMemcpyFromSymbol(&e, g_conv_err, sizeof(int)));
    if (e) {
        const int zero = 0;
        CPMDP_CUDA(cudaMemcpyToSymbol(g_conv_err, &zero, sizeof(int)));
        set_error("a tensor-core wait in a warm-start convolution ran out");
        return CPMDP_ETIMEOUT;
    }
    return CPMDP_OK;
}

}  // extern "C"
