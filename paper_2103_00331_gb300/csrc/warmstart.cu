// Learned warm start for value iteration: a fully convolutional 3-D network
// maps coarse features of a GridWorld (cells of 4 x 4 x 4 states: mean
// reward of the non-obstacle states, obstacle fraction, largest terminal
// reward, -log(1 - gamma) / 5) to an estimate of V* per coarse cell; value
// iteration then starts from that estimate upsampled to the full grid. The
// solver is unchanged: a poor estimate only costs sweeps.
//
// Kernels (BF16 storage, FP32 accumulation, channels-last activations with
// 64 channels, "same" dilated 3 x 3 x 3 convolutions, tap t = (dz+1) * 9 +
// (dy+1) * 3 + (dx+1)):
//   conv_tc_kernel   y[v, n] = sum_t sum_k x[v + s d off(t), k] B_t[n, k] (+ b, ReLU, mask)
//                    on the tcgen05 tensor cores: forward (s = +1, B_t[co, ci] =
//                    W[t, co, ci]) and data gradient (s = -1, B_t[ci, co] =
//                    W[t, co, ci], times the ReLU mask of the layer input),
//                    a 128-voxel x 64-channel tile per CTA
//   conv_dw_kernel   dW[t, co, ci] = sum_v dy[v, co] x[v + d off(t), ci] (SIMT)
//   plus features / targets / upsampling from a packed batch, the loss
//   gradient, Adam and the FP32 -> BF16 weight casts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

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

// ---------------------------------------------------------------------------
// convolution (forward and data gradient) on the tcgen05 tensor cores
//
// Implicit GEMM per tap: D[v, n] += sum_k A_t[v, k] B_t[n, k] with
// A_t[v, k] = x[v + s d off(t), k] (zero outside the grid) and B_t the tap's
// 64 x 64 weight tile; 27 taps x 4 K-steps of 16 accumulate into one TMEM
// tile of 128 voxels x 64 channels (FP32). One warpgroup per CTA, thread i
// owns voxel row i: it gathers that voxel's 128 contiguous bytes of the tap
// (channels-last) into the 128-byte-swizzled K-major A tile, and the tap's
// B tile, pre-swizzled by the weight cast, arrives by one bulk copy. Two
// buffers: the gather of tap t + 1 runs under the MMAs of tap t. Every
// mbarrier wait is bounded; one that runs out records an error (read by
// cpmdp_ws_sync) and the CTA stops.

constexpr int kCvThreads = 128;
constexpr int kCvATile = 128 * 128;                  // 128 voxels x 64 bf16
constexpr int kCvBTile = 64 * 128;                   // 64 channels x 64 bf16
constexpr int kCvOffA = 0;
constexpr int kCvOffB = 2 * kCvATile;
constexpr int kCvOffBar = kCvOffB + 2 * kCvBTile;
constexpr int kCvSmem = kCvOffBar + 64 + 1024;
constexpr long long kCvWaitCycles = 2000000000LL;    // about 1 s at 2 GHz

__device__ int g_conv_err = 0;

// Element offset of (row r, k) in a 64-wide bf16 tile with 128-byte rows
// and the 128-byte swizzle (16-byte chunk k / 8 of row r at chunk
// (k / 8) ^ (r % 8)).
__host__ __device__ __forceinline__ int sw_elem(int r, int k) { return r * 64 + ((((k >> 3) ^ (r & 7)) & 7) << 3) + (k & 7); }

__global__ void __launch_bounds__(kCvThreads, 4) conv_tc_kernel(const __nv_bfloat16 *__restrict__ x,
                                                             const uint8_t *__restrict__ wimg,
                                                             const float *__restrict__ bias,
                                                             const __nv_bfloat16 *__restrict__ mask_act,
                                                             __nv_bfloat16 *__restrict__ y, float *__restrict__ y0,
                                                             Dims dm, int dil, int sign, int relu) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bfull = reinterpret_cast<uint64_t *>(sm + kCvOffBar);   // [2] weight tile in
    uint64_t *mdone = bfull + 2;                                      // [2] MMAs of the buffer done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bfull + 4);
    volatile int *sflag = reinterpret_cast<volatile int *>(bfull + 5);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < 4; i++) tc::mbar_init(&bfull[i], 1);
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 64);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t aA = tc::smem_u32(sm + kCvOffA), aB = tc::smem_u32(sm + kCvOffB);
    const int nvox = dm.nvox();
    const int v = blockIdx.x * kCvThreads + tid;
    const bool valid = v < nvox;
    int xx = 0, yy = 0, zz = 0, nn = 0;
    if (valid) {
        int r = v;
        xx = r % dm.x; r /= dm.x;
        yy = r % dm.y; r /= dm.y;
        zz = r % dm.z; nn = r / dm.z;
    }
    int last = -1;             // thread 0: last tap whose MMAs were committed
    int ptap0 = -1, ptap1 = -1;   // thread 0: tap of a weight copy (buffer 0 / 1) not yet waited for
    bool ok = true;
    for (int t = 0; t < 27; t++) {
        const int b = t & 1;
        // the MMAs of tap t - 2 read buffer b
        if (t >= 2 && !tc::mbar_wait(&mdone[b], (uint32_t)(((t >> 1) - 1) & 1), kCvWaitCycles)) *sflag = 1;
        if (tid == 0 && !*sflag) {
            tc::mbar_expect_tx(&bfull[b], kCvBTile);
            tc::bulk_g2s(aB + b * kCvBTile, wimg + (size_t)t * kCvBTile, kCvBTile, &bfull[b]);
            if (b) ptap1 = t; else ptap0 = t;
        }
        const int oz = sign * dil * (t / 9 - 1), oy = sign * dil * ((t / 3) % 3 - 1), ox = sign * dil * (t % 3 - 1);
        const int z2 = zz + oz, y2 = yy + oy, x2 = xx + ox;
        uint4 row[8];
        if (valid && z2 >= 0 && z2 < dm.z && y2 >= 0 && y2 < dm.y && x2 >= 0 && x2 < dm.x) {
            const uint4 *src = reinterpret_cast<const uint4 *>(x + ((size_t)((nn * dm.z + z2) * dm.y + y2) * dm.x + x2) * kC);
#pragma unroll
            for (int j = 0; j < 8; j++) row[j] = src[j];
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++) row[j] = make_uint4(0u, 0u, 0u, 0u);
        }
        uint8_t *arow = sm + kCvOffA + b * kCvATile + tid * 128;
#pragma unroll
        for (int j = 0; j < 8; j++) *reinterpret_cast<uint4 *>(arow + ((j ^ (tid & 7)) << 4)) = row[j];
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (*sflag) { ok = false; break; }
        if (tid == 0) {
            if (!tc::mbar_wait(&bfull[b], (uint32_t)((t >> 1) & 1), kCvWaitCycles)) {
                *sflag = 1;
            } else {
                if (b) ptap1 = -1; else ptap0 = -1;
#pragma unroll
                for (int ks = 0; ks < 4; ks++)
                    tc::mma(tmem, tc::sdesc(aA + b * kCvATile + ks * 32), tc::sdesc(aB + b * kCvBTile + ks * 32),
                            tc::kIdescM128N64, (t > 0 || ks > 0) ? 1u : 0u);
                tc::commit(&mdone[b]);
                last = t;
            }
        }
    }
    // tap 26 (buffer 0, its 14th use) completes after every earlier MMA
    if (ok && !tc::mbar_wait(&mdone[0], 1u, kCvWaitCycles)) *sflag = 1;
    __syncthreads();
    if (*sflag) {
        if (tid == 0) {
            atomicExch(&g_conv_err, 1);
            // let copies and MMAs still in flight finish before the CTA's shared memory goes
            if (ptap0 >= 0) tc::mbar_wait(&bfull[0], (uint32_t)((ptap0 >> 1) & 1), kCvWaitCycles);
            if (ptap1 >= 0) tc::mbar_wait(&bfull[1], (uint32_t)((ptap1 >> 1) & 1), kCvWaitCycles);
            if (last >= 0) tc::mbar_wait(&mdone[last & 1], (uint32_t)((last >> 1) & 1), kCvWaitCycles);
        }
    } else {
        tc::fence_after();
        float acc[64];
        tc::tmem_ld64(tmem + ((uint32_t)(32 * warp) << 16), acc);
        if (valid) {
#pragma unroll
            for (int n = 0; n < 64; n++) acc[n] += bias ? bias[n] : 0.f;
            if (mask_act) {
                const uint4 *mrow = reinterpret_cast<const uint4 *>(mask_act + (size_t)v * kC);
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const uint4 m = mrow[j];
                    const uint32_t w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                    for (int h = 0; h < 8; h++) {
                        const uint16_t bits = (uint16_t)(w[h >> 1] >> (16 * (h & 1)));
                        if (!(bf(__ushort_as_bfloat16(bits)) > 0.f)) acc[8 * j + h] = 0.f;
                    }
                }
            }
            uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)v * kC);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    float a0 = acc[8 * j + 2 * h], a1 = acc[8 * j + 2 * h + 1];
                    if (relu) { a0 = fmaxf(a0, 0.f); a1 = fmaxf(a1, 0.f); }
                    if (j == 0 && h == 0 && y0) y0[v] = a0;
                    w[h] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a0)) |
                           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a1)) << 16);
                }
                dst[j] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
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
        for (int z = cz * kF; z < min((cz + 1) * kF, I.shape[0]); z++)
            for (int y = cy * kF; y < min((cy + 1) * kF, I.shape[1]); y++)
                for (int x = cx * kF; x < min((cx + 1) * kF, I.shape[2]); x++) {
                    const long long s = I.offset + (long long)z * I.stride[0] + y * I.stride[1] + x;
                    const unsigned c = code[s];
                    n++;
                    if (c & ob) { obst++; continue; }
                    live++;
                    rsum += R[s];
                    if (c & tb) { tmax = any_t ? fmaxf(tmax, R[s]) : R[s]; any_t = 1; }
                }
        __nv_bfloat16 *f = feat + g * kC;
        f[0] = __float2bfloat16_rn(live ? rsum / live : 0.f);
        f[1] = __float2bfloat16_rn((float)obst / (float)n);
        f[2] = __float2bfloat16_rn(any_t ? tmax : 0.f);
        f[3] = __float2bfloat16_rn(-logf(1.f - I.gamma) / 5.f);
        for (int c = 4; c < kC; c++) f[c] = __float2bfloat16_rn(0.f);
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

// Coarse estimate (plus base, if given) at the cell centres, interpolated
// trilinearly to every fine state: a fine coordinate x sits at
// (x + 0.5) / 4 - 0.5 in cell units, clamped to the outermost centres.
// Terminals take R(t), obstacles 0.
__global__ void upsample_kernel(const BatchInst *__restrict__ inst, const uint8_t *__restrict__ code,
                                const float *__restrict__ R, int first, int count, int cells,
                                const float *__restrict__ coarse, const float *__restrict__ base,
                                float *__restrict__ V) {
    const BatchInst I0 = inst[first];
    const long long per = I0.nstates;
    const long long total = (long long)count * per;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / per);
        const int s = (int)(g % per);
        const BatchInst I = inst[first + i];
        const int z = s / I.stride[0], y = (s / I.stride[1]) % I.shape[1], x = s % I.shape[2];
        const int zc = (I.shape[0] + kF - 1) / kF, yc = (I.shape[1] + kF - 1) / kF, xc = (I.shape[2] + kF - 1) / kF;
        const unsigned c = code[I.offset + s];
        float v;
        if (c & (1u << (2 * I.ndim))) {
            v = 0.f;
        } else if (c & (1u << (2 * I.ndim + 1))) {
            v = R[I.offset + s];
        } else {
            int lo[3], hi[3];
            float t[3];
            const int pos[3] = {z, y, x}, nc[3] = {zc, yc, xc};
#pragma unroll
            for (int d = 0; d < 3; d++) {
                float u = ((float)pos[d] + 0.5f) / (float)kF - 0.5f;
                u = fminf(fmaxf(u, 0.f), (float)(nc[d] - 1));
                lo[d] = (int)floorf(u);
                hi[d] = min(lo[d] + 1, nc[d] - 1);
                t[d] = u - (float)lo[d];
            }
            const float *cv = coarse + (long long)i * cells;
            const float *bv = base ? base + (long long)i * cells : nullptr;
            v = 0.f;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int cz = (k & 4) ? hi[0] : lo[0], cy = (k & 2) ? hi[1] : lo[1], cx = (k & 1) ? hi[2] : lo[2];
                const float w = ((k & 4) ? t[0] : 1.f - t[0]) * ((k & 2) ? t[1] : 1.f - t[1]) *
                                ((k & 1) ? t[2] : 1.f - t[2]);
                const int cell = (cz * yc + cy) * xc + cx;
                v += w * (cv[cell] + (bv ? bv[cell] : 0.f));
            }
        }
        V[I.offset + s] = v;
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

__device__ __forceinline__ unsigned float_key(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void __launch_bounds__(kCoarseThreads) coarse_vi_kernel(const BatchInst *__restrict__ inst,
                                                                   const uint8_t *__restrict__ code,
                                                                   const float *__restrict__ R, int first, int cells,
                                                                   float tol, int max_sweeps,
                                                                   float *__restrict__ coarse_v,
                                                                   __nv_bfloat16 *__restrict__ feat) {
    extern __shared__ uint8_t smem_raw[];
    int *n_obst = reinterpret_cast<int *>(smem_raw);                 // later: V (even sweeps)
    int *n_free = n_obst + cells;                                    // later: V (odd sweeps)
    float *rsum = reinterpret_cast<float *>(n_free + cells);         // later: coarse reward
    unsigned *tkey = reinterpret_cast<unsigned *>(rsum + cells);     // largest terminal reward (0: none)
    uint8_t *kind = reinterpret_cast<uint8_t *>(tkey + cells);      // bits 0-5 blocked moves, 6 obstacle, 7 terminal
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const BatchInst I = inst[first + i];
    const int zc = (I.shape[0] + kF - 1) / kF, yc = (I.shape[1] + kF - 1) / kF, xc = (I.shape[2] + kF - 1) / kF;
    for (int c = tid; c < cells; c += kCoarseThreads) {
        n_obst[c] = 0;
        n_free[c] = 0;
        rsum[c] = 0.f;
        tkey[c] = 0u;
    }
    __syncthreads();
    const unsigned ob = 1u << (2 * I.ndim), tb = 1u << (2 * I.ndim + 1);
    for (int s = tid; s < I.nstates; s += kCoarseThreads) {   // coalesced over the fine states
        const int z = s / I.stride[0], y = (s / I.stride[1]) % I.shape[1], x = s % I.shape[2];
        const int c = ((z / kF) * yc + y / kF) * xc + x / kF;
        const unsigned cs = code[I.offset + s];
        if (cs & ob) { atomicAdd(&n_obst[c], 1); continue; }
        const float r = R[I.offset + s];
        if (cs & tb) { atomicMax(&tkey[c], float_key(r)); continue; }
        atomicAdd(&n_free[c], 1);
        atomicAdd(&rsum[c], r);
    }
    __syncthreads();
    const float g = I.gamma;
    const float gc = g * g * g * g, steps = 1.f + g + g * g + g * g * g;
    for (int c = tid; c < cells; c += kCoarseThreads) {
        const int cz = c / (yc * xc), cy = (c / xc) % yc, cx = c % xc;
        const int n = (min((cz + 1) * kF, I.shape[0]) - cz * kF) * (min((cy + 1) * kF, I.shape[1]) - cy * kF) *
                      (min((cx + 1) * kF, I.shape[2]) - cx * kF);
        uint8_t k = 0;
        float r = 0.f;
        if (2 * n_obst[c] >= n) k = 0x40;
        else if (tkey[c]) { k = 0x80; r = key_float(tkey[c]); }
        else r = n_free[c] ? rsum[c] / (float)n_free[c] * steps : 0.f;
        kind[c] = k;
        rsum[c] = r;
    }
    __syncthreads();
    float *va = reinterpret_cast<float *>(n_obst), *vb = reinterpret_cast<float *>(n_free);
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
// must be 3-D and of one shape; returns the coarse cell count.
static cpmdp_status batch_range(const cpmdp_batch *B, int first, int count, int *cells) {
    if (!B || count < 1 || first < 0 || first + count > B->ninst) { set_error("instance range outside the batch"); return CPMDP_EINVAL; }
    const BatchInst &I0 = B->inst[(size_t)first];
    if (I0.ndim != 3) { set_error("the warm start takes 3-D instances"); return CPMDP_EINVAL; }
    for (int i = first; i < first + count; i++) {
        const BatchInst &I = B->inst[(size_t)i];
        if (I.ndim != 3 || I.shape[0] != I0.shape[0] || I.shape[1] != I0.shape[1] || I.shape[2] != I0.shape[2] ||
            I.offset != I0.offset + (long long)(i - first) * I0.nstates) {
            set_error("instances %d..%d must share one shape and be contiguous", first, first + count - 1);
            return CPMDP_EINVAL;
        }
    }
    *cells = ((I0.shape[0] + kF - 1) / kF) * ((I0.shape[1] + kF - 1) / kF) * ((I0.shape[2] + kF - 1) / kF);
    return CPMDP_OK;
}

static cudaError_t launch_conv(const __nv_bfloat16 *x, const uint8_t *wimg, const float *bias,
                               const __nv_bfloat16 *mask_act, __nv_bfloat16 *y, float *y0, Dims dm, int dil, int sign,
                               int relu, cudaStream_t st) {
    const cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCvSmem);
    if (e != cudaSuccess) return e;
    conv_tc_kernel<<<(dm.nvox() + kCvThreads - 1) / kCvThreads, kCvThreads, kCvSmem, st>>>(x, wimg, bias, mask_act, y,
                                                                                         y0, dm, dil, sign, relu);
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
    const long long n = (long long)count * B->inst[(size_t)first].nstates;
    upsample_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, B->d_R, first, count,
                                                                        cells, coarse, base, V);
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
    const size_t smem = (size_t)cells * 17;
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
