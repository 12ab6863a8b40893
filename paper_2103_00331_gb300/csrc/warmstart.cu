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
//   conv_kernel      y[v, n] = sum_t sum_k x[v + s d off(t), k] w[t, k, n] (+ b, ReLU, mask)
//                    forward (s = +1, w = W^T per tap) and data gradient
//                    (s = -1, w = W per tap, times the ReLU mask of the
//                    layer input), a 64-voxel x 64-channel tile per block
//   conv_dw_kernel   dW[t, co, ci] = sum_v dy[v, co] x[v + d off(t), ci]
//   plus features / targets / upsampling from a packed batch, the loss
//   gradient, Adam and the FP32 -> BF16 weight casts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "batch_internal.h"

namespace cpmdp {

constexpr int kC = 64;        // channels of every activation
constexpr int kF = 4;         // coarsening factor per dimension

struct Dims {
    int n, z, y, x;           // instances and coarse grid
    __host__ __device__ int nvox() const { return n * z * y * x; }
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------------------
// convolution (forward and data gradient)

__global__ void __launch_bounds__(256) conv_kernel(const __nv_bfloat16 *__restrict__ x,
                                                   const __nv_bfloat16 *__restrict__ wk,
                                                   const float *__restrict__ bias,
                                                   const __nv_bfloat16 *__restrict__ mask_act,
                                                   __nv_bfloat16 *__restrict__ y, float *__restrict__ y0,
                                                   Dims dm, int dil, int sign, int relu) {
    __shared__ float sA[64][65];   // [voxel][k]
    __shared__ float sB[64][65];   // [k][n]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int v0 = blockIdx.x * 64;
    const int nvox = dm.nvox();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
    for (int t = 0; t < 27; t++) {
        const int oz = sign * dil * (t / 9 - 1), oy = sign * dil * ((t / 3) % 3 - 1), ox = sign * dil * (t % 3 - 1);
        for (int e = tid; e < 64 * 64; e += 256) {
            const int vv = e >> 6, k = e & 63;
            const int v = v0 + vv;
            float val = 0.f;
            if (v < nvox) {
                int r = v;
                const int xx = r % dm.x; r /= dm.x;
                const int yy = r % dm.y; r /= dm.y;
                const int zz = r % dm.z; const int nn = r / dm.z;
                const int z2 = zz + oz, y2 = yy + oy, x2 = xx + ox;
                if (z2 >= 0 && z2 < dm.z && y2 >= 0 && y2 < dm.y && x2 >= 0 && x2 < dm.x)
                    val = bf(x[((size_t)((nn * dm.z + z2) * dm.y + y2) * dm.x + x2) * kC + k]);
            }
            sA[vv][k] = val;
            sB[vv][k] = bf(wk[(size_t)t * kC * kC + e]);   // e = k_row * 64 + n
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 64; k++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = sA[ty + 16 * i][k];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = sB[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int v = v0 + ty + 16 * i;
        if (v >= nvox) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int n = tx + 16 * j;
            float val = acc[i][j] + (bias ? bias[n] : 0.f);
            if (mask_act && !(bf(mask_act[(size_t)v * kC + n]) > 0.f)) val = 0.f;
            if (relu) val = fmaxf(val, 0.f);
            y[(size_t)v * kC + n] = __float2bfloat16_rn(val);
            if (y0 && n == 0) y0[v] = val;
        }
    }
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

// W [t][co][ci] (FP32) -> wf [t][ci][co] (forward operand) and wb [t][co][ci] (data gradient operand)
__global__ void cast_weights_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf,
                                    __nv_bfloat16 *__restrict__ wb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / (kC * kC), r = i % (kC * kC), co = r / kC, ci = r % kC;
        const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
        wb[i] = h;
        wf[t * kC * kC + ci * kC + co] = h;
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
                               float *__restrict__ target, float *__restrict__ mask) {
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
        target[g] = live ? s / live : 0.f;
        mask[g] = live ? 1.f : 0.f;
    }
}

__global__ void upsample_kernel(const BatchInst *__restrict__ inst, const uint8_t *__restrict__ code,
                                const float *__restrict__ R, int first, int count, int cells,
                                const float *__restrict__ coarse, float *__restrict__ V) {
    const BatchInst I0 = inst[first];
    const long long per = I0.nstates;
    const long long total = (long long)count * per;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / per);
        const int s = (int)(g % per);
        const BatchInst I = inst[first + i];
        const int z = s / I.stride[0], y = (s / I.stride[1]) % I.shape[1], x = s % I.shape[2];
        const int xc = (I.shape[2] + kF - 1) / kF, yc = (I.shape[1] + kF - 1) / kF;
        const int cell = ((z / kF) * yc + y / kF) * xc + x / kF;
        const unsigned c = code[I.offset + s];
        float v = coarse[(long long)i * cells + cell];
        if (c & (1u << (2 * I.ndim + 1))) v = R[I.offset + s];
        if (c & (1u << (2 * I.ndim))) v = 0.f;
        V[I.offset + s] = v;
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

cpmdp_status cpmdp_ws_targets(const cpmdp_batch *B, const float *V, int32_t first, int32_t count, float *target,
                              float *mask, void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    const long long n = (long long)count * cells;
    targets_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, V, first, count, cells,
                                                                       target, mask);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_ws_upsample(const cpmdp_batch *B, const float *coarse, int32_t first, int32_t count, float *V,
                               void *stream) {
    int cells = 0;
    cpmdp_status s = batch_range(B, first, count, &cells);
    if (s != CPMDP_OK) return s;
    const long long n = (long long)count * B->inst[(size_t)first].nstates;
    upsample_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(B->d_inst, B->d_code, B->d_R, first, count,
                                                                        cells, coarse, V);
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
    conv_kernel<<<(dm.nvox() + 63) / 64, 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)wf, bias, nullptr, (__nv_bfloat16 *)y, y0, dm, dilation, 1,
        relu);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

cpmdp_status cpmdp_conv3d_backward_data(const uint16_t *dy, const uint16_t *wb, const uint16_t *act_in, uint16_t *dx,
                                        int32_t n, int32_t z, int32_t yy, int32_t xx, int32_t dilation, void *stream) {
    cpmdp_status s = dims_ok(n, z, yy, xx, dilation);
    if (s != CPMDP_OK) return s;
    if (!dy || !wb || !dx) { set_error("dy, w and dx are required"); return CPMDP_EINVAL; }
    Dims dm{n, z, yy, xx};
    conv_kernel<<<(dm.nvox() + 63) / 64, 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)dy, (const __nv_bfloat16 *)wb, nullptr, (const __nv_bfloat16 *)act_in,
        (__nv_bfloat16 *)dx, nullptr, dm, dilation, -1, 0);
    CPMDP_CUDA(cudaGetLastError());
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

}  // extern "C"
