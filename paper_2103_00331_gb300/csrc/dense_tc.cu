// Dense CP backup on the tcgen05 tensor cores, BF16x3 (shapes 64^4).
//
// E_a[V] = sum_r lambda_{a,r} V x_1 U_{a,r,1} x_2 U_{a,r,2} x_3 U_{a,r,3} x_4 U_{a,r,4}
// (the CP form applied per action; Eq. 1 then takes R + gamma max_a E_a).
// Matricise V as a 4096 x 4096 matrix with rows (i1,i2) and columns (i3,i4):
// E = (U_1 (x) U_2) V (U_3 (x) U_4)^T. Two passes, each applying two modes
// to 64 x 64 slabs entirely on chip:
//
//  pass A, per chain c = (a, r) and slab b = (i1,i2) of V (rows i3, cols i4):
//    Z = X U_4^T            (GEMM 1, M = 2 slabs x 64 rows, N = 64, K = 64)
//    Y^T = Z^T U_3^T        (GEMM 2, A operand = Z^T written by the threads)
//    T_c[(i3',i4')][(i1,i2)] = Y[i3',i4']   (bf16 hi/lo pairs, 4 bytes)
//  pass B, per slab q = (i3',i4') of T_c (rows i1, cols i2), ranks of one
//  action accumulated in TMEM (lambda is folded into U_1):
//    W = Z U_2^T, E^T += W^T (lambda U_1)^T
//    then max / argmax over actions in registers, V' = R + gamma max_a E_a
//    (exact: rounding is monotone and gamma >= 0), residual max |V' - V|.
//
// Each GEMM is D = A B^T with K-major 128B-swizzled tiles, run as BF16x3
// (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation in TMEM): about 16
// significant bits per operand. Value iteration corrects the remaining error
// against a base expectation E_a(V_base) computed in FP32 (defect
// correction: E_a(V) = E_a(V_base) + E_a^{bf16x3}(V - V_base)); the base is
// refreshed when the residual stops falling. One FP64 sweep certifies the
// result.
//
// One warpgroup per CTA (thread t owns TMEM lane t). Every mbarrier wait is
// bounded; a wait that runs out sets the error word and the CTA stops.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace cpmdp {

constexpr int kN = 64;
constexpr int kSlab = 4096;               // elements of one 64 x 64 slab
constexpr long long kS = 16777216LL;      // 64^4 states
constexpr int kTileBytes = 8192;          // 64 x 64 bf16 tile
constexpr int kPairBytes = 16384;         // 128 x 64 bf16 tile
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

// U tiles in global memory, pre-split and pre-swizzled:
// ((c * 4 + d) * 2 + part) * 8192 bytes, part 0 = hi, 1 = lo; d = 0 holds lambda U_1.
__device__ __forceinline__ const uint8_t *utile(const uint8_t *U, int c, int d, int part) {
    return U + ((size_t)(c * 4 + d) * 2 + part) * kTileBytes;
}

__device__ __forceinline__ void put_bf16(uint8_t *tile, uint32_t row, uint32_t k, uint16_t v) {
    *reinterpret_cast<uint16_t *>(tile + tc::sw128_off(row, k)) = v;
}

// Uniform wait: every thread waits; the CTA continues only if all succeeded.
__device__ __forceinline__ bool wait_all(uint64_t *mbar, uint32_t &phase, int *err) {
    const bool ok = tc::mbar_wait(mbar, phase, kWaitCycles);
    phase ^= 1u;
    const int all = __syncthreads_and(ok ? 1 : 0);
    if (!all && threadIdx.x == 0) atomicExch(err, (int)CPMDP_ETIMEOUT);
    return all != 0;
}

__device__ __forceinline__ void sync_for_async() {
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// Intermediate layout: for chain c and pass-B slab pair P (slabs q = 2P and
// 2P + 1, q = (i3', i4')), a 32 KB tile of 64 rows (i1) x 16 quad pairs;
// quad j of row i1 of slab q (16 bytes at (c * 4096 + 2P) * 16384 +
// ((i1 * 16 + j) * 2 + (q & 1)) * 16) holds the bf16 hi parts of
// k = i2 = 4j .. 4j+3 followed by their lo parts. Pass A writes whole quads,
// the two slabs of a pair side by side, so two adjacent lanes fill one
// 32-byte sector; pass B copies a slab pair (32 KB, contiguous) with one
// bulk copy.
constexpr int kQuadTileBytes = 16384;

// Quads of one staged item (chain c, slab group starting at b0), those with
// q in [q_lo, q_hi): the stage buffer holds the FP32 results ([slab][q]);
// each quad is split into bf16 hi / lo parts (split_bf16 on each value) and
// written as one 16-byte unit of the intermediate layout.
__device__ __forceinline__ void write_quads(uint8_t *T, const uint32_t *stage, int c, int b0, int q_lo, int q_hi,
                                            int tid, int nthreads) {
    uint8_t *Tc = T + (size_t)c * kSlab * kQuadTileBytes + (size_t)((b0 >> 6) * 16 + ((b0 & 63) >> 2)) * 32;
    for (int q = q_lo + tid; q < q_hi; q += nthreads) {
        const float x0 = __uint_as_float(stage[q]), x1 = __uint_as_float(stage[kSlab + q]);
        const float x2 = __uint_as_float(stage[2 * kSlab + q]), x3 = __uint_as_float(stage[3 * kSlab + q]);
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(x0, x1), h23 = __floats2bfloat162_rn(x2, x3);
        const __nv_bfloat162 l01 = __floats2bfloat162_rn(x0 - __low2float(h01), x1 - __high2float(h01));
        const __nv_bfloat162 l23 = __floats2bfloat162_rn(x2 - __low2float(h23), x3 - __high2float(h23));
        uint4 v;
        v.x = *reinterpret_cast<const uint32_t *>(&h01);
        v.y = *reinterpret_cast<const uint32_t *>(&h23);
        v.z = *reinterpret_cast<const uint32_t *>(&l01);
        v.w = *reinterpret_cast<const uint32_t *>(&l23);
        *reinterpret_cast<uint4 *>(Tc + (size_t)(q >> 1) * (2 * kQuadTileBytes) + (q & 1) * 16) = v;
    }
}

// ---------------------------------------------------------------------------
// pass A: slabs of V (minus V_base when given) -> T_c for every chain c
//
// Warp-specialised in three roles. An item is (slab group g, chain c); per
// item and pair p of the group's two slab pairs:
//   GEMM 1 (D1[p]) = X_p U_4^T            rows (s2, i3), cols i4'
//   CONV (group C): D1[p] -> A2 (bf16 hi/lo, MN-major: each thread writes
//        its own accumulator row as 16-byte chunks, no transpose)
//   GEMM 2 (D2[p]) = A2 U_3^T             rows (s2, i4'), cols i3'
//   EPI (group E): D2[p] -> stage (FP32); after both pairs, the item's
//        quads (split to bf16 hi / lo) -> T.
// One control thread issues the GEMMs (the next item's GEMM 1 ahead of this
// item's GEMM 2) and the factor copies (U_3 and U_4 rings, refilled as soon
// as the GEMM that read a slot completes). The two converter groups (8 warps
// of 8 and 16 warps, two and four per TMEM lane quarter) never wait for each other: group C works
// on one item's conversions while group E writes out another's quads, and
// the tensor core runs the GEMMs in between. Within a group the warps decide
// every wait together (named AND barrier of the group), so a wait that runs
// out stops the whole group and no named barrier is left half-entered; the
// error word is set and every role leaves its loop.

constexpr int kAGroupC = 256;                        // group C: 8 warps, 32 accumulator columns per thread
constexpr int kAGroupE = 512;                        // group E: 16 warps, 16 columns per thread
constexpr int kAThreads = kAGroupC + kAGroupE + 32;  // + the control warp
constexpr int kAColsC = 64 * 128 / kAGroupC, kAColsE = 64 * 128 / kAGroupE;
constexpr int kAOffX = 0;                            // 2 pairs x {hi, lo} x 16 KB, K-major
constexpr int kAOffA2 = 4 * kPairBytes;              // {hi, lo} x 16 KB, MN-major
constexpr int kAOffU = kAOffA2 + 2 * kPairBytes;     // U3 slots 0, 1 then U4 slots 0, 1 ({hi, lo} each)
constexpr int kAOffStage = kAOffU + 2 * 4 * kTileBytes;  // 4 slabs x 4096 FP32 results
constexpr int kAOffBar = kAOffStage + 4 * kSlab * 4;
constexpr int kASmem = kAOffBar + 192 + 1024;
constexpr uint32_t kBarC = 1, kBarE = 2;             // named barriers of the two groups

// Group-side wait: lane 0 of every warp of the group polls the mbarrier
// (bounded); the group (n threads) then agrees on the outcome (named AND
// barrier).
__device__ __forceinline__ bool group_wait(uint64_t *mbar, uint32_t parity, int lane, uint32_t bar, uint32_t n) {
    bool ok = true;
    if (lane == 0) ok = tc::mbar_wait(mbar, parity, kWaitCycles);
    ok = __shfl_sync(0xFFFFFFFFu, ok ? 1 : 0, 0) != 0;
    return tc::named_and(bar, n, ok);
}

// Stage the group's 4 slabs (b0 .. b0+3) of V (- V_base) as two K-major
// pair tiles, bf16 hi / lo: row = (s % 2) * 64 + i3, k = i4 (by the
// kAGroupC threads of group C, gtid = 0 .. kAGroupC - 1).
__device__ __forceinline__ void stage_x(uint8_t *sX, const float *V, const float *Vbase, int b0, int gtid) {
    for (int e4 = gtid; e4 < kSlab; e4 += kAGroupC) {   // 4 consecutive elements per step
        const int s = e4 >> 10, rem = (e4 & 1023) * 4;
        const size_t gi = (size_t)(b0 + s) * kSlab + rem;
        float4 x = *reinterpret_cast<const float4 *>(V + gi);
        if (Vbase) {
            const float4 y = *reinterpret_cast<const float4 *>(Vbase + gi);
            x.x -= y.x; x.y -= y.y; x.z -= y.z; x.w -= y.w;
        }
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(x.x, x.y), h1 = __floats2bfloat162_rn(x.z, x.w);
        const __nv_bfloat162 l0 = __floats2bfloat162_rn(x.x - __low2float(h0), x.y - __high2float(h0));
        const __nv_bfloat162 l1 = __floats2bfloat162_rn(x.z - __low2float(h1), x.w - __high2float(h1));
        uint8_t *tile = sX + (s >> 1) * 2 * kPairBytes;
        const uint32_t off = tc::sw128_off((uint32_t)((s & 1) * 64 + (rem >> 6)), (uint32_t)(rem & 63));
        *reinterpret_cast<uint2 *>(tile + off) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1));
        *reinterpret_cast<uint2 *>(tile + kPairBytes + off) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&l0), *reinterpret_cast<const uint32_t *>(&l1));
    }
}

__global__ void __launch_bounds__(kAThreads, 1) dense_pass_a(const float *__restrict__ V, const float *__restrict__ Vbase,
                                                       const uint8_t *__restrict__ U, uint8_t *__restrict__ T,
                                                       int nchains, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sX = sm + kAOffX;
    uint8_t *sA2 = sm + kAOffA2;
    uint32_t *stage = reinterpret_cast<uint32_t *>(sm + kAOffStage);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kAOffBar);
    uint64_t *d1_full = bars + 0, *d1_empty = bars + 2, *d2_full = bars + 4, *d2_empty = bars + 6;
    uint64_t *a2_full = bars + 8, *u3_full = bars + 10, *u3_free = bars + 12, *u4_full = bars + 14;
    uint64_t *u4_free = bars + 16, *x_full = bars + 18, *fin = bars + 19;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kAOffBar + 160);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        // d1_empty, d2_empty and a2_full take one arrival per warp of their group
        for (int i = 0; i < 20; i++) {
            const bool by_c = (i >= 2 && i < 4) || (i >= 8 && i < 10), by_e = i >= 6 && i < 8;
            tc::mbar_init(&bars[i], by_c ? kAGroupC / 32 : by_e ? kAGroupE / 32 : 1);
        }
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;   // D1[p] at column 64 p, D2[p] at 128 + 64 p
    const int ngroups = kSlab / 4;
    const int my_groups = blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int nitems = my_groups * nchains;
    // converter threads: accumulator row (TMEM lane; warp w reads lane quarter w % 4)
    const int row = tid & 127;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int s2 = row >> 6, r63 = row & 63;

    if (warp == (kAGroupC + kAGroupE) / 32) {
        // ---------------- control thread ----------------
        // Issue order: GEMM 1 of item 0, then per item it: GEMM 2 (it, p0),
        // GEMM 1 (it+1, p0), GEMM 2 (it, p1), GEMM 1 (it+1, p1) (at a group
        // change both GEMM 2 first: X is restaged after this item's CONV).
        if (lane == 0 && nitems > 0) {
            const uint32_t aX = tc::smem_u32(sX), aA2 = tc::smem_u32(sA2), aU = tc::smem_u32(sm + kAOffU);
            int issued3 = 0, landed3 = 0, issued4 = 0, landed4 = 0;   // factor copies issued / waited for
            auto issue_u3 = [&]() {
                const int j = issued3++, sl = j & 1;
                tc::mbar_expect_tx(&u3_full[sl], 2 * kTileBytes);
                tc::bulk_g2s(aU + sl * 2 * kTileBytes, utile(U, j % nchains, 2, 0), 2 * kTileBytes, &u3_full[sl]);
            };
            auto issue_u4 = [&]() {
                const int j = issued4++, sl = j & 1;
                tc::mbar_expect_tx(&u4_full[sl], 2 * kTileBytes);
                tc::bulk_g2s(aU + (2 + sl) * 2 * kTileBytes, utile(U, j % nchains, 3, 0), 2 * kTileBytes,
                             &u4_full[sl]);
            };
            // GEMM 1 (j, p) once group C has read D1[p] of item j-1; for p = 0
            // also X (first chain of a group) and U4 of item j
            auto gemm1 = [&](int j, int p) -> bool {
                const int sl = j & 1;
                if (p == 0) {
                    if (j % nchains == 0 && !tc::mbar_wait(x_full, (uint32_t)((j / nchains) & 1), kWaitCycles))
                        return false;
                    if (!tc::mbar_wait(&u4_full[sl], (uint32_t)((j >> 1) & 1), kWaitCycles)) return false;
                    landed4++;
                }
                if (!tc::mbar_wait(&d1_empty[p], (uint32_t)((j & 1) ^ 1), kWaitCycles)) return false;
                tc::fence_after();
                const uint32_t xa = aX + p * 2 * kPairBytes, u4 = aU + (2 + sl) * 2 * kTileBytes;
                tc::mma_bf16x3(tmem + 64 * p, xa, xa + kPairBytes, u4, u4 + kTileBytes, 0);
                tc::commit(&d1_full[p]);
                if (p == 1) tc::commit(&u4_free[sl]);
                return true;
            };
            // GEMM 2 (it, p) once group C wrote A2 and group E has read D2[p] of item it-1
            auto gemm2 = [&](int it, int p) -> bool {
                const int sl = it & 1;
                if (!tc::mbar_wait(&a2_full[p], (uint32_t)(it & 1), kWaitCycles)) return false;
                if (!tc::mbar_wait(&d2_empty[p], (uint32_t)((it & 1) ^ 1), kWaitCycles)) return false;
                tc::fence_after();
                const uint32_t u3 = aU + sl * 2 * kTileBytes;
                tc::mma_bf16x3_amn(tmem + 128 + 64 * p, aA2, aA2 + kPairBytes, u3, u3 + kTileBytes, 0);
                tc::commit(&d2_full[p]);
                if (p == 1) tc::commit(&u3_free[sl]);
                return true;
            };
            issue_u4();
            issue_u3();
            if (nitems > 1) {
                issue_u4();
                issue_u3();
            }
            bool ok = gemm1(0, 0) && gemm1(0, 1);
            for (int it = 0; it < nitems && ok; it++) {
                const int sl = it & 1;
                ok = tc::mbar_wait(&u3_full[sl], (uint32_t)((it >> 1) & 1), kWaitCycles);
                if (!ok) break;
                landed3++;
                const bool next = it + 1 < nitems, newgroup = next && (it + 1) % nchains == 0;
                ok = gemm2(it, 0);
                // U3 of item it+1 into the slot GEMM 2 (it-1) has finished with
                if (ok && it >= 1 && next) {
                    ok = tc::mbar_wait(&u3_free[sl ^ 1], (uint32_t)(((it - 1) >> 1) & 1), kWaitCycles);
                    if (ok) issue_u3();
                }
                if (ok && next && !newgroup) ok = gemm1(it + 1, 0);
                ok = ok && gemm2(it, 1);
                if (ok && newgroup) ok = gemm1(it + 1, 0);
                if (ok && next) ok = gemm1(it + 1, 1);
                // U4 of item it+2 into the slot GEMM 1 (it) has finished with (issued an item
                // ago, so this wait rarely blocks; item it+2's GEMM 1 is an item away)
                if (ok && it + 2 < nitems) {
                    ok = tc::mbar_wait(&u4_free[sl], (uint32_t)((it >> 1) & 1), kWaitCycles);
                    if (ok) issue_u4();
                }
            }
            // the last item's commit: every MMA of this CTA has completed
            if (ok) ok = tc::mbar_wait(&u3_free[(nitems - 1) & 1], (uint32_t)(((nitems - 1) >> 1) & 1), kWaitCycles);
            if (!ok) {
                atomicExch(err, (int)CPMDP_ETIMEOUT);
                // let the MMAs and copies already issued finish before the CTA leaves
                tc::commit(fin);
                tc::mbar_wait(fin, 0, kWaitCycles);
                for (int j = landed3; j < issued3; j++)
                    tc::mbar_wait(&u3_full[j & 1], (uint32_t)((j >> 1) & 1), kWaitCycles);
                for (int j = landed4; j < issued4; j++)
                    tc::mbar_wait(&u4_full[j & 1], (uint32_t)((j >> 1) & 1), kWaitCycles);
            }
        }
        __syncwarp();
    } else if (warp < kAGroupC / 32 && nitems > 0) {
        // ---------------- group C: D1 -> A2 ----------------
        // columns cbase .. cbase + 31 of this thread's row, in two halves of 16
        const int cbase = kAColsC * ((warp >> 2) & 1);
        // MN-major A2: this thread's row (s2, i3 = r63) -> k = i3, m = s2 * 64 + i4'
        const uint32_t a2_off = (uint32_t)s2 * 8192u + (uint32_t)(r63 >> 3) * 1024u + (uint32_t)(r63 & 7) * 128u;
        auto store_a2 = [&](int col0, const uint32_t (&hi)[2][4], const uint32_t (&lo)[2][4]) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t chunk = (uint32_t)((col0 >> 3) + h);
                const uint32_t off = a2_off + (((chunk ^ (uint32_t)(r63 & 7)) & 7u) << 4);
                *reinterpret_cast<uint4 *>(sA2 + off) = make_uint4(hi[h][0], hi[h][1], hi[h][2], hi[h][3]);
                *reinterpret_cast<uint4 *>(sA2 + kPairBytes + off) = make_uint4(lo[h][0], lo[h][1], lo[h][2], lo[h][3]);
            }
        };
        bool ok = true;
        stage_x(sX, V, Vbase, 4 * blockIdx.x, tid);
        tc::fence_proxy_async();
        tc::named_sync(kBarC, kAGroupC);
        if (tid == 0) tc::mbar_arrive(x_full);
        for (int it = 0; it < nitems && ok; it++) {
            const int c = it % nchains, gi = it / nchains;
            for (int p = 0; p < 2; p++) {
                ok = group_wait(&d1_full[p], (uint32_t)(it & 1), lane, kBarC, kAGroupC);
                if (!ok) break;
                tc::fence_after();
                float z0[16], z1[16];
                tc::tmem_ld16(tmem + lane_off + 64 * p + cbase, z0);        // row (s2, i3), cols i4'
                tc::tmem_ld16(tmem + lane_off + 64 * p + cbase + 16, z1);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&d1_empty[p]);
                uint32_t hi0[2][4], lo0[2][4], hi1[2][4], lo1[2][4];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    tc::split8_bf16(z0 + 8 * h, hi0[h], lo0[h]);
                    tc::split8_bf16(z1 + 8 * h, hi1[h], lo1[h]);
                }
                // A2 is free once the GEMM 2 that read it last completed: (it-1, p1) before p0, (it, p0) before p1
                if (p == 0 && it >= 1) ok = group_wait(&d2_full[1], (uint32_t)((it - 1) & 1), lane, kBarC, kAGroupC);
                if (p == 1) ok = group_wait(&d2_full[0], (uint32_t)(it & 1), lane, kBarC, kAGroupC);
                if (!ok) break;
                store_a2(cbase, hi0, lo0);
                store_a2(cbase + 16, hi1, lo1);
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&a2_full[p]);
            }
            // last chain of the group: both GEMM 1 of this item are complete, restage X
            if (ok && c == nchains - 1 && gi + 1 < my_groups) {
                stage_x(sX, V, Vbase, 4 * (blockIdx.x + (gi + 1) * gridDim.x), tid);
                tc::fence_proxy_async();
                tc::named_sync(kBarC, kAGroupC);
                if (tid == 0) tc::mbar_arrive(x_full);
            }
        }
        if (!ok && tid == 0) atomicExch(err, (int)CPMDP_ETIMEOUT);
    } else if (warp < (kAGroupC + kAGroupE) / 32 && nitems > 0) {
        // ---------------- group E: D2 -> stage -> quads of T ----------------
        const int etid = tid - kAGroupC;
        const int cbase = kAColsE * ((warp - kAGroupC / 32) >> 2);
        bool ok = true;
        for (int it = 0; it < nitems && ok; it++) {
            const int c = it % nchains, gi = it / nchains;
            const int b0 = 4 * (blockIdx.x + gi * gridDim.x);
            for (int p = 0; p < 2; p++) {
                ok = group_wait(&d2_full[p], (uint32_t)(it & 1), lane, kBarE, kAGroupE);
                if (!ok) break;
                tc::fence_after();
                float y[kAColsE];
                tc::tmem_ld16(tmem + lane_off + 128 + 64 * p + cbase, y);   // row (s2, i4'), cols i3'
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&d2_empty[p]);
                uint32_t *dst = stage + (2 * p + s2) * kSlab + cbase * 64 + r63;
#pragma unroll
                for (int jj = 0; jj < kAColsE; jj++) dst[jj * 64] = __float_as_uint(y[jj]);
            }
            if (!ok) break;
            tc::named_sync(kBarE, kAGroupE);   // the item's four slabs are staged
            write_quads(T, stage, c, b0, 0, kSlab, etid, kAGroupE);
            tc::named_sync(kBarE, kAGroupE);   // and read: the stage is free again
        }
        if (!ok && etid == 0) atomicExch(err, (int)CPMDP_ETIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// pass B: slabs of T_c -> E_a accumulated over ranks -> max over actions
//
// About 106 KB of shared memory, so that two CTAs share an SM and each
// fills the other's MMA and copy waits: one raw slab-pair buffer and one
// factor buffer (each refilled as soon as it is consumed, each with its
// own mbarrier), and one operand buffer that holds Z for the first GEMM and
// then the second GEMM's A operand (Z is consumed once the first GEMM has
// completed).

constexpr int kBOffRaw = 0;                              // raw slab pair, 32 KB
constexpr int kBOffU = kBOffRaw + 2 * kQuadTileBytes;    // U1 hi, lo, U2 hi, lo: 32 KB
constexpr int kBOffZ = kBOffU + 4 * kTileBytes;          // Z / A2 {hi, lo} x 16 KB
constexpr int kBOffArg = kBOffZ + 2 * kPairBytes;        // 64 x 128 argmax bytes
constexpr int kBOffBar = kBOffArg + 64 * 128;
constexpr int kBSmem = kBOffBar + 64 + 1024;

// Two warpgroups per CTA: thread t owns accumulator row t % 128 and
// columns 32 (t / 128) .. +31 (16 warps per SM with two CTAs).
constexpr int kBThreads = 256;
constexpr int kBCols = 64 * 128 / kBThreads;

// eval_pi (policy evaluation, nullable): instead of the max over actions,
// each state keeps the expectation of its own action eval_pi[s] (staged in
// the argmax bytes of shared memory, so no registers are added).
__global__ void __launch_bounds__(kBThreads, 2) dense_pass_b(const uint8_t *__restrict__ T, const uint8_t *__restrict__ U,
                                                       const float *__restrict__ RB, const float *__restrict__ EB,
                                                       const float *__restrict__ Vin, float *__restrict__ Vout,
                                                       uint8_t *__restrict__ pi, const uint8_t *__restrict__ eval_pi,
                                                       int nact, int nrank, float gamma, unsigned long long *res,
                                                       int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sZ = sm + kBOffZ;
    uint8_t *sArg = sm + kBOffArg;
    uint64_t *full_raw = reinterpret_cast<uint64_t *>(sm + kBOffBar);
    uint64_t *full_u = reinterpret_cast<uint64_t *>(sm + kBOffBar + 8);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + kBOffBar + 16);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kBOffBar + 24);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        tc::mbar_init(full_raw, 1);
        tc::mbar_init(full_u, 1);
        tc::mbar_init(mbar, 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sync_for_async();
    const uint32_t tmem = *tslot;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int row = tid & 127, cbase = kBCols * (tid >> 7);   // accumulator row, first column
    uint32_t mph = 0, rph = 0, uph = 0;
    // a copy issued and not yet waited for (its phase is flipped already
    // when its own wait ran out)
    bool alive = true, raw_pending = false, u_pending = false, raw_failed = false, u_failed = false;
    const uint32_t aRaw = tc::smem_u32(sm + kBOffRaw), aU = tc::smem_u32(sm + kBOffU), aZ = tc::smem_u32(sZ);
    const int npairs = kSlab / 2, nchains = nact * nrank;
    double local_res = 0.0;

    auto issue_raw = [&](int P, int c) {
        tc::mbar_expect_tx(full_raw, 2 * kQuadTileBytes);
        tc::bulk_g2s(aRaw, T + ((size_t)c * kSlab + 2 * P) * kQuadTileBytes, 2 * kQuadTileBytes, full_raw);
    };
    auto issue_u = [&](int c) {
        tc::mbar_expect_tx(full_u, 4 * kTileBytes);
        tc::bulk_g2s(aU, utile(U, c, 0, 0), 4 * kTileBytes, full_u);
    };
    if (tid == 0 && blockIdx.x < npairs) {
        issue_raw(blockIdx.x, 0);
        issue_u(0);
    }
    raw_pending = u_pending = blockIdx.x < npairs;
    for (int P = blockIdx.x; P < npairs && alive; P += gridDim.x) {
        const int q0 = 2 * P;
        float best[kBCols];
#pragma unroll
        for (int j = 0; j < kBCols; j++) best[j] = 0.f;
        if (eval_pi) {
            // this pair's actions, at the positions the epilogue reads
            const int qq = q0 + (row >> 6), i2 = row & 63;
#pragma unroll 8
            for (int jj = 0; jj < kBCols; jj++) {
                const int j = cbase + jj;
                sArg[j * 128 + row] = eval_pi[(size_t)(j * 64 + i2) * kSlab + qq];
            }
        }
        for (int a = 0; a < nact && alive; a++) {
            for (int r = 0; r < nrank && alive; r++) {
                const int c = a * nrank + r;
                int nc = c + 1, nP = P;
                if (nc == nchains) { nc = 0; nP = P + gridDim.x; }
                const bool has_next = nP < npairs;
                // raw slab pair -> swizzled hi / lo Z tiles (the operand
                // buffer is free: the previous item's second GEMM completed)
                if (!wait_all(full_raw, rph, err)) { raw_failed = true; alive = false; break; }
                raw_pending = false;
                {
                    const uint4 *raw = reinterpret_cast<const uint4 *>(sm + kBOffRaw);
#pragma unroll 4
                    for (int idx = tid; idx < 2 * 1024; idx += kBThreads) {
                        const uint4 w = raw[idx];
                        const uint32_t s2 = idx & 1, i1 = idx >> 5, j = (idx >> 1) & 15;
                        const uint32_t row = s2 * 64 + i1, k = j * 4;
                        const uint32_t off = tc::sw128_off(row, k);
                        *reinterpret_cast<uint2 *>(sZ + off) = make_uint2(w.x, w.y);
                        *reinterpret_cast<uint2 *>(sZ + kPairBytes + off) = make_uint2(w.z, w.w);
                    }
                }
                sync_for_async();
                // the raw buffer is free: fetch the next item's slab pair
                if (has_next) {
                    if (tid == 0) issue_raw(nP, nc);
                    raw_pending = true;
                }
                if (!wait_all(full_u, uph, err)) { u_failed = true; alive = false; break; }
                u_pending = false;
                const uint32_t u1 = aU, u2 = aU + 2 * kTileBytes;
                if (tid == 0) {
                    tc::mma_bf16x3(tmem, aZ, aZ + kPairBytes, u2, u2 + kTileBytes, 0);
                    tc::commit(mbar);
                }
                if (!wait_all(mbar, mph, err)) { alive = false; break; }
                tc::fence_after();
                float w1[kBCols];
                tc::tmem_ld32(tmem + lane_off + cbase, w1);   // row = (s2, i1), cols i2' = cbase ..
                {
                    // the second GEMM's A operand, MN-major into the operand
                    // buffer: k = i1 (this thread's row), m = s2 * 64 + i2'
                    const uint32_t s2 = row >> 6, i1 = row & 63;
                    const uint32_t a4_off = s2 * 8192u + (i1 >> 3) * 1024u + (i1 & 7u) * 128u;
#pragma unroll
                    for (int h = 0; h < kBCols / 8; h++) {
                        uint32_t hi[4], lo[4];
                        tc::split8_bf16(w1 + 8 * h, hi, lo);
                        const uint32_t chunk = (uint32_t)((cbase >> 3) + h);
                        const uint32_t off = a4_off + (((chunk ^ (i1 & 7u)) & 7u) << 4);
                        *reinterpret_cast<uint4 *>(sZ + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                        *reinterpret_cast<uint4 *>(sZ + kPairBytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                sync_for_async();
                if (tid == 0) {
                    tc::mma_bf16x3_amn(tmem + 64, aZ, aZ + kPairBytes, u1, u1 + kTileBytes, r > 0 ? 1u : 0u);
                    tc::commit(mbar);
                }
                if (!wait_all(mbar, mph, err)) { alive = false; break; }
                // the factor buffer is free: fetch the next item's factors
                if (has_next) {
                    if (tid == 0) issue_u(nc);
                    u_pending = true;
                }
            }
            if (!alive) break;
            tc::fence_after();
            float e[kBCols];
            tc::tmem_ld32(tmem + lane_off + 64 + cbase, e);   // row = (s2, i2'), cols i1' = cbase ..
            const int q = q0 + (row >> 6), i2 = row & 63;
            if (EB) {
                const float *eb = EB + (size_t)a * kS + (size_t)q * kSlab + i2;
#pragma unroll
                for (int jj = 0; jj < kBCols; jj++) e[jj] += eb[(cbase + jj) * 64];
            }
            if (eval_pi) {
#pragma unroll
                for (int jj = 0; jj < kBCols; jj++)
                    if (sArg[(cbase + jj) * 128 + row] == (uint8_t)a) best[jj] = e[jj];
            } else {
#pragma unroll
                for (int jj = 0; jj < kBCols; jj++) {
                    if (a == 0 || e[jj] > best[jj]) {
                        best[jj] = e[jj];
                        sArg[(cbase + jj) * 128 + row] = (uint8_t)a;
                    }
                }
            }
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
        }
        if (!alive) break;
        // V'(s) = R(s) + gamma max_a E_a(s); state s = (i1' * 64 + i2') * 4096 + q
        const int q = q0 + (row >> 6), i2 = row & 63;
        const float *rb = RB + (size_t)q * kSlab + i2;
#pragma unroll
        for (int jj = 0; jj < kBCols; jj++) {
            const int j = cbase + jj;
            const size_t s = (size_t)(j * 64 + i2) * kSlab + q;
            const float v = rb[j * 64] + gamma * best[jj];
            if (Vout) Vout[s] = v;
            if (pi && !eval_pi) pi[s] = sArg[j * 128 + row];
            if (res) local_res = fmax(local_res, fabs((double)v - (double)Vin[s]));
        }
        __syncthreads();
    }
    if (res) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) local_res = fmax(local_res, __shfl_xor_sync(0xFFFFFFFFu, local_res, o));
        if ((tid & 31) == 0 && local_res > 0.0) atomicMax(res, (unsigned long long)__double_as_longlong(local_res));
    }
    // a copy may still be in flight when this CTA stopped early: wait for it
    if (!alive && tid == 0) {
        if (raw_pending) tc::mbar_wait(full_raw, raw_failed ? rph ^ 1u : rph, kWaitCycles);
        if (u_pending) tc::mbar_wait(full_u, u_failed ? uph ^ 1u : uph, kWaitCycles);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// host side

static uint16_t host_bf16_rn(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static float host_bf16_to_f(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

bool dense_tc_supported(const Factors &F) {
    if (F.kind != CPMDP_DENSE_CP || F.ndim != 4 || F.nactions > 16) return false;
    for (int d = 0; d < 4; d++)
        if (F.shape[d] != kN) return false;
    return true;
}

// Device buffers of the tensor-core path, allocated on first use.
static cpmdp_status tc_prepare(Factors &F) {
    if (F.d_Ubf) return CPMDP_OK;
    const int C = F.nactions * F.rank;
    // factor tiles: hi / lo split, swizzled; mode 1 carries lambda
    std::vector<uint8_t> tiles((size_t)C * 4 * 2 * kTileBytes, 0);
    for (int c = 0; c < C; c++) {
        const int a = c / F.rank, r = c % F.rank;
        const double lam = F.lambda[(size_t)a * F.rank + r];
        for (int d = 0; d < 4; d++) {
            const double *Ud = &F.dense_factors[(size_t)F.factor_off[((size_t)a * F.rank + r) * 4 + d]];
            uint8_t *hi = &tiles[((size_t)(c * 4 + d) * 2 + 0) * kTileBytes];
            uint8_t *lo = &tiles[((size_t)(c * 4 + d) * 2 + 1) * kTileBytes];
            for (int i = 0; i < kN; i++)
                for (int k = 0; k < kN; k++) {
                    const float x = (float)(d == 0 ? lam * Ud[i * kN + k] : Ud[i * kN + k]);
                    const uint16_t h = host_bf16_rn(x);
                    const uint16_t l = host_bf16_rn(x - host_bf16_to_f(h));
                    const uint32_t off = tc::sw128_off((uint32_t)i, (uint32_t)k);
                    memcpy(hi + off, &h, 2);
                    memcpy(lo + off, &l, 2);
                }
        }
    }
    // rewards in the pass-B layout: RB[q * 4096 + (i1,i2)] = R[(i1,i2) * 4096 + q]
    std::vector<float> rb((size_t)kS);
    for (long long col = 0; col < kSlab; col++)
        for (long long q = 0; q < kSlab; q++) rb[(size_t)(q * kSlab + col)] = (float)F.reward[(size_t)(col * kSlab + q)];
    Factors &Fm = F;
    CPMDP_CUDA(cudaMalloc(&Fm.d_Ubf, tiles.size()));
    CPMDP_CUDA(cudaMemcpy(Fm.d_Ubf, tiles.data(), tiles.size(), cudaMemcpyHostToDevice));
    CPMDP_CUDA(cudaMalloc(&Fm.d_RB, (size_t)kS * sizeof(float)));
    CPMDP_CUDA(cudaMemcpy(Fm.d_RB, rb.data(), (size_t)kS * sizeof(float), cudaMemcpyHostToDevice));
    CPMDP_CUDA(cudaMalloc(&Fm.d_T, (size_t)C * kS * sizeof(uint32_t)));
    CPMDP_CUDA(cudaMalloc(&Fm.d_EB, (size_t)F.nactions * kS * sizeof(float)));
    CPMDP_CUDA(cudaMalloc(&Fm.d_Vbase, (size_t)kS * sizeof(float)));
    if (!Fm.d_tc_err) CPMDP_CUDA(cudaMalloc(&Fm.d_tc_err, sizeof(int)));
    CPMDP_CUDA(cudaFuncSetAttribute(dense_pass_a, cudaFuncAttributeMaxDynamicSharedMemorySize, kASmem));
    CPMDP_CUDA(cudaFuncSetAttribute(dense_pass_b, cudaFuncAttributeMaxDynamicSharedMemorySize, kBSmem));
    return CPMDP_OK;
}

// One BF16x3 backup: Vout = R + gamma max_a (EB_a + E_a(Vin - Vbase)), or
// with eval_pi the expectation of the action eval_pi[s] instead of the max.
static cpmdp_status tc_sweep(const Factors &F, const float *Vin, float *Vout, uint8_t *pi, bool use_base,
                             unsigned long long *res, cudaStream_t st, const uint8_t *eval_pi = nullptr) {
    const int C = F.nactions * F.rank;
    int *err = F.d_tc_err;
    const int grid = F.num_sms > 0 ? F.num_sms : 148;
    dense_pass_a<<<grid, kAThreads, kASmem, st>>>(Vin, use_base ? F.d_Vbase : nullptr, (const uint8_t *)F.d_Ubf,
                                            (uint8_t *)F.d_T, C, err);
    CPMDP_CUDA(cudaGetLastError());
    // pass B: two CTAs per SM (about 106 KB of shared memory each)
    dense_pass_b<<<2 * grid, kBThreads, kBSmem, st>>>((const uint8_t *)F.d_T, (const uint8_t *)F.d_Ubf, F.d_RB,
                                            use_base ? F.d_EB : nullptr, Vin, Vout, pi, eval_pi, F.nactions,
                                            F.rank, (float)F.gamma, res, err);
    CPMDP_CUDA(cudaGetLastError());
    return CPMDP_OK;
}

static cpmdp_status tc_check_err(const Factors &F, cudaStream_t st) {
    int h = 0;
    CPMDP_CUDA(cudaMemcpyAsync(&h, F.d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CPMDP_CUDA(cudaStreamSynchronize(st));
    if (h != 0) {
        set_error("a tensor-core wait exceeded its limit; results are undefined");
        return CPMDP_ETIMEOUT;
    }
    return CPMDP_OK;
}

cpmdp_status dense_tc_backup(const Factors &F, const float *Vin, float *Vout, uint8_t *pi, double *res,
                             cudaStream_t st) {
    if (!dense_tc_supported(F)) {
        set_error("BF16X3 needs a dense model with 4 dimensions of size 64 and at most 16 actions");
        return CPMDP_EINVAL;
    }
    cpmdp_status s = tc_prepare(const_cast<Factors &>(F));
    if (s != CPMDP_OK) return s;
    CPMDP_CUDA(cudaMemsetAsync(F.d_tc_err, 0, sizeof(int), st));
    unsigned long long *rb = reinterpret_cast<unsigned long long *>(res);
    if (rb) CPMDP_CUDA(cudaMemsetAsync(rb, 0, sizeof(double), st));
    s = tc_sweep(F, Vin, Vout, pi, false, rb, st);
    if (s != CPMDP_OK) return s;
    return tc_check_err(F, st);
}

// FP32 SIMT expectation of every action, stored in the pass-B layout (dense.cu).
cpmdp_status dense_store_expectation(const Factors &F, const float *V, float *EB, cudaStream_t st);
// FP64 SIMT backup of a float value tensor (dense.cu).
cpmdp_status dense_certify(const Factors &F, const float *V, uint8_t *pi, double *res, cudaStream_t st);

// Value iteration with BF16x3 sweeps and defect correction against an FP32
// base expectation, stopped by an FP64 residual, as one CUDA graph launch.
//
// The working residual max |V' - V| of float iterates bottoms out at one to
// three units in the last place of the largest |V| (rounding of V' flips
// from sweep to sweep), so once it is below tol it no longer shows the
// geometric part of the error, which still shrinks by gamma per sweep. With
// certify on, the solve therefore runs ceil(ln 2 / ln(1 / gamma)) more
// sweeps (halving that part), then one FP64 backup of V gives the certified
// residual max |T(V) - V| and the FP64 argmax policy; if the certified
// residual is not below tol either, it runs as many sweeps again and
// certifies again (within max_iter). The returned V then meets the value
// iteration stopping rule evaluated in FP64. eval_sweeps in the result
// counts the FP64 certifying sweeps.
//
// The whole loop stays on the device: a conditional WHILE node repeats a
// body of two sweeps (V -> scratch, scratch -> V); after each sweep a
// one-thread control kernel reads the residual, keeps the last eight, and
// sets the conditions of the nodes that follow it: refresh the FP32 base
// (the residual stopped falling: no lower than 0.9 of its value five sweeps
// earlier, six sweeps or more after the last refresh), take the FP64 check,
// run the second sweep, repeat. Every sweep uses the base (zero until the
// first refresh, which subtracts and adds exact zeros). The host reads the
// control block once, after the graph. The graph is recorded once per
// (V, policy, tol, max_iter, certify, trace) and replayed.
static_assert(sizeof(DensePiCtl) <= kLoopCtlBytes, "loop control block");

struct DenseLoopCtl {
    int k;              // sweeps done
    int last_rebase;    // sweep of the last base refresh
    int rebases;
    int extra;          // -1: working residual not below tol yet; else sweeps left before the FP64 check
    int certs;          // FP64 checks taken
    int conv;           // FP64 residual below tol
    int stop;
    int which;          // buffer of the current iterate: 0 = V, 1 = scratch
    double res;         // last working residual
    double hist[8];     // last eight working residuals (sweep k - 1 at k - 1 mod 8)
};
static_assert(sizeof(DenseLoopCtl) <= kLoopCtlBytes, "loop control block");

__global__ void dense_loop_ctl_kernel(DenseLoopCtl *c, unsigned long long *res_slot, const int *err, double tol,
                                      int max_iter, int certify, int halve, double *trace, int step,
                                      cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_rebase,
                                      cudaGraphConditionalHandle h_cert, cudaGraphConditionalHandle h_second) {
    if (c->stop || *(volatile const int *)err) {
        c->stop = 1;
        cudaGraphSetConditional(h_rebase, 0u);
        cudaGraphSetConditional(h_cert, 0u);
        if (step == 0) cudaGraphSetConditional(h_second, 0u);
        cudaGraphSetConditional(h_loop, 0u);
        return;
    }
    double r;
    memcpy(&r, res_slot, sizeof(r));
    *res_slot = 0ull;
    if (trace) trace[c->k] = r;
    c->hist[c->k & 7] = r;
    c->k++;
    c->res = r;
    c->which = step == 0 ? 1 : 0;
    unsigned rebase = 0, cert = 0;
    if (c->extra < 0 && r < tol) {
        if (!certify) { c->conv = 1; c->stop = 1; }
        else c->extra = halve;
    }
    if (!c->stop) {
        if (c->extra > 0) {
            if (--c->extra == 0) cert = 1;
        } else if (c->k - c->last_rebase >= 6 && r > 0.9 * c->hist[(c->k - 6) & 7] && c->rebases < 64) {
            rebase = 1;
            c->last_rebase = c->k;
            c->rebases++;
        }
        if (!cert && c->k >= max_iter) c->stop = 1;
    }
    cudaGraphSetConditional(h_rebase, rebase);
    cudaGraphSetConditional(h_cert, cert);
    if (step == 0) cudaGraphSetConditional(h_second, (!c->stop && !cert) ? 1u : 0u);
    cudaGraphSetConditional(h_loop, c->stop ? 0u : 1u);
}

// After an FP64 check: stop below tol, else go on for `halve` more sweeps.
__global__ void dense_cert_check_kernel(DenseLoopCtl *c, const double *cert, double tol, int max_iter, int halve,
                                        int step, cudaGraphConditionalHandle h_loop,
                                        cudaGraphConditionalHandle h_second) {
    double v;
    memcpy(&v, cert, sizeof(v));
    c->certs++;
    if (v < tol) {
        c->conv = 1;
        c->stop = 1;
    } else {
        c->extra = halve;
        if (c->k >= max_iter) c->stop = 1;
    }
    if (step == 0) cudaGraphSetConditional(h_second, c->stop ? 0u : 1u);
    cudaGraphSetConditional(h_loop, c->stop ? 0u : 1u);
}

// Nodes of g that no other node depends on.
cudaError_t graph_leaves(cudaGraph_t g, std::vector<cudaGraphNode_t> &out) {
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && (e = cudaGraphGetNodes(g, nodes.data(), &n)) != cudaSuccess) return e;
    out.clear();
    for (cudaGraphNode_t nd : nodes) {
        size_t m = 0;
        if ((e = cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &m)) != cudaSuccess) return e;
        if (m == 0) out.push_back(nd);
    }
    return cudaSuccess;
}

// Add a conditional node (IF or WHILE) after `deps` in g; returns its body.
cudaError_t add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps,
                                   cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                   cudaGraphNode_t *node, cudaGraph_t *body) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
    if (e != cudaSuccess) return e;
    *body = p.conditional.phGraph_out[0];
    return cudaSuccess;
}

cpmdp_status dense_certify(const Factors &F, const float *V, uint8_t *pi, double *res, cudaStream_t st);
cpmdp_status dense_store_expectation(const Factors &F, const float *V, float *EB, cudaStream_t st);

// Record the loop into a new graph (see above).
static cpmdp_status record_dense_vi(Factors &F, float *V, uint8_t *pi, const SolveOpts &o, int halve,
                                    cudaGraph_t *out) {
    float *W = (float *)F.d_scratch;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    double *cert = (double *)((char *)F.d_ctrl + offsetof(Ctrl, certify_residual));
    DenseLoopCtl *c = reinterpret_cast<DenseLoopCtl *>(F.d_dense_loop);
    cudaGraph_t G = nullptr;
    cudaStream_t cap = nullptr;
    cpmdp_status s = CPMDP_OK;
    cudaError_t e = cudaGraphCreate(&G, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraphConditionalHandle h_loop = 0, h_reb0 = 0, h_cert0 = 0, h_second = 0, h_reb1 = 0, h_cert1 = 0;
    cudaGraph_t body = nullptr, sbody = nullptr;
    cudaGraphNode_t node;
    std::vector<cudaGraphNode_t> leaves;
    auto capture = [&](cudaGraph_t g, auto &&fn) -> cpmdp_status {
        cudaError_t ce = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return cuda_fail(ce, "begin capture");
        cpmdp_status cs = fn();
        cudaGraph_t gg = g;
        ce = cudaStreamEndCapture(cap, &gg);
        if (cs != CPMDP_OK) return cs;
        if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
        return CPMDP_OK;
    };
    // one sweep from `in` to `out`, then the control kernel of that step
    auto sweep_ctl = [&](const float *in, float *out, int step, cudaGraphConditionalHandle hr,
                         cudaGraphConditionalHandle hc) -> cpmdp_status {
        cudaError_t ce = cudaMemsetAsync(rb, 0, sizeof(*rb), cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "memset");
        cpmdp_status cs = tc_sweep(F, in, out, nullptr, true, rb, cap);
        if (cs != CPMDP_OK) return cs;
        dense_loop_ctl_kernel<<<1, 1, 0, cap>>>(c, rb, F.d_tc_err, o.tol, o.max_iter, o.certify, halve, o.trace, step,
                                                h_loop, hr, hc, h_second);
        ce = cudaGetLastError();
        return ce == cudaSuccess ? CPMDP_OK : cuda_fail(ce, "control kernel");
    };
    auto rebase_body = [&](const float *cur) -> cpmdp_status {
        cudaError_t ce = cudaMemcpyAsync(F.d_Vbase, cur, (size_t)kS * sizeof(float), cudaMemcpyDeviceToDevice, cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "base copy");
        return dense_store_expectation(F, cur, F.d_EB, cap);
    };
    auto cert_body = [&](const float *cur, int step) -> cpmdp_status {
        cpmdp_status cs = dense_certify(F, cur, pi, cert, cap);
        if (cs != CPMDP_OK) return cs;
        dense_cert_check_kernel<<<1, 1, 0, cap>>>(c, cert, o.tol, o.max_iter, halve, step, h_loop, h_second);
        cudaError_t ce = cudaGetLastError();
        return ce == cudaSuccess ? CPMDP_OK : cuda_fail(ce, "check kernel");
    };
    if (e != cudaSuccess) { s = cuda_fail(e, "graph setup"); goto done; }
    // root: WHILE(loop)
    if ((e = cudaGraphConditionalHandleCreate(&h_loop, G, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = add_conditional(G, {}, h_loop, cudaGraphCondTypeWhile, &node, &body)) != cudaSuccess) goto fail;
    // body: sweep V -> W, control, IF(refresh), IF(check), IF(second sweep)
    if ((e = cudaGraphConditionalHandleCreate(&h_reb0, body, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = cudaGraphConditionalHandleCreate(&h_cert0, body, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = cudaGraphConditionalHandleCreate(&h_second, body, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((s = capture(body, [&] { return sweep_ctl(V, W, 0, h_reb0, h_cert0); })) != CPMDP_OK) goto done;
    {
        cudaGraph_t b1, b2, b3;
        cudaGraphNode_t n1, n2, n3;
        if ((e = graph_leaves(body, leaves)) != cudaSuccess) goto fail;
        if ((e = add_conditional(body, leaves, h_reb0, cudaGraphCondTypeIf, &n1, &b1)) != cudaSuccess) goto fail;
        if ((e = add_conditional(body, {n1}, h_cert0, cudaGraphCondTypeIf, &n2, &b2)) != cudaSuccess) goto fail;
        if ((e = add_conditional(body, {n2}, h_second, cudaGraphCondTypeIf, &n3, &b3)) != cudaSuccess) goto fail;
        if ((s = capture(b1, [&] { return rebase_body(W); })) != CPMDP_OK) goto done;
        if ((s = capture(b2, [&] { return cert_body(W, 0); })) != CPMDP_OK) goto done;
        sbody = b3;
    }
    // second sweep W -> V, control, IF(refresh), IF(check)
    if ((e = cudaGraphConditionalHandleCreate(&h_reb1, sbody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = cudaGraphConditionalHandleCreate(&h_cert1, sbody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((s = capture(sbody, [&] { return sweep_ctl(W, V, 1, h_reb1, h_cert1); })) != CPMDP_OK) goto done;
    {
        cudaGraph_t b1, b2;
        cudaGraphNode_t n1, n2;
        if ((e = graph_leaves(sbody, leaves)) != cudaSuccess) goto fail;
        if ((e = add_conditional(sbody, leaves, h_reb1, cudaGraphCondTypeIf, &n1, &b1)) != cudaSuccess) goto fail;
        if ((e = add_conditional(sbody, {n1}, h_cert1, cudaGraphCondTypeIf, &n2, &b2)) != cudaSuccess) goto fail;
        if ((s = capture(b1, [&] { return rebase_body(V); })) != CPMDP_OK) goto done;
        if ((s = capture(b2, [&] { return cert_body(V, 1); })) != CPMDP_OK) goto done;
    }
    goto done;
fail:
    s = cuda_fail(e, "recording the dense value iteration graph");
done:
    if (cap) cudaStreamDestroy(cap);
    if (s != CPMDP_OK) {
        if (G) cudaGraphDestroy(G);
        return s;
    }
    *out = G;
    return CPMDP_OK;
}

cpmdp_status dense_tc_solve(const Factors &F, float *V, uint8_t *pi, const SolveOpts &o, Ctrl *hc, cudaStream_t st) {
    if (!dense_tc_supported(F)) {
        set_error("BF16X3 needs a dense model with 4 dimensions of size 64 and at most 16 actions");
        return CPMDP_EINVAL;
    }
    cpmdp_status s = tc_prepare(const_cast<Factors &>(F));
    if (s != CPMDP_OK) return s;
    Factors &M = const_cast<Factors &>(F);
    // buffers the recorded graph uses must exist before the recording
    if (!M.d_dense_loop) CPMDP_CUDA(cudaMalloc(&M.d_dense_loop, kLoopCtlBytes));
    if (!M.d_Vd) CPMDP_CUDA(cudaMalloc(&M.d_Vd, (size_t)F.nstates * sizeof(double)));
    const int halve = F.gamma > 0.0 && F.gamma < 1.0 ? (int)ceil(log(2.0) / log(1.0 / F.gamma)) : 1;
    const bool same = M.dense_graph && M.dense_graph_V == (void *)V && M.dense_graph_pi == (void *)pi &&
                      M.dense_graph_tol == o.tol && M.dense_graph_max_iter == o.max_iter &&
                      M.dense_graph_certify == o.certify && M.dense_graph_trace == (void *)o.trace;
    if (!same) {
        if (M.dense_graph) { cudaGraphExecDestroy(M.dense_graph); M.dense_graph = nullptr; }
        cudaGraph_t g = nullptr;
        s = record_dense_vi(M, V, pi, o, halve, &g);
        if (s != CPMDP_OK) return s;
        cudaError_t e = cudaGraphInstantiate(&M.dense_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { M.dense_graph = nullptr; CPMDP_CUDA(e); }
        M.dense_graph_V = (void *)V;
        M.dense_graph_pi = (void *)pi;
        M.dense_graph_tol = o.tol;
        M.dense_graph_max_iter = o.max_iter;
        M.dense_graph_certify = o.certify;
        M.dense_graph_trace = (void *)o.trace;
    }
    // start: zero base (E of a zero base is zero), control block, residual slot
    DenseLoopCtl c0;
    memset(&c0, 0, sizeof(c0));
    c0.extra = -1;
    CPMDP_CUDA(cudaMemcpyAsync(M.d_dense_loop, &c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_Vbase, 0, (size_t)kS * sizeof(float), st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_EB, 0, (size_t)F.nactions * kS * sizeof(float), st));
    CPMDP_CUDA(cudaMemsetAsync(&F.d_ctrl->res_slot[0], 0, sizeof(unsigned long long), st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_tc_err, 0, sizeof(int), st));
    if (o.trace) CPMDP_CUDA(cudaMemsetAsync(o.trace, 0, (size_t)o.max_iter * sizeof(double), st));
    CPMDP_CUDA(cudaGraphLaunch(M.dense_graph, st));
    DenseLoopCtl c;
    CPMDP_CUDA(cudaMemcpyAsync(&c, M.d_dense_loop, sizeof(c), cudaMemcpyDeviceToHost, st));
    s = tc_check_err(F, st);
    if (s != CPMDP_OK) return s;
    float *W = (float *)F.d_scratch;
    if (c.which == 1) CPMDP_CUDA(cudaMemcpyAsync(V, W, (size_t)kS * sizeof(float), cudaMemcpyDeviceToDevice, st));
    int certs = c.certs;
    double *cert = (double *)((char *)F.d_ctrl + offsetof(Ctrl, certify_residual));
    if (o.certify && !c.conv) {
        // max_iter ran out: certify what is returned
        s = dense_certify(F, V, pi, cert, st);
        if (s != CPMDP_OK) return s;
        certs++;
    } else if (!o.certify && pi) {
        s = tc_sweep(F, V, W, pi, true, nullptr, st);
        if (s != CPMDP_OK) return s;
    }
    hc->iterations = c.k;
    hc->rounds = c.rebases;
    hc->eval_sweeps = certs;
    hc->converged = c.conv;
    hc->last_residual = c.res;
    hc->backups = (long long)c.k * kS * F.nactions;
    return CPMDP_OK;
}

// Policy improvement from Q of the current action (Qold, an evaluation
// sweep's output) and the best Q with its argmax (Qbest, pib, a max sweep's
// output): switch to the argmax only when it beats the current action by
// more than margin (1 + |Qold|); count the switches.
__global__ void dense_improve_kernel(const float *__restrict__ Qold, const float *__restrict__ Qbest,
                                     const uint8_t *__restrict__ pib, uint8_t *__restrict__ pi, float margin,
                                     long long n, unsigned *changed) {
    unsigned c = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const float qo = Qold[s], qb = Qbest[s];
        const uint8_t b = pib[s];
        if (b != pi[s] && qb > qo + margin * (1.f + fabsf(qo))) {
            pi[s] = b;
            c++;
        }
    }
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(changed, c);
}

// Policy iteration with BF16x3 sweeps and the defect correction of value
// iteration (background section: evaluate the fixed policy, improve
// greedily, stop when no action changes), in the modified form of the
// GridWorld solvers: evaluations capped at partial_eval sweeps until an
// improvement changes no action, then to eval_tol. An evaluation sweep is
// the tensor-core backup with each state's own action; an improvement is
// one evaluation-mode sweep (Q of the current action), one max sweep (best
// Q and its argmax) and dense_improve_kernel (keep margin 1e-6 (1 + |Q|)).
// The FP32 base expectation is refreshed when an evaluation's residual
// stops falling. With certify on, one FP64 backup of the result gives the
// certified residual max |T(V) - V| (the policy is left as PI found it).
// ---------------------------------------------------------------------------
// BF16x3 policy iteration as one CUDA graph launch (nested conditional
// nodes; the same steps and decisions as a host-driven loop):
//   greedy sweep (max mode: the initial policy), then WHILE(round):
//     round start (evaluation cap: partial_eval sweeps while the policy
//     changes, max_eval_iter once a full evaluation is asked for)
//     WHILE(eval): sweep V -> W in evaluation mode, control, IF(base
//       refresh), IF(second: sweep W -> V, control, IF(base refresh))
//     IF(odd count: copy W -> V)
//     improvement: Q of the current action, best Q and its argmax, compare
//     with the keep margin; round end (stop rules of modified PI)

__global__ void pi_init_kernel(DensePiCtl *c, const int *err, int max_rounds, cudaGraphConditionalHandle h_round) {
    if (*(volatile const int *)err || max_rounds <= 0) c->stop = 1;
    cudaGraphSetConditional(h_round, c->stop ? 0u : 1u);
}

__global__ void pi_round_start_kernel(DensePiCtl *c, int partial_eval, int max_eval_iter,
                                      cudaGraphConditionalHandle h_eval) {
    c->e = 0;
    c->ok = 0;
    c->last_rebase = 0;
    c->which = 0;
    c->cap = c->full ? max_eval_iter : min(partial_eval, max_eval_iter);
    cudaGraphSetConditional(h_eval, c->cap > 0 ? 1u : 0u);
}

// After evaluation sweep `step` (0: V -> W, 1: W -> V).
// can_rebase = 0 (SIMT paths): no base refresh, h_rebase is not touched.
__global__ void pi_eval_ctl_kernel(DensePiCtl *c, unsigned long long *res_slot, const int *err, double eval_tol,
                                   int step, int can_rebase, cudaGraphConditionalHandle h_eval,
                                   cudaGraphConditionalHandle h_rebase, cudaGraphConditionalHandle h_second) {
    unsigned rebase = 0;
    bool done;
    if (*(volatile const int *)err) {
        c->stop = 1;
        done = true;
    } else {
        double r;
        memcpy(&r, res_slot, sizeof(r));
        *res_slot = 0ull;
        c->hist[c->e & 7] = r;
        c->e++;
        c->total++;
        c->res = r;
        c->which = step == 0 ? 1 : 0;
        done = false;
        if (r < eval_tol) {
            c->ok = 1;
            done = true;
        } else {
            if (can_rebase && c->e - c->last_rebase >= 6 && r > 0.9 * c->hist[(c->e - 6) & 7] && c->rebases < 256) {
                rebase = 1;
                c->last_rebase = c->e;
                c->rebases++;
            }
            if (c->e >= c->cap) done = true;
        }
    }
    if (can_rebase) cudaGraphSetConditional(h_rebase, rebase);
    if (step == 0) cudaGraphSetConditional(h_second, done ? 0u : 1u);
    cudaGraphSetConditional(h_eval, done ? 0u : 1u);
}

__global__ void pi_after_eval_kernel(const DensePiCtl *c, cudaGraphConditionalHandle h_odd) {
    cudaGraphSetConditional(h_odd, c->which == 1 ? 1u : 0u);
}

__global__ void pi_round_end_kernel(DensePiCtl *c, const unsigned *changed, const int *err, int max_rounds,
                                    cudaGraphConditionalHandle h_round) {
    const unsigned nchg = *changed;
    c->evals += c->e;
    c->total++;
    c->rounds++;
    if (*(volatile const int *)err) {
        c->stop = 1;
    } else if (nchg == 0) {
        if (c->ok) {
            c->conv = 1;
            c->stop = 1;
        } else if (c->full) {
            c->stop = 1;
        } else {
            c->full = 1;
        }
    } else if (!c->ok && c->full) {
        c->stop = 1;
    }
    if (c->rounds >= max_rounds) c->stop = 1;
    cudaGraphSetConditional(h_round, c->stop ? 0u : 1u);
}

static cpmdp_status record_dense_pi(Factors &F, float *V, uint8_t *pi, const SolveOpts &o, cudaGraph_t *out) {
    float *W = (float *)F.d_scratch;
    unsigned long long *rb = &F.d_ctrl->res_slot[0];
    unsigned *cb = &F.d_ctrl->changed_slot[0];
    float *Qold = reinterpret_cast<float *>(F.d_pi_work), *Qbest = Qold + kS;
    uint8_t *pib = reinterpret_cast<uint8_t *>(Qbest + kS);
    DensePiCtl *c = reinterpret_cast<DensePiCtl *>(F.d_dense_loop);
    const int grid = F.num_sms > 0 ? F.num_sms * 8 : 1216;
    cudaGraph_t G = nullptr;
    cudaStream_t cap = nullptr;
    cpmdp_status s = CPMDP_OK;
    cudaError_t e = cudaGraphCreate(&G, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraphConditionalHandle h_round = 0, h_eval = 0, h_odd = 0, h_reb0 = 0, h_second = 0, h_reb1 = 0;
    cudaGraph_t rbody = nullptr, ebody = nullptr, obody = nullptr, sbody = nullptr;
    cudaGraphNode_t n_round, n_eval, n_odd;
    std::vector<cudaGraphNode_t> leaves;
    // capture fn's work into g, after the nodes deps
    auto capture = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, auto &&fn) -> cpmdp_status {
        cudaError_t ce = cudaStreamBeginCaptureToGraph(cap, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                                       deps.size(), cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return cuda_fail(ce, "begin capture");
        cpmdp_status cs = fn();
        cudaGraph_t gg = g;
        ce = cudaStreamEndCapture(cap, &gg);
        if (cs != CPMDP_OK) return cs;
        if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
        return CPMDP_OK;
    };
    auto launched = [&](const char *what) -> cpmdp_status {
        cudaError_t ce = cudaGetLastError();
        return ce == cudaSuccess ? CPMDP_OK : cuda_fail(ce, what);
    };
    // one evaluation sweep from `in` to `out` (each state's own action), then its control kernel
    auto eval_ctl = [&](const float *in, float *outv, int step, cudaGraphConditionalHandle hr) -> cpmdp_status {
        cudaError_t ce = cudaMemsetAsync(rb, 0, sizeof(*rb), cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "memset");
        cpmdp_status cs = tc_sweep(F, in, outv, nullptr, true, rb, cap, pi);
        if (cs != CPMDP_OK) return cs;
        pi_eval_ctl_kernel<<<1, 1, 0, cap>>>(c, rb, F.d_tc_err, o.eval_tol, step, 1, h_eval, hr, h_second);
        return launched("evaluation control kernel");
    };
    auto rebase_body = [&](const float *cur) -> cpmdp_status {
        cudaError_t ce = cudaMemcpyAsync(F.d_Vbase, cur, (size_t)kS * sizeof(float), cudaMemcpyDeviceToDevice, cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "base copy");
        return dense_store_expectation(F, cur, F.d_EB, cap);
    };
    if (e != cudaSuccess) { s = cuda_fail(e, "graph setup"); goto done; }
    if ((e = cudaGraphConditionalHandleCreate(&h_round, G, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    // root: greedy sweep (max mode: its argmax is the initial policy), the stop test, WHILE(round)
    if ((s = capture(G, {}, [&]() -> cpmdp_status {
             cpmdp_status cs = tc_sweep(F, V, W, pi, true, nullptr, cap);
             if (cs != CPMDP_OK) return cs;
             pi_init_kernel<<<1, 1, 0, cap>>>(c, F.d_tc_err, o.max_rounds, h_round);
             return launched("init kernel");
         })) != CPMDP_OK)
        goto done;
    if ((e = graph_leaves(G, leaves)) != cudaSuccess) goto fail;
    if ((e = add_conditional(G, leaves, h_round, cudaGraphCondTypeWhile, &n_round, &rbody)) != cudaSuccess) goto fail;
    // round body: start kernel, WHILE(eval), IF(odd: copy W -> V), improvement, end kernel
    if ((e = cudaGraphConditionalHandleCreate(&h_eval, rbody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = cudaGraphConditionalHandleCreate(&h_odd, rbody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((s = capture(rbody, {}, [&]() -> cpmdp_status {
             pi_round_start_kernel<<<1, 1, 0, cap>>>(c, o.partial_eval, o.max_eval_iter, h_eval);
             return launched("round start kernel");
         })) != CPMDP_OK)
        goto done;
    if ((e = graph_leaves(rbody, leaves)) != cudaSuccess) goto fail;
    if ((e = add_conditional(rbody, leaves, h_eval, cudaGraphCondTypeWhile, &n_eval, &ebody)) != cudaSuccess) goto fail;
    if ((s = capture(rbody, {n_eval}, [&]() -> cpmdp_status {
             pi_after_eval_kernel<<<1, 1, 0, cap>>>(c, h_odd);
             return launched("after-evaluation kernel");
         })) != CPMDP_OK)
        goto done;
    if ((e = graph_leaves(rbody, leaves)) != cudaSuccess) goto fail;
    if ((e = add_conditional(rbody, leaves, h_odd, cudaGraphCondTypeIf, &n_odd, &obody)) != cudaSuccess) goto fail;
    if ((s = capture(obody, {}, [&]() -> cpmdp_status {
             cudaError_t ce = cudaMemcpyAsync(V, W, (size_t)kS * sizeof(float), cudaMemcpyDeviceToDevice, cap);
             return ce == cudaSuccess ? CPMDP_OK : cuda_fail(ce, "iterate copy");
         })) != CPMDP_OK)
        goto done;
    if ((s = capture(rbody, {n_odd}, [&]() -> cpmdp_status {
             cpmdp_status cs = tc_sweep(F, V, Qold, nullptr, true, nullptr, cap, pi);
             if (cs != CPMDP_OK) return cs;
             if ((cs = tc_sweep(F, V, Qbest, pib, true, nullptr, cap)) != CPMDP_OK) return cs;
             cudaError_t ce = cudaMemsetAsync(cb, 0, sizeof(*cb), cap);
             if (ce != cudaSuccess) return cuda_fail(ce, "memset");
             dense_improve_kernel<<<grid, 256, 0, cap>>>(Qold, Qbest, pib, pi, 1e-6f, kS, cb);
             if ((cs = launched("improvement kernel")) != CPMDP_OK) return cs;
             pi_round_end_kernel<<<1, 1, 0, cap>>>(c, cb, F.d_tc_err, o.max_rounds, h_round);
             return launched("round end kernel");
         })) != CPMDP_OK)
        goto done;
    // evaluation body: sweep V -> W, control, IF(refresh from W), IF(second)
    if ((e = cudaGraphConditionalHandleCreate(&h_reb0, ebody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((e = cudaGraphConditionalHandleCreate(&h_second, ebody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((s = capture(ebody, {}, [&] { return eval_ctl(V, W, 0, h_reb0); })) != CPMDP_OK) goto done;
    {
        cudaGraph_t b1, b2;
        cudaGraphNode_t n1, n2;
        if ((e = graph_leaves(ebody, leaves)) != cudaSuccess) goto fail;
        if ((e = add_conditional(ebody, leaves, h_reb0, cudaGraphCondTypeIf, &n1, &b1)) != cudaSuccess) goto fail;
        if ((e = add_conditional(ebody, {n1}, h_second, cudaGraphCondTypeIf, &n2, &b2)) != cudaSuccess) goto fail;
        if ((s = capture(b1, {}, [&] { return rebase_body(W); })) != CPMDP_OK) goto done;
        sbody = b2;
    }
    // second sweep W -> V, control, IF(refresh from V)
    if ((e = cudaGraphConditionalHandleCreate(&h_reb1, sbody, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) goto fail;
    if ((s = capture(sbody, {}, [&] { return eval_ctl(W, V, 1, h_reb1); })) != CPMDP_OK) goto done;
    {
        cudaGraph_t b1;
        cudaGraphNode_t n1;
        if ((e = graph_leaves(sbody, leaves)) != cudaSuccess) goto fail;
        if ((e = add_conditional(sbody, leaves, h_reb1, cudaGraphCondTypeIf, &n1, &b1)) != cudaSuccess) goto fail;
        if ((s = capture(b1, {}, [&] { return rebase_body(V); })) != CPMDP_OK) goto done;
    }
    goto done;
fail:
    s = cuda_fail(e, "recording the dense policy iteration graph");
done:
    if (cap) cudaStreamDestroy(cap);
    if (s != CPMDP_OK) {
        if (G) cudaGraphDestroy(G);
        return s;
    }
    *out = G;
    return CPMDP_OK;
}

cpmdp_status dense_tc_policy_iteration(const Factors &F, float *V, uint8_t *pi, const SolveOpts &o, Ctrl *hc,
                                       cudaStream_t st) {
    if (!dense_tc_supported(F)) {
        set_error("BF16X3 needs a dense model with 4 dimensions of size 64 and at most 16 actions");
        return CPMDP_EINVAL;
    }
    cpmdp_status s = tc_prepare(const_cast<Factors &>(F));
    if (s != CPMDP_OK) return s;
    Factors &M = const_cast<Factors &>(F);
    // buffers the recorded graph uses must exist before the recording
    if (!M.d_pi_work) CPMDP_CUDA(cudaMalloc(&M.d_pi_work, (size_t)kS * (2 * sizeof(float) + 1)));
    if (!M.d_dense_loop) CPMDP_CUDA(cudaMalloc(&M.d_dense_loop, kLoopCtlBytes));
    const bool same = M.dense_pi_graph && M.dense_pi_graph_V == (void *)V && M.dense_pi_graph_pi == (void *)pi &&
                      M.dense_pi_graph_eval_tol == o.eval_tol && M.dense_pi_graph_rounds == o.max_rounds &&
                      M.dense_pi_graph_eval_iter == o.max_eval_iter && M.dense_pi_graph_partial == o.partial_eval;
    if (!same) {
        if (M.dense_pi_graph) { cudaGraphExecDestroy(M.dense_pi_graph); M.dense_pi_graph = nullptr; }
        cudaGraph_t g = nullptr;
        s = record_dense_pi(M, V, pi, o, &g);
        if (s != CPMDP_OK) return s;
        cudaError_t e = cudaGraphInstantiate(&M.dense_pi_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { M.dense_pi_graph = nullptr; CPMDP_CUDA(e); }
        M.dense_pi_graph_V = (void *)V;
        M.dense_pi_graph_pi = (void *)pi;
        M.dense_pi_graph_eval_tol = o.eval_tol;
        M.dense_pi_graph_rounds = o.max_rounds;
        M.dense_pi_graph_eval_iter = o.max_eval_iter;
        M.dense_pi_graph_partial = o.partial_eval;
    }
    // start: zero base (E of a zero base is zero), control block (one sweep: the greedy start)
    DensePiCtl c0;
    memset(&c0, 0, sizeof(c0));
    c0.full = o.partial_eval <= 0;
    c0.total = 1;
    CPMDP_CUDA(cudaMemcpyAsync(M.d_dense_loop, &c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_Vbase, 0, (size_t)kS * sizeof(float), st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_EB, 0, (size_t)F.nactions * kS * sizeof(float), st));
    CPMDP_CUDA(cudaMemsetAsync(&F.d_ctrl->res_slot[0], 0, sizeof(unsigned long long), st));
    CPMDP_CUDA(cudaMemsetAsync(F.d_tc_err, 0, sizeof(int), st));
    CPMDP_CUDA(cudaGraphLaunch(M.dense_pi_graph, st));
    DensePiCtl c;
    CPMDP_CUDA(cudaMemcpyAsync(&c, M.d_dense_loop, sizeof(c), cudaMemcpyDeviceToHost, st));
    s = tc_check_err(F, st);
    if (s != CPMDP_OK) return s;
    if (o.certify) {
        double *cert = (double *)((char *)F.d_ctrl + offsetof(Ctrl, certify_residual));
        s = dense_certify(F, V, nullptr, cert, st);
        if (s != CPMDP_OK) return s;
    }
    hc->iterations = c.total;
    hc->rounds = c.rounds;
    hc->eval_sweeps = c.evals;
    hc->converged = c.conv;
    hc->last_residual = c.rounds > 0 ? c.res : INFINITY;
    hc->backups = (long long)(1 + c.rounds) * kS * F.nactions + (long long)c.evals * kS;
    return CPMDP_OK;
}

}  // namespace cpmdp
