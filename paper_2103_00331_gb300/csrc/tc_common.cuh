// Blackwell (sm_103a) tensor-core primitives used by the dense CP kernels:
// tcgen05 MMA with operands in shared memory and the accumulator in tensor
// memory (TMEM), completion through an mbarrier, TMEM -> register loads.
//
// Operand tiles are K-major with the 128-byte swizzle: a tile row holds 64
// bf16 values (128 bytes) of one M (or N) index along K; 16-byte chunk c of
// row r is stored at chunk position c ^ (r % 8); 8-row groups are 1024
// bytes apart; tiles start on 1024-byte boundaries.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cpmdp {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a K-major 128B-swizzled bf16 tile.
__host__ __device__ __forceinline__ uint32_t sw128_off(uint32_t row, uint32_t k) {
    return row * 128u + ((((k >> 3) ^ (row & 7u)) & 7u) << 4) + ((k & 7u) << 1);
}

// Shared-memory matrix descriptor: start address, leading byte offset
// (unused for swizzled K-major tiles), stride byte offset (8-row groups,
// 1024 B), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Descriptor of an MN-major 128B-swizzled bf16 tile: a 1024-byte atom holds
// 8 K indices (128-byte rows) x 64 MN indices (8 chunks of 16 bytes, chunk c
// of row r at position c ^ r); atoms along MN are `mn_stride` bytes apart
// (leading byte offset), atoms along K 1024 bytes (stride byte offset).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t addr, uint32_t mn_stride) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((mn_stride >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Byte offset of element (m, k) in an MN-major 128B-swizzled bf16 tile of
// 128 MN indices x 64 K indices (two MN atoms 8192 bytes apart).
__host__ __device__ __forceinline__ uint32_t sw128_mn_off(uint32_t m, uint32_t k) {
    return (m >> 6) * 8192u + (k >> 3) * 1024u + (k & 7u) * 128u + (((((m >> 3) & 7u) ^ (k & 7u)) & 7u) << 4) +
           ((m & 7u) << 1);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N = 64, M = 128.
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
// The same with A MN-major (transpose-A bit).
constexpr uint32_t kIdescM128N64AMN = kIdescM128N64 | (1u << 15);

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// D (+)= A * B^T for 128 x 64 (A) and 64 x 64 (B) K-major tiles with K = 64,
// as BF16x3: A_hi B_hi + A_hi B_lo + A_lo B_hi (4 K-steps of 16 each).
// Issued by one thread. accumulate = 0 starts D from zero.
__device__ __forceinline__ void mma_bf16x3(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                           uint32_t b_lo, uint32_t accumulate) {
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        const uint32_t o = ks * 32;
        mma(d_tmem, sdesc(a_hi + o), sdesc(b_hi + o), kIdescM128N64, (accumulate || ks > 0) ? 1u : 0u);
        mma(d_tmem, sdesc(a_hi + o), sdesc(b_lo + o), kIdescM128N64, 1u);
        mma(d_tmem, sdesc(a_lo + o), sdesc(b_hi + o), kIdescM128N64, 1u);
    }
}

// The same with A an MN-major 128 x 64 tile (sw128_mn_off): a K-step of 16
// is two 1024-byte K atoms.
__device__ __forceinline__ void mma_bf16x3_amn(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                               uint32_t b_lo, uint32_t accumulate) {
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        const uint32_t oa = ks * 2048, ob = ks * 32;
        mma(d_tmem, sdesc_mn(a_hi + oa, 8192), sdesc(b_hi + ob), kIdescM128N64AMN, (accumulate || ks > 0) ? 1u : 0u);
        mma(d_tmem, sdesc_mn(a_hi + oa, 8192), sdesc(b_lo + ob), kIdescM128N64AMN, 1u);
        mma(d_tmem, sdesc_mn(a_lo + oa, 8192), sdesc(b_hi + ob), kIdescM128N64AMN, 1u);
    }
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

// One test of the phase; the thread may be suspended in hardware for up to
// about 0.1 ms while the phase is still incomplete (woken when it completes),
// so a waiting thread issues few instructions.
__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(phase), "r"(100000u)
        : "memory");
    return ok != 0;
}

// Wait for the given phase with a limit in SM clock cycles; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase, long long limit_cycles) {
    const long long t0 = clock64();
    while (!mbar_try(mbar, phase))
        if (clock64() - t0 > limit_cycles) return false;
    return true;
}

// One-dimensional bulk copy global -> shared through the copy engine,
// completing `bytes` of transaction count on the mbarrier. Addresses
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// Tiled tensor copy global -> shared of one box of a 5-D tensor map (the
// map is a __grid_constant__ kernel parameter), completing the box's bytes
// on the mbarrier. Coordinates are element indices, innermost first; parts
// of the box outside the tensor are filled with zeros. The innermost
// coordinate times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void *tmap, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(mbar))
        : "memory");
}

// Arrive on the mbarrier and expect `bytes` of transactions in this phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// Plain arrive (count 1) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Named barrier `id` over `n` threads (a multiple of 32), and the same with
// an AND of a predicate over those threads.
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool named_and(uint32_t id, uint32_t n, bool pred) {
    uint32_t out;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %3, 0;\nbar.red.and.pred q, %1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(out)
        : "r"(id), "r"(n), "r"((uint32_t)pred)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 32 lanes x 64 columns of 32-bit values: this warp's 32 TMEM lanes
// (lane offset in bits 31..16 of taddr), one row of 64 values per thread.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 64; j++) v[j] = __uint_as_float(r[j]);
}

// 32 lanes x 32 columns: this warp's 32 TMEM lanes, 32 values per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
}

// 32 lanes x 16 columns: this warp's 32 TMEM lanes, 16 values per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// 32 lanes x 16 columns issued without waiting: the registers may be read
// only after tmem_wait16 on the same array (the wait names them, so the
// compiler keeps every use of them after it).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// x = hi + lo with hi = bf16(x) and lo = bf16(x - hi) (round to nearest):
// hi + lo carries about 16 significant bits of x.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Eight values as bf16 hi and lo parts (split_bf16 on each), packed two per
// 32-bit word in order: hi[0..3] and lo[0..3] hold x[0..7].
__device__ __forceinline__ void split8_bf16(const float *x, uint32_t (&hi)[4], uint32_t (&lo)[4]) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * i] - __low2float(h), x[2 * i + 1] - __high2float(h));
        hi[i] = *reinterpret_cast<const uint32_t *>(&h);
        lo[i] = *reinterpret_cast<const uint32_t *>(&l);
    }
}

__device__ __forceinline__ uint32_t pack_hilo(float x) {
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    return (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
}

}  // namespace tc
}  // namespace cpmdp
