// Fused dense 3-way CP pass on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Same computation and partial-sum layouts as the FP32 pass (CPContr^(n) of P and Q,
// Section 6.1; Theorem "CP block multiplicative update"; Xhat never stored).  A CTA owns a
// tile of 128 rows j, a block of KB columns k (128, or 256 for the KL single-TF32 variants)
// and a range of slabs i, walked as a sequence of 64-column chunks (KB / 64 per slab).
// Warps are specialised and hand off through mbarriers only:
//   warp 17 (producer, one thread): X chunks into a shared-memory ring by TMA (chunks further
//     ahead into L2 by bulk prefetch) and GEMM1 of every chunk;
//   warp 16 (issuer, one thread; owns the TMEM allocation): the contractions (GEMM2);
//   warps 18, 19 (builders): per slab, the GEMM1 rows R = A_i (.) B_j (TF32) and the column
//     contraction's KRn^T = (A_i (.) B_j)^T (BF16), into rings of NR / NK buffers, one slab
//     ahead of their use;
//   warps 0..15 (epilogue): two groups of eight warps that take the chunks in turn (group
//     g = chunk parity).  Thread (warp w, lane l) owns tile row 32 (w % 4) + l (its TMEM
//     lane) and the 32 columns 32 ((w / 4) % 2) of its group's chunks; while one group runs
//     the MUFU-bound powers of a chunk, the other loads, hands off and folds.
//
// Per chunk n (slab i, columns k0 + 64 q):
//   TMA       X chunk (128 x 64 FP32, two 32-column boxes) into a 2- or 3-stage ring;
//   GEMM1     Xhat = R C^T on TF32 operands rounded to nearest, M128 N64 K32, into TMEM
//             buffer n % 2 as soon as that buffer's previous chunk has been read; with S3 the
//             operands are split into hi / lo TF32 parts (hi*lo + lo*hi + hi*hi);
//   epilogue  Xhat from TMEM (tcgen05.ld), X from shared memory, P = X Y^(beta-2),
//             Q = Y^(beta-1) (Y = max(Xhat, eps)) and the objective terms in FP32 registers;
//             P, Q stored once as BF16 tiles [rows][64 cols] (buffer n % NP);
//   GEMM2     rows: W[j][r] += sum_k P[j][k] Cn[k][r]   (A = P K-major, B = Cn^T)
//             cols: N3^T[r][k] += sum_j KRn^T[r][j] P[j][k]  (A = KRn^T with the rank
//             padded to M = 128, B = the P tile read MN-major; with four P buffers the P
//             tiles of a chunk pair, adjacent in shared memory, are one N = 128 operand),
//             BF16 operands, FP32 accumulation in TMEM.
// W of slab i (double-buffered by slab parity) is folded by both groups, each for 16 of the
// 32 ranks, early in slab i + 1: mode 1 reduces sum_j W[j][r] Bn[j][r] over each warp's 32
// rows (shuffle reduce-scatter, one partial per 32-row quarter, summed in fixed order
// later), mode 2 accumulates An[i][r] W[j][r] per row.  Every wait on an mbarrier is bounded;
// a wait that runs out raises a shared abort flag that ends the other waits at once; the
// kernel then sets the context's status word, waits (bounded) for its copies and MMAs, frees
// its TMEM and returns.
//
// With RX (explicit rows: the Tucker passes of Appendix C), the GEMM1 rows of slab i are
// rrow[i*J + j] (the mode-3 partial tensor B^(3) of eq. (block_Bn)) instead of A_i (.) B_j,
// the column contraction's operand is nrow[i*J + j] (and drow) instead of A_i (.) B_j, and
// the rows contraction W[j][r] of each slab is written out ([column block][I*J][RP]
// partials, summed over the column blocks afterwards) instead of being folded into modes
// 1 and 2.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <type_traits>

#include "ntf_internal.h"

namespace ntf {
namespace tc {

constexpr int ROWS = 128;  // tile rows
constexpr int KBLK = 128;  // columns per CTA block (256 for the KL / single-TF32 variants)
constexpr int CH = 64;     // columns per chunk
constexpr int RP = 32;
constexpr int CW = 32;     // columns per epilogue thread and chunk
constexpr int EW = 512;    // epilogue threads (two groups of eight warps)
constexpr int GW = EW / 2; // threads per group
constexpr int BW = 64;     // builder threads
constexpr int NT = EW + 64 + BW;  // + the issuer and producer warps + the builders
constexpr int PF = 6;      // X chunks prefetched into L2 ahead of the shared-memory ring

struct Layout {
    int x, p, q, r, rl, c, cl, cnt, cdt, knt, kdt, misc, total;
    int ns;  // X stages (2)
    int np;  // P / Q buffers (2: one per epilogue group; 4: two per group)
    int nk;  // KRn^T / KRd^T buffers
    int nr;  // R buffers
};

// 1024-aligned regions.  The column contraction reads KRn^T as an M = 128 operand whose
// rows 32..127 are padding: those rows only feed accumulator rows that are never read, so
// only the 32 real rows are stored (two 4 KB K-atoms per buffer) and the padding reads fall
// on the 16 KB or more that follow (the C / R tiles), which stay inside the allocation.
// kb: columns per CTA block; the C tile is kb x 32 TF32 (128 bytes a column) and the
// contraction's C^T operand 32 x kb BF16.
__host__ __device__ constexpr int layout_bytes(bool rows, bool m3, bool den, bool s3, int ns, int np, int nk, int nr,
                                               int kb) {
    return ns * 32768 + np * 16384 * (den ? 2 : 1) + (s3 ? 2 : 1) * kb * 128 + nr * (s3 ? 2 : 1) * 16384 +
           (rows ? kb * 64 : 0) + ((rows && den) ? kb * 64 : 0) + (m3 ? nk * 8192 : 0) + ((m3 && den) ? nk * 8192 : 0) +
           512 + 1024;
}

__host__ __device__ constexpr Layout make_layout(bool rows, bool m3, bool den, bool s3, int kb) {
    Layout L{};
    constexpr int kMax = 231424;  // opt-in shared memory per CTA (227 KB), less 1 KB of margin
    L.ns = 2;
    L.np = 2;
    L.nk = 1;
    L.nr = 1;
    if (layout_bytes(rows, m3, den, s3, 2, 2, 1, 2, kb) <= kMax) L.nr = 2;
    if (m3 && layout_bytes(rows, m3, den, s3, 2, 2, 2, L.nr, kb) <= kMax) L.nk = 2;
    if (layout_bytes(rows, m3, den, s3, 2, 4, L.nk, L.nr, kb) <= kMax) L.np = 4;
    // two X stages: chunk n uses slot n % 2, so each slot serves one epilogue group, whose parity
    // wait on it then always follows its own wait on the slot's previous phase
    int o = 0;
    L.x = o; o += L.ns * 32768;
    L.p = o; o += L.np * 16384;
    L.q = o; o += den ? L.np * 16384 : 0;
    L.knt = o; o += m3 ? L.nk * 8192 : 0;            // padding rows read the C tiles below
    L.c = o; o += kb * 128;
    L.cl = o; o += s3 ? kb * 128 : 0;
    L.kdt = o; o += (m3 && den) ? L.nk * 8192 : 0;   // padding rows read the R tiles below
    L.r = o; o += L.nr * 16384;
    L.rl = o; o += s3 ? L.nr * 16384 : 0;
    L.cnt = o; o += rows ? kb * 64 : 0;
    L.cdt = o; o += (rows && den) ? kb * 64 : 0;
    L.misc = o; o += 512;
    L.total = o + 1024;  // alignment slack of the dynamic base
    return L;
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, 128-byte swizzle: lbo = stride between 128-byte atoms
// along the contiguous dimension (MN-major only), sbo = stride between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo = 16, uint32_t sbo = 1024) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// instruction descriptors (D = F32, M = 128): TF32 K-major; BF16 with B K- or MN-major
__device__ __forceinline__ uint32_t idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ uint32_t idesc_bf16(int N, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float *v) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t addr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
}
// a 16-column load whose registers are only read after tmem_ld_wait16 on them: the wait
// names them as operands, so no use can be scheduled before it
__device__ __forceinline__ void tmem_ld16_issue(uint32_t addr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_ld_wait16(uint32_t *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :: "memory");
}
// two 16-column loads under one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t addr0, uint32_t addr1, float *v) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr0));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(addr1));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t addr, float *v) {
    if (N == 32) tmem_ld32(addr, v);
    else if (N == 16) tmem_ld16(addr, v);
    else tmem_ld8(addr, v);
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

constexpr int WAIT_LIMIT = 1 << 22;  // polls (a second or so at worst) before a wait gives up

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (int it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ float tf32_rna(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// element offsets inside 128-byte swizzled atoms (8-row period)
__device__ __forceinline__ int swf(int row, int k) { return row * 32 + ((((k >> 2) ^ (row & 7)) << 2) | (k & 3)); }
__device__ __forceinline__ int swh(int row, int k) { return row * 64 + ((((k >> 3) ^ (row & 7)) << 3) | (k & 7)); }

__device__ __forceinline__ void tma_2d(const CUtensorMap *map, uint32_t dst, uint32_t bar, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar) : "memory");
}
// shared -> global tensor store (bulk group); elements outside the tensor are not written
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n"
                 :: "l"(map), "r"(x), "r"(y), "r"(z), "r"(src) : "memory");
}
__device__ __forceinline__ void tma_3d(const CUtensorMap *map, uint32_t dst, uint32_t bar, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];\n" :: "l"(map), "r"(x), "r"(y) : "memory");
}
__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(bar), "r"(bytes) : "memory");
}

// Hardware approximate transcendentals (single MUFU instructions, denormals flushed).
__device__ __forceinline__ float mufu_rcp(float x) { float r; asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float mufu_rsqrt(float x) { float r; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float mufu_sqrt(float x) { float r; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float mufu_lg2(float x) { float r; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float mufu_ex2(float x) { float r; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }

// Packed pairs of FP32 values (one FMA-pipe instruction for both lanes of the pair).
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n mul.rn.ftz.f32x2 d, a, b;\n"
        " mov.b64 {%0, %1}, d;\n}\n" : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n .reg .b64 a, b, c, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n mov.b64 c, {%6, %7};\n"
        " fma.rn.ftz.f32x2 d, a, b, c;\n mov.b64 {%0, %1}, d;\n}\n"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n add.rn.ftz.f32x2 d, a, b;\n"
        " mov.b64 {%0, %1}, d;\n}\n" : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n sub.rn.ftz.f32x2 d, a, b;\n"
        " mov.b64 {%0, %1}, d;\n}\n" : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// One entry of the epilogue: P, Q (stored in BF16) and, with OBJ, the terms of d_beta(x|y)
// (Section 3.2) split so that the per-entry work is a few MUFU / FMA instructions:
//   KL : d = ln2 * x lg2 P + (y - x), P = x / y          -> o1 += x lg2 P,          o2 += y - x
//   IS : d = u - ln2 lg2 u - 1, u = x / y                -> o1 += lg2 u,            o2 += u - 1
//   1/2: d = -4 (sqrt x - y / 2 sqrt y - x / 2 sqrt y)  -> o2 += d
//   3/2: d = (x sqrt x + y sqrt y / 2 - 3 x sqrt y / 2) / (3/4)  -> o2 += d
//   else: beta (beta - 1) d with ex2 / lg2                -> o2 += beta (beta - 1) d
// The chunk's objective is o1 * ln2 + o2 (KL), o2 - o1 * ln2 (IS), o2 / (beta (beta - 1))
// for the general class and o2 for 1/2, 3/2.  These
// are the definition evaluated directly: where x ~ y its terms cancel, which costs about
// u_fp32 * x^beta / d relative accuracy per entry (the FP32 path keeps log1p / expm1 forms).
template <int BK, bool OBJ>
__device__ __forceinline__ void point(float beta, float x, float y, float &P, float &Q, float &o1, float &o2) {
    if (BK == BK_KL) {
        P = x * mufu_rcp(y);
        Q = 1.0f;
        if (OBJ) {  // x log(x / y) = x log P; the floor only keeps 0 * log 0 at 0
            o1 = fmaf(x, mufu_lg2(fmaxf(P, 1e-30f)), o1);
            o2 += y - x;
        }
    } else if (BK == BK_IS) {
        const float r = mufu_rcp(y);
        Q = r;
        P = x * r * r;
        if (OBJ) {
            const float u = x * r;
            o1 += mufu_lg2(u);
            o2 += u - 1.0f;
        }
    } else if (BK == BK_HALF) {
        const float sr = mufu_rsqrt(y);
        Q = sr;
        P = x * sr * sr * sr;
        if (OBJ) o2 += -4.0f * (mufu_sqrt(x) - 0.5f * y * sr - 0.5f * x * sr);
    } else if (BK == BK_THREEHALF) {
        const float sr = mufu_rsqrt(y), sy = y * sr;
        Q = sy;
        P = x * sr;
        if (OBJ) o2 += (x * mufu_sqrt(x) + 0.5f * y * sy - 1.5f * x * sy) * (1.0f / 0.75f);
    } else {
        const float ly = mufu_lg2(y);
        Q = mufu_ex2((beta - 1.0f) * ly);
        P = x * Q * mufu_rcp(y);
        if (OBJ) {
            const float yb = mufu_ex2(beta * ly);
            const float xb = x > 0.0f ? mufu_ex2(beta * mufu_lg2(x)) : 0.0f;
            o2 += xb + (beta - 1.0f) * yb - beta * x * Q;
        }
    }
}

template <int BK>
__device__ __forceinline__ float obj_combine(float beta, float o1, float o2) {
    const float ln2 = 0.6931471805599453f;
    if (BK == BK_KL) return fmaf(o1, ln2, o2);
    if (BK == BK_IS) return fmaf(-o1, ln2, o2);
    if (BK == BK_GEN) return o2 / (beta * (beta - 1.0f));
    return o2;
}

// sum over the 32 lanes of v[k] for k < N: afterwards lane l holds the sum for k = l % N
template <int N>
__device__ __forceinline__ float reduce_scatter(float v[N]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = N / 2; k >= 1; k >>= 1) {
        const bool upper = (lane & k) != 0;
#pragma unroll
        for (int q = 0; q < k; ++q) {
            const float send = upper ? v[q] : v[q + k];
            const float keep = upper ? v[q + k] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, k);
        }
    }
    float s = v[0];
#pragma unroll
    for (int o = N; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// eight BF16 values s * v[e] as one 16-byte word
__device__ __forceinline__ uint4 pack8(const float *v, float s) {
    __nv_bfloat162 h0 = __floats2bfloat162_rn(s * v[0], s * v[1]), h1 = __floats2bfloat162_rn(s * v[2], s * v[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(s * v[4], s * v[5]), h3 = __floats2bfloat162_rn(s * v[6], s * v[7]);
    uint4 u;
    u.x = *reinterpret_cast<uint32_t *>(&h0); u.y = *reinterpret_cast<uint32_t *>(&h1);
    u.z = *reinterpret_cast<uint32_t *>(&h2); u.w = *reinterpret_cast<uint32_t *>(&h3);
    return u;
}

template <int MS, int BK, bool S3, bool RX, int KB, bool WC = false>
__global__ void __launch_bounds__(NT, 1) cp3_pass_tc(const __grid_constant__ CUtensorMap xmap,
                                                      const __grid_constant__ CUtensorMap pcmap,
                                                      const __grid_constant__ CUtensorMap qcmap, const Cp3Args a) {
    constexpr bool DEN = BK != BK_KL;
    constexpr bool M1 = (MS & PM_M1) != 0, M2 = (MS & PM_M2) != 0, M3 = (MS & PM_M3) != 0;
    constexpr bool OBJ = (MS & PM_OBJ) != 0, RW = M1 || M2;
    // X-free pass (the dense part of a sparse tensor's update, Section 6.3): every entry is x = 0,
    // so no X chunk is copied (the producer's arrival takes the copy's place on chunk_ready), P
    // vanishes and Q = Xhat^(beta - 1) and the objective term d_beta(0 | Xhat) remain
    constexpr bool NX = (MS & PM_NOX) != 0;
    static_assert(!NX || (DEN && !RX && !WC), "the X-free pass is the denominator side of a CP pass");
    constexpr int CPS = KB / CH;  // chunks per slab (2 or 4)
    // 256-column blocks: single TF32, and either the KL CP passes or the explicit-rows W pass (no
    // column contraction: its N3 / N3d tensor-memory columns are free)
    static_assert(KB == 128 || (KB == 256 && !S3 && ((!DEN && !RX) || (RX && !M3))),
                  "256-column blocks: single TF32, KL CP passes or the explicit-rows W pass");
    constexpr Layout L = make_layout(RW, M3, DEN, S3, KB);
    constexpr int NS = L.ns, NP = L.np, NK = L.nk, NR = L.nr;
    constexpr bool PAIR = M3 && NP == 4;  // column contraction on chunk pairs (N = 128)
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const float *Xs = (const float *)(sm + L.x);
    __nv_bfloat16 *Ps = (__nv_bfloat16 *)(sm + L.p);
    __nv_bfloat16 *Qs = (__nv_bfloat16 *)(sm + L.q);
    float *Rs = (float *)(sm + L.r);
    float *Rl = (float *)(sm + L.rl);
    float *Cs = (float *)(sm + L.c);
    float *Cl = (float *)(sm + L.cl);
    __nv_bfloat16 *CnT = (__nv_bfloat16 *)(sm + L.cnt);
    __nv_bfloat16 *CdT = (__nv_bfloat16 *)(sm + L.cdt);
    __nv_bfloat16 *KnT = (__nv_bfloat16 *)(sm + L.knt);
    __nv_bfloat16 *KdT = (__nv_bfloat16 *)(sm + L.kdt);
    // mbarriers.  Per X ring slot (chunk % NS): chunk_ready (the X stage landed and X-hat
    // computed: the TMA bytes plus the GEMM1 commit), inputs_free (the chunk's group has read
    // the stage and the X-hat buffer).  Per P buffer (chunk % NP): p_full (the group's eight
    // warps), g2_done (the contractions that read it are complete).  Per R / KR buffer
    // (slab % NR, slab % NK): *_full (both builder warps), *_free (the slab's last GEMM1 /
    // GEMM2 complete).
    uint64_t *bars = (uint64_t *)(sm + L.misc);
    uint64_t *chunk_ready = bars, *inputs_free = bars + 3, *p_full = bars + 6, *g2_done = bars + 10;
    uint64_t *r_free = bars + 14, *r_full = bars + 16, *k_free = bars + 18, *k_full = bars + 20;
    uint64_t *probe_bar = bars + 22;  // nothing arrives on it (the timeout probe)
    constexpr int NBAR = 23;
    uint32_t *tslot = (uint32_t *)(sm + L.misc + 192);
    volatile int *abort_flag = (volatile int *)(sm + L.misc + 200);
    double *dred = (double *)(sm + L.misc + 256);  // [EW / 32] (128 bytes)

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const bool issuer = warp == EW / 32, producer = warp == EW / 32 + 1, builder = warp >= EW / 32 + 2;
    const int quarter = warp & 3, half = (warp >> 2) & 1, grp = (warp >> 3) & 1;
    const int row = 32 * quarter + lane;  // tile row = TMEM lane (epilogue warps)
    int b = blockIdx.x;
    const int is = b % a.n_is;
    b /= a.n_is;
    const int kb = b % a.n_kb;
    const int jt = b / a.n_kb;
    const int i0 = (int)((int64_t)is * a.I / a.n_is);
    const int i1 = (int)((int64_t)(is + 1) * a.I / a.n_is);
    const int J = a.J, K = a.K;
    const int j0 = jt * ROWS, k0 = kb * KB;
    const int j = j0 + row;
    const bool epi = warp < EW / 32;
    const bool jv = epi && j < J;
    const int NSL = i1 - i0;  // slabs of this CTA
    const int NC = CPS * NSL;
    const int rf = 16 * grp + 8 * half;  // this thread's 8 ranks of the folds

    const int wlim = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT;
    auto wait = [&](uint64_t *bar, uint32_t phase) -> bool {
        const uint32_t ba = su32(bar);
        for (int it = 0; it < wlim; ++it) {
            uint32_t done;
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(done) : "r"(ba), "r"(phase) : "memory");
            if (done) return true;
            if (*abort_flag) return false;
        }
        *abort_flag = 1;
        return false;
    };
    auto arrive = [&](uint64_t *bar) {  // one arrival per warp, after the warp's accesses
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(su32(bar)) : "memory");
    };

    // ---- per-CTA constants (epilogue threads): the row factors of the mode-1 fold ----------
    float bn[8], bd[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        bn[r] = (jv && M1 && !RX) ? __ldg(a.num[1] + (int64_t)j * RP + rf + r) : 0.0f;
        bd[r] = (jv && M1 && DEN && !RX) ? __ldg(a.den[1] + (int64_t)j * RP + rf + r) : 0.0f;
    }
    if (epi) {
        // C tile (GEMM1 B operand, TF32 hi / lo) and Cn^T / Cd^T (rows contraction B operand)
        const int cr0 = 8 * (warp >> 2);
#pragma unroll 1
        for (int cc = row; cc < KB; cc += ROWS) {  // block column cc
            const int kc = k0 + cc;
            const bool kv = kc < K;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float v = kv ? __ldg(a.rec[2] + (int64_t)kc * RP + cr0 + 4 * q + e) : 0.0f;
                    h[e] = tf32_rna(v);
                    l[e] = S3 ? tf32_rna(v - h[e]) : 0.0f;
                }
                *reinterpret_cast<float4 *>(Cs + swf(cc, cr0 + 4 * q)) = make_float4(h[0], h[1], h[2], h[3]);
                if (S3) *reinterpret_cast<float4 *>(Cl + swf(cc, cr0 + 4 * q)) = make_float4(l[0], l[1], l[2], l[3]);
            }
            if (RW) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int rr = cr0 + r;
                    CnT[(cc >> 6) * 2048 + swh(rr, cc & 63)] =
                        __float2bfloat16_rn(kv ? __ldg(a.num[2] + (int64_t)kc * RP + rr) : 0.0f);
                    if (DEN)
                        CdT[(cc >> 6) * 2048 + swh(rr, cc & 63)] =
                            __float2bfloat16_rn(kv ? __ldg(a.den[2] + (int64_t)kc * RP + rr) : 0.0f);
                }
            }
        }
    }
    if (t == EW) {
        for (int q = 0; q < NBAR; ++q) {
            // chunk_ready: expect_tx + GEMM1 commit; g2_done, r_free, k_free: one commit;
            // r_full, k_full: the two builder warps; inputs_free, p_full: a group's eight warps;
            // probe_bar: one (never given)
            const uint32_t cnt = q < 3 ? 2 : q < 10 ? GW / 32 : q < 16 ? 1 : q < 18 ? 2 : q < 20 ? 1 : q < 22 ? 2 : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(su32(bars + q)), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        *abort_flag = 0;
    }
    __syncthreads();
    if (issuer) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" :: "r"(su32(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    // TMEM columns: X-hat [2][64] | W, Wd of even / odd slabs [2][32 + 32] | N3 [KB] | N3d [128]
    const uint32_t t_d1 = tmem, t_w = tmem + 128, t_wd = tmem + 160, t_n3 = tmem + 256, t_n3d = tmem + 384;

    float acc2[8], acc2d[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc2[r] = acc2d[r] = 0.0f;
    double obj_acc = 0.0;

    if (producer) {
        // ---- producer thread: X chunks into the ring, PF chunks ahead into L2, GEMM1 ------
        if (lane == 0 && NC > 0) {
            auto prefetch_x = [&](int n) {
                if (NX) return;
                const int i = i0 + n / CPS, x = k0 + CH * (n % CPS);
                // only boxes that start inside the tensor (a ragged block's last chunk may not)
                if (x < K) tma_prefetch_2d(&xmap, x, i * J + j0);
                if (x + 32 < K) tma_prefetch_2d(&xmap, x + 32, i * J + j0);
            };
            auto load_x = [&](int n) {
                const int i = i0 + n / CPS, q = n % CPS;
                const uint32_t bar = su32(chunk_ready + n % NS);
                const uint32_t dst = su32(Xs) + (n % NS) * 32768;
                if (NX) {  // nothing to copy: the arrival alone
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(bar) : "memory");
                    return;
                }
                expect_tx(bar, 32768);
                tma_2d(&xmap, dst, bar, k0 + CH * q, i * J + j0);
                tma_2d(&xmap, dst + 16384, bar, k0 + CH * q + 32, i * J + j0);
            };
            // GEMM1 descriptors: A = R rows (K-major, 4 K-steps of 8 TF32), B = C columns
            const uint32_t id1 = idesc_tf32(CH);
            const uint64_t dR = sdesc(su32(Rs)), dRl = sdesc(su32(Rl)), dC = sdesc(su32(Cs)), dCl = sdesc(su32(Cl));
            // the timeout probe: one bounded wait that runs out before anything is issued
            const bool go = !a.timeout_probe || wait(probe_bar, 0);
            if (go)
                for (int c = 0; c < NS && c < NC; ++c) load_x(c);
            if (go)
                for (int c = NS; c < NS + PF && c < NC; ++c) prefetch_x(c);
            for (int n = 0; n < NC && go; ++n) {
                if (n >= 2) {
                    // chunk n - 2 has been read: X-hat buffer n % 2 and ring slot (n - 2) % NS
                    // free; the X chunk first (the longer path), then GEMM1 of chunk n
                    if (!wait(inputs_free + (n - 2) % NS, ((n - 2) / NS) & 1) || *abort_flag) break;
                    const int c = n - 2 + NS;
                    if (c < NC) load_x(c);
                    if (c + PF < NC) prefetch_x(c + PF);
                }
                const int s = n / CPS, q = n % CPS;
                if (q == 0 && !wait(r_full + s % NR, (s / NR) & 1)) break;
                if (*abort_flag) break;  // nothing is issued once a wait has given up
                fence_after();
                const uint32_t d = t_d1 + 64 * (n & 1);
                const uint32_t ro = (uint32_t)(s % NR) * 1024u;  // 16 KB R buffer, in 16-byte units
                const uint32_t co = (uint32_t)q * 512u;           // 8 KB of C per chunk
                if (S3) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) mma_tf32(d, dRl + ro + 2 * k, dC + co + 2 * k, id1, k > 0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) mma_tf32(d, dR + ro + 2 * k, dCl + co + 2 * k, id1, 1);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) mma_tf32(d, dR + ro + 2 * k, dC + co + 2 * k, id1, S3 || k > 0);
                mma_commit(su32(chunk_ready + n % NS));
                if (q == CPS - 1) mma_commit(su32(r_free + s % NR));  // R of slab s read once done
            }
        }
        __syncwarp();
    } else if (issuer) {
        // ---- issuer thread: the contractions of every chunk, in chunk order ----------------
        if (lane == 0 && NC > 0) {
            const uint32_t idr = idesc_bf16(RP, false), idc = idesc_bf16(PAIR ? 2 * CH : CH, true);
            const uint64_t dP = sdesc(su32(Ps)), dQ = sdesc(su32(Qs)), dCn = sdesc(su32(CnT)), dCd = sdesc(su32(CdT));
            const uint64_t dPm = sdesc(su32(Ps), 16384, 1024), dQm = sdesc(su32(Qs), 16384, 1024);
            const uint64_t dKn = sdesc(su32(KnT)), dKd = sdesc(su32(KdT));
            for (int n = 0; n < NC; ++n) {
                const int s = n / CPS, q = n % CPS, pb = n % NP;
                if (!wait(p_full + pb, (n / NP) & 1)) break;
                if (M3 && q == 0 && !wait(k_full + s % NK, (s / NK) & 1)) break;
                if (*abort_flag) break;  // nothing is issued once a wait has given up
                fence_after();
                const uint32_t po = (uint32_t)pb * 1024u;  // P / Q buffer (16 KB) in 16-byte units
                if (RW) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t acc = (q > 0 || k > 0) ? 1u : 0u;
                        mma_bf16(t_w + 64 * (s & 1), dP + po + 2 * k, dCn + q * 256 + 2 * k, idr, acc);
                        if (DEN) mma_bf16(t_wd + 64 * (s & 1), dQ + po + 2 * k, dCd + q * 256 + 2 * k, idr, acc);
                    }
                }
                if (M3 && (!PAIR || (n & 1))) {
                    // one chunk (N = 64), or the pair n - 1, n (N = 128: the two P buffers are
                    // the operand's two 64-column atoms, 16 KB apart)
                    const int qq = PAIR ? q - 1 : q;
                    const uint32_t pp = PAIR ? po - 1024u : po;
                    const uint32_t ko = (uint32_t)(s % NK) * 512u;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t ao = ko + (k >> 2) * 256 + (k & 3) * 2;
                        const uint32_t acc = (s > 0 || k > 0) ? 1u : 0u;
                        mma_bf16(t_n3 + 64 * qq, dKn + ao, dPm + pp + k * 128, idc, acc);
                        if (DEN) mma_bf16(t_n3d + 64 * qq, dKd + ao, dQm + pp + k * 128, idc, acc);
                    }
                    if (PAIR) mma_commit(su32(g2_done + (n - 1) % NP));
                }
                if (WC) {
                    // the chunk's P~ / Q~ tiles into the cache by TMA; they must be read out of
                    // shared memory before the buffer's g2_done, which the epilogue waits on
                    // before it rewrites the buffer
                    fence_async_smem();
                    tma_store_3d(&pcmap, su32(Ps) + pb * 16384, k0 + CH * q, j0, i0 + s);
                    if (DEN) tma_store_3d(&qcmap, su32(Qs) + pb * 16384, k0 + CH * q, j0, i0 + s);
                    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                }
                if (!PAIR || (n & 1)) mma_commit(su32(g2_done + pb));
                if (M3 && q == CPS - 1) mma_commit(su32(k_free + s % NK));  // KR of slab s read once done
            }
            if (WC) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");  // the cache writes done
        }
        __syncwarp();
    } else if (builder) {
        // ---- builder warps: R and KRn^T / KRd^T of every slab, one slab ahead -------------
        // thread bt owns the tile rows 2 bt and 2 bt + 1 (R rows; KR^T columns); every global
        // load of a 16-rank half is issued before its first use (one latency per half)
        const int bt = t - (EW + 64), jr0 = 2 * bt;
        const bool v0 = j0 + jr0 < J, v1 = j0 + jr0 + 1 < J;
        const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        auto mul4 = [](float4 x, float4 y) { return make_float4(x.x * y.x, x.y * y.y, x.z * y.z, x.w * y.w); };
        // rank half h of rows j0 + jr0, + 1 of slab i: A_i (.) B_j from the factors f0 / f1, or
        // the explicit rows xr[i * J + j]
        auto rows2 = [&](const float *f0, const float *f1, const float *xr, int i, int h, float4 *x0, float4 *x1) {
            if (RX) {
                const float4 *p = reinterpret_cast<const float4 *>(xr + ((int64_t)i * J + j0 + jr0) * RP + 16 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x0[q] = v0 ? __ldg(p + q) : z4;
                    x1[q] = v1 ? __ldg(p + RP / 4 + q) : z4;
                }
            } else {
                const float4 *pa = reinterpret_cast<const float4 *>(f0 + (int64_t)i * RP + 16 * h);
                const float4 *pb = reinterpret_cast<const float4 *>(f1 + (int64_t)(j0 + jr0) * RP + 16 * h);
                float4 av[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    av[q] = __ldg(pa + q);
                    x0[q] = v0 ? __ldg(pb + q) : z4;
                    x1[q] = v1 ? __ldg(pb + RP / 4 + q) : z4;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x0[q] = mul4(av[q], x0[q]);
                    x1[q] = mul4(av[q], x1[q]);
                }
            }
        };
        // KR^T entries (r, jr0) and (r, jr0 + 1) for the 16 ranks of half h, as BF16 pairs
        auto store_kt = [&](__nv_bfloat16 *kt, int h, const float4 *x0, const float4 *x1) {
            __nv_bfloat16 *base = kt + (jr0 >> 6) * 2048;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float a0[4] = {x0[q].x, x0[q].y, x0[q].z, x0[q].w}, a1[4] = {x1[q].x, x1[q].y, x1[q].z, x1[q].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(a0[e], a1[e]);
                    *reinterpret_cast<__nv_bfloat162 *>(base + swh(16 * h + 4 * q + e, jr0 & 63)) = pr;
                }
            }
        };
        for (int s = 0; s < NSL; ++s) {
            const int i = i0 + s;
            if (s >= NR && !wait(r_free + s % NR, ((s - NR) / NR) & 1)) break;
            {
                // R [128 rows][32 ranks] TF32 (hi / lo)
                float *rh = Rs + (s % NR) * 4096, *rl = Rl + (s % NR) * 4096;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float4 x0[4], x1[4];
                    rows2(a.rec[0], a.rec[1], a.rrow, i, h, x0, x1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float4 v = e ? x1[q] : x0[q];
                            const float h0 = tf32_rna(v.x), h1 = tf32_rna(v.y), h2 = tf32_rna(v.z), h3 = tf32_rna(v.w);
                            *reinterpret_cast<float4 *>(rh + swf(jr0 + e, 16 * h + 4 * q)) = make_float4(h0, h1, h2, h3);
                            if (S3)
                                *reinterpret_cast<float4 *>(rl + swf(jr0 + e, 16 * h + 4 * q)) =
                                    make_float4(tf32_rna(v.x - h0), tf32_rna(v.y - h1), tf32_rna(v.z - h2), tf32_rna(v.w - h3));
                        }
                    }
                }
            }
            fence_async_smem();
            arrive(r_full + s % NR);
            if (M3) {
                if (s >= NK && !wait(k_free + s % NK, ((s - NK) / NK) & 1)) break;
                // KRn^T / KRd^T [32 ranks][128 rows] BF16
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float4 x0[4], x1[4];
                    rows2(a.num[0], a.num[1], a.nrow, i, h, x0, x1);
                    store_kt(KnT + (s % NK) * 4096, h, x0, x1);
                    if (DEN) {
                        rows2(a.den[0], a.den[1], a.drow, i, h, x0, x1);
                        store_kt(KdT + (s % NK) * 4096, h, x0, x1);
                    }
                }
                fence_async_smem();
                arrive(k_full + s % NK);
            }
        }
    } else {
        // ---- epilogue warps ---------------------------------------------------------------
        auto fold = [&](int s, const float *an, const float *ad) {  // modes 1 and 2 from W of slab offset s
            const int i = i0 + s;
            const uint32_t wb = 64 * (s & 1);
            float w[8], wd[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) w[r] = wd[r] = 0.0f;
            if (!__any_sync(0xffffffffu, *abort_flag != 0)) {  // warp-uniform before tcgen05.ld
                tmem_ld8(t_w + wb + lane_off + rf, w);
                if (DEN) tmem_ld8(t_wd + wb + lane_off + rf, wd);
            }
            if (RX) {  // W rows of slab i for this column block: [kb][i * J + j][RP] partials
                if (jv && !*abort_flag) {
                    const int64_t o = (((int64_t)kb * a.I + i) * J + j) * RP + rf;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        reinterpret_cast<float4 *>(a.p1n + o)[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
                        if (DEN)
                            reinterpret_cast<float4 *>(a.p1d + o)[q] =
                                make_float4(wd[4 * q], wd[4 * q + 1], wd[4 * q + 2], wd[4 * q + 3]);
                    }
                }
                return;
            }
            if (M2) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    acc2[r] = fmaf(an[r], w[r], acc2[r]);
                    if (DEN) acc2d[r] = fmaf(ad[r], wd[r], acc2d[r]);
                }
            }
            if (M1) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    w[r] *= bn[r];
                    if (DEN) wd[r] *= bd[r];
                }
                // one partial per warp (its 32 rows of the tile), summed later in fixed order
                const float sr = reduce_scatter<8>(w);
                const float sd = DEN ? reduce_scatter<8>(wd) : 0.0f;
                if (lane < 8 && !*abort_flag) {
                    const int64_t slot = (((int64_t)(jt * a.n_kb + kb) * 4 + quarter) * a.I + i) * RP + rf + lane;
                    a.p1n[slot] = sr;
                    if (DEN) a.p1d[slot] = sd;
                }
            }
        };
        // W of slab s is folded by each group once the contractions of the slab's last chunk
        // L = CPS (s + 1) - 1 are complete, and before slab s + 2's first contraction rewrites
        // it (that contraction is issued after the P tile of chunk CPS (s + 2)).  Where that
        // leaves room, a group folds at its first chunk n >= L + NP, whose own P-buffer wait
        // (chunk n - NP) covers chunk L; otherwise group 1 folds at L + 2 and group 0 at L + 3
        // after an explicit wait for chunk L (that barrier cannot have moved on by two phases:
        // chunk L + NP's contraction needs a P tile of this chunk or a later one).
        int fold_next = 0;
        auto fold_chunk = [&](int s) {
            const int last = CPS * (s + 1) - 1;
            if (last + NP + 1 <= CPS * (s + 2)) return last + NP + ((grp ^ (last + NP)) & 1);
            return last + 3 - grp;
        };
        // shared-memory offsets of this thread's X and P / Q entries within a stage / tile
        int xo[CW / 4], po[CW / 8];
#pragma unroll
        for (int g = 0; g < CW / 4; ++g) xo[g] = half * 4096 + swf(row, 4 * g);
#pragma unroll
        for (int g = 0; g < CW / 8; ++g) po[g] = swh(row, CW * half + 8 * g);
        float osum = 0.0f, ocomp = 0.0f;  // objective of this thread's chunks: compensated FP32 sum
        for (int n = grp; n < NC; n += 2) {
            const int s = n / CPS, q = n % CPS;
            const int pb = n % NP;
            const bool fold_now = RW && fold_next < s && fold_chunk(fold_next) <= n;
            float an[8], ad[8];  // the folded slab's factor row, loaded before the waits
            if (fold_now && M2 && !RX) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    an[r] = __ldg(a.num[0] + (int64_t)(i0 + fold_next) * RP + rf + r);
                    ad[r] = DEN ? __ldg(a.den[0] + (int64_t)(i0 + fold_next) * RP + rf + r) : 0.0f;
                }
            }
            if (n >= NP) wait(g2_done + pb, ((n - NP) / NP) & 1);  // P tile pb free again
            if (fold_now) {
                const int last = CPS * (fold_next + 1) - 1;
                if (n - NP < last) wait(g2_done + last % NP, (last / NP) & 1);
                fence_after();
                fold(fold_next++, an, ad);
                fence_before();
            }
            const bool ready = __all_sync(0xffffffffu, wait(chunk_ready + n % NS, (n / NS) & 1));
            fence_after();
            // the thread's 32 columns as two halves of 16: X-hat of the second half is loaded
            // from TMEM while the first half's powers run; X of each half from shared memory
            // just before its powers
            float xh0[16], xh1[16], xv[CW / 2];
            uint32_t xr1[16];
            const uint32_t ta = t_d1 + 64 * (n & 1) + lane_off + CW * half;
            if (ready) {  // warp-uniform before tcgen05.ld
                tmem_ld16(ta, xh0);
                tmem_ld16_issue(ta + 16, xr1);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) xh0[c] = 0.0f;
            }
            const float *xa = Xs + (n % NS) * 8192;
            auto load_x = [&](int h) {
#pragma unroll
                for (int g = 0; g < CW / 8; ++g) {
                    const float4 v = NX ? make_float4(0.0f, 0.0f, 0.0f, 0.0f)
                                        : *reinterpret_cast<const float4 *>(xa + xo[4 * h + g]);
                    xv[4 * g] = v.x; xv[4 * g + 1] = v.y; xv[4 * g + 2] = v.z; xv[4 * g + 3] = v.w;
                }
            };
            __nv_bfloat16 *pa = Ps + pb * 8192;
            __nv_bfloat16 *qa = Qs + pb * 8192;
            const int kc0 = k0 + CH * q + CW * half;
            float o1 = 0.0f, o2 = 0.0f;
            float2 u1 = make_float2(0.0f, 0.0f), u2 = make_float2(0.0f, 0.0f);  // packed KL sums
            // powers of half h (columns kc0 + 16 h ..); full strip of a valid row: no masks
            auto body = [&](auto full_tag, int h) {
                constexpr bool FULL = decltype(full_tag)::value;
                const int kc = kc0 + 16 * h;
                const float *xhh = h ? xh1 : xh0;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    float pv[8], qv[8];
                    if (FULL && BK == BK_KL) {
                        // the KL point function on pairs of entries; P = x / y + 1e-30 keeps
                        // the logarithm of an x = 0 entry finite (0 * lg2(1e-30) = 0)
#pragma unroll
                        for (int c = 0; c < 8; c += 2) {
                            const float2 x2 = make_float2(xv[8 * g + c], xv[8 * g + c + 1]);
                            const float2 y2 = make_float2(fmaxf(xhh[8 * g + c], a.eps), fmaxf(xhh[8 * g + c + 1], a.eps));
                            const float2 P2 = fma2(x2, make_float2(mufu_rcp(y2.x), mufu_rcp(y2.y)),
                                                   make_float2(1e-30f, 1e-30f));
                            pv[c] = P2.x;
                            pv[c + 1] = P2.y;
                            if (OBJ) {
                                const float2 l2 = make_float2(mufu_lg2(P2.x), mufu_lg2(P2.y));
                                u1 = fma2(x2, l2, u1);
                                u2 = add2(u2, sub2(y2, x2));
                            }
                        }
                    } else
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float x = xv[8 * g + c];
                        if (BK == BK_IS) x = fmaxf(x, a.eps_x);
                        const float y = fmaxf(xhh[8 * g + c], a.eps);
                        if (FULL) {
                            point<BK, OBJ>(a.beta, x, y, pv[c], qv[c], o1, o2);
                        } else {
                            float P, Q, e1 = 0.0f, e2 = 0.0f;
                            point<BK, OBJ>(a.beta, x, y, P, Q, e1, e2);
                            const bool v = jv && (kc + 8 * g + c) < K;
                            pv[c] = v ? P : 0.0f;
                            qv[c] = v ? Q : 0.0f;
                            if (OBJ && v) { o1 += e1; o2 += e2; }
                        }
                    }
                    *reinterpret_cast<uint4 *>(pa + po[2 * h + g]) = pack8(pv, 1.0f);
                    if (DEN) *reinterpret_cast<uint4 *>(qa + po[2 * h + g]) = pack8(qv, 1.0f);

                }
            };
            load_x(0);
            if (jv && kc0 + 16 <= K) body(std::true_type{}, 0);
            else body(std::false_type{}, 0);
            if (ready) tmem_ld_wait16(xr1);
#pragma unroll
            for (int c = 0; c < 16; ++c) xh1[c] = ready ? __uint_as_float(xr1[c]) : 0.0f;
            load_x(1);
            fence_before();
            arrive(inputs_free + n % NS);
            if (jv && kc0 + 32 <= K) body(std::true_type{}, 1);
            else body(std::false_type{}, 1);
            if (OBJ) {
                if (BK == BK_KL) {
                    o1 += u1.x + u1.y;
                    o2 += u2.x + u2.y;
                }
                const float oy = obj_combine<BK>(a.beta, o1, o2) - ocomp;  // Kahan summation
                const float ot = osum + oy;
                ocomp = (ot - osum) - oy;
                osum = ot;
            }
            fence_async_smem();
            arrive(p_full + pb);
        }
        if (OBJ) obj_acc = (double)osum - (double)ocomp;
        if (NC > 0) {
            // every contraction complete.  A parity wait on a barrier is valid only while the
            // barrier's previous phase is complete and its next one is not: the last NP chunks
            // (one per P buffer, none after them) are waited for in increasing order; the
            // first one's previous phase (chunk NC - 2 NP) is covered by this thread's last
            // P-buffer wait, each later one's by the wait before it (in-order completion)
            for (int m = NC - NP > 0 ? NC - NP : 0; m < NC; ++m) wait(g2_done + m % NP, (m / NP) & 1);
            fence_after();
            if (RW) {
                while (fold_next < NSL) {
                    float an[8], ad[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        an[r] = (M2 && !RX) ? __ldg(a.num[0] + (int64_t)(i0 + fold_next) * RP + rf + r) : 0.0f;
                        ad[r] = (M2 && DEN && !RX) ? __ldg(a.den[0] + (int64_t)(i0 + fold_next) * RP + rf + r) : 0.0f;
                    }
                    fold(fold_next++, an, ad);
                }
            }
        }
        // ---- CTA outputs ------------------------------------------------------------------
        const bool good = !__any_sync(0xffffffffu, *abort_flag != 0);
        if (M2 && jv && !RX) {
            const int64_t base = ((int64_t)(kb * a.n_is + is) * J + j) * RP + rf;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                a.p2n[base + r] = acc2[r];
                if (DEN) a.p2d[base + r] = acc2d[r];
            }
        }
        if (M3 && quarter == 0) {
            const int cg4 = warp >> 2;
            const int64_t base = (int64_t)(jt * a.n_is + is) * K;
#pragma unroll 1
            for (int g = 0; g < KB / 128; ++g) {
                float v[32], vd[32];
                const bool have = good && NC > 0;
                const int cb = (KB / 4) * cg4 + 32 * g;
                if (have) {
                    tmem_ld32(t_n3 + cb, v);
                    if (DEN) tmem_ld32(t_n3d + cb, vd);
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int kc = k0 + cb + c;
                    if (kc < K) {
                        a.p3n[(base + kc) * RP + lane] = have ? v[c] : 0.0f;
                        if (DEN) a.p3d[(base + kc) * RP + lane] = have ? vd[c] : 0.0f;
                    }
                }
            }
        }
        if (OBJ) {
            double v = obj_acc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) dred[warp] = v;
            asm volatile("bar.sync 1, %0;\n" :: "n"(EW) : "memory");
            if (t == 0) {
                double s2 = 0.0;
                for (int w = 0; w < EW / 32; ++w) s2 += dred[w];
                a.obj[blockIdx.x] = s2;
            }
        }
    }
    fence_before();
    __syncthreads();
    if (*abort_flag && t == EW) {
        // bounded waits (without the abort shortcut) for copies and MMAs still in flight
        const int clim = wlim < (1 << 20) ? wlim : (1 << 20);
        for (int q = 0; q < NBAR; ++q) {
            for (int ph = 0; ph < 2; ++ph) {
                for (int it = 0; it < clim; ++it) {
                    uint32_t done;
                    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                                 : "=r"(done) : "r"(su32(bars + q)), "r"(ph) : "memory");
                    if (done) break;
                }
            }
        }
        if (a.err) atomicExch(a.err, 1);
    }
    __syncthreads();
    if (issuer) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" :: "r"(tmem));
    }
}

cudaError_t launch_x_map(const Cp3Args &a, CUtensorMap *map);
// P~ / Q~ cache as a 3-D BF16 tensor [I][J][K] with row stride kp; boxes of 64 x 128 x 1 with the
// 128-byte swizzle of the operand buffers (rows past J and columns past K are outside the tensor)
cudaError_t cache_map(void *base, const Cp3Args &a, CUtensorMap *map);

template <int MS, int BK, bool S3, bool RX, int KB = KBLK, bool WC = false>
cudaError_t launch_t(const Cp3Plan &p, const Cp3Args &a, cudaStream_t s) {
    constexpr Layout L = make_layout((MS & (PM_M1 | PM_M2)) != 0, (MS & PM_M3) != 0, BK != BK_KL, S3, KB);
    CUtensorMap map{}, pm{}, qm{};
    cudaError_t e = (MS & PM_NOX) ? cudaSuccess : launch_x_map(a, &map);  // the X-free pass reads no X
    if (e == cudaSuccess && WC) e = cache_map(a.pc, a, &pm);
    if (e == cudaSuccess && WC && BK != BK_KL) e = cache_map(a.qc, a, &qm);
    if (e != cudaSuccess) return e;
    auto k = cp3_pass_tc<MS, BK, S3, RX, KB, WC>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < NT) return cudaErrorLaunchOutOfResources;  // registers x NT beyond the SM
    k<<<p.grid, NT, L.total, s>>>(map, pm, qm, a);
    return cudaGetLastError();
}

template <int BK, bool S3>
cudaError_t launch_bk(const Cp3Plan &p, const Cp3Args &a, int ms, cudaStream_t s) {
    if (a.pc) {  // J-CoMM first pass that also writes the P~ / Q~ cache (beta != 1)
        if constexpr (BK != BK_KL) {
            if (p.KB == KBLK && ms == (PM_M1 | PM_OBJ)) return launch_t<PM_M1 | PM_OBJ, BK, S3, false, KBLK, true>(p, a, s);
            if (p.KB == KBLK && ms == PM_M1) return launch_t<PM_M1, BK, S3, false, KBLK, true>(p, a, s);
        }
        return cudaErrorInvalidValue;
    }
    if (ms & PM_NOX) {  // X-free denominator passes of a sparse tensor at beta != 1
        if constexpr (BK != BK_KL) {
            if (p.KB != KBLK) return cudaErrorInvalidValue;
            switch (ms) {
                case PM_M1 | PM_NOX: return launch_t<PM_M1 | PM_NOX, BK, S3, false>(p, a, s);
                case PM_M1 | PM_OBJ | PM_NOX: return launch_t<PM_M1 | PM_OBJ | PM_NOX, BK, S3, false>(p, a, s);
                case PM_M2 | PM_NOX: return launch_t<PM_M2 | PM_NOX, BK, S3, false>(p, a, s);
                case PM_M3 | PM_NOX: return launch_t<PM_M3 | PM_NOX, BK, S3, false>(p, a, s);
                default: break;
            }
        }
        return cudaErrorInvalidValue;
    }
    if (a.rrow) {  // explicit rows (Tucker): W rows out, or the column contraction
        if constexpr (!S3) {
            if (p.KB == 256) {
                switch (ms) {
                    case PM_M1 | PM_M2: return launch_t<PM_M1 | PM_M2, BK, S3, true, 256>(p, a, s);
                    case PM_M1 | PM_M2 | PM_OBJ: return launch_t<PM_M1 | PM_M2 | PM_OBJ, BK, S3, true, 256>(p, a, s);
                    default: return cudaErrorInvalidValue;
                }
            }
        }
        if (p.KB != KBLK) return cudaErrorInvalidValue;
        switch (ms) {
            case PM_M1 | PM_M2: return launch_t<PM_M1 | PM_M2, BK, S3, true>(p, a, s);
            case PM_M1 | PM_M2 | PM_OBJ: return launch_t<PM_M1 | PM_M2 | PM_OBJ, BK, S3, true>(p, a, s);
            case PM_M3: return launch_t<PM_M3, BK, S3, true>(p, a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if constexpr (BK == BK_KL && !S3) {
        if (p.KB == 256) {
            switch (ms) {
                case PM_M1: return launch_t<PM_M1, BK, S3, false, 256>(p, a, s);
                case PM_M1 | PM_OBJ: return launch_t<PM_M1 | PM_OBJ, BK, S3, false, 256>(p, a, s);
                case PM_M2: return launch_t<PM_M2, BK, S3, false, 256>(p, a, s);
                case PM_M3: return launch_t<PM_M3, BK, S3, false, 256>(p, a, s);
                case PM_M1 | PM_M2 | PM_M3 | PM_OBJ: return launch_t<PM_M1 | PM_M2 | PM_M3 | PM_OBJ, BK, S3, false, 256>(p, a, s);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    if (p.KB != KBLK) return cudaErrorInvalidValue;
    switch (ms) {
        case PM_M1: return launch_t<PM_M1, BK, S3, false>(p, a, s);
        case PM_M1 | PM_OBJ: return launch_t<PM_M1 | PM_OBJ, BK, S3, false>(p, a, s);
        case PM_M2: return launch_t<PM_M2, BK, S3, false>(p, a, s);
        case PM_M3: return launch_t<PM_M3, BK, S3, false>(p, a, s);
        case PM_M1 | PM_M2 | PM_M3 | PM_OBJ:
            if constexpr (BK == BK_KL) return launch_t<PM_M1 | PM_M2 | PM_M3 | PM_OBJ, BK_KL, S3, false>(p, a, s);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
}  // namespace ntf
