// Fused dense 3-way CP pass on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Same computation and partial-sum layouts as the FP32 pass (CPContr^(n) of P and Q,
// Section 6.1; Theorem "CP block multiplicative update"; Xhat never stored).  A CTA owns a
// tile of 128 rows j, a block of 128 columns k and a range of slabs i, walked as a sequence
// of 64-column chunks (two per slab).  Warps are specialised: warp 4 CG + 1 streams X
// chunks into a shared-memory ring by TMA (and PF chunks further ahead into L2 by bulk
// prefetch); warp 4 CG issues every MMA, in chunk order; warps 0..4 CG - 1 are the epilogue,
// thread (warp w, lane l) owning tile row 32 (w % 4) + l (its TMEM lane), the column group
// w / 4 (64 / CG columns) of each chunk and the rank slice w / 4 (32 / CG ranks) of the
// row-side constants and folds.  The epilogue warps signal per warp, on mbarriers, when an
// X stage, an X-hat buffer, a P tile or the next slab's R operand is free / ready; the only
// block-wide wait is one named barrier per slab.
//
// Per chunk n (slab i, columns k0 + 64 q):
//   TMA       X chunk (128 x 64 FP32) into a 2- or 3-stage ring, issued that far ahead;
//   GEMM1     Xhat = R C^T on TF32 operands rounded to nearest, M128 N64 K32, into one of
//             two TMEM buffers, issued one chunk ahead; with S3 the operands are split into
//             hi / lo TF32 parts and GEMM1 is hi*lo + lo*hi + hi*hi (about FP32 accuracy);
//   epilogue  Xhat from TMEM (tcgen05.ld), X from shared memory, P = X Y^(beta-2),
//             Q = Y^(beta-1) (Y = max(Xhat, eps)) and the objective terms in FP32
//             registers; P, Q stored once as BF16 tiles [rows][64 cols];
//   GEMM2     rows: W[j][r] += sum_k P[j][k] Cn[k][r]   (A = P K-major, B = Cn^T)
//             cols: N3^T[r][k] += sum_j KRn^T[r][j] P[j][k]  (A = KRn^T with the rank
//             padded to M = 128, B = the same P tile read MN-major),
//             BF16 operands, FP32 accumulation in TMEM, overlapping the next epilogue.
// W and KRn^T are double-buffered per slab: during the second chunk of slab i, mode 1
// reduces sum_j W[j][r] Bn[j][r] of slab i - 1 over each warp's 32 rows (shuffle
// reduce-scatter; one partial per 32-row quarter, summed in fixed order later) and mode 2
// accumulates An[i-1][r] W[j][r] per row, while the contractions of slab i proceed.  Every wait on an mbarrier is bounded;
// a wait that runs out raises a shared abort flag that ends the other waits at once; the
// kernel then sets the context's status word, waits (bounded) for its copies and MMAs,
// frees its TMEM and returns.
//
// With RX (explicit rows: the Tucker passes of Appendix C), the GEMM1 rows of slab i are
// rrow[i*J + j] (the mode-3 partial tensor B^(3) of eq. (block_Bn)) instead of A_i (.) B_j,
// the column contraction's operand is nrow[i*J + j] (and drow) instead of A_i (.) B_j, and
// the rows contraction W[j][r] of each slab is written out ([column block][I*J][RP]
// partials, summed over the column blocks afterwards) instead of being folded into modes
// 1 and 2.  Row values are loaded from global memory two chunks before they are staged.
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
constexpr int CG = 4;      // column groups per chunk (epilogue warps = 4 CG)
constexpr int CW = CH / CG;  // columns per epilogue thread and chunk
constexpr int RS = RP / CG;  // ranks per epilogue thread in the row-side work
constexpr int EW = 128 * CG;  // epilogue threads
constexpr int NT = EW + 64;   // + the MMA issuer warp + the TMA producer warp
constexpr int PF = 6;         // X chunks prefetched into L2 ahead of the shared-memory ring
static_assert(CW % 8 == 0 && RS % 4 == 0 && 32 % CW == 0, "column groups");

struct Layout {
    int x, p, q, r, rl, c, cl, cnt, cdt, knt, kdt, misc, total;
    int ns;  // X stages
    int np;  // P / Q buffers
    int nk;  // KRn^T / KRd^T buffers (2: slab i + 1's is written while slab i's is read)
};

// 1024-aligned regions.  The column contraction reads KRn^T as an M = 128 operand whose
// rows 32..127 are padding: those rows only feed accumulator rows that are never read, so
// only the 32 real rows are stored (two 4 KB K-atoms per buffer) and the padding reads fall
// on the 16 KB that follow (the Crec / R tiles), which stay inside the allocation.
// kb: columns per CTA block; the C tile is kb x 32 TF32 (128 bytes a column) and the
// contraction's C^T operand 32 x kb BF16
__host__ __device__ constexpr int layout_bytes(bool rows, bool m3, bool den, bool s3, int ns, int np, int nk, int kb) {
    return ns * 32768 + np * 16384 * (den ? 2 : 1) + (s3 ? 2 : 1) * kb * 128 + (s3 ? 2 : 1) * 16384 +
           (rows ? kb * 64 : 0) + ((rows && den) ? kb * 64 : 0) + (m3 ? nk * 8192 : 0) + ((m3 && den) ? nk * 8192 : 0) +
           4096 + 1024;
}

__host__ __device__ constexpr Layout make_layout(bool rows, bool m3, bool den, bool s3, int kb) {
    Layout L{};
    constexpr int kMax = 232448;  // opt-in shared memory per CTA
    L.ns = 2;
    L.np = 1;
    L.nk = 1;
    if (layout_bytes(rows, m3, den, s3, 2, 2, 1, kb) <= kMax) L.np = 2;
    if (layout_bytes(rows, m3, den, s3, 2, L.np, 2, kb) <= kMax) L.nk = 2;
    if (layout_bytes(rows, m3, den, s3, 3, L.np, L.nk, kb) <= kMax) L.ns = 3;
    int o = 0;
    L.x = o; o += L.ns * 32768;
    L.p = o; o += L.np * 16384;
    L.q = o; o += den ? L.np * 16384 : 0;
    L.knt = o; o += m3 ? L.nk * 8192 : 0;            // padding rows read the C tiles below
    L.c = o; o += kb * 128;
    L.cl = o; o += s3 ? kb * 128 : 0;
    L.kdt = o; o += (m3 && den) ? L.nk * 8192 : 0;   // padding rows read the R tiles below
    L.r = o; o += 16384;
    L.rl = o; o += s3 ? 16384 : 0;
    L.cnt = o; o += rows ? kb * 64 : 0;
    L.cdt = o; o += (rows && den) ? kb * 64 : 0;
    L.misc = o; o += 4096;
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
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t addr, float *v) {
    if (N == 32) tmem_ld32(addr, v);
    else if (N == 16) tmem_ld16(addr, v);
    else tmem_ld8(addr, v);
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

constexpr int WAIT_LIMIT = 1 << 26;  // polls (seconds at worst) before a wait gives up

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

template <int MS, int BK, bool S3, bool RX, int KB>
__global__ void __launch_bounds__(NT, 1) cp3_pass_tc(const __grid_constant__ CUtensorMap xmap, const Cp3Args a) {
    constexpr bool DEN = BK != BK_KL;
    constexpr bool M1 = (MS & PM_M1) != 0, M2 = (MS & PM_M2) != 0, M3 = (MS & PM_M3) != 0;
    constexpr bool OBJ = (MS & PM_OBJ) != 0, RW = M1 || M2;
    constexpr int CPS = KB / CH;  // chunks per slab
    static_assert(KB == 128 || (KB == 256 && !DEN && !S3 && !RX), "256-column blocks: KL, single TF32");
    constexpr Layout L = make_layout(RW, M3, DEN, S3, KB);
    constexpr int NP = L.np, NS = L.ns, NK = L.nk;
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
    // mbarriers, per ring slot s = chunk % NS: chunk_ready (X stage landed and X-hat computed:
    // the TMA bytes plus the GEMM1 commit), inputs_free (every epilogue warp has read the X
    // stage and the X-hat buffer); per P buffer: p_full, g2_done (its contractions complete);
    // r_full (R holds the next slab)
    uint64_t *bars = (uint64_t *)(sm + L.misc);
    uint64_t *chunk_ready = bars, *inputs_free = bars + 4, *p_full = bars + 8, *g2_done = bars + 10;
    uint64_t *r_full = bars + 12;
    constexpr int NBAR = 13;
    uint32_t *tslot = (uint32_t *)(sm + L.misc + 128);
    volatile int *abort_flag = (volatile int *)(sm + L.misc + 136);
    double *dred = (double *)(sm + L.misc + 192 + 1024);  // [EW / 32]
    float *srow = (float *)(sm + L.misc + 2048);          // [4 slabs][rec0, num0, den0][32]

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const bool issuer = warp == EW / 32, producer = warp == EW / 32 + 1, epi = warp < EW / 32;
    const int quarter = warp & 3, cg = warp >> 2;
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
    const bool jv = epi && j < J;
    const int NC = CPS * (i1 - i0);
    const int r0 = RS * cg;

    auto wait = [&](uint64_t *bar, uint32_t phase) -> bool {
        const uint32_t ba = su32(bar);
        for (int it = 0; it < WAIT_LIMIT; ++it) {
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
    auto epi_sync = [&]() { asm volatile("bar.sync 1, %0;\n" :: "n"(EW) : "memory"); };

    // ---- per-CTA constants (epilogue threads) ----------------------------------------------
    float brec[RS], bn[RS], bd[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        brec[r] = (jv && !RX) ? __ldg(a.rec[1] + (int64_t)j * RP + r0 + r) : 0.0f;
        bn[r] = (jv && M1 && !RX) ? __ldg(a.num[1] + (int64_t)j * RP + r0 + r) : 0.0f;
        bd[r] = (jv && M1 && DEN && !RX) ? __ldg(a.den[1] + (int64_t)j * RP + r0 + r) : 0.0f;
    }
    // KRn^T / KRd^T side (mode 3): epilogue thread t owns rank t % 32 and the eight tile rows
    // 8 (t / 32) .. 8 (t / 32) + 7, so that a slab's KR tile is one 16-byte store per thread
    const int kr_r = t & 31, kr_j = 8 * (t >> 5);
    float bk[8], bkd[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const bool v = M3 && !RX && epi && j0 + kr_j + e < J;
        bk[e] = v ? __ldg(a.num[1] + (int64_t)(j0 + kr_j + e) * RP + kr_r) : 0.0f;
        bkd[e] = (v && DEN) ? __ldg(a.den[1] + (int64_t)(j0 + kr_j + e) * RP + kr_r) : 0.0f;
    }
    if (epi) {
#pragma unroll 1
        for (int cc = row; cc < KB; cc += ROWS) {  // block column cc
            const int kc = k0 + cc;
            const bool kv = kc < K;
#pragma unroll
            for (int q = 0; q < RS / 4; ++q) {
                float h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float v = kv ? __ldg(a.rec[2] + (int64_t)kc * RP + r0 + 4 * q + e) : 0.0f;
                    h[e] = tf32_rna(v);
                    l[e] = S3 ? tf32_rna(v - h[e]) : 0.0f;
                }
                *reinterpret_cast<float4 *>(Cs + swf(cc, r0 + 4 * q)) = make_float4(h[0], h[1], h[2], h[3]);
                if (S3) *reinterpret_cast<float4 *>(Cl + swf(cc, r0 + 4 * q)) = make_float4(l[0], l[1], l[2], l[3]);
            }
            if (RW) {
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    const int rr = r0 + r;
                    CnT[(cc >> 6) * 2048 + swh(rr, cc & 63)] =
                        __float2bfloat16_rn(kv ? __ldg(a.num[2] + (int64_t)kc * RP + rr) : 0.0f);
                    if (DEN)
                        CdT[(cc >> 6) * 2048 + swh(rr, cc & 63)] =
                            __float2bfloat16_rn(kv ? __ldg(a.den[2] + (int64_t)kc * RP + rr) : 0.0f);
                }
            }
        }
    }
    // Factor rows of slab i for R / KR / folds, in a ring of 4: slot (i + 2) % 4 is written at
    // the start of slab i, after the barrier there, and its previous slab (i - 2) was last
    // read by the fold during slab i - 1, before every warp reached that barrier; the first
    // reader of slab i + 2 (R during slab i + 1) comes after the barrier of slab i + 1.
    // Slabs i0 .. i0 + 2 are staged before the loop; at the start of slab i (after its
    // barrier) threads 0..95 store slab i + 2 from a register loaded a slab earlier.
    auto row_val = [&](int i) -> float {  // thread t < 96: entry t of slab i's staged rows
        const int f = t >> 5, r = t & 31;
        const float *src = f == 0 ? a.rec[0] : f == 1 ? a.num[0] : a.den[0];
        return (f == 2 && !DEN) ? 0.0f : __ldg(src + (int64_t)i * RP + r);
    };
    auto stage_rows = [&](int i) {
        if (t < 96 && !RX) srow[(i & 3) * 96 + t] = row_val(i);
    };
    // RX: this thread's entries of the next slabs' explicit rows, loaded ahead
    float rx[RS], kx[8], kxd[8];
    auto rx_load = [&](int i) {  // GEMM1 rows of slab i: row `row`, rank slice r0
#pragma unroll
        for (int q = 0; q < RS / 4; ++q) {
            const float4 v = jv ? __ldg(reinterpret_cast<const float4 *>(a.rrow + ((int64_t)i * J + j) * RP + r0) + q)
                                : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            rx[4 * q] = v.x; rx[4 * q + 1] = v.y; rx[4 * q + 2] = v.z; rx[4 * q + 3] = v.w;
        }
    };
    auto kx_load = [&](int i) {  // column-contraction rows of slab i: rank kr_r, rows kr_j ..
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const bool v = epi && j0 + kr_j + e < J;
            const int64_t o = ((int64_t)i * J + j0 + kr_j + e) * RP + kr_r;
            kx[e] = v ? __ldg(a.nrow + o) : 0.0f;
            kxd[e] = (v && DEN) ? __ldg(a.drow + o) : 0.0f;
        }
    };
    auto slab_rows = [&](int i) {  // R (hi/lo) of slab i: row `row`, rank slice r0
        const float *ar = srow + (i & 3) * 96 + r0;
#pragma unroll
        for (int q = 0; q < RS / 4; ++q) {
            float h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float v = RX ? rx[4 * q + e] : ar[4 * q + e] * brec[4 * q + e];
                h[e] = tf32_rna(v);
                l[e] = S3 ? tf32_rna(v - h[e]) : 0.0f;
            }
            *reinterpret_cast<float4 *>(Rs + swf(row, r0 + 4 * q)) = make_float4(h[0], h[1], h[2], h[3]);
            if (S3) *reinterpret_cast<float4 *>(Rl + swf(row, r0 + 4 * q)) = make_float4(l[0], l[1], l[2], l[3]);
        }
    };
    auto pack8 = [](const float *v, float s) {  // eight BF16 values s * v[e] as one uint4
        __nv_bfloat162 h0 = __floats2bfloat162_rn(s * v[0], s * v[1]), h1 = __floats2bfloat162_rn(s * v[2], s * v[3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(s * v[4], s * v[5]), h3 = __floats2bfloat162_rn(s * v[6], s * v[7]);
        uint4 u;
        u.x = *reinterpret_cast<uint32_t *>(&h0); u.y = *reinterpret_cast<uint32_t *>(&h1);
        u.z = *reinterpret_cast<uint32_t *>(&h2); u.w = *reinterpret_cast<uint32_t *>(&h3);
        return u;
    };
    auto slab_kr = [&](int i) {  // KRn^T / KRd^T of slab i: row kr_r, columns kr_j .. kr_j + 7
        const float *an = srow + (i & 3) * 96 + 32;
        const int off = (kr_j >> 6) * 2048 + swh(kr_r, kr_j & 63);
        *reinterpret_cast<uint4 *>(KnT + ((i - i0) % NK) * 4096 + off) = RX ? pack8(kx, 1.0f) : pack8(bk, an[kr_r]);
        if (DEN)
            *reinterpret_cast<uint4 *>(KdT + ((i - i0) % NK) * 4096 + off) = RX ? pack8(kxd, 1.0f) : pack8(bkd, an[32 + kr_r]);
    };
    if (t == EW) {
        for (int q = 0; q < NBAR; ++q) {
            const uint32_t cnt = q < 4 ? 2 : q < 10 || q == 12 ? EW / 32 : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(su32(bars + q)), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        *abort_flag = 0;
    }
    float rnext = 0.0f;  // slab i0 + 3's staged-row entry (threads t < 96)
    if (NC > 0) {
        for (int i = i0; i < i0 + 3 && i < i1; ++i) stage_rows(i);
        if (t < 96 && i0 + 3 < i1 && !RX) rnext = row_val(i0 + 3);
    }
    __syncthreads();
    if (issuer) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" :: "r"(su32(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    } else if (epi && NC > 0) {
        if (RX) rx_load(i0);
        slab_rows(i0);
        if (RX && i0 + 1 < i1) rx_load(i0 + 1);
        if (M3) {
            if (RX) kx_load(i0);
            slab_kr(i0);
            if (RX && i0 + 1 < i1) kx_load(i0 + 1);
        }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    // TMEM columns: X-hat [2][64] | W, Wd of even / odd slabs [2][32 + 32] | N3 [128] | N3d [128]
    const uint32_t t_d1 = tmem, t_w = tmem + 128, t_wd = tmem + 160, t_n3 = tmem + 256, t_n3d = tmem + 384;

    float acc2[RS], acc2d[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) acc2[r] = acc2d[r] = 0.0f;
    double obj_acc = 0.0;

    if (producer) {
        // ---- producer warp: X chunks into the shared-memory ring, PF chunks ahead into L2 ----
        if (lane == 0 && NC > 0) {
            auto prefetch_x = [&](int n) {
                const int i = i0 + n / CPS, x = k0 + CH * (n % CPS);
                // only boxes that start inside the tensor (a ragged block's last chunk may not)
                if (x < K) tma_prefetch_2d(&xmap, x, i * J + j0);
                if (x + 32 < K) tma_prefetch_2d(&xmap, x + 32, i * J + j0);
            };
            for (int c = NS; c < NS + PF && c < NC; ++c) prefetch_x(c);
            int xs = 0;        // ring slot of chunk n
            uint32_t xph = 0;  // parity of its phase, (n / NS) & 1
            for (int n = 0; n < NC; ++n) {
                // chunk n - NS used this slot with the other parity
                if (n >= NS && !wait(inputs_free + xs, xph ^ 1)) break;
                const int i = i0 + n / CPS, q = n % CPS;
                const uint32_t bar = su32(chunk_ready + xs);
                const uint32_t dst = su32(Xs) + xs * 32768;
                expect_tx(bar, 32768);
                tma_2d(&xmap, dst, bar, k0 + CH * q, i * J + j0);
                tma_2d(&xmap, dst + 16384, bar, k0 + CH * q + 32, i * J + j0);
                if (n >= NS && n + PF < NC) prefetch_x(n + PF);
                if (++xs == NS) {
                    xs = 0;
                    xph ^= 1;
                }
            }
        }
        __syncwarp();
    } else if (issuer) {
        // ---- issuer warp: GEMM1 and the contractions, in chunk order ----------------------
        if (lane == 0 && NC > 0) {
            auto issue_g1 = [&](int n) {
                const int q = n % CPS;
                const uint32_t d = t_d1 + 64 * (n & 1);
                const uint32_t id = idesc_tf32(CH);
                const uint32_t cb = su32(Cs) + q * 8192, cbl = su32(Cl) + q * 8192;
                if (S3) {
#pragma unroll
                    for (int s = 0; s < 4; ++s) mma_tf32(d, sdesc(su32(Rl) + s * 32), sdesc(cb + s * 32), id, s > 0);
#pragma unroll
                    for (int s = 0; s < 4; ++s) mma_tf32(d, sdesc(su32(Rs) + s * 32), sdesc(cbl + s * 32), id, 1);
                }
#pragma unroll
                for (int s = 0; s < 4; ++s) mma_tf32(d, sdesc(su32(Rs) + s * 32), sdesc(cb + s * 32), id, S3 || s > 0);
                mma_commit(su32(chunk_ready + n % NS));
            };
            auto issue_g2 = [&](int n) {
                const int q = n % CPS, sb = (n / CPS) & 1;
                const uint32_t kn = su32(KnT) + ((n / CPS) % NK) * 8192, kd = su32(KdT) + ((n / CPS) % NK) * 8192;
                const uint32_t pb = su32(Ps) + (n % NP) * 16384, qb = su32(Qs) + (n % NP) * 16384;
                if (RW) {
                    const uint32_t id = idesc_bf16(RP, false);
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint32_t acc = (q > 0 || s > 0) ? 1u : 0u;
                        mma_bf16(t_w + 64 * sb, sdesc(pb + s * 32), sdesc(su32(CnT) + q * 4096 + s * 32), id, acc);
                        if (DEN) mma_bf16(t_wd + 64 * sb, sdesc(qb + s * 32), sdesc(su32(CdT) + q * 4096 + s * 32), id, acc);
                    }
                }
                if (M3) {
                    const uint32_t id = idesc_bf16(CH, true);
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        const uint32_t ao = (s >> 2) * 4096 + (s & 3) * 32;
                        const uint32_t acc = (n >= CPS || s > 0) ? 1u : 0u;
                        mma_bf16(t_n3 + 64 * q, sdesc(kn + ao), sdesc(pb + s * 2048, 16384, 1024), id, acc);
                        if (DEN) mma_bf16(t_n3d + 64 * q, sdesc(kd + ao), sdesc(qb + s * 2048, 16384, 1024), id, acc);
                    }
                }
                mma_commit(su32(g2_done + (n % NP)));
            };
            fence_after();
            issue_g1(0);
            for (int n = 0; n < NC && !*abort_flag; ++n) {
                const int m = n + 1;
                if (m < NC) {
                    bool ok = true;
                    // X-hat buffer m & 1 was last read by chunk m - 2
                    if (m >= 2) ok = wait(inputs_free + (m - 2) % NS, ((m - 2) / NS) & 1);
                    if (ok && m % CPS == 0) ok = wait(r_full, (m / CPS - 1) & 1);
                    if (!ok) break;
                    fence_after();
                    issue_g1(m);
                }
                if (!wait(p_full + (n % NP), (n / NP) & 1)) break;
                fence_after();
                issue_g2(n);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps ---------------------------------------------------------------
        auto fold = [&](int i) {  // modes 1 and 2 from W of slab i (its contractions complete)
            const uint32_t wb = 64 * ((i - i0) & 1);
            float w[RS], wd[RS];
#pragma unroll
            for (int r = 0; r < RS; ++r) w[r] = wd[r] = 0.0f;
            if (!__any_sync(0xffffffffu, *abort_flag != 0)) {  // warp-uniform before tcgen05.ld
                tmem_ld<RS>(t_w + wb + lane_off + r0, w);
                if (DEN) tmem_ld<RS>(t_wd + wb + lane_off + r0, wd);
            }
            if (RX) {  // W rows of slab i for this column block: [kb][i * J + j][RP] partials
                if (jv && !*abort_flag) {
                    const int64_t o = (((int64_t)kb * a.I + i) * J + j) * RP + r0;
#pragma unroll
                    for (int q = 0; q < RS / 4; ++q) {
                        reinterpret_cast<float4 *>(a.p1n + o)[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
                        if (DEN)
                            reinterpret_cast<float4 *>(a.p1d + o)[q] =
                                make_float4(wd[4 * q], wd[4 * q + 1], wd[4 * q + 2], wd[4 * q + 3]);
                    }
                }
                return;
            }
            if (M2) {
                const float *an = srow + (i & 3) * 96 + 32 + r0, *ad = an + 32;
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    acc2[r] = fmaf(an[r], w[r], acc2[r]);
                    if (DEN) acc2d[r] = fmaf(ad[r], wd[r], acc2d[r]);
                }
            }
            if (M1) {
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    w[r] *= bn[r];
                    if (DEN) wd[r] *= bd[r];
                }
                // one partial per warp (its 32 rows of the tile), summed later in fixed order
                const float sr = reduce_scatter<RS>(w);
                const float sd = DEN ? reduce_scatter<RS>(wd) : 0.0f;
                if (lane < RS && !*abort_flag) {
                    const int64_t slot = (((int64_t)(jt * a.n_kb + kb) * 4 + quarter) * a.I + i) * RP + r0 + lane;
                    a.p1n[slot] = sr;
                    if (DEN) a.p1d[slot] = sd;
                }
            }
        };
        // shared-memory offsets of this thread's X and P / Q entries within a stage / tile
        int xo[CW / 4], po[CW / 8];
#pragma unroll
        for (int g = 0; g < CW / 4; ++g) xo[g] = ((CW * cg) >> 5) * 4096 + swf(row, ((CW * cg) & 31) + 4 * g);
#pragma unroll
        for (int g = 0; g < CW / 8; ++g) po[g] = swh(row, CW * cg + 8 * g);
        int xs = 0;        // ring slot of chunk n
        uint32_t xph = 0;  // parity of its phase, (n / NS) & 1
        for (int n = 0; n < NC; ++n) {
            const int i = i0 + n / CPS, q = n % CPS;
            const int pb = n % NP;
            if (n >= NP) wait(g2_done + pb, ((n - NP) / NP) & 1);  // P tile pb free again
            if (q == 0 && n > 0) {
                // slab boundary: rows of slab i + 2 staged; KRn^T of slab i written into the
                // buffer last read by the contractions of slab i - NK, which are complete (the
                // wait above covers chunk n - 1 or n - 2, and MMAs complete in order)
                if (M3 && NK == 1 && NP == 2) {
                    wait(g2_done + ((n - 1) % NP), ((n - 1) / NP) & 1);
                }
                fence_after();
                epi_sync();  // rows of slab i + 1 (stored at the previous boundary) visible
                if (t < 96 && i + 2 < i1) {
                    if (!RX) srow[((i + 2) & 3) * 96 + t] = rnext;
                    if (i + 3 < i1 && !RX) rnext = row_val(i + 3);
                }
                if (M3) {
                    slab_kr(i);
                    if (RX && i + 1 < i1) kx_load(i + 1);
                }
            }
            if (RW && q == 1 && n > CPS) {
                // fold slab i - 1: its last contraction (chunk n - 2) is complete, as the
                // P-tile wait above covers chunk n - NP >= n - 2; W of slab i - 1 is rewritten
                // by slab i + 1, whose contractions start only after this chunk's P tile
                fence_after();
                fold(i - 1);
                fence_before();
            }
            const bool ready = __all_sync(0xffffffffu, wait(chunk_ready + xs, xph));
            fence_after();
            float xh[CW], xv[CW];
            if (ready) {  // warp-uniform before tcgen05.ld
                tmem_ld<CW>(t_d1 + 64 * (n & 1) + lane_off + CW * cg, xh);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c) xh[c] = 0.0f;
            }
            {
                // the X stage holds two 128 x 32 halves; this group's columns lie in one
                const float *xa = Xs + xs * 8192;
#pragma unroll
                for (int g = 0; g < CW / 4; ++g) {
                    const float4 v = *reinterpret_cast<const float4 *>(xa + xo[g]);
                    xv[4 * g] = v.x; xv[4 * g + 1] = v.y; xv[4 * g + 2] = v.z; xv[4 * g + 3] = v.w;
                }
            }
            fence_before();
            arrive(inputs_free + xs);
            if (++xs == NS) {
                xs = 0;
                xph ^= 1;
            }
            if (q == CPS - 1 && n + 1 < NC) {
                // this chunk's GEMM1 is complete, so R can take slab i + 1 (needed by GEMM1 of
                // the next chunk, which the issuer starts once every warp has arrived)
                slab_rows(i + 1);
                if (RX && i + 2 < i1) rx_load(i + 2);
                fence_async_smem();
                arrive(r_full);
            }
            __nv_bfloat16 *pa = Ps + pb * 8192;
            __nv_bfloat16 *qa = Qs + pb * 8192;
            const int kc = k0 + CH * q + CW * cg;
            float o1 = 0.0f, o2 = 0.0f;
            float2 u1 = make_float2(0.0f, 0.0f), u2 = make_float2(0.0f, 0.0f);  // packed KL sums
            // full strip of a valid row: no per-entry masks
            auto body = [&](auto full_tag) {
                constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
                for (int g = 0; g < CW / 8; ++g) {
                    float pv[8], qv[8];
                    if (FULL && BK == BK_KL) {
                        // the KL point function on pairs of entries
#pragma unroll
                        for (int c = 0; c < 8; c += 2) {
                            const float2 x2 = make_float2(xv[8 * g + c], xv[8 * g + c + 1]);
                            const float2 y2 = make_float2(fmaxf(xh[8 * g + c], a.eps), fmaxf(xh[8 * g + c + 1], a.eps));
                            const float2 P2 = mul2(x2, make_float2(mufu_rcp(y2.x), mufu_rcp(y2.y)));
                            pv[c] = P2.x;
                            pv[c + 1] = P2.y;
                            if (OBJ) {
                                const float2 l2 = make_float2(mufu_lg2(fmaxf(P2.x, 1e-30f)), mufu_lg2(fmaxf(P2.y, 1e-30f)));
                                u1 = fma2(x2, l2, u1);
                                u2 = add2(u2, sub2(y2, x2));
                            }
                        }
                    } else
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float x = xv[8 * g + c];
                        if (BK == BK_IS) x = fmaxf(x, a.eps_x);
                        const float y = fmaxf(xh[8 * g + c], a.eps);
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
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(pv[0], pv[1]), h1 = __floats2bfloat162_rn(pv[2], pv[3]);
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(pv[4], pv[5]), h3 = __floats2bfloat162_rn(pv[6], pv[7]);
                    uint4 u;
                    u.x = *reinterpret_cast<uint32_t *>(&h0); u.y = *reinterpret_cast<uint32_t *>(&h1);
                    u.z = *reinterpret_cast<uint32_t *>(&h2); u.w = *reinterpret_cast<uint32_t *>(&h3);
                    *reinterpret_cast<uint4 *>(pa + po[g]) = u;
                    if (DEN) {
                        h0 = __floats2bfloat162_rn(qv[0], qv[1]); h1 = __floats2bfloat162_rn(qv[2], qv[3]);
                        h2 = __floats2bfloat162_rn(qv[4], qv[5]); h3 = __floats2bfloat162_rn(qv[6], qv[7]);
                        u.x = *reinterpret_cast<uint32_t *>(&h0); u.y = *reinterpret_cast<uint32_t *>(&h1);
                        u.z = *reinterpret_cast<uint32_t *>(&h2); u.w = *reinterpret_cast<uint32_t *>(&h3);
                        *reinterpret_cast<uint4 *>(qa + po[g]) = u;
                    }
                }
            };
            if (jv && kc + CW <= K) body(std::true_type{});
            else body(std::false_type{});
            if (BK == BK_KL) {
                o1 += u1.x + u1.y;
                o2 += u2.x + u2.y;
            }
            const float objf = OBJ ? obj_combine<BK>(a.beta, o1, o2) : 0.0f;
            if (OBJ) obj_acc += (double)objf;
            fence_async_smem();
            arrive(p_full + pb);
        }
        if (NC > 0) {
            wait(g2_done + (NC - 1) % NP, ((NC - 1) / NP) & 1);
            fence_after();
            if (RW) fold(i1 - 1);
        }
        // ---- CTA outputs ------------------------------------------------------------------
        const bool good = !__any_sync(0xffffffffu, *abort_flag != 0);
        if (M2 && jv && !RX) {
            const int64_t base = ((int64_t)(kb * a.n_is + is) * J + j) * RP + r0;
#pragma unroll
            for (int r = 0; r < RS; ++r) {
                a.p2n[base + r] = acc2[r];
                if (DEN) a.p2d[base + r] = acc2d[r];
            }
        }
        if (M3 && quarter == 0) {
            const int64_t base = (int64_t)(jt * a.n_is + is) * K;
#pragma unroll 1
            for (int g = 0; g < KB / (32 * CG); ++g) {
                float v[32], vd[32];
                const bool have = good && NC > 0;
                const int cb = (KB / CG) * cg + 32 * g;
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
            epi_sync();
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
        for (int q = 0; q < NBAR; ++q) {
            for (int ph = 0; ph < 2; ++ph) {
                for (int it = 0; it < (1 << 20); ++it) {
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

template <int MS, int BK, bool S3, bool RX, int KB = KBLK>
cudaError_t launch_t(const Cp3Plan &p, const Cp3Args &a, cudaStream_t s) {
    constexpr Layout L = make_layout((MS & (PM_M1 | PM_M2)) != 0, (MS & PM_M3) != 0, BK != BK_KL, S3, KB);
    CUtensorMap map;
    cudaError_t e = launch_x_map(a, &map);
    if (e != cudaSuccess) return e;
    auto k = cp3_pass_tc<MS, BK, S3, RX, KB>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    k<<<p.grid, NT, L.total, s>>>(map, a);
    return cudaGetLastError();
}

template <int BK, bool S3>
cudaError_t launch_bk(const Cp3Plan &p, const Cp3Args &a, int ms, cudaStream_t s) {
    if (a.rrow) {  // explicit rows (Tucker): W rows out, or the column contraction
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
            if (BK == BK_KL) return launch_t<PM_M1 | PM_M2 | PM_M3 | PM_OBJ, BK_KL, S3, false>(p, a, s);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
}  // namespace ntf
