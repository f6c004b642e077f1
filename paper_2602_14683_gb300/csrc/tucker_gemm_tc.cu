// The small contractions of the Tucker updates on the 5th-generation tensor cores (tcgen05).
//
// The partial tensor B^(3) = G x_1 A^(1) x_2 A^(2) (eq. (block_Bn)), the core contractions of
// eq. (block_core_num_den) and the factor contractions of eqs. (block_factor_num/den) are all
// strided batched products C[bt] = sum_k A(bt, m, k) B(bt, k, n) (the Gemm of ntf_tucker.h).
// Here one CTA of four warps computes a 128 x NTT tile of one batch over one reduction range:
//   * per chunk of 32 reduction indices, the threads gather the A and B tiles with plain loads
//     (any strides), round them to TF32 (and, for 3xTF32, the remainders too) and store them into
//     128-byte-swizzled K-major tiles (one 128-byte row per m or n) of a two-stage ring in shared
//     memory.  An operand whose rows are contiguous (unit m or n stride) is read with consecutive
//     lanes on consecutive rows, any other with consecutive lanes on consecutive reduction
//     indices (on 32-column tiles, four consecutive indices per lane with 16-byte loads and
//     shared stores when the layout is aligned for it), so that a warp's load touches as few
//     lines as the layout allows; the loads of chunk c + 1 are issued into registers before
//     chunk c's MMAs;
//   * thread 0 issues the chunk's tcgen05.mma.kind::tf32 (M 128, N NTT, K 8 four times; with the
//     split hi*hi + hi*lo + lo*hi) into one TMEM accumulator and commits to the stage's mbarrier,
//     which the threads wait on before they refill that stage two chunks later;
//   * after the last chunk each warp reads its 32 TMEM lanes (rows), transposes them through
//     shared memory and stores whole rows (consecutive lanes on consecutive columns); with a
//     second index folded into the rows (C's rows contiguous, its columns not) each thread stores
//     its own row instead.
// Every wait is bounded; a wait that runs out sets the context's status word, and the kernel then
// writes nothing, waits (bounded) for its MMAs and frees its TMEM.
#include "cp3_tc.cuh"
#include "ntf_tucker.h"

namespace ntf {
namespace tgemm {

using tc::fence_after;
using tc::fence_async_smem;
using tc::fence_before;
using tc::idesc_tf32;
using tc::mbar_wait;
using tc::mma_commit;
using tc::mma_tf32;
using tc::sdesc;
using tc::su32;
using tc::swf;
using tc::tf32_rna;
using tc::tmem_ld32;

constexpr int NTH = 128;
constexpr int KC = 32;  // reduction indices per chunk: one 128-byte TF32 row of each tile

template <int NTT, bool S3>
struct Geo {
    static constexpr int ABYTES = 128 * KC * 4;  // 16 KB
    static constexpr int BBYTES = NTT * KC * 4;  // NTT rows of 128 bytes
    static constexpr int STAGE = (ABYTES + BBYTES) * (S3 ? 2 : 1);
    static constexpr int SMEM = 2 * STAGE + 64 + 1024;  // + barriers, TMEM slot, flags; + alignment slack
};

// One operand tile (NR rows x 32 reduction indices k0 .. k0 + 31) of a chunk: element (row r,
// index kk) = base[r srow + k1 sk1 + k2 sk2] with k0 + kk = k1 K2 + k2, zero outside rows < nrow or
// indices < kend.  Each thread holds NR / 4 elements: with unit row stride (rowmode) thread t takes
// row t % NR (consecutive lanes, consecutive rows) and a run of consecutive indices; otherwise its
// lane is the index and the warps take rows in turn (mode 0), or (mode 2) each group of eight
// lanes takes one row, four consecutive indices per lane.  load_tile issues the global loads into
// registers (a chunk ahead of its use), store_tile rounds them to TF32 and writes the swizzled
// K-major tiles hi (and lo).
template <int NR>
struct TileMap {
    static constexpr int TPR = NR >= NTH ? 1 : NTH / NR;  // rowmode: threads per row
    static constexpr int RK = KC / TPR;                  // rowmode: indices per thread and row
    static constexpr int RPT = NR >= NTH ? NR / NTH : 1;  // rowmode: rows per thread
    static constexpr int PER = NR / 4;                   // elements per thread (both modes)
};

// Offset of tile row r (global row row0 + r): (row / nin) sblk + (row % nin) srow when the batch
// is folded into the rows (nin > 0), else row srow.
__device__ __forceinline__ int64_t row_off(int row, int64_t srow, int nin, int64_t sblk) {
    if (nin > 0) {
        const int b = row / nin;
        return (int64_t)b * sblk + (int64_t)(row - b * nin) * srow;
    }
    return (int64_t)row * srow;
}

template <int NR, bool V>
__device__ __forceinline__ void load_tile(float (&v)[NR / 4], int mode, const float *base, int row0, int64_t srow,
                                          int nin, int64_t sblk, int64_t sk1, int64_t sk2, int K2, int k0, int kend,
                                          int nrow, int t) {
    using T = TileMap<NR>;
    if (V && mode == 2) {  // eight lanes per row, four consecutive indices each, four rows per warp load
        const int lane = t & 31, warp = t >> 5;
        const int k = k0 + 4 * (lane & 7);
        const bool kv = k < kend;
        const int64_t ko = kv ? (K2 == 1 ? (int64_t)k * sk1 : (int64_t)(k / K2) * sk1 + (int64_t)(k % K2) * sk2) : 0;
#pragma unroll
        for (int s = 0; s < NR / 16; ++s) {
            const int r = 16 * s + 4 * warp + (lane >> 3);
            float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (kv && r < nrow) x = __ldg(reinterpret_cast<const float4 *>(base + row_off(row0 + r, srow, nin, sblk) + ko));
            v[4 * s] = x.x;
            v[4 * s + 1] = x.y;
            v[4 * s + 2] = x.z;
            v[4 * s + 3] = x.w;
        }
        return;
    }
    const bool rowmode = mode == 1;
    if (rowmode) {
#pragma unroll
        for (int p = 0; p < T::RPT; ++p) {
            const int r = NR >= NTH ? t + NTH * p : t % NR;
            const int kk0 = NR >= NTH ? 0 : (t / NR) * T::RK;
            int k = k0 + kk0, k1 = K2 == 1 ? k : k / K2, k2 = k - k1 * K2;
            const bool rv = r < nrow;
            const float *br = base + (rv ? row_off(row0 + r, srow, nin, sblk) : 0);
#pragma unroll
            for (int q = 0; q < T::RK; ++q) {
                v[p * T::RK + q] = (rv && k + q < kend) ? __ldg(br + (int64_t)k1 * sk1 + (int64_t)k2 * sk2) : 0.0f;
                if (++k2 == K2) {
                    k2 = 0;
                    ++k1;
                }
            }
        }
    } else {
        const int lane = t & 31, warp = t >> 5;
        const int k = k0 + lane;
        const bool kv = k < kend;
        int k1 = 0, k2 = 0;
        if (kv) {
            k1 = K2 == 1 ? k : k / K2;
            k2 = k - k1 * K2;
        }
        const float *p = base + (int64_t)k1 * sk1 + (int64_t)k2 * sk2;
#pragma unroll
        for (int i = 0; i < T::PER; ++i) {
            const int r = 4 * i + warp;
            v[i] = (kv && r < nrow) ? __ldg(p + row_off(row0 + r, srow, nin, sblk)) : 0.0f;
        }
    }
}

template <int NR, bool S3, bool V>
__device__ __forceinline__ void store_tile(const float (&v)[NR / 4], int mode, float *hi, float *lo, int t) {
    using T = TileMap<NR>;
    if (V && mode == 2) {
        const int lane = t & 31, warp = t >> 5;
        const int kk = 4 * (lane & 7);
#pragma unroll
        for (int s = 0; s < NR / 16; ++s) {
            const int r = 16 * s + 4 * warp + (lane >> 3);
            float h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                h[e] = tf32_rna(v[4 * s + e]);
                l[e] = S3 ? tf32_rna(v[4 * s + e] - h[e]) : 0.0f;
            }
            *reinterpret_cast<float4 *>(hi + swf(r, kk)) = make_float4(h[0], h[1], h[2], h[3]);
            if (S3) *reinterpret_cast<float4 *>(lo + swf(r, kk)) = make_float4(l[0], l[1], l[2], l[3]);
        }
        return;
    }
    const bool rowmode = mode == 1;
    if (rowmode) {
#pragma unroll
        for (int p = 0; p < T::RPT; ++p) {
            const int r = NR >= NTH ? t + NTH * p : t % NR;
            const int kk0 = NR >= NTH ? 0 : (t / NR) * T::RK;
#pragma unroll
            for (int q = 0; q < T::RK; ++q) {
                const float x = v[p * T::RK + q], h = tf32_rna(x);
                hi[swf(r, kk0 + q)] = h;
                if (S3) lo[swf(r, kk0 + q)] = tf32_rna(x - h);
            }
        }
    } else {
        const int lane = t & 31, warp = t >> 5;
#pragma unroll
        for (int i = 0; i < T::PER; ++i) {
            const int r = 4 * i + warp;
            const float x = v[i], h = tf32_rna(x);
            hi[swf(r, lane)] = h;
            if (S3) lo[swf(r, lane)] = tf32_rna(x - h);
        }
    }
}

// RF: rows folded (g.mfold > 0) in A and C; each thread then stores its own row of C (or, over
// several reduction ranges, of the transposed partials [range][n][m]), so that a warp's store of
// one column covers 32 consecutive rows.
template <int NTT, bool S3, bool V, bool RF>
__global__ void __launch_bounds__(NTH, 1) gemm_tc_kernel(const Gemm g) {
    using G = Geo<NTT, S3>;
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * G::STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    int *last_issued = abort_flag + 1;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int n0 = blockIdx.x * NTT, m0 = blockIdx.y * 128;
    const int bt = blockIdx.z % g.batch, sp = blockIdx.z / g.batch;
    const int K = g.K1 * g.K2;
    const int kbeg = sp * g.kchunks * KC, kend = min(K, kbeg + g.kchunks * KC);
    const int nch = kend > kbeg ? (kend - kbeg + KC - 1) / KC : 0;

    if (t == 0) {
        for (int q = 0; q < 2; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(su32(bars + q)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        *abort_flag = 0;
        *last_issued = -1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(su32(tslot)), "n"(NTT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t id = idesc_tf32(NTT);
    const int64_t abase = (int64_t)bt * g.sab, bbase = (int64_t)bt * g.sbb;

    const float *Abase = g.A + abase, *Bbase = g.B + bbase;
    // operand modes: rows contiguous (1); else one index per lane (0), or with V (the launcher has
    // checked the alignment) runs of four indices per lane (2)
    const int arow = g.sam == 1 ? 1 : V ? 2 : 0;
    const int brow = g.sbn == 1 ? 1 : V ? 2 : 0;
    float va[32], vb[NTT / 4];  // the next chunk's operands, loaded a chunk ahead
    if (nch > 0) {
        load_tile<128, V>(va, arow, Abase, m0, g.sam, RF ? g.mfold : 0, g.samb, g.sak1, g.sak2, g.K2, kbeg, kend, g.M - m0, t);
        load_tile<NTT, V>(vb, brow, Bbase, n0, g.sbn, g.nin, g.sbb, g.sbk1, g.sbk2, g.K2, kbeg, kend, g.N - n0, t);
    }
    for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        uint8_t *st = sm + s * G::STAGE;
        float *Ah = reinterpret_cast<float *>(st), *Bh = reinterpret_cast<float *>(st + G::ABYTES);
        float *Al = reinterpret_cast<float *>(st + G::ABYTES + G::BBYTES);
        float *Bl = reinterpret_cast<float *>(st + 2 * G::ABYTES + G::BBYTES);
        // the MMAs of chunk c - 2 read this stage
        if (c >= 2 && !mbar_wait(su32(bars + s), ((c - 2) >> 1) & 1)) *abort_flag = 1;
        store_tile<128, S3, V>(va, arow, Ah, Al, t);
        store_tile<NTT, S3, V>(vb, brow, Bh, Bl, t);
        if (c + 1 < nch) {  // in flight while this chunk is handed to the tensor cores
            const int k0 = kbeg + (c + 1) * KC;
            load_tile<128, V>(va, arow, Abase, m0, g.sam, RF ? g.mfold : 0, g.samb, g.sak1, g.sak2, g.K2, k0, kend, g.M - m0, t);
            load_tile<NTT, V>(vb, brow, Bbase, n0, g.sbn, g.nin, g.sbb, g.sbk1, g.sbk2, g.K2, k0, kend, g.N - n0, t);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (*abort_flag) break;  // uniform: read after the barrier
        if (t == 0) {
            fence_after();
            const uint64_t da = sdesc(su32(Ah)), db = sdesc(su32(Bh));
            if (S3) {
                const uint64_t dal = sdesc(su32(Al)), dbl = sdesc(su32(Bl));
#pragma unroll
                for (int q = 0; q < 4; ++q) mma_tf32(tmem, dal + 2 * q, db + 2 * q, id, (c > 0 || q > 0) ? 1u : 0u);
#pragma unroll
                for (int q = 0; q < 4; ++q) mma_tf32(tmem, da + 2 * q, dbl + 2 * q, id, 1u);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) mma_tf32(tmem, da + 2 * q, db + 2 * q, id, (S3 || c > 0 || q > 0) ? 1u : 0u);
            mma_commit(su32(bars + s));
            *last_issued = c;
        }
    }
    __syncthreads();
    // the last chunk's commit covers every MMA issued before it
    const int li = *last_issued;
    if (li >= 0 && !*abort_flag && !mbar_wait(su32(bars + (li & 1)), (li >> 1) & 1)) *abort_flag = 1;
    __syncthreads();
    fence_after();
    const bool aborted = *abort_flag != 0;
    if (RF && !aborted) {
        // each thread stores its own row (TMEM lane): C's row m (scm = 1 within a fold block), or
        // row m of the range's transposed partial [n][m]
        const int m = m0 + 32 * warp + lane;
        const bool part = g.splits > 1;
        float *base = part ? g.part + ((int64_t)sp * g.batch + bt) * g.M * g.N : g.C;
        const int64_t ro = part ? (int64_t)m : (int64_t)bt * g.scb + row_off(m, 1, g.mfold, g.scmb);
        const int64_t cs = part ? (int64_t)g.M : g.scn;
#pragma unroll 1
        for (int j = 0; j < NTT / 32; ++j) {
            float v[32];
            if (li >= 0) {
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * j, v);
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.0f;  // empty reduction range
            }
            if (m < g.M) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int n = n0 + 32 * j + q;
                    if (n < g.N) base[ro + (int64_t)n * cs] = v[q];
                }
            }
        }
    } else if (!aborted) {
        // warp w holds TMEM lanes 32 w .. 32 w + 31 (rows m0 + 32 w + lane); each 32-column block
        // goes through a 32 x 33 staging tile of the warp's own (the operand ring is free now), and
        // the warp then stores its rows one at a time, lane = column
        float *stg = reinterpret_cast<float *>(sm) + warp * 32 * 33;
        const int64_t sn = g.splits > 1 ? 1 : g.scn;
#pragma unroll 1
        for (int j = 0; j < NTT / 32; ++j) {
            float v[32];
            if (li >= 0) {
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * j, v);
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.0f;  // empty reduction range
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) stg[lane * 33 + q] = v[q];
            __syncwarp();
            const int n = n0 + 32 * j + lane;
            if (n < g.N) {
                // this lane's column: its offset in C (batch block and column when folded); the
                // warp's rows then follow at a fixed stride
                const int mw = m0 + 32 * warp, mcnt = min(32, g.M - mw);
                float *dst = g.splits > 1 ? g.part + (((int64_t)sp * g.batch + bt) * g.M + mw) * g.N + n
                                          : g.C + (int64_t)bt * g.scb + (int64_t)mw * g.scm + row_off(n, sn, g.nin, g.scb);
                const int64_t rstep = g.splits > 1 ? (int64_t)g.N : g.scm;
#pragma unroll 4
                for (int i = 0; i < mcnt; ++i, dst += rstep) *dst = stg[i * 33 + lane];
            }
            __syncwarp();
        }
    } else if (t == 0) {
        if (g.err) atomicExch(g.err, 1);
        if (li >= 0) {  // bounded wait for the MMAs still in flight before the TMEM is freed
            for (int it = 0; it < (1 << 20); ++it) {
                uint32_t done;
                asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                             : "=r"(done) : "r"(su32(bars + (li & 1))), "r"((li >> 1) & 1) : "memory");
                if (done) break;
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "n"(NTT));
    }
}

template <int NTT, bool S3, bool V = false, bool RF = false>
cudaError_t launch_t(const Gemm &g, cudaStream_t s) {
    using G = Geo<NTT, S3>;
    auto k = gemm_tc_kernel<NTT, S3, V, RF>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((g.N + NTT - 1) / NTT), (unsigned)((g.M + 127) / 128), (unsigned)(g.batch * g.splits));
    k<<<grid, NTH, G::SMEM, s>>>(g);
    return cudaGetLastError();
}

// Runs of four reduction indices per lane (16-byte loads and shared stores) for an operand whose
// rows are not contiguous: the runs, the row, batch and fold offsets and the base all 16-byte
// aligned, K % 4 == 0 (a run is then either inside the range or past its end).  Operands with
// contiguous rows keep their own mapping.
static bool vec_ok(const float *p, int64_t sbat, int64_t srow, int nin, int64_t sblk, int64_t sk1, int64_t sk2,
                   int K2, int K) {
    if (srow == 1) return true;
    const bool runs = (K2 == 1 && sk1 == 1) || (sk2 == 1 && K2 % 4 == 0 && sk1 % 4 == 0);
    return runs && K % 4 == 0 && srow % 4 == 0 && sbat % 4 == 0 && (nin == 0 || sblk % 4 == 0) &&
           (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

}  // namespace tgemm

cudaError_t gemm_tc_launch(const Gemm &g, bool s3, int ntt, cudaStream_t s) {
    if (g.M < 1 || g.N < 1 || g.batch < 1 || g.splits < 1 || g.kchunks < 1) return cudaErrorInvalidValue;
    const int K = g.K1 * g.K2;
    if (g.mfold > 0) {  // rows folded: 32-column tiles, C's rows contiguous within a fold block
        if (ntt != 32 || g.scm != 1 || g.nin != 0) return cudaErrorInvalidValue;
        return s3 ? tgemm::launch_t<32, true, false, true>(g, s) : tgemm::launch_t<32, false, false, true>(g, s);
    }
    // the 16-byte form only for 32-column tiles (the long-reduction factor contractions): in the
    // wider tiles its extra registers cost a resident CTA per SM
    const bool v = ntt == 32 && (g.sam != 1 || g.sbn != 1) &&
                   tgemm::vec_ok(g.A, g.sab, g.sam, g.mfold, g.samb, g.sak1, g.sak2, g.K2, K) &&
                   tgemm::vec_ok(g.B, g.sbb, g.sbn, g.nin, g.sbb, g.sbk1, g.sbk2, g.K2, K);
    if (v) return s3 ? tgemm::launch_t<32, true, true>(g, s) : tgemm::launch_t<32, false, true>(g, s);
    switch (ntt) {
        case 32: return s3 ? tgemm::launch_t<32, true>(g, s) : tgemm::launch_t<32, false>(g, s);
        case 64: return s3 ? tgemm::launch_t<64, true>(g, s) : tgemm::launch_t<64, false>(g, s);
        case 128: return s3 ? tgemm::launch_t<128, true>(g, s) : tgemm::launch_t<128, false>(g, s);
        case 256: return s3 ? tgemm::launch_t<256, true>(g, s) : tgemm::launch_t<256, false>(g, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntf
