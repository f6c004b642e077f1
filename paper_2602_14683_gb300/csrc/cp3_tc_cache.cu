// Contraction-only tensor-core pass of J-CoMM's inner block updates over cached reference-
// powered tensors (Section 5.3, "Reference-powered tensors": P~ = X (.) X~^(beta-2) and
// Q~ = X~^(beta-1) are fixed during the inner loop; Algorithm 2).
//
// The first pass of an outer iteration (the tensor-core pass with the cache outputs set)
// stores the BF16 P~ / Q~ tiles that its contractions consume, by TMA, as [I][J][kp] tensors.
// Every later block pass of the outer iteration runs this kernel instead: P~ and Q~ tiles come
// from HBM by TMA straight into the shared-memory operand buffers (128-byte swizzle, the layout
// the epilogue writes), and only the contractions remain -- no X stream, no reconstruction
// GEMM, no powers.  The contractions (the column contraction on chunk pairs, N = 128) and the
// partial-sum layouts are those of the recomputing pass with the same plan, so the results are
// the same bit for bit.  Bytes per pass: 2 + 2 per tensor entry (the recomputing pass reads 4
// of X).
//
// Warps: 17 (producer, one thread) loads the P~ / Q~ chunk pairs into a ring of NPC buffers;
// 16 (issuer, one thread; owns TMEM) issues the contractions; 18, 19 (builders) write
// KRn^T / KRd^T of every slab; 0..15 fold W of every slab into modes 1 and 2 (8 ranks per
// thread, its TMEM lane quadrant) and write the mode-3 partials at the end.
#include "cp3_tc.cuh"

namespace ntf {
namespace tc {

constexpr int NPC = 4;  // P~ / Q~ chunk buffers

struct CLayout {
    int p, q, cnt, cdt, knt, kdt, misc, total;
};

__host__ __device__ constexpr CLayout make_clayout(bool rows, bool m3, int kb) {
    CLayout L{};
    int o = 0;
    // KR^T first: the M = 128 operand's padding rows read the 16 KB that follow each K-atom
    L.knt = o; o += m3 ? 2 * 8192 : 0;
    L.kdt = o; o += m3 ? 2 * 8192 : 0;
    L.p = o; o += NPC * 16384;
    L.q = o; o += NPC * 16384;
    L.cnt = o; o += rows ? kb * 64 : 0;
    L.cdt = o; o += rows ? kb * 64 : 0;
    L.misc = o; o += 512;
    L.total = o + 1024;
    return L;
}

template <int MS, int KB>
__global__ void __launch_bounds__(NT, 1) cp3_contract_tc(const __grid_constant__ CUtensorMap pmap,
                                                          const __grid_constant__ CUtensorMap qmap, const Cp3Args a) {
    constexpr bool M1 = (MS & PM_M1) != 0, M2 = (MS & PM_M2) != 0, M3 = (MS & PM_M3) != 0, RW = M1 || M2;
    constexpr int CPS = KB / CH;
    constexpr int NK = 2;
    constexpr CLayout L = make_clayout(RW, M3, KB);
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16 *Ps = (__nv_bfloat16 *)(sm + L.p);
    __nv_bfloat16 *Qs = (__nv_bfloat16 *)(sm + L.q);
    __nv_bfloat16 *CnT = (__nv_bfloat16 *)(sm + L.cnt);
    __nv_bfloat16 *CdT = (__nv_bfloat16 *)(sm + L.cdt);
    __nv_bfloat16 *KnT = (__nv_bfloat16 *)(sm + L.knt);
    __nv_bfloat16 *KdT = (__nv_bfloat16 *)(sm + L.kdt);
    // mbarriers: per chunk buffer p_full (the TMA bytes), g2_done (its contractions complete);
    // per KR buffer k_full (both builder warps), k_free (the slab's last contraction complete);
    // per W buffer w_ready (the slab's last contraction complete), w_free (the 16 fold warps);
    // all_done (every contraction complete)
    uint64_t *bars = (uint64_t *)(sm + L.misc);
    uint64_t *p_full = bars, *g2_done = bars + 4, *k_full = bars + 8, *k_free = bars + 10;
    uint64_t *w_ready = bars + 12, *w_free = bars + 14, *all_done = bars + 16;
    constexpr int NBAR = 17;
    uint32_t *tslot = (uint32_t *)(sm + L.misc + 192);
    volatile int *abort_flag = (volatile int *)(sm + L.misc + 200);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const bool issuer = warp == EW / 32, producer = warp == EW / 32 + 1, builder = warp >= EW / 32 + 2;
    const bool epi = warp < EW / 32;
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
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
    const int NSL = i1 - i0;
    const int NC = CPS * NSL;
    const int rf = 8 * (warp >> 2);  // this thread's 8 ranks of the folds

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
    auto arrive = [&](uint64_t *bar) {
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(su32(bar)) : "memory");
    };

    float bn[8], bd[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        bn[r] = (jv && M1) ? __ldg(a.num[1] + (int64_t)j * RP + rf + r) : 0.0f;
        bd[r] = (jv && M1) ? __ldg(a.den[1] + (int64_t)j * RP + rf + r) : 0.0f;
    }
    if (epi && RW) {
        // Cn^T / Cd^T (rows contraction B operand), as in the recomputing pass
#pragma unroll 1
        for (int cc = row; cc < KB; cc += ROWS) {
            const int kc = k0 + cc;
            const bool kv = kc < K;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int rr = rf + r;
                CnT[(cc >> 6) * 2048 + swh(rr, cc & 63)] = __float2bfloat16_rn(kv ? __ldg(a.num[2] + (int64_t)kc * RP + rr) : 0.0f);
                CdT[(cc >> 6) * 2048 + swh(rr, cc & 63)] = __float2bfloat16_rn(kv ? __ldg(a.den[2] + (int64_t)kc * RP + rr) : 0.0f);
            }
        }
    }
    if (t == EW) {
        for (int q = 0; q < NBAR; ++q) {
            const uint32_t cnt = q < 8 ? 1 : q < 10 ? 2 : q < 14 ? 1 : q < 16 ? EW / 32 : 1;
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
    // TMEM columns: W, Wd of even / odd slabs at 128 + [2][32 + 32] | N3 [KB] | N3d [128]
    const uint32_t t_w = tmem + 128, t_wd = tmem + 160, t_n3 = tmem + 256, t_n3d = tmem + 384;

    if (producer) {
        if (lane == 0 && NC > 0) {
            for (int n = 0; n < NC; ++n) {
                const int pb = n % NPC, i = i0 + n / CPS, q = n % CPS;
                // the buffer's previous chunk has been contracted (waited in chunk order)
                if (n >= NPC && !wait(g2_done + pb, ((n - NPC) / NPC) & 1)) break;
                if (*abort_flag) break;
                const uint32_t bar = su32(p_full + pb);
                expect_tx(bar, 2 * 16384);
                tma_3d(&pmap, su32(Ps) + pb * 16384, bar, k0 + CH * q, j0, i);
                tma_3d(&qmap, su32(Qs) + pb * 16384, bar, k0 + CH * q, j0, i);
            }
        }
        __syncwarp();
    } else if (issuer) {
        if (lane == 0 && NC > 0) {
            const uint32_t idr = idesc_bf16(RP, false), idc = idesc_bf16(2 * CH, true);
            const uint64_t dP = sdesc(su32(Ps)), dQ = sdesc(su32(Qs)), dCn = sdesc(su32(CnT)), dCd = sdesc(su32(CdT));
            const uint64_t dPm = sdesc(su32(Ps), 16384, 1024), dQm = sdesc(su32(Qs), 16384, 1024);
            const uint64_t dKn = sdesc(su32(KnT)), dKd = sdesc(su32(KdT));
            for (int n = 0; n < NC; ++n) {
                const int s = n / CPS, q = n % CPS, pb = n % NPC;
                if (!wait(p_full + pb, (n / NPC) & 1)) break;
                if (M3 && q == 0 && !wait(k_full + s % NK, (s / NK) & 1)) break;
                // W of slab s - 2 (the same TMEM buffer) has been folded
                if (RW && q == 0 && s >= 2 && !wait(w_free + (s & 1), ((s - 2) >> 1) & 1)) break;
                if (*abort_flag) break;
                fence_after();
                const uint32_t po = (uint32_t)pb * 1024u;
                if (RW) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t acc = (q > 0 || k > 0) ? 1u : 0u;
                        mma_bf16(t_w + 64 * (s & 1), dP + po + 2 * k, dCn + q * 256 + 2 * k, idr, acc);
                        mma_bf16(t_wd + 64 * (s & 1), dQ + po + 2 * k, dCd + q * 256 + 2 * k, idr, acc);
                    }
                }
                if (M3 && (n & 1)) {
                    // chunks n - 1, n: their P tiles are adjacent buffers, one N = 128 operand
                    const uint32_t ko = (uint32_t)(s % NK) * 512u, pp = po - 1024u;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t ao = ko + (k >> 2) * 256 + (k & 3) * 2;
                        const uint32_t acc = (s > 0 || k > 0) ? 1u : 0u;
                        mma_bf16(t_n3 + 64 * (q - 1), dKn + ao, dPm + pp + k * 128, idc, acc);
                        mma_bf16(t_n3d + 64 * (q - 1), dKd + ao, dQm + pp + k * 128, idc, acc);
                    }
                    mma_commit(su32(g2_done + (n - 1) % NPC));
                }
                if (!M3 || (n & 1)) mma_commit(su32(g2_done + pb));
                if (q == CPS - 1) {
                    if (M3) mma_commit(su32(k_free + s % NK));
                    if (RW) mma_commit(su32(w_ready + (s & 1)));
                }
            }
            mma_commit(su32(all_done));
        }
        __syncwarp();
    } else if (builder) {
        if (M3) {
            // KRn^T / KRd^T of every slab (thread bt owns tile rows 2 bt, 2 bt + 1), as in the
            // recomputing pass
            const int bt = t - (EW + 64), jr0 = 2 * bt;
            const bool v0 = j0 + jr0 < J, v1 = j0 + jr0 + 1 < J;
            for (int s = 0; s < NSL; ++s) {
                const int i = i0 + s;
                if (s >= NK && !wait(k_free + s % NK, ((s - NK) / NK) & 1)) break;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        const float *f0 = f ? a.den[0] : a.num[0], *f1 = f ? a.den[1] : a.num[1];
                        const float4 *pa = reinterpret_cast<const float4 *>(f0 + (int64_t)i * RP + 16 * h);
                        const float4 *pb = reinterpret_cast<const float4 *>(f1 + (int64_t)(j0 + jr0) * RP + 16 * h);
                        float4 av[4], x0[4], x1[4];
                        const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            av[q] = __ldg(pa + q);
                            x0[q] = v0 ? __ldg(pb + q) : z4;
                            x1[q] = v1 ? __ldg(pb + RP / 4 + q) : z4;
                        }
                        __nv_bfloat16 *base = (f ? KdT : KnT) + (s % NK) * 4096 + (jr0 >> 6) * 2048;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float a4[4] = {av[q].x, av[q].y, av[q].z, av[q].w};
                            const float b0[4] = {x0[q].x, x0[q].y, x0[q].z, x0[q].w}, b1[4] = {x1[q].x, x1[q].y, x1[q].z, x1[q].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                *reinterpret_cast<__nv_bfloat162 *>(base + swh(16 * h + 4 * q + e, jr0 & 63)) =
                                    __floats2bfloat162_rn(a4[e] * b0[e], a4[e] * b1[e]);
                        }
                    }
                }
                fence_async_smem();
                arrive(k_full + s % NK);
            }
        }
    } else {
        // ---- fold warps ---------------------------------------------------------------------
        float acc2[8], acc2d[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) acc2[r] = acc2d[r] = 0.0f;
        if (RW) {
            for (int s = 0; s < NSL; ++s) {
                const int i = i0 + s;
                float an[8], ad[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    an[r] = M2 ? __ldg(a.num[0] + (int64_t)i * RP + rf + r) : 0.0f;
                    ad[r] = M2 ? __ldg(a.den[0] + (int64_t)i * RP + rf + r) : 0.0f;
                }
                const bool ok = __all_sync(0xffffffffu, wait(w_ready + (s & 1), (s >> 1) & 1));
                fence_after();
                float w[8], wd[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) w[r] = wd[r] = 0.0f;
                if (ok) {
                    tmem_ld8(t_w + 64 * (s & 1) + lane_off + rf, w);
                    tmem_ld8(t_wd + 64 * (s & 1) + lane_off + rf, wd);
                }
                fence_before();
                arrive(w_free + (s & 1));
                if (M2) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        acc2[r] = fmaf(an[r], w[r], acc2[r]);
                        acc2d[r] = fmaf(ad[r], wd[r], acc2d[r]);
                    }
                }
                if (M1) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        w[r] *= bn[r];
                        wd[r] *= bd[r];
                    }
                    const float sr = reduce_scatter<8>(w);
                    const float sd = reduce_scatter<8>(wd);
                    if (lane < 8 && !*abort_flag) {
                        const int64_t slot = (((int64_t)(jt * a.n_kb + kb) * 4 + quarter) * a.I + i) * RP + rf + lane;
                        a.p1n[slot] = sr;
                        a.p1d[slot] = sd;
                    }
                }
            }
        }
        if (NC > 0) wait(all_done, 0);
        fence_after();
        const bool good = !__any_sync(0xffffffffu, *abort_flag != 0);
        if (M2 && jv) {
            const int64_t base = ((int64_t)(kb * a.n_is + is) * J + j) * RP + rf;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                a.p2n[base + r] = acc2[r];
                a.p2d[base + r] = acc2d[r];
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
                    tmem_ld32(t_n3d + cb, vd);
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int kc = k0 + cb + c;
                    if (kc < K) {
                        a.p3n[(base + kc) * RP + lane] = have ? v[c] : 0.0f;
                        a.p3d[(base + kc) * RP + lane] = have ? vd[c] : 0.0f;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (*abort_flag && t == EW) {
        const int clim = wlim < (1 << 20) ? wlim : (1 << 20);
        for (int q = 0; q < NBAR; ++q)
            for (int ph = 0; ph < 2; ++ph)
                for (int it = 0; it < clim; ++it) {
                    uint32_t done;
                    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                                 : "=r"(done) : "r"(su32(bars + q)), "r"(ph) : "memory");
                    if (done) break;
                }
        if (a.err) atomicExch(a.err, 1);
    }
    __syncthreads();
    if (issuer) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" :: "r"(tmem));
    }
}

template <int MS>
static cudaError_t launch_c(const Cp3Plan &p, const Cp3Args &a, cudaStream_t s) {
    constexpr CLayout L = make_clayout((MS & (PM_M1 | PM_M2)) != 0, (MS & PM_M3) != 0, KBLK);
    CUtensorMap pm, qm;
    cudaError_t e = cache_map(a.pc, a, &pm);
    if (e == cudaSuccess) e = cache_map(a.qc, a, &qm);
    if (e != cudaSuccess) return e;
    auto k = cp3_contract_tc<MS, KBLK>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    k<<<p.grid, NT, L.total, s>>>(pm, qm, a);
    return cudaGetLastError();
}

}  // namespace tc

cudaError_t cp3_tc_contract_launch(const Cp3Plan &p, const Cp3Args &a, int ms, cudaStream_t s) {
    if (!p.tc || p.RP != 32 || p.KB != tc::KBLK || !a.pc || !a.qc || a.kp % 8 != 0) return cudaErrorInvalidValue;
    switch (ms) {
        case PM_M1: return tc::launch_c<PM_M1>(p, a, s);
        case PM_M2: return tc::launch_c<PM_M2>(p, a, s);
        case PM_M3: return tc::launch_c<PM_M3>(p, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntf
