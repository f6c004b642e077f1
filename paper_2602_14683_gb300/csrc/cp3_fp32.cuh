// Fused dense 3-way CP pass on CUDA cores (FP32 FMA), the parity path.
//
// One CTA (256 threads) owns a row tile of TJ = 64 rows j in [j0, j0+TJ), a column block of
// KB = 64 columns k in [k0, k0+KB) and a slab range i in [i0, i1).  For each i it walks
// the column block in chunks of KC = 32 columns:
//   GEMM1  Xhat[j][k] = sum_r Arec[i][r] Brec[j][r] Crec[k][r]        (reduction over R)
//   powers P = X * max(Xhat,eps)^(beta-2), Q = max(Xhat,eps)^(beta-1)  (registers)
//   rows   W[j][r]   += sum_k P[j][k] Cn[k][r]   (feeds modes 1 and 2; reduction over k)
//   cols   N3[k][r]  += sum_j P[j][k] An[i][r] Bn[j][r]                  (mode 3)
// then, at the end of each i, mode 1 reduces sum_j W[j][r] Bn[j][r] into a partial row
// for i and mode 2 accumulates An[i][r] W[j][r] per j.  The same with Q and the
// denominator factors when DEN.  This is CPContr^(n) of Section 6.1 applied to P and Q
// (Theorem "CP block multiplicative update", Algorithm 1) with Xhat never stored.
// Partial sums go to per-CTA slots and are reduced in a fixed order by the epilogue, so
// results are deterministic.  Xhat tiles come from GEMM1 on the fly; X tiles are
// double-buffered in shared memory with cp.async.
#pragma once

#include "ntf_internal.h"

namespace ntf {
namespace fp32 {

constexpr int NT = 256;
constexpr int KC = 32;
constexpr int KB = 64;
constexpr int NCH = KB / KC;
constexpr int XS = KC + 4;

// Tiles of 64 rows: at RP <= 32 the shared-memory layout then stays under 100 KB and two CTAs
// (16 warps) share an SM, which the latency-bound loops below need more than the longer register
// tiles that 128-row tiles allow
template <int RP>
struct Geo {
    static constexpr int TJ = 64;
    static constexpr int MINB = (RP == 64) ? 1 : 2;  // resident CTAs per SM the launch bounds ask for
    static constexpr int RW = TJ / 32;  // rows per thread in GEMM1 / rows-GEMM2
    static constexpr int RG = RP / 8;   // rank columns per thread in the GEMM2s
    static constexpr int TS = TJ / 4;   // rows per slice in the cols-GEMM2
    static constexpr int RS = RP + 4;   // padded stride of [row][r] buffers
    static constexpr int TT = TJ + 4;   // padded stride of [r][row] buffers
};

struct Layout {
    int xs, ps, qs, rrT, brT, bn, bd, krn, krd, crT, cn, cd, red, end;
};

template <int RP, bool DEN, int MS>
__host__ __device__ constexpr Layout layout() {
    using G = Geo<RP>;
    Layout L{};
    int o = 0;
    L.xs = o; o += 2 * G::TJ * XS;
    L.ps = o; o += G::TJ * XS;
    L.qs = o; o += DEN ? G::TJ * XS : 0;
    L.rrT = o; o += RP * G::TT;
    L.brT = o; o += RP * G::TT;
    L.bn = o; o += (MS & (PM_M1 | PM_M3)) ? G::TJ * G::RS : 0;
    L.bd = o; o += ((MS & (PM_M1 | PM_M3)) && DEN) ? G::TJ * G::RS : 0;
    L.krn = o; o += (MS & PM_M3) ? G::TJ * G::RS : 0;
    L.krd = o; o += ((MS & PM_M3) && DEN) ? G::TJ * G::RS : 0;
    L.crT = o; o += NCH * RP * KC;
    L.cn = o; o += (MS & (PM_M1 | PM_M2)) ? KB * G::RS : 0;
    L.cd = o; o += ((MS & (PM_M1 | PM_M2)) && DEN) ? KB * G::RS : 0;
    L.red = o; o += 2 * 8 * RP + 2 * 8 * 2;  // mode-1 reduction + 8 doubles
    L.end = o;
    return L;
}

template <int N>
struct VecLd;
template <>
struct VecLd<1> {
    __device__ static void ld(const float *p, float *v) { v[0] = p[0]; }
};
template <>
struct VecLd<2> {
    __device__ static void ld(const float *p, float *v) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
};
template <>
struct VecLd<4> {
    __device__ static void ld(const float *p, float *v) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <>
struct VecLd<8> {
    __device__ static void ld(const float *p, float *v) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        float4 u = *reinterpret_cast<const float4 *>(p + 4);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        v[4] = u.x; v[5] = u.y; v[6] = u.z; v[7] = u.w;
    }
};

__device__ __forceinline__ void cp_async16(float *dst, const float *src, int src_bytes) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Stage the X tile for slab i, column chunk starting at kc into xs (TJ x KC, stride XS).
// Rows j >= J and columns k >= K are zero-filled.
template <int TJ>
__device__ __forceinline__ void load_x_tile(const Cp3Args &a, float *xs, int i, int j0, int kc) {
    const int tid = threadIdx.x;
    const int64_t rowbase = (int64_t)i * a.J;
    if (a.vec16) {
        constexpr int SEG = KC / 4;  // 16-byte segments per row
        for (int s = tid; s < TJ * SEG; s += NT) {
            int row = s / SEG, seg = s % SEG;
            int j = j0 + row, k = kc + seg * 4;
            int bytes = 0;
            const float *src = a.X;
            if (j < a.J && k < a.K) {
                int n = a.K - k;
                bytes = (n >= 4 ? 4 : n) * 4;
                src = a.X + (rowbase + j) * a.K + k;
            }
            cp_async16(xs + row * XS + seg * 4, src, bytes);
        }
    } else {
        for (int s = tid; s < TJ * KC; s += NT) {
            int row = s / KC, c = s % KC;
            int j = j0 + row, k = kc + c;
            const float *src = a.X;
            int bytes = 0;
            if (j < a.J && k < a.K) {
                bytes = 4;
                src = a.X + (rowbase + j) * a.K + k;
            }
            cp_async4(xs + row * XS + c, src, bytes);
        }
    }
}

// The pass over one CTA's share (work item `blk` of the plan's grid): the kernel below runs
// item blockIdx.x; the batched kernel runs the items of many jobs' plans in one launch.
template <int RP, bool DEN, int MS>
__device__ __forceinline__ void cp3_fp32_body(const Cp3Args &a, const int blk) {
    using G = Geo<RP>;
    constexpr int TJ = G::TJ, RW = G::RW, RG = G::RG, TS = G::TS, RS = G::RS, TT = G::TT;
    constexpr bool M1 = (MS & PM_M1) != 0, M2 = (MS & PM_M2) != 0, M3 = (MS & PM_M3) != 0;
    constexpr bool OBJ = (MS & PM_OBJ) != 0;
    constexpr bool NOX = (MS & PM_NOX) != 0;  // X == 0, not read; denominator side only
    constexpr bool ROWS = M1 || M2;
    constexpr Layout L = layout<RP, DEN, MS>();

    extern __shared__ __align__(16) float sm[];
    float *const xs0 = sm + L.xs;
    float *const ps = sm + L.ps;
    float *const qs = sm + L.qs;
    float *const rrT = sm + L.rrT;
    float *const brT = sm + L.brT;
    float *const bn = sm + L.bn;
    float *const bd = sm + L.bd;
    float *const krn = sm + L.krn;
    float *const krd = sm + L.krd;
    float *const crT = sm + L.crT;
    float *const cn = sm + L.cn;
    float *const cd = sm + L.cd;
    float *const red = sm + L.red;

    const int tid = threadIdx.x;
    const int tr = tid >> 3, tc = tid & 7;
    const int slice = tid >> 6, gc = (tid & 63) >> 3, gr = tid & 7;

    int b = blk;
    const int is = b % a.n_is;
    b /= a.n_is;
    const int kb = b % a.n_kb;
    const int jt = b / a.n_kb;
    const int i0 = (int)((int64_t)is * a.I / a.n_is);
    const int i1 = (int)((int64_t)(is + 1) * a.I / a.n_is);
    const int j0 = jt * TJ, k0 = kb * KB;
    const int J = a.J, K = a.K;

    // ---- per-CTA constants: column-factor chunks and row-factor rows -------------
    for (int t = tid; t < NCH * RP * KC; t += NT) {
        int ch = t / (RP * KC), rem = t % (RP * KC);
        int r = rem / KC, c = rem % KC;
        int k = k0 + ch * KC + c;
        float v = (k < K) ? a.rec[2][(int64_t)k * RP + r] : 0.0f;
        // column c is stored at position (c % 8) * 4 + c / 8 so that thread tc reads
        // columns tc, tc+8, tc+16, tc+24 with one 16-byte load
        crT[(ch * RP + r) * KC + (c & 7) * 4 + (c >> 3)] = v;
    }
    if (ROWS) {
        for (int t = tid; t < KB * RP; t += NT) {
            int kk = t / RP, r = t % RP, k = k0 + kk;
            cn[kk * RS + r] = (k < K) ? a.num[2][(int64_t)k * RP + r] : 0.0f;
            if (DEN) cd[kk * RS + r] = (k < K) ? a.den[2][(int64_t)k * RP + r] : 0.0f;
        }
    }
    for (int t = tid; t < TJ * RP && !a.rrow; t += NT) {
        int row = t / RP, r = t % RP, j = j0 + row;
        brT[r * TT + row] = (j < J) ? a.rec[1][(int64_t)j * RP + r] : 0.0f;
        if (M1 || M3) {
            bn[row * RS + r] = (j < J) ? a.num[1][(int64_t)j * RP + r] : 0.0f;
            if (DEN) bd[row * RS + r] = (j < J) ? a.den[1][(int64_t)j * RP + r] : 0.0f;
        }
    }
    __syncthreads();

    float W[RW][RG], Wd[RW][RG];
    float acc2[RW][RG], acc2d[RW][RG];
    float acc3[NCH][4][RG], acc3d[NCH][4][RG];
#pragma unroll
    for (int x = 0; x < RW; ++x)
#pragma unroll
        for (int q = 0; q < RG; ++q) W[x][q] = Wd[x][q] = acc2[x][q] = acc2d[x][q] = 0.0f;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int q = 0; q < RG; ++q) acc3[ch][c][q] = acc3d[ch][c][q] = 0.0f;
    double obj_acc = 0.0;

    if (!NOX && i0 < i1) load_x_tile<TJ>(a, xs0, i0, j0, k0);
    cp_async_commit();

    int buf = 0;
    for (int i = i0; i < i1; ++i) {
        // per-slab row factors: Rrec[j] = Arec[i] * Brec[j], KRn[j] = An[i] * Bn[j]
        // (Brec, Bn, Bd rows of the tile are resident in shared memory), or explicit rows
        if (a.rrow) {
            const int64_t rb = (int64_t)i * J + j0;
            for (int t = tid; t < TJ * RP; t += NT) {
                int row = t / RP, r = t % RP;
                rrT[r * TT + row] = (j0 + row < J) ? __ldg(a.rrow + (rb + row) * RP + r) : 0.0f;
            }
            if (M3) {
                for (int t = tid; t < TJ * RP; t += NT) {
                    int row = t / RP, r = t % RP;
                    const bool v = j0 + row < J;
                    krn[row * RS + r] = v ? __ldg(a.nrow + (rb + row) * RP + r) : 0.0f;
                    if (DEN) krd[row * RS + r] = v ? __ldg(a.drow + (rb + row) * RP + r) : 0.0f;
                }
            }
        } else {
            for (int t = tid; t < TJ * RP; t += NT) {
                int row = t % TJ, r = t / TJ;
                rrT[r * TT + row] = __ldg(a.rec[0] + (int64_t)i * RP + r) * brT[r * TT + row];
            }
            if (M3) {
                for (int t = tid; t < TJ * RP; t += NT) {
                    int row = t / RP, r = t % RP;
                    krn[row * RS + r] = __ldg(a.num[0] + (int64_t)i * RP + r) * bn[row * RS + r];
                    if (DEN) krd[row * RS + r] = __ldg(a.den[0] + (int64_t)i * RP + r) * bd[row * RS + r];
                }
            }
        }
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            // prefetch the next tile of the (i, chunk) sequence into the other buffer
            {
                int ni = (ch + 1 < NCH) ? i : i + 1;
                int nch = (ch + 1 < NCH) ? ch + 1 : 0;
                if (!NOX && ni < i1) load_x_tile<TJ>(a, xs0 + (buf ^ 1) * TJ * XS, ni, j0, k0 + nch * KC);
                cp_async_commit();
            }
            cp_async_wait<1>();
            __syncthreads();
            const float *xs = xs0 + buf * TJ * XS;
            const int kc = k0 + ch * KC;

            // ---- GEMM1: Xhat micro tile (RW rows x 4 columns) ----------------------
            float xh[RW][4];
#pragma unroll
            for (int x = 0; x < RW; ++x)
#pragma unroll
                for (int c = 0; c < 4; ++c) xh[x][c] = 0.0f;
            const float *crc = crT + ch * RP * KC + tc * 4;
#pragma unroll 8
            for (int r = 0; r < RP; ++r) {
                float ra[RW], cb[4];
                VecLd<RW>::ld(rrT + r * TT + tr * RW, ra);
                VecLd<4>::ld(crc + r * KC, cb);
#pragma unroll
                for (int x = 0; x < RW; ++x)
#pragma unroll
                    for (int c = 0; c < 4; ++c) xh[x][c] = fmaf(ra[x], cb[c], xh[x][c]);
            }

            // ---- powers (and objective terms) in registers --------------------------
            float objf = 0.0f;
#pragma unroll
            for (int x = 0; x < RW; ++x) {
                const int row = tr * RW + x;
                const bool rv = (j0 + row) < J;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int col = tc + 8 * c;
                    const bool v = rv && (kc + col) < K;
                    float xv = NOX ? 0.0f : xs[row * XS + col];
                    if (!NOX && a.bkind == BK_IS) xv = fmaxf(xv, a.eps_x);
                    const float y = fmaxf(xh[x][c], a.eps);
                    float P = 0.0f, Q = 0.0f;
                    if (M1 || M2 || M3) pq_powers(a.bkind, a.beta, xv, y, P, Q);
                    if (!v) { P = 0.0f; Q = 0.0f; }
                    if (OBJ && v) objf += dbeta_stable(a.bkind, a.beta, xv, y);
                    if (M1 || M2 || M3) {
                        if (!NOX) ps[row * XS + col] = P;
                        if (DEN) qs[row * XS + col] = Q;
                    }
                }
            }
            if (OBJ) obj_acc += (double)objf;
            __syncthreads();

            // ---- rows GEMM2: W += P Cn (and Wd += Q Cd) ----------------------------
            if (ROWS) {
                const float *cnc = cn + ch * KC * RS + tc * RG;
                const float *cdc = cd + ch * KC * RS + tc * RG;
#pragma unroll 2
                for (int c4 = 0; c4 < KC / 4; ++c4) {
                    float p[RW][4], qv[RW][4];
#pragma unroll
                    for (int x = 0; x < RW; ++x) {
                        if (!NOX) VecLd<4>::ld(ps + (tr * RW + x) * XS + c4 * 4, p[x]);
                        if (DEN) VecLd<4>::ld(qs + (tr * RW + x) * XS + c4 * 4, qv[x]);
                    }
#pragma unroll
                    for (int cq = 0; cq < 4; ++cq) {
                        float cv[RG], dv[RG];
                        if (!NOX) VecLd<RG>::ld(cnc + (c4 * 4 + cq) * RS, cv);
                        if (DEN) VecLd<RG>::ld(cdc + (c4 * 4 + cq) * RS, dv);
#pragma unroll
                        for (int x = 0; x < RW; ++x)
#pragma unroll
                            for (int q = 0; q < RG; ++q) {
                                if (!NOX) W[x][q] = fmaf(p[x][cq], cv[q], W[x][q]);
                                if (DEN) Wd[x][q] = fmaf(qv[x][cq], dv[q], Wd[x][q]);
                            }
                    }
                }
            }
            // ---- cols GEMM2 (mode 3): N3 += P^T KRn (and Q^T KRd) -------------------
            if (M3) {
#pragma unroll 4
                for (int rr = 0; rr < TS; ++rr) {
                    const int row = slice * TS + rr;
                    float p[4], qv[4], kv[RG], kd[RG];
                    if (!NOX) {
                        VecLd<4>::ld(ps + row * XS + gc * 4, p);
                        VecLd<RG>::ld(krn + row * RS + gr * RG, kv);
                    }
                    if (DEN) {
                        VecLd<4>::ld(qs + row * XS + gc * 4, qv);
                        VecLd<RG>::ld(krd + row * RS + gr * RG, kd);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
#pragma unroll
                        for (int q = 0; q < RG; ++q) {
                            if (!NOX) acc3[ch][c][q] = fmaf(p[c], kv[q], acc3[ch][c][q]);
                            if (DEN) acc3d[ch][c][q] = fmaf(qv[c], kd[q], acc3d[ch][c][q]);
                        }
                }
            }
            __syncthreads();
            buf ^= 1;
        }

        // ---- end of slab i: fold W into the mode-1 and mode-2 accumulators --------
        if (M2) {
            float an[RG], ad[RG];
#pragma unroll
            for (int q = 0; q < RG; ++q) {
                an[q] = NOX ? 0.0f : a.num[0][(int64_t)i * RP + tc * RG + q];
                ad[q] = DEN ? a.den[0][(int64_t)i * RP + tc * RG + q] : 0.0f;
            }
#pragma unroll
            for (int x = 0; x < RW; ++x)
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    if (!NOX) acc2[x][q] = fmaf(an[q], W[x][q], acc2[x][q]);
                    if (DEN) acc2d[x][q] = fmaf(ad[q], Wd[x][q], acc2d[x][q]);
                }
        }
        if (M1) {
            float s[RG], sd[RG];
#pragma unroll
            for (int q = 0; q < RG; ++q) {
                s[q] = 0.0f;
                sd[q] = 0.0f;
#pragma unroll
                for (int x = 0; x < RW; ++x) {
                    if (!NOX) s[q] = fmaf(W[x][q], bn[(tr * RW + x) * RS + tc * RG + q], s[q]);
                    if (DEN) sd[q] = fmaf(Wd[x][q], bd[(tr * RW + x) * RS + tc * RG + q], sd[q]);
                }
                // lanes with the same tc: lane = (tr & 3) * 8 + tc
                if (!NOX) {
                    s[q] += __shfl_xor_sync(0xffffffffu, s[q], 8);
                    s[q] += __shfl_xor_sync(0xffffffffu, s[q], 16);
                }
                if (DEN) {
                    sd[q] += __shfl_xor_sync(0xffffffffu, sd[q], 8);
                    sd[q] += __shfl_xor_sync(0xffffffffu, sd[q], 16);
                }
            }
            const int warp = tid >> 5, lane = tid & 31;
            if (lane < 8) {
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    if (!NOX) red[warp * RP + lane * RG + q] = s[q];
                    if (DEN) red[8 * RP + warp * RP + lane * RG + q] = sd[q];
                }
            }
            __syncthreads();
            if (tid < RP) {
                float t = 0.0f, td = 0.0f;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    if (!NOX) t += red[w * RP + tid];
                    if (DEN) td += red[8 * RP + w * RP + tid];
                }
                const int64_t slot = ((int64_t)(jt * a.n_kb + kb) * a.I + i) * RP + tid;
                if (!NOX) a.p1n[slot] = t;
                if (DEN) a.p1d[slot] = td;
            }
            __syncthreads();
        }
        if (ROWS) {
#pragma unroll
            for (int x = 0; x < RW; ++x)
#pragma unroll
                for (int q = 0; q < RG; ++q) W[x][q] = Wd[x][q] = 0.0f;
        }
    }
    cp_async_wait<0>();

    // ---- CTA outputs ------------------------------------------------------------------
    if (M2) {
        const int64_t base = (int64_t)(kb * a.n_is + is) * J;
#pragma unroll
        for (int x = 0; x < RW; ++x) {
            const int j = j0 + tr * RW + x;
            if (j < J) {
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    if (!NOX) a.p2n[(base + j) * RP + tc * RG + q] = acc2[x][q];
                    if (DEN) a.p2d[(base + j) * RP + tc * RG + q] = acc2d[x][q];
                }
            }
        }
    }
    if (M3) {
        // the four row slices hold partial sums of the same outputs: add them in slice
        // order through shared memory, then store the column block
        float *acc_s = xs0;  // KB x RP floats, fits in the X double buffer
        __syncthreads();
        for (int pass = NOX ? 1 : 0; pass < (DEN ? 2 : 1); ++pass) {
            for (int sl = 0; sl < 4; ++sl) {
                if (slice == sl) {
#pragma unroll
                    for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
                        for (int c = 0; c < 4; ++c)
#pragma unroll
                            for (int q = 0; q < RG; ++q) {
                                const int kk = ch * KC + gc * 4 + c, r = gr * RG + q;
                                const float v = pass == 0 ? acc3[ch][c][q] : acc3d[ch][c][q];
                                if (sl == 0) acc_s[kk * RP + r] = v;
                                else acc_s[kk * RP + r] += v;
                            }
                }
                __syncthreads();
            }
            float *dst = pass == 0 ? a.p3n : a.p3d;
            const int64_t base = (int64_t)(jt * a.n_is + is) * K;
            for (int t = tid; t < KB * RP; t += NT) {
                const int kk = t / RP, r = t % RP, k = k0 + kk;
                if (k < K) dst[(base + k) * RP + r] = acc_s[t];
            }
            __syncthreads();
        }
    }
    if (OBJ) {
        double v = obj_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        double *dred = reinterpret_cast<double *>(red + 2 * 8 * RP);
        __syncthreads();
        if ((tid & 31) == 0) dred[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += dred[w];
            a.obj[blk] = t;
        }
    }
}

template <int RP, bool DEN, int MS>
__global__ void __launch_bounds__(NT, Geo<RP>::MINB) cp3_pass_fp32(const Cp3Args a) {
    cp3_fp32_body<RP, DEN, MS>(a, blockIdx.x);
}

// Many jobs' passes in one launch: a persistent grid walks the items of the work table (job j
// owns items [pfx[j], pfx[j+1]) of its own plan), skipping jobs that have stopped.  Each item
// does exactly the arithmetic of the single-job kernel, so a job's partial sums do not depend
// on the other jobs of the table.
template <int RP, bool DEN, int MS>
__global__ void __launch_bounds__(NT, Geo<RP>::MINB) cp3_pass_fp32_batched(const BatchTable<Cp3Args> t) {
    const int n = *t.n;
    const int total = n > 0 ? t.pfx[n] : 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = batch_job_of(t.pfx, n, item);
        if (t.state[j].done) continue;  // uniform over the CTA
        const Cp3Args a = t.args[j];
        cp3_fp32_body<RP, DEN, MS>(a, item - t.pfx[j]);
        __syncthreads();
    }
}

template <int RP, bool DEN, int MS>
cudaError_t launch_one(const Cp3Plan &p, const Cp3Args &a, cudaStream_t s) {
    constexpr Layout L = layout<RP, DEN, MS>();
    const size_t bytes = (size_t)L.end * sizeof(float);
    auto k = cp3_pass_fp32<RP, DEN, MS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k<<<p.grid, NT, bytes, s>>>(a);
    return cudaGetLastError();
}

// All mode sets used by the library for one rank padding.
template <int RP>
cudaError_t launch_rp(const Cp3Plan &p, const Cp3Args &a, int ms, int den, cudaStream_t s) {
    if (den) {
        switch (ms) {
            case PM_M1: return launch_one<RP, true, PM_M1>(p, a, s);
            case PM_M1 | PM_OBJ: return launch_one<RP, true, PM_M1 | PM_OBJ>(p, a, s);
            case PM_M2: return launch_one<RP, true, PM_M2>(p, a, s);
            case PM_M3: return launch_one<RP, true, PM_M3>(p, a, s);
            case PM_M1 | PM_NOX: return launch_one<RP, true, PM_M1 | PM_NOX>(p, a, s);
            case PM_M1 | PM_OBJ | PM_NOX: return launch_one<RP, true, PM_M1 | PM_OBJ | PM_NOX>(p, a, s);
            case PM_M2 | PM_NOX: return launch_one<RP, true, PM_M2 | PM_NOX>(p, a, s);
            case PM_M3 | PM_NOX: return launch_one<RP, true, PM_M3 | PM_NOX>(p, a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (ms) {
        case PM_M1: return launch_one<RP, false, PM_M1>(p, a, s);
        case PM_M1 | PM_OBJ: return launch_one<RP, false, PM_M1 | PM_OBJ>(p, a, s);
        case PM_M2: return launch_one<RP, false, PM_M2>(p, a, s);
        case PM_M3: return launch_one<RP, false, PM_M3>(p, a, s);
        case PM_M1 | PM_M2 | PM_M3 | PM_OBJ:
            return launch_one<RP, false, PM_M1 | PM_M2 | PM_M3 | PM_OBJ>(p, a, s);
        case PM_OBJ: return launch_one<RP, false, PM_OBJ>(p, a, s);
        case PM_OBJ | PM_NOX: return launch_one<RP, false, PM_OBJ | PM_NOX>(p, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int RP, bool DEN, int MS>
cudaError_t launch_batched_one(const BatchTable<Cp3Args> &t, int grid, cudaStream_t s) {
    constexpr Layout L = layout<RP, DEN, MS>();
    const size_t bytes = (size_t)L.end * sizeof(float);
    auto k = cp3_pass_fp32_batched<RP, DEN, MS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {  // persistent grid: every CTA that fits on the device at once
        int per_sm = 0, dev = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, bytes)) != cudaSuccess) return e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid = per_sm * sms;
    }
    k<<<grid, NT, bytes, s>>>(t);
    return cudaGetLastError();
}

// The pass variants of the batched iterations: the first pass of an iteration (mode 1 with
// the objective), modes 2 and 3, and the KL J-CoMM pass (all numerators and the objective).
template <int RP>
cudaError_t launch_batched_rp(const BatchTable<Cp3Args> &t, int ms, int den, int grid, cudaStream_t s) {
    if (den) {
        switch (ms) {
            case PM_M1 | PM_OBJ: return launch_batched_one<RP, true, PM_M1 | PM_OBJ>(t, grid, s);
            case PM_M2: return launch_batched_one<RP, true, PM_M2>(t, grid, s);
            case PM_M3: return launch_batched_one<RP, true, PM_M3>(t, grid, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (ms) {
        case PM_M1 | PM_OBJ: return launch_batched_one<RP, false, PM_M1 | PM_OBJ>(t, grid, s);
        case PM_M2: return launch_batched_one<RP, false, PM_M2>(t, grid, s);
        case PM_M3: return launch_batched_one<RP, false, PM_M3>(t, grid, s);
        case PM_M1 | PM_M2 | PM_M3 | PM_OBJ:
            return launch_batched_one<RP, false, PM_M1 | PM_M2 | PM_M3 | PM_OBJ>(t, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fp32
}  // namespace ntf
