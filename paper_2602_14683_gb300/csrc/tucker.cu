// Dense 3-way Tucker: block MM (Theorem "Tucker block multiplicative updates",
// Appendix C.2) and J-CoMM (Algorithm 2, Appendix C.3).
//
// Every block update reads X once through a fused pass:
//   * Xhat rows come from the mode-3 partial tensor B3[i][j][c] = sum_{a,b} G[a,b,c]
//     A1[i,a] A2[j,b] (eq. (block_Bn) for n = 3), materialised as an I1*I2 x J3 matrix
//     (20 MB at 400^3, J = 32) by two small GEMMs, and the columns of A3:
//     Xhat[i,j,k] = sum_c B3[i,j,c] A3[k,c].
//   * Core and modes 1, 2: the "rows" pass writes W[i,j,c] = sum_k P[i,j,k] A3n[k,c] (and
//     Wd with Q and A3d).  The remaining sums of eqs. (block_core_num_den),
//     (block_factor_num/den) are then small GEMMs over W:
//       Num1[i,a]   = sum_{j,c} W[i,j,c] H[j,a,c],    H[j,a,c]   = sum_b G[a,b,c] A2[j,b]
//       Num2[j,b]   = sum_{i,c} W[i,j,c] GA1[i,b,c],  GA1[i,b,c] = sum_a A1[i,a] G[a,b,c]
//       Pcore[a,b,c] = sum_i A1[i,a] sum_j A2[j,b] W[i,j,c]
//   * Mode 3: the CP pass in mode 3 with explicit rows, Num3[k,c] = sum_{i,j} P B3n[i,j,c].
// J-CoMM uses the reference blocks to rebuild Xtilde and chi1 / chi2 transforms of the
// current blocks (and of the core) on the numerator / denominator side; since W depends
// on the third factor only, one rows pass serves the core and modes 1 and 2 of an inner
// sweep, so an inner sweep reads X twice instead of four times.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <string>

#include "cp3_fp32.cuh"
#include "ntf_coo.h"
#include "ntf_tucker.h"

namespace ntf {

// ----------------------------------------------------------------------------------
// Strided batched GEMM with a two-level reduction index (FP32 FMA, FP64 carry):
//   C[bt][m][n] = sum_{k1 < K1, k2 < K2} A(bt, m, k1, k2) * B(bt, k1, k2, n)
// The reduction index k = k1 * K2 + k2 may be split into `splits` contiguous ranges, one
// CTA per (tile, batch, range); each range's sum goes to `part` (FP32), and the ranges are
// then added in order, in FP64, by a second kernel (a fixed order for every run).  Within a
// range, products are summed in FP32 over blocks of GCARRY * GK terms and the blocks in
// FP64; a range of one block never touches FP64 (a slow pipe on this part).
// ----------------------------------------------------------------------------------
constexpr int GK = 16;   // reduction chunk
constexpr int GCARRY = 16;  // chunks summed in FP32 before the FP64 carry

// Output tiles of TM x TN for NBT batches at once (64 x 64; 128 x 32 for outputs at most 32
// columns wide, 256 x 16 for at most 16, 512 x 8 for at most 8; 32 x 32, 64 x 16 or 128 x 8 for
// four batches of at most that many outputs);
// each of the 256 threads holds a 4 x 4 block of contiguous rows and columns of one batch, read
// from the k-major shared tiles with one 16-byte load each.  Tile elements are fetched with
// consecutive threads on the operand's unit-stride index (m or n when that stride is 1, else k),
// and the next chunk's elements are prefetched into registers while this chunk computes.  Within a
// reduction range every output sums its k terms in increasing k; the number of ranges follows the
// tile count (gemm()), so a change of tile shape can move results in the last bits.
template <int TM, int TN, int NBT>
__global__ void __launch_bounds__(256) gemm2k_kernel(const Gemm g) {
    static_assert(TM * TN * NBT == 4096, "256 threads x 16 outputs");
    constexpr int CT = TN / 4, TPB = 256 / NBT;  // thread columns, threads per batch
    constexpr int LA = TM + 4, LB = TN + 4;       // padded rows (16-byte aligned)
    __shared__ __align__(16) float As[NBT][GK][LA];
    __shared__ __align__(16) float Bs[NBT][GK][LB];
    const int nbg = (g.batch + NBT - 1) / NBT;
    const int bg = blockIdx.z % nbg, sp = blockIdx.z / nbg;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int tid = threadIdx.x, bs = tid / TPB, tl = tid % TPB, tm = tl / CT, tn = tl % CT;
    const int bt = bg * NBT + bs;  // this thread's batch (outputs only when < batch)
    const int K = g.K1 * g.K2;
    const int kbeg = sp * g.kchunks * GK, kend = min(K, kbeg + g.kchunks * GK);
    const bool carry = (kend - kbeg + GK - 1) / GK > GCARRY;  // more than one FP32 block
    float acc[4][4];
    double tot[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f, tot[x][y] = 0.0;
    // (k1, k2) of k = k0 + kk from k0's quotient and remainder (one division per chunk)
    auto split = [&](int q0, int r0, int kk, int &k1, int &k2) {
        if (g.K2 == 1) {
            k1 = q0 + kk;
            k2 = 0;
            return;
        }
        k2 = r0 + kk;
        k1 = q0;
        if (k2 >= g.K2) {
            if (g.K2 >= GK) {
                k2 -= g.K2;
                k1 += 1;
            } else {
                k1 += k2 / g.K2;
                k2 %= g.K2;
            }
        }
    };
    const bool a_mfast = g.sam == 1, b_nfast = g.sbn == 1;
    constexpr int TOTA = NBT * GK * TM, TOTB = NBT * GK * TN;  // tile elements
    constexpr int NA = (TOTA + 255) / 256, NB = (TOTB + 255) / 256;
    float ra[NA], rb[NB];
    // element e of this thread: batch slot, k offset and m (or n) offset within the tile
    auto a_idx = [&](int e, int &sb, int &kk, int &mm) {
        const int t = tid + 256 * e;
        sb = t / (GK * TM);
        const int u = t % (GK * TM);
        if (a_mfast) { kk = u / TM; mm = u % TM; } else { mm = u / GK; kk = u % GK; }
    };
    auto b_idx = [&](int e, int &sb, int &kk, int &nn) {
        const int t = tid + 256 * e;
        sb = t / (GK * TN);
        const int u = t % (GK * TN);
        if (b_nfast) { kk = u / TN; nn = u % TN; } else { nn = u / GK; kk = u % GK; }
    };
    auto load = [&](int k0) {
        const int q0 = k0 / g.K2, r0 = k0 - q0 * g.K2;
#pragma unroll
        for (int e = 0; e < NA; ++e) {
            int sb, kk, mm;
            a_idx(e, sb, kk, mm);
            const int k = k0 + kk, b = bg * NBT + sb;
            float va = 0.0f;
            if (tid + 256 * e < TOTA && k < kend && m0 + mm < g.M && b < g.batch) {
                int k1, k2;
                split(q0, r0, kk, k1, k2);
                va = g.A[b * g.sab + (m0 + mm) * g.sam + k1 * g.sak1 + k2 * g.sak2];
            }
            ra[e] = va;
        }
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            int sb, kk, nn;
            b_idx(e, sb, kk, nn);
            const int k = k0 + kk, b = bg * NBT + sb;
            float vb = 0.0f;
            if (tid + 256 * e < TOTB && k < kend && n0 + nn < g.N && b < g.batch) {
                int k1, k2;
                split(q0, r0, kk, k1, k2);
                vb = g.B[b * g.sbb + k1 * g.sbk1 + k2 * g.sbk2 + (n0 + nn) * g.sbn];
            }
            rb[e] = vb;
        }
    };
    if (kbeg < kend) load(kbeg);
    int chunk = 0;
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
        for (int e = 0; e < NA; ++e) {
            int sb, kk, mm;
            a_idx(e, sb, kk, mm);
            if (tid + 256 * e < TOTA) As[sb][kk][mm] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            int sb, kk, nn;
            b_idx(e, sb, kk, nn);
            if (tid + 256 * e < TOTB) Bs[sb][kk][nn] = rb[e];
        }
        __syncthreads();
        if (k0 + GK < kend) load(k0 + GK);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 av = *reinterpret_cast<const float4 *>(&As[bs][kk][4 * tm]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[bs][kk][4 * tn]);
            const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
        if (carry && ++chunk == GCARRY) {
            chunk = 0;
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) tot[x][y] += (double)acc[x][y], acc[x][y] = 0.0f;
        }
    }
    if (bt >= g.batch) return;
    // outputs: four consecutive columns as one 16-byte store where the layout allows
    const int nb = n0 + 4 * tn;
    const bool vec = nb + 3 < g.N &&
                     (g.splits > 1 ? (g.N % 4 == 0)
                                   : (g.scn == 1 && g.scm % 4 == 0 && g.scb % 4 == 0 &&
                                      (reinterpret_cast<uintptr_t>(g.C) & 15) == 0));
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int m = m0 + 4 * tm + x;
        if (m >= g.M) continue;
        float v[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) v[y] = carry ? (float)(tot[x][y] + (double)acc[x][y]) : acc[x][y];
        float *dst = g.splits > 1 ? g.part + (((int64_t)sp * g.batch + bt) * g.M + m) * g.N + nb
                                  : g.C + bt * g.scb + m * g.scm + nb * g.scn;
        if (vec) {
            *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int y = 0; y < 4; ++y)
                if (nb + y < g.N) dst[y * (g.splits > 1 ? 1 : g.scn)] = v[y];
        }
    }
}

// C = sum over the reduction ranges.  With L = 4 (many ranges) four consecutive threads per output
// each add a quarter of the ranges in range order (loads eight at a time) and the four quarter
// sums are added in quarter order; with L = 1 (at most eight ranges) one thread adds them all in
// range order.  In FP64 for the FP32 GEMM (its accuracy carry), in FP32 for the tensor-core one
// (TF32 operands; a few ranges, and the GB300 FP64 pipe, conversions included, is slow).  With the
// batch folded into the columns (g.nin > 0), column b nin + n goes to batch block b of C; with a
// second index folded into the rows (g.mfold > 0) the partials are [n][m].  A bounded grid strides
// over the outputs (32 / L per warp and step, warp-uniform loop).
template <typename T, int L>
__global__ void gemm_split_sum_kernel(const Gemm g) {
    const int64_t total = (int64_t)g.M * g.N * g.batch;
    const int qid = L == 1 ? 0 : (int)(threadIdx.x & 3);
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) / L;
    const int per = (g.splits + L - 1) / L, s0 = qid * per, s1 = min(g.splits, s0 + per);
    const int64_t first = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / L;  // the warp's first output
    for (int64_t w0 = first; w0 < total; w0 += step) {
        const int64_t t = w0 + (threadIdx.x & 31) / L;
        const bool live = t < total;
        T v = 0;
        if (live) {
            for (int sp0 = s0; sp0 < s1; sp0 += 8) {
                float x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = sp0 + q < s1 ? g.part[(int64_t)(sp0 + q) * total + t] : 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (sp0 + q < s1) v += (T)x[q];
            }
        }
        T tot = v;
        if (L == 4) {
            const T v1 = __shfl_down_sync(0xffffffffu, v, 1), v2 = __shfl_down_sync(0xffffffffu, v, 2),
                    v3 = __shfl_down_sync(0xffffffffu, v, 3);
            tot = ((v + v1) + v2) + v3;
        }
        if (qid != 0 || !live) continue;
        // output t: [batch][M][N] order, or [batch][N][M] for the row-folded form (its partials'
        // order, m contiguous in C)
        const int inner = g.mfold > 0 ? g.M : g.N, outer = g.mfold > 0 ? g.N : g.M;
        int bt, o, r;
        if (total < (1ll << 31)) {  // 32-bit index arithmetic
            const int ti = (int)t, q = ti / inner;
            r = ti - q * inner;
            bt = q / outer;
            o = q - bt * outer;
        } else {
            const int64_t q = t / inner;
            r = (int)(t - q * inner);
            bt = (int)(q / outer);
            o = (int)(q - (int64_t)bt * outer);
        }
        const int m = g.mfold > 0 ? r : o, n = g.mfold > 0 ? o : r;
        int64_t mo = (int64_t)m * g.scm;  // row m's offset (second index folded into the rows: mfold > 0)
        if (g.mfold > 0) {
            const int f = m / g.mfold;
            mo = (int64_t)f * g.scmb + (int64_t)(m - f * g.mfold) * g.scm;
        }
        int64_t c;
        if (g.nin > 0) {
            const int b = n / g.nin;
            c = mo + (int64_t)b * g.scb + (int64_t)(n - b * g.nin) * g.scn;
        } else {
            c = (int64_t)bt * g.scb + mo + (int64_t)n * g.scn;
        }
        g.C[c] = (float)tot;
    }
}

static cudaError_t split_sum(const Gemm &g, cudaStream_t s, bool fp64, int sms) {
    const int64_t total = (int64_t)g.M * g.N * g.batch;
    const int L = g.splits <= 8 ? 1 : 4;
    const unsigned blocks = (unsigned)std::min<int64_t>((L * total + 255) / 256, 8 * (int64_t)sms);
    if (fp64) {
        if (L == 1) gemm_split_sum_kernel<double, 1><<<blocks, 256, 0, s>>>(g);
        else gemm_split_sum_kernel<double, 4><<<blocks, 256, 0, s>>>(g);
    } else {
        if (L == 1) gemm_split_sum_kernel<float, 1><<<blocks, 256, 0, s>>>(g);
        else gemm_split_sum_kernel<float, 4><<<blocks, 256, 0, s>>>(g);
    }
    return cudaGetLastError();
}

// Tensor-core plans timed by the autotuner: process-wide, keyed by device, shape, strides and
// arithmetic; the value is (tile width, reduction ranges).
struct GemmKey {
    int dev, M, N, K1, K2, batch, mode, mfold;
    int64_t sab, sam, samb, sak1, sak2, sbb, sbk1, sbk2, sbn;
    bool operator<(const GemmKey &o) const {
        return std::tie(dev, M, N, K1, K2, batch, mode, mfold, sab, sam, samb, sak1, sak2, sbb, sbk1, sbk2, sbn) <
               std::tie(o.dev, o.M, o.N, o.K1, o.K2, o.batch, o.mode, o.mfold, o.sab, o.sam, o.samb, o.sak1, o.sak2,
                        o.sbb, o.sbk1, o.sbk2, o.sbn);
    }
};
std::mutex g_gemm_mu;
std::map<GemmKey, std::pair<int, int>> g_gemm_tuned;

// reduction ranges for a tile width: up to about two CTAs per SM (rounded down, so that the
// CTAs fit one wave), at least two chunks each
static int tc_splits(const Gemm &f, int w, int sms) {
    const int nchunks = std::max(1, (f.K1 * f.K2 + 31) / 32);
    const int64_t want = 2 * (int64_t)sms;
    const int64_t tiles = (int64_t)((f.N + w - 1) / w) * ((f.M + 127) / 128) * f.batch;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want / tiles, nchunks / 2));
}

// One tensor-core product with the given plan (launch, and the range sum when split).
static int gemm_tc_run(ntf_ctx *ctx, Gemm f, int ntt, int splits, int mode, cudaStream_t s) {
    const int nchunks = std::max(1, (f.K1 * f.K2 + 31) / 32);
    f.kchunks = std::max(1, (nchunks + splits - 1) / splits);
    f.splits = std::max(1, (nchunks + f.kchunks - 1) / f.kchunks);
    if ((int64_t)f.batch * f.splits > 65535 || (f.M + 127) / 128 > 65535) return NTF_ERR_UNSUPPORTED;
    f.err = ctx_status(ctx);
    if (f.splits > 1) {
        f.part = (float *)ctx_ws(ctx, "gemm_split", sizeof(float) * (size_t)f.splits * f.batch * f.M * f.N);
        if (!f.part) return ctx_fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    }
    cudaError_t e = gemm_tc_launch(f, mode == 2, ntt, s);
    if (e == cudaSuccess && f.splits > 1) {
        e = split_sum(f, s, false, ctx_num_sms(ctx));
        ctx_count(ctx, 1);
    }
    if (e != cudaSuccess) return ctx_fail(ctx, NTF_ERR_CUDA, cudaGetErrorString(e));
    ctx_count(ctx, 1);
    return NTF_OK;
}

// Splits the reduction when the output tiles alone would leave most SMs idle: about two
// CTAs per SM, at least four GK-chunks per range (two 32-index chunks on the tensor cores).
// mode: 0 FP32 CUDA cores, 1 tcgen05 on TF32 operands, 2 tcgen05 on split (3xTF32) operands.
// tune (tensor cores): on the first call for a shape, time every tile width with its rule's
// ranges, and the rule's width with half and twice its ranges, and keep the fastest for the
// process (not while the stream is being captured: the rule's plan then).
static int gemm(ntf_ctx *ctx, Gemm g, cudaStream_t s, int mode = 0, bool tune = false) {
    if (mode) {
        // tensor cores: an A shared by every batch (sab = 0) serves several batches per tile, with
        // the batch folded into the columns (the B^(3) build, Y = A2^T W, H); then the widest tile
        // whose split plan still gives about two CTAs per SM (else 32 columns)
        Gemm f = g;
        if (g.sab == 0 && g.batch > 1 && g.N < 256 && (int64_t)g.N * g.batch < (1ll << 30)) {
            f.nin = g.N;
            f.N = g.N * g.batch;
            f.batch = 1;
        }
        const int sms = ctx_num_sms(ctx);
        const int64_t want = 2 * (int64_t)sms;
        int ntt = 32, splits = 1;
        for (int w = 256; w >= 32; w >>= 1) {
            if (w > 32 && f.N <= w / 2) continue;
            const int64_t tiles = (int64_t)((f.N + w - 1) / w) * ((f.M + 127) / 128) * f.batch;
            const int sp = tc_splits(f, w, sms);
            if (tiles * sp >= want || w == 32) {
                ntt = w;
                splits = sp;
                break;
            }
        }
        if (tune) {
            int dev = 0;
            cudaGetDevice(&dev);
            const GemmKey key{dev,   f.M,   f.N,    f.K1,  f.K2,  f.batch, mode,  f.mfold, f.sab,
                              f.sam, f.samb, f.sak1, f.sak2, f.sbb, f.sbk1,  f.sbk2, f.sbn};
            bool found = false;
            {
                std::lock_guard<std::mutex> lk(g_gemm_mu);
                auto it = g_gemm_tuned.find(key);
                if (it != g_gemm_tuned.end()) {
                    ntt = it->second.first;
                    splits = it->second.second;
                    found = true;
                }
            }
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (!found && cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
                std::vector<std::pair<int, int>> cand;
                for (int w = 256; w >= 32; w >>= 1)
                    if (w == 32 || f.N > w / 2) cand.push_back({w, tc_splits(f, w, sms)});
                cand.push_back({ntt, std::max(1, splits / 2)});
                cand.push_back({ntt, splits * 2});
                cudaEvent_t e0, e1;
                if (cudaEventCreate(&e0) != cudaSuccess) return ctx_fail(ctx, NTF_ERR_CUDA, "event creation failed");
                if (cudaEventCreate(&e1) != cudaSuccess) {
                    cudaEventDestroy(e0);
                    return ctx_fail(ctx, NTF_ERR_CUDA, "event creation failed");
                }
                float best = -1.0f;
                int rc = NTF_OK;
                for (const auto &c : cand) {
                    int r = gemm_tc_run(ctx, f, c.first, c.second, mode, s);  // untimed: code and caches
                    if (r == NTF_ERR_UNSUPPORTED) continue;
                    if (!r && cudaEventRecord(e0, s) != cudaSuccess) r = NTF_ERR_CUDA;
                    if (r) {
                        rc = r;
                        break;
                    }
                    for (int q = 0; q < 2 && !r; ++q) r = gemm_tc_run(ctx, f, c.first, c.second, mode, s);
                    float ms = 0.0f;
                    if (r || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = r ? r : NTF_ERR_CUDA;
                        break;
                    }
                    if (best < 0.0f || ms < best) {
                        best = ms;
                        ntt = c.first;
                        splits = c.second;
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (rc == NTF_ERR_CUDA) return ctx_fail(ctx, rc, "autotuning a contraction failed");
                if (rc) return rc;
                std::lock_guard<std::mutex> lk(g_gemm_mu);
                g_gemm_tuned[key] = {ntt, splits};
            }
        }
        const int r = gemm_tc_run(ctx, f, ntt, splits, mode, s);
        if (r != NTF_ERR_UNSUPPORTED) return r;
        // past the grid's z extent (batch x splits): the CUDA-core kernel below
    }
    if (g.mfold > 0) return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "row-folded contraction past the tensor-core grid");
    // tile shape: four batches per CTA for outputs of at most 32 x 32, 64 x 16 or 128 x 8, else by
    // width
    const bool multi = g.batch >= 4 && ((g.M <= 32 && g.N <= 32) || (g.M <= 64 && g.N <= 16) ||
                                        (g.M <= 128 && g.N <= 8));
    const int NBT = multi ? 4 : 1;
    const int TN = g.N <= 8 ? 8 : g.N <= 16 ? 16 : g.N <= 32 ? 32 : 64, TM = 4096 / (TN * NBT);
    const int nbg = (g.batch + NBT - 1) / NBT;
    const int tiles = ((g.N + TN - 1) / TN) * ((g.M + TM - 1) / TM) * nbg;
    const int nchunks = (g.K1 * g.K2 + GK - 1) / GK;
    int splits = (2 * ctx_num_sms(ctx) + tiles - 1) / tiles;
    splits = std::max(1, std::min(splits, nchunks / 4));
    g.kchunks = (nchunks + splits - 1) / splits;
    g.splits = (nchunks + g.kchunks - 1) / g.kchunks;
    if (g.splits > 1) {
        g.part = (float *)ctx_ws(ctx, "gemm_split", sizeof(float) * (size_t)g.splits * g.batch * g.M * g.N);
        if (!g.part) return ctx_fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    }
    dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, nbg * g.splits);
    if (multi && TN == 8)
        gemm2k_kernel<128, 8, 4><<<grid, 256, 0, s>>>(g);
    else if (multi && TN == 16)
        gemm2k_kernel<64, 16, 4><<<grid, 256, 0, s>>>(g);
    else if (multi)
        gemm2k_kernel<32, 32, 4><<<grid, 256, 0, s>>>(g);
    else if (TN == 8)
        gemm2k_kernel<512, 8, 1><<<grid, 256, 0, s>>>(g);
    else if (TN == 16)
        gemm2k_kernel<256, 16, 1><<<grid, 256, 0, s>>>(g);
    else if (TN == 32)
        gemm2k_kernel<128, 32, 1><<<grid, 256, 0, s>>>(g);
    else
        gemm2k_kernel<64, 64, 1><<<grid, 256, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && g.splits > 1) {
        e = split_sum(g, s, true, ctx_num_sms(ctx));
        ctx_count(ctx, 1);
    }
    if (e != cudaSuccess) return ctx_fail(ctx, NTF_ERR_CUDA, cudaGetErrorString(e));
    ctx_count(ctx, 1);
    return NTF_OK;
}

// ----------------------------------------------------------------------------------
// Rows pass: W[i][j][c] = sum_k P[i,j,k] Cn[k,c], Wd with Q and Cd, over all k.
// Xhat[i,j,k] = sum_c Rrow[i*J+j][c] Crec[k][c].  One CTA owns a tile of TJ rows j and a
// range of slabs i; column chunks of the third factors are staged with the X tile.
// ----------------------------------------------------------------------------------
struct RowsArgs {
    Cp3Args a;      // X, sizes, bkind/beta/eps, rrow, rec[2] (= Crec), num[2], den[2], obj
    float *Wn, *Wd; // [I*J][RP]
    int n_is;
};

// NOX (the dense part of a sparse tensor's update at beta != 1, Section 6.3): every entry is x = 0,
// no X tile is staged, and only Wd (Q against the den columns) and the objective terms
// d_beta(0 | Xhat) are computed.
template <int RP, bool DEN, bool OBJ, bool NOX = false>
__global__ void __launch_bounds__(fp32::NT, fp32::Geo<RP>::MINB) tucker_rows_kernel(const RowsArgs ra) {
    using namespace fp32;
    using G = Geo<RP>;
    constexpr int TJ = G::TJ, RW = G::RW, RG = G::RG, RS = G::RS, TT = G::TT;
    const Cp3Args &a = ra.a;
    extern __shared__ __align__(16) float sm[];
    float *xs0 = sm;                          // 2 x TJ x XS
    float *ps = xs0 + 2 * TJ * XS;            // TJ x XS
    float *qs = ps + TJ * XS;                 // TJ x XS (DEN)
    float *rrT = qs + (DEN ? TJ * XS : 0);    // RP x TT
    float *ct0 = rrT + RP * TT;               // 2 x RP x KC  (Crec chunk, permuted)
    float *cn0 = ct0 + 2 * RP * KC;           // 2 x KC x RS
    float *cd0 = cn0 + 2 * KC * RS;           // 2 x KC x RS (DEN)
    double *dred = reinterpret_cast<double *>(cd0 + (DEN ? 2 * KC * RS : 0));

    const int tid = threadIdx.x, tr = tid >> 3, tc = tid & 7;
    const int is = blockIdx.x % ra.n_is, jt = blockIdx.x / ra.n_is;
    const int i0 = (int)((int64_t)is * a.I / ra.n_is), i1 = (int)((int64_t)(is + 1) * a.I / ra.n_is);
    const int j0 = jt * TJ, J = a.J, K = a.K;
    const int nch = (K + KC - 1) / KC;

    auto stage = [&](int buf, int i, int q) {
        const int kc = q * KC;
        if (!NOX) load_x_tile<TJ>(a, xs0 + buf * TJ * XS, i, j0, kc);
        float *ct = ct0 + buf * RP * KC;
        for (int t = tid; t < RP * KC; t += NT) {
            const int r = t / KC, c = t % KC, k = kc + c;
            const bool v = k < K;
            cp_async4(ct + r * KC + (c & 7) * 4 + (c >> 3), v ? a.rec[2] + (int64_t)k * RP + r : a.rec[2], v ? 4 : 0);
        }
        float *cn = cn0 + buf * KC * RS;
        float *cd = cd0 + buf * KC * RS;
        for (int t = tid; t < KC * (RP / 4); t += NT) {
            const int c = t / (RP / 4), seg = t % (RP / 4), k = kc + c;
            const bool v = k < K;
            cp_async16(cn + c * RS + seg * 4, v ? a.num[2] + (int64_t)k * RP + seg * 4 : a.num[2], v ? 16 : 0);
            if (DEN) cp_async16(cd + c * RS + seg * 4, v ? a.den[2] + (int64_t)k * RP + seg * 4 : a.den[2], v ? 16 : 0);
        }
    };

    double obj_acc = 0.0;
    const int total = (i1 - i0) * nch;
    if (total > 0) stage(0, i0, 0);
    cp_async_commit();
    int buf = 0;
    float W[RW][RG], Wd[RW][RG];
    for (int it = 0; it < total; ++it) {
        const int i = i0 + it / nch, q = it % nch;
        if (q == 0) {
            const int64_t rb = (int64_t)i * J + j0;
            for (int t = tid; t < TJ * RP; t += NT) {
                const int row = t / RP, r = t % RP;
                rrT[r * TT + row] = (j0 + row < J) ? __ldg(a.rrow + (rb + row) * RP + r) : 0.0f;
            }
#pragma unroll
            for (int x = 0; x < RW; ++x)
#pragma unroll
                for (int y = 0; y < RG; ++y) W[x][y] = Wd[x][y] = 0.0f;
        }
        if (it + 1 < total) stage(buf ^ 1, i0 + (it + 1) / nch, (it + 1) % nch);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const float *xs = xs0 + buf * TJ * XS;
        const float *ct = ct0 + buf * RP * KC;
        const float *cn = cn0 + buf * KC * RS;
        const float *cd = cd0 + buf * KC * RS;
        const int kc = q * KC;

        float xh[RW][4];
#pragma unroll
        for (int x = 0; x < RW; ++x)
#pragma unroll
            for (int c = 0; c < 4; ++c) xh[x][c] = 0.0f;
#pragma unroll 8
        for (int r = 0; r < RP; ++r) {
            float rv[RW], cb[4];
            VecLd<RW>::ld(rrT + r * TT + tr * RW, rv);
            VecLd<4>::ld(ct + r * KC + tc * 4, cb);
#pragma unroll
            for (int x = 0; x < RW; ++x)
#pragma unroll
                for (int c = 0; c < 4; ++c) xh[x][c] = fmaf(rv[x], cb[c], xh[x][c]);
        }
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
                float P, Q;
                pq_powers(a.bkind, a.beta, xv, y, P, Q);
                if (!v) { P = 0.0f; Q = 0.0f; }
                if (OBJ && v) objf += dbeta_stable(a.bkind, a.beta, xv, y);
                if (!NOX) ps[row * XS + col] = P;
                if (DEN) qs[row * XS + col] = Q;
            }
        }
        if (OBJ) obj_acc += (double)objf;
        __syncthreads();
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
                if (!NOX) VecLd<RG>::ld(cn + (c4 * 4 + cq) * RS + tc * RG, cv);
                if (DEN) VecLd<RG>::ld(cd + (c4 * 4 + cq) * RS + tc * RG, dv);
#pragma unroll
                for (int x = 0; x < RW; ++x)
#pragma unroll
                    for (int y = 0; y < RG; ++y) {
                        if (!NOX) W[x][y] = fmaf(p[x][cq], cv[y], W[x][y]);
                        if (DEN) Wd[x][y] = fmaf(qv[x][cq], dv[y], Wd[x][y]);
                    }
            }
        }
        if (q == nch - 1) {
            const int64_t rb = (int64_t)i * J + j0;
#pragma unroll
            for (int x = 0; x < RW; ++x) {
                const int row = tr * RW + x;
                if (j0 + row < J) {
#pragma unroll
                    for (int y = 0; y < RG; ++y) {
                        if (!NOX) ra.Wn[(rb + row) * RP + tc * RG + y] = W[x][y];
                        if (DEN) ra.Wd[(rb + row) * RP + tc * RG + y] = Wd[x][y];
                    }
                }
            }
        }
        __syncthreads();  // buffers of this iteration are restaged two iterations later
        buf ^= 1;
    }
    cp_async_wait<0>();
    if (OBJ) {
        double v = obj_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((tid & 31) == 0) dred[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += dred[w];
            a.obj[blockIdx.x] = t;
        }
    }
}

template <int RP, bool DEN, bool OBJ, bool NOX = false>
static cudaError_t rows_launch_t(const RowsArgs &ra, int grid, cudaStream_t s) {
    using namespace fp32;
    using G = Geo<RP>;
    const size_t floats = 2 * G::TJ * XS + G::TJ * XS + (DEN ? G::TJ * XS : 0) + RP * G::TT + 2 * RP * KC +
                          2 * KC * G::RS + (DEN ? 2 * KC * G::RS : 0) + 2 * 32;
    const size_t bytes = floats * sizeof(float);
    auto k = tucker_rows_kernel<RP, DEN, OBJ, NOX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, bytes, s>>>(ra);
    return cudaGetLastError();
}

template <int RP>
static cudaError_t rows_launch_rp(const RowsArgs &ra, int grid, bool obj, cudaStream_t s, bool nox) {
    if (nox) return obj ? rows_launch_t<RP, true, true, true>(ra, grid, s) : rows_launch_t<RP, true, false, true>(ra, grid, s);
    return obj ? rows_launch_t<RP, true, true>(ra, grid, s) : rows_launch_t<RP, true, false>(ra, grid, s);
}

static cudaError_t rows_launch(int RP, const RowsArgs &ra, int grid, bool obj, cudaStream_t s, bool nox = false) {
    switch (RP) {
        case 8: return rows_launch_rp<8>(ra, grid, obj, s, nox);
        case 16: return rows_launch_rp<16>(ra, grid, obj, s, nox);
        case 32: return rows_launch_rp<32>(ra, grid, obj, s, nox);
        case 64: return rows_launch_rp<64>(ra, grid, obj, s, nox);
        default: return cudaErrorInvalidValue;
    }
}

// ----------------------------------------------------------------------------------
// small elementwise kernels
// ----------------------------------------------------------------------------------
// out[t] = sum over the parts of parts[p][t], in part order (loads issued eight at a time)
__global__ void sum_parts_kernel(const float *parts, int n_parts, int64_t n, float *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float acc = 0.0f;
    for (int p0 = 0; p0 < n_parts; p0 += 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = p0 + k < n_parts ? parts[(int64_t)(p0 + k) * n + t] : 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (p0 + k < n_parts) acc += v[k];
    }
    out[t] = acc;
}

// The same sum, four consecutive elements per thread (n4 = n / 4 float4 groups, 16-byte
// aligned arrays); blockIdx.y picks one of two independent sums (W and Wd in one launch).
__global__ void sum_parts4_kernel(const float *pa, float *oa, const float *pb, float *ob, int n_parts, int64_t n4) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n4) return;
    const float4 *parts = reinterpret_cast<const float4 *>(blockIdx.y ? pb : pa);
    float4 acc = parts[t];
    for (int p = 1; p < n_parts; ++p) {
        const float4 v = parts[(int64_t)p * n4 + t];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    reinterpret_cast<float4 *>(blockIdx.y ? ob : oa)[t] = acc;
}

// Extrapolation of one flat block (Section "Going beyond: Majorization-Minimization with
// Extrapolation"): D = [A - Aprev]_+ and FP64 partial sums of D^2 per CTA, Aprev <- A; then
// E = max(A + alpha D, eps), alpha = min(alpha_nes, cap / (||D||_F + delta)), every CTA
// summing the partials in the same order.
constexpr int XB = 64;  // CTAs of the flat extrapolation kernels

__global__ void extrap_flat_prep_kernel(const float *A, float *Aprev, float *D, int64_t n, double *part) {
    __shared__ double sh[256];
    double s2 = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float a = A[t];
        const float d = fmaxf(a - Aprev[t], 0.0f);
        Aprev[t] = a;
        D[t] = d;
        s2 += (double)d * (double)d;
    }
    sh[threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void extrap_flat_apply_kernel(const float *A, const float *D, int64_t n, const double *part, float alpha_nes,
                                         float cap, float delta, float eps, float *E) {
    __shared__ float alpha_s;
    if (threadIdx.x == 0) {
        double s2 = 0.0;
        for (int b = 0; b < XB; ++b) s2 += part[b];
        const double c = (double)cap / (sqrt(s2) + (double)delta);
        alpha_s = (float)((double)alpha_nes < c ? (double)alpha_nes : c);
    }
    __syncthreads();
    const float alpha = alpha_s;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        E[t] = fmaxf(fmaf(alpha, D[t], A[t]), eps);
}

// Order N >= 4 on the 3-way kernels (modes cut into three runs of consecutive modes): the
// factor of a run of several modes is the Kronecker product of the run's factors, rows and
// columns both row-major over the run (the memory order of X and of the core):
//   V[(i_a, i_b, ...)][(j_a, j_b, ...)] = prod_m A_m[i_m][j_m], columns >= cols up to ld zero.
struct KronArgs {
    const float *L[8];  // the run's factors, I[m] x J[m] row-major
    int I[8], J[8];
    int M, rows, cols, ld;
    float *out;
};

__global__ void kron_build_kernel(KronArgs k) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)k.rows * k.ld) return;
    int row = (int)(t / k.ld), c = (int)(t % k.ld);
    if (c >= k.cols) {
        k.out[t] = 0.0f;
        return;
    }
    float v = 1.0f;
    for (int m = k.M - 1; m >= 0; --m) {
        const int im = row % k.I[m], jm = c % k.J[m];
        row /= k.I[m];
        c /= k.J[m];
        v *= k.L[m][(int64_t)im * k.J[m] + jm];
    }
    k.out[t] = v;
}

// out[i_n][j_n] = sum over the run's other (i, j) index pairs of
//   S[(i ...)][(j ...)] * prod_{m != n} A_m[i_m][j_m]
// -- the Tucker factor contraction of mode n from the run's contraction S; one block of 256
// threads per output, the threads striding the pairs with FP64 sums added as a fixed tree.
struct KronFoldArgs {
    const float *S;  // [rows][ld]
    int ld;
    const float *L[8];
    int I[8], J[8];
    int M, n;
    float *out;      // [I[n]][J[n]]
};

__global__ void kron_fold_kernel(KronFoldArgs f) {
    __shared__ double sh[256];
    const int64_t t = blockIdx.x;  // one block per output
    const int in = (int)(t / f.J[f.n]), jn = (int)(t % f.J[f.n]);
    int64_t oi = 1, oj = 1;
    for (int m = 0; m < f.M; ++m)
        if (m != f.n) {
            oi *= f.I[m];
            oj *= f.J[m];
        }
    double acc = 0.0;
    for (int64_t q = threadIdx.x; q < oi * oj; q += blockDim.x) {
        int64_t ri = q / oj, rj = q % oj, row = 0, col = 0, mi = 1, mj = 1;
        float w = 1.0f;
        for (int m = f.M - 1; m >= 0; --m) {
            int im = in, jm = jn;
            if (m != f.n) {
                im = (int)(ri % f.I[m]);
                ri /= f.I[m];
                jm = (int)(rj % f.J[m]);
                rj /= f.J[m];
                w *= f.L[m][(int64_t)im * f.J[m] + jm];
            }
            row += im * mi;
            col += jm * mj;
            mi *= f.I[m];
            mj *= f.J[m];
        }
        acc += (double)f.S[row * f.ld + col] * (double)w;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {  // fixed tree
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) f.out[t] = (float)sh[0];
}

__global__ void mu_plain_kernel(const float *pre, const float *num, const float *den, int64_t n, float gamma,
                                float eps, float *out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float ratio = __fdiv_rn(num[t], den[t]);
    const float m = gamma == 1.0f ? ratio : (gamma == 0.5f ? sqrtf(ratio) : powf(ratio, gamma));
    out[t] = fmaxf(pre[t] * m, eps);
}

__global__ void chi_kernel(const float *z, const float *zt, int64_t n, float beta, float *c1, float *c2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    c1[t] = chi1_f(beta, z[t], zt[t]);
    c2[t] = chi2_f(beta, z[t], zt[t]);
}

// Column sums of a [rows][RP] matrix in two launches: CSB blocks each sum a strided set of row
// groups (FP32 within a thread, FP64 across the block's groups), then one block adds the CSB
// partials (lane groups striding the blocks, the groups added in order).
constexpr int CSB = 256;

__global__ void colsum_part_kernel(const float *src, int64_t rows, int RP, double *part) {
    __shared__ double sh[256];
    const int G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    float s = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * G + g; i < rows; i += (int64_t)gridDim.x * G) s += src[i * RP + r];
    sh[t] = (double)s;
    __syncthreads();
    if (t < RP) {
        double tot = 0.0;
        for (int k = 0; k < G; ++k) tot += sh[k * RP + t];
        part[(int64_t)blockIdx.x * RP + t] = tot;
    }
}

__global__ void colsum_final_kernel(const double *part, int nb, int RP, float *out) {
    __shared__ double sh[256];
    const int G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    double s = 0.0;
    for (int b = g; b < nb; b += G) s += part[(int64_t)b * RP + r];
    sh[t] = s;
    __syncthreads();
    if (t < RP) {
        double tot = 0.0;
        for (int k = 0; k < G; ++k) tot += sh[k * RP + t];
        out[t] = (float)tot;
    }
}

// out[p][row][c] = (p == 0 ? v[c] : 0) for p < parts, row < rows, c < RP
__global__ void bcast_rows_kernel(const float *v, int64_t rows, int RP, int parts, float *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)parts * rows * RP) return;
    out[t] = t < rows * RP ? v[t % RP] : 0.0f;
}

// row index of the (i, j) pair of a stored entry in the I1*I2 x I3 view of a 3-way COO tensor
__global__ void pair_index_kernel(const int32_t *i, const int32_t *j, int64_t nnz, int I2, int32_t *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) out[t] = i[t] * I2 + j[t];
}

__global__ void pad_cols_kernel(const float *src, int rows, int cols, int ld, float *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * ld) return;
    const int i = (int)(t / ld), c = (int)(t % ld);
    dst[t] = c < cols ? src[(int64_t)i * cols + c] : 0.0f;
}

__global__ void unpad_cols_kernel(const float *src, int rows, int cols, int ld, float *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * cols) return;
    const int i = (int)(t / cols), c = (int)(t % cols);
    dst[t] = src[(int64_t)i * ld + c];
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

// ----------------------------------------------------------------------------------
// orchestration
// ----------------------------------------------------------------------------------
namespace {

struct Blocks {  // one Tucker parameter set on the device (A3 padded to RP columns)
    float *G, *A1, *A2, *A3p;
};

struct TuckerWs {
    int I1, I2, I3, J1, J2, J3, RP;
    float *Brec, *Bn, *Bd;  // [I1*I2][RP]
    float *GA1, *H;         // [I1][J2*J3], [I2][J1*J3]
    float *Wn, *Wd;         // [I1*I2][RP]
    float *Y;               // [I1][J2*J3]
    float *num, *den;       // max(I_n*J_n, J1*J2*J3)
    float *pn3, *pd3;       // mode-3 partials
    double *obj;
    Cp3Plan plan3;
    int rows_grid, rows_is;
    // tensor-core passes (TF32 / 3xTF32 reconstruction, BF16 contractions): plan, W partials
    // per 128-column block [n_kb][I1*I2][RP], and the partial counts of the passes in use
    bool tc;
    Cp3Plan tplan;   // rows pass (W, Wd): 256-column blocks with single TF32, else 128
    Cp3Plan tplan3;  // mode-3 pass: 128-column blocks
    // the passes' view of X as tI slabs of tJ rows: with explicit rows only the row index
    // i I2 + j matters, so when 128 divides I1 I2 the rows are cut into slabs of exactly 128
    // (no ragged row tile); otherwise (I1, I2)
    int tI, tJ;
    float *Wpn, *Wpd;
    int parts3, obj_n;
    float *cs;                // [RP] column sums (closed-form denominators at beta = 1)
    double *cs_part;          // [CSB][RP] their partials
    Blocks cur, ref, t1, t2;  // current, reference, chi1 and chi2 transforms
    int gemm_mode;            // small contractions: 0 FP32, 1 TF32 tensor cores, 2 3xTF32 tensor cores
    bool gemm_tune;           // time the tensor-core contraction plans (ntf_opts.autotune)
    // sparse (COO) X at beta = 1: the stored entries as a 2-way COO tensor with rows (i, j) -> i I2 + j
    // and columns k, on which Xhat[(i, j), k] = sum_c B3[(i, j), c] A3[k, c] is a 2-way CP model
    bool coo;
    ntf_tensor X2;
    int64_t dims2[2];
    const int32_t *idx2[2];
    float *pd3x;     // beta != 1: the X-free mode-3 pass's Den3 partials [plan3.parts3][I3][RP]
    double *obj_tot; // the sparse objective (stored + dense parts), one value
};

// The source COO tensor of each context's 2-way view: the view's row indices live in the
// context's workspace, and the COO orders built for the view are cached by that pointer, so a
// different source tensor rebuilds both.
struct CooSrc {
    const void *idx[3], *vals;
    int64_t nnz, dims[3];
    bool operator==(const CooSrc &o) const {
        return idx[0] == o.idx[0] && idx[1] == o.idx[1] && idx[2] == o.idx[2] && vals == o.vals && nnz == o.nnz &&
               dims[0] == o.dims[0] && dims[1] == o.dims[1] && dims[2] == o.dims[2];
    }
};
std::mutex g_coo_src_mu;
std::map<const ntf_ctx *, CooSrc> g_coo_src;

#define TK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return ctx_fail(ctx, NTF_ERR_CUDA, cudaGetErrorString(e_)); \
        ctx_count(ctx, 1);                                                         \
    } while (0)

int rank_pad(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : 64; }

float *wsf(ntf_ctx *ctx, const char *name, int64_t n, bool &ok) {
    float *p = (float *)ctx_ws(ctx, name, sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (!p) ok = false;
    return p;
}

// B3[i][j][c] = sum_b A2[j,b] sum_a A1[i,a] G[a,b,c], padded to RP columns (pad kept 0)
// B3 = (A1 x_1 G) x_2 A2 into out; with ga1_ready, w.GA1 already holds A1 x_1 G of these blocks
int build_b3(ntf_ctx *ctx, TuckerWs &w, const Blocks &b, float *out, cudaStream_t st, bool ga1_ready = false) {
    // the product writes columns c < J3 of every row; padding columns (J3 < RP) must read zero
    if (w.J3 < w.RP) TK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)w.I1 * w.I2 * w.RP, st));
    Gemm g{};
    g.A = b.A1; g.B = b.G; g.C = w.GA1;
    g.M = w.I1; g.N = w.J2 * w.J3; g.K1 = w.J1; g.K2 = 1; g.batch = 1;
    g.sam = w.J1; g.sak1 = 1; g.sbk1 = (int64_t)w.J2 * w.J3; g.sbn = 1; g.scm = (int64_t)w.J2 * w.J3; g.scn = 1;
    if (!ga1_ready) { const int rc_ = gemm(ctx, g, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
    Gemm h{};
    h.A = b.A2; h.B = w.GA1; h.C = out;
    h.M = w.I2; h.N = w.J3; h.K1 = w.J2; h.K2 = 1; h.batch = w.I1;
    h.sab = 0; h.sam = w.J2; h.sak1 = 1;
    h.sbb = (int64_t)w.J2 * w.J3; h.sbk1 = w.J3; h.sbn = 1;
    h.scb = (int64_t)w.I2 * w.RP; h.scm = w.RP; h.scn = 1;
    { const int rc_ = gemm(ctx, h, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
    return NTF_OK;
}

Cp3Args base_args(const ntf_tensor *X, const TuckerWs &w, const ntf_opts &o, float beta) {
    Cp3Args a{};
    a.X = X->values;
    a.I = w.I1; a.J = w.I2; a.K = w.I3;
    a.bkind = beta_kind(beta);
    a.beta = beta;
    a.eps = (float)o.eps;
    a.eps_x = (float)o.eps_x;
    a.vec16 = (w.I3 % 4 == 0) && ((reinterpret_cast<uintptr_t>(X->values) & 15) == 0);
    a.obj = w.obj;
    return a;
}

int colsum_rows(ntf_ctx *ctx, TuckerWs &w, const float *src, int64_t rows, cudaStream_t st) {
    colsum_part_kernel<<<CSB, 256, 0, st>>>(src, rows, w.RP, w.cs_part);
    TK(cudaGetLastError());
    colsum_final_kernel<<<1, 256, 0, st>>>(w.cs_part, CSB, w.RP, w.cs);
    TK(cudaGetLastError());
    return NTF_OK;
}

// W (and Wd) from P, Q with third-factor columns n3 / d3; Xhat from rrow, A3rec.
int rows_pass(ntf_ctx *ctx, TuckerWs &w, const ntf_tensor *X, const ntf_opts &o, float beta, const float *rrow,
              const float *a3rec, const float *n3, const float *d3, bool obj, cudaStream_t st) {
    if (w.coo) {
        // W over the stored entries: the 2-way view's rows contraction, W[(i, j)][c] = sum_k P A3n[k][c]
        // (Section 6.3: P vanishes where X does); with obj the whole KL objective (stored entries +
        // sum of Xhat = sum_c colsum(B3)_c colsum(A3)_c) into w.obj[0]
        const float *rec[2] = {rrow, a3rec}, *num[2] = {rrow, n3};
        double *objp = nullptr;
        int nobj = 0;
        int rc = coo_num_rows(ctx, &w.X2, 0, w.RP, rec, num, beta, (float)o.eps, w.Wn, obj ? &objp : nullptr, &nobj, st);
        if (rc) return rc;
        if (beta_kind(beta) == BK_KL) {
            if (obj && (rc = coo_kl_objective_total(ctx, &w.X2, rec, w.J3, w.RP, objp, nobj, w.obj, st))) return rc;
            // Q = 1: Wd[(i, j)][c] = sum_k d3[k][c] for every row
            if ((rc = colsum_rows(ctx, w, d3, w.I3, st))) return rc;
            const int64_t n = (int64_t)w.I1 * w.I2 * w.RP;
            bcast_rows_kernel<<<nblk(n), 256, 0, st>>>(w.cs, (int64_t)w.I1 * w.I2, w.RP, 1, w.Wd);
            TK(cudaGetLastError());
            return NTF_OK;
        }
        // Q = Xhat^(beta - 1) is dense: Wd over the whole index space from the X-free rows pass,
        // which also sums the objective's dense part d_beta(0 | Xhat) (rows_grid partials)
        RowsArgs ra{};
        ra.a = base_args(X, w, o, beta);
        ra.a.X = nullptr;
        ra.a.vec16 = 0;
        ra.a.rrow = rrow;
        ra.a.rec[2] = a3rec;
        ra.a.num[2] = d3;
        ra.a.den[2] = d3;
        ra.Wn = w.Wd;  // not written by the X-free pass
        ra.Wd = w.Wd;
        ra.n_is = w.rows_is;
        TK(rows_launch(w.RP, ra, w.rows_grid, obj, st, /*nox=*/true));
        if (obj) {  // stored-entry part + dense part, as one partial for the caller's sum
            TK(reduce_objective2(objp, nobj, w.obj, w.rows_grid, w.obj_tot, st));
            TK(cudaMemcpyAsync(w.obj, w.obj_tot, sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        return NTF_OK;
    }
    if (w.tc) {
        Cp3Args a = base_args(X, w, o, beta);
        a.I = w.tI;
        a.J = w.tJ;
        a.rrow = rrow;
        a.rec[2] = a3rec;
        a.num[2] = n3;
        a.den[2] = d3;
        a.n_jt = w.tplan.n_jt;
        a.n_kb = w.tplan.n_kb;
        a.n_is = w.tplan.n_is;
        // one column block: the pass writes W (and Wd) directly
        const bool one = w.tplan.n_kb == 1;
        a.p1n = one ? w.Wn : w.Wpn;
        a.p1d = one ? w.Wd : w.Wpd;
        ctx_wait_opts(ctx, a);
        const bool kl = beta_kind(beta) == BK_KL;
        TK(cp3_tc_launch(w.tplan, a, PM_M1 | PM_M2 | (obj ? PM_OBJ : 0), kl ? 0 : 1, st));
        // W (and Wd) = sum over the column blocks, in block order
        const int64_t n = (int64_t)w.I1 * w.I2 * w.RP;
        if (!one) {
            const dim3 grid(nblk(n / 4), kl ? 1 : 2);
            sum_parts4_kernel<<<grid, 256, 0, st>>>(w.Wpn, w.Wn, w.Wpd, w.Wd, w.tplan.n_kb, n / 4);
            TK(cudaGetLastError());
        }
        if (kl) {
            // Q = 1: Wd[i][j][c] = sum_k d3[k][c], the same for every row
            int rc = colsum_rows(ctx, w, d3, w.I3, st);
            if (rc) return rc;
            bcast_rows_kernel<<<nblk(n), 256, 0, st>>>(w.cs, (int64_t)w.I1 * w.I2, w.RP, 1, w.Wd);
            TK(cudaGetLastError());
        }
        return NTF_OK;
    }
    RowsArgs ra{};
    ra.a = base_args(X, w, o, beta);
    ra.a.rrow = rrow;
    ra.a.rec[2] = a3rec;
    ra.a.num[2] = n3;
    ra.a.den[2] = d3;
    ra.Wn = w.Wn;
    ra.Wd = w.Wd;
    ra.n_is = w.rows_is;
    TK(rows_launch(w.RP, ra, w.rows_grid, obj, st));
    return NTF_OK;
}

// Num1 / Num2 / Pcore from W with the (possibly transformed) blocks b; with same_blocks the
// W-free factor (H of block 1, GA1 of block 2) of the previous call, made from the same b, is
// reused
int contract_from_w(ntf_ctx *ctx, TuckerWs &w, int block, const Blocks &b, const float *W, float *out,
                    cudaStream_t st, bool same_blocks = false) {
    if (block == 0) {  // core: Y[i][b][c] = sum_j A2[j,b] W[i,j,c]; Pcore = sum_i A1[i,a] Y[i]
        Gemm g{};
        // tensor cores: W is the 128-row operand, rows (i, c) folded (m = i J3 + c), so that no tile
        // row is padding (J2 alone fills a quarter of one), while its row tiles fit the grid
        if (w.gemm_mode && ((int64_t)w.I1 * w.J3 + 127) / 128 <= 65535) {
            g.A = W; g.B = b.A2; g.C = w.Y;
            g.M = w.I1 * w.J3; g.N = w.J2; g.K1 = w.I2; g.K2 = 1; g.batch = 1;
            g.mfold = w.J3; g.sam = 1; g.samb = (int64_t)w.I2 * w.RP; g.sak1 = w.RP;
            g.sbk1 = w.J2; g.sbn = 1;
            g.scm = 1; g.scmb = (int64_t)w.J2 * w.J3; g.scn = w.J3;
        } else {
            g.A = b.A2; g.B = W; g.C = w.Y;
            g.M = w.J2; g.N = w.J3; g.K1 = w.I2; g.K2 = 1; g.batch = w.I1;
            g.sam = 1; g.sak1 = w.J2;
            g.sbb = (int64_t)w.I2 * w.RP; g.sbk1 = w.RP; g.sbn = 1;
            g.scb = (int64_t)w.J2 * w.J3; g.scm = w.J3; g.scn = 1;
        }
        { const int rc_ = gemm(ctx, g, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
        Gemm h{};
        h.A = b.A1; h.B = w.Y; h.C = out;
        h.M = w.J1; h.N = w.J2 * w.J3; h.K1 = w.I1; h.K2 = 1; h.batch = 1;
        h.sam = 1; h.sak1 = w.J1; h.sbk1 = (int64_t)w.J2 * w.J3; h.sbn = 1;
        h.scm = (int64_t)w.J2 * w.J3; h.scn = 1;
        { const int rc_ = gemm(ctx, h, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
    } else if (block == 1) {  // H[j][a][c] = sum_b A2[j,b] G[a,b,c]; Num1 = sum_{j,c} W H
        Gemm g{};
        g.A = b.A2; g.B = b.G; g.C = w.H;
        g.M = w.I2; g.N = w.J3; g.K1 = w.J2; g.K2 = 1; g.batch = w.J1;
        g.sam = w.J2; g.sak1 = 1;
        g.sbb = (int64_t)w.J2 * w.J3; g.sbk1 = w.J3; g.sbn = 1;
        g.scb = w.J3; g.scm = (int64_t)w.J1 * w.J3; g.scn = 1;
        if (!same_blocks) { const int rc_ = gemm(ctx, g, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
        Gemm h{};
        h.A = W; h.B = w.H; h.C = out;
        h.M = w.I1; h.N = w.J1; h.K1 = w.I2; h.K2 = w.J3; h.batch = 1;
        h.sam = (int64_t)w.I2 * w.RP; h.sak1 = w.RP; h.sak2 = 1;
        h.sbk1 = (int64_t)w.J1 * w.J3; h.sbk2 = 1; h.sbn = w.J3;
        h.scm = w.J1; h.scn = 1;
        { const int rc_ = gemm(ctx, h, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
    } else {  // GA1[i][b][c] = sum_a A1[i,a] G[a,b,c]; Num2 = sum_{i,c} W GA1
        Gemm g{};
        g.A = b.A1; g.B = b.G; g.C = w.GA1;
        g.M = w.I1; g.N = w.J2 * w.J3; g.K1 = w.J1; g.K2 = 1; g.batch = 1;
        g.sam = w.J1; g.sak1 = 1; g.sbk1 = (int64_t)w.J2 * w.J3; g.sbn = 1; g.scm = (int64_t)w.J2 * w.J3; g.scn = 1;
        if (!same_blocks) { const int rc_ = gemm(ctx, g, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
        Gemm h{};
        h.A = W; h.B = w.GA1; h.C = out;
        h.M = w.I2; h.N = w.J2; h.K1 = w.I1; h.K2 = w.J3; h.batch = 1;
        h.sam = w.RP; h.sak1 = (int64_t)w.I2 * w.RP; h.sak2 = 1;
        h.sbk1 = (int64_t)w.J2 * w.J3; h.sbk2 = 1; h.sbn = w.J3;
        h.scm = w.J2; h.scn = 1;
        { const int rc_ = gemm(ctx, h, st, w.gemm_mode, w.gemm_tune); if (rc_) return rc_; }
    }
    return NTF_OK;
}

int setup(ntf_ctx *ctx, const ntf_tensor *X, const int64_t *core_dims, bool jcomm, TuckerWs &w, const ntf_opts &o,
          float beta, cudaStream_t st_setup = nullptr) {
    w.I1 = (int)X->dims[0]; w.I2 = (int)X->dims[1]; w.I3 = (int)X->dims[2];
    w.J1 = (int)core_dims[0]; w.J2 = (int)core_dims[1]; w.J3 = (int)core_dims[2];
    // tensor cores when asked for and the shapes fit them: third core dimension <= 32
    // (padded to 32), a 16-byte aligned X with I3 % 4 == 0; at beta = 1 (Q = 1) the passes
    // carry no denominator side and its sums are column sums (closed_den)
    w.tc = o.precision != NTF_PREC_FP32 && w.J3 <= 32 && cp3_tc_eligible(32, w.I3, X->values) &&
           (int64_t)w.I1 * w.I2 < (1ll << 31);
    w.coo = X->kind == NTF_COO;
    if (w.coo) w.tc = false;  // the stored-entry passes run on CUDA cores; their rows are 32 or 64 wide
    w.RP = w.tc ? 32 : w.coo ? (w.J3 <= 32 ? 32 : 64) : rank_pad(w.J3);
    // the small contractions follow the passes: tensor cores when the passes use them
    w.gemm_mode = !w.tc ? 0 : o.precision == NTF_PREC_3XTF32 ? 2 : 1;
    w.gemm_tune = o.autotune != 0;
    const int64_t IJ = (int64_t)w.I1 * w.I2, Jc = (int64_t)w.J1 * w.J2 * w.J3;
    bool ok = true;
    w.Brec = wsf(ctx, "tkBrec", IJ * w.RP, ok);
    w.Bn = jcomm ? wsf(ctx, "tkBn", IJ * w.RP, ok) : w.Brec;
    w.Bd = jcomm ? wsf(ctx, "tkBd", IJ * w.RP, ok) : w.Brec;
    w.GA1 = wsf(ctx, "tkGA1", (int64_t)w.I1 * w.J2 * w.J3, ok);
    w.H = wsf(ctx, "tkH", (int64_t)w.I2 * w.J1 * w.J3, ok);
    w.Wn = wsf(ctx, "tkWn", IJ * w.RP, ok);
    w.Wd = wsf(ctx, "tkWd", IJ * w.RP, ok);
    w.Y = wsf(ctx, "tkY", (int64_t)w.I1 * w.J2 * w.J3, ok);
    int64_t mx = Jc;
    const int64_t In[3] = {w.I1, w.I2, w.I3}, Jn[3] = {w.J1, w.J2, w.J3};
    for (int n = 0; n < 3; ++n) mx = mx > In[n] * Jn[n] ? mx : In[n] * Jn[n];
    w.num = wsf(ctx, "tkNum", mx, ok);
    w.den = wsf(ctx, "tkDen", mx, ok);
    w.plan3 = cp3_plan(w.I1, w.I2, w.I3, w.RP, ctx_num_sms(ctx));
    if (w.tc) {
        // the rows pass carries no column contraction, so with single TF32 operands its tensor
        // memory and shared memory allow 256-column blocks: half as many W partials to add
        const int kb_rows = o.precision == NTF_PREC_TF32 ? 256 : 128;
        const int TR = 128;  // row tile of the tensor-core passes
        const bool flat = IJ % TR == 0;
        w.tI = flat ? (int)(IJ / TR) : w.I1;
        w.tJ = flat ? TR : w.I2;
        w.tplan = cp3_plan(w.tI, w.tJ, w.I3, w.RP, ctx_num_sms(ctx), kb_rows);
        w.tplan.s3 = o.precision == NTF_PREC_3XTF32;
        w.tplan3 = cp3_plan(w.tI, w.tJ, w.I3, w.RP, ctx_num_sms(ctx), 128);
        w.tplan3.s3 = w.tplan.s3;
        w.Wpn = wsf(ctx, "tkWpn", (int64_t)w.tplan.n_kb * IJ * w.RP, ok);
        w.Wpd = wsf(ctx, "tkWpd", (int64_t)w.tplan.n_kb * IJ * w.RP, ok);
    }
    w.parts3 = w.coo ? 1 : w.tc ? w.tplan3.parts3 : w.plan3.parts3;
    w.pn3 = wsf(ctx, "tkPn3", (int64_t)w.parts3 * w.I3 * w.RP, ok);
    w.pd3 = wsf(ctx, "tkPd3", (int64_t)w.parts3 * w.I3 * w.RP, ok);
    // the FP32 rows kernel's tile (fp32::Geo) and about one wave of its resident CTAs (two per SM
    // at RP <= 32)
    const int TJ = 64, per_sm = w.RP == 64 ? 1 : 2;
    const int n_jt = (w.I2 + TJ - 1) / TJ;
    int is = (per_sm * ctx_num_sms(ctx) + n_jt - 1) / n_jt;
    if (is > w.I1) is = w.I1;
    w.rows_is = is;
    w.rows_grid = n_jt * is;
    w.obj_n = w.coo ? 1 : w.tc ? w.tplan.grid : w.rows_grid;
    int gmax = std::max(std::max(w.rows_grid, w.plan3.grid), w.tc ? std::max(w.tplan.grid, w.tplan3.grid) : 0);
    w.obj = (double *)ctx_ws(ctx, "tkObj", sizeof(double) * (size_t)gmax);
    if (!w.obj) ok = false;
    w.cs = wsf(ctx, "tkCs", 64, ok);
    w.cs_part = (double *)ctx_ws(ctx, "tkCsPart", sizeof(double) * CSB * 64);
    if (!w.cs_part) ok = false;
    const char *names[4][4] = {{"tkG", "tkA1", "tkA2", "tkA3"}, {"tkGt", "tkA1t", "tkA2t", "tkA3t"},
                               {"tkG1", "tkA11", "tkA21", "tkA31"}, {"tkG2", "tkA12", "tkA22", "tkA32"}};
    Blocks *bs[4] = {&w.cur, &w.ref, &w.t1, &w.t2};
    for (int q = 0; q < (jcomm ? 4 : 1); ++q) {
        bs[q]->G = wsf(ctx, names[q][0], Jc, ok);
        bs[q]->A1 = wsf(ctx, names[q][1], (int64_t)w.I1 * w.J1, ok);
        bs[q]->A2 = wsf(ctx, names[q][2], (int64_t)w.I2 * w.J2, ok);
        bs[q]->A3p = wsf(ctx, names[q][3], (int64_t)w.I3 * w.RP, ok);
    }
    if (!ok) return ctx_fail(ctx, NTF_ERR_OOM, "Tucker workspace allocation failed");
    if (w.coo) {
        if ((int64_t)w.I1 * w.I2 >= (1ll << 31)) return ctx_fail(ctx, NTF_ERR_SHAPE, "I1 * I2 exceeds 32-bit indices");
        bool ok2 = true;
        w.pd3x = beta_kind(beta) == BK_KL ? nullptr : wsf(ctx, "tkPd3x", (int64_t)w.plan3.parts3 * w.I3 * w.RP, ok2);
        w.obj_tot = (double *)ctx_ws(ctx, "tkObjTot", sizeof(double));
        if (!ok2 || !w.obj_tot) return ctx_fail(ctx, NTF_ERR_OOM, "Tucker workspace allocation failed");
        int32_t *rows = (int32_t *)ctx_ws(ctx, "tkCooRows", sizeof(int32_t) * (size_t)(X->nnz + 1));
        if (!rows) return ctx_fail(ctx, NTF_ERR_OOM, "Tucker workspace allocation failed");
        w.dims2[0] = (int64_t)w.I1 * w.I2;
        w.dims2[1] = w.I3;
        w.idx2[0] = rows;
        w.idx2[1] = X->idx[2];
        w.X2 = *X;
        w.X2.order = 2;
        w.X2.dims = w.dims2;
        w.X2.idx = w.idx2;
        const CooSrc src{{X->idx[0], X->idx[1], X->idx[2]}, X->values, X->nnz, {X->dims[0], X->dims[1], X->dims[2]}};
        bool same;
        {
            std::lock_guard<std::mutex> lk(g_coo_src_mu);
            auto it = g_coo_src.find(ctx);
            same = it != g_coo_src.end() && it->second == src;
            g_coo_src[ctx] = src;
        }
        if (!same) {  // a new source tensor: its pair rows, and the view's orders rebuilt on first use
            coo_release(ctx);
            if (X->nnz > 0) {
                pair_index_kernel<<<nblk(X->nnz), 256, 0, st_setup>>>(X->idx[0], X->idx[1], X->nnz, w.I2, rows);
                TK(cudaGetLastError());
            }
        }
    }
    return NTF_OK;
}

int load_blocks(ntf_ctx *ctx, TuckerWs &w, const float *core, const float *const *A, Blocks &b, cudaStream_t st) {
    const int64_t Jc = (int64_t)w.J1 * w.J2 * w.J3;
    TK(cudaMemcpyAsync(b.G, core, sizeof(float) * Jc, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(b.A1, A[0], sizeof(float) * w.I1 * w.J1, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(b.A2, A[1], sizeof(float) * w.I2 * w.J2, cudaMemcpyDeviceToDevice, st));
    pad_cols_kernel<<<nblk((int64_t)w.I3 * w.RP), 256, 0, st>>>(A[2], w.I3, w.J3, w.RP, b.A3p);
    TK(cudaGetLastError());
    return NTF_OK;
}

int copy_blocks(ntf_ctx *ctx, TuckerWs &w, const Blocks &s, Blocks &d, cudaStream_t st) {
    const int64_t Jc = (int64_t)w.J1 * w.J2 * w.J3;
    TK(cudaMemcpyAsync(d.G, s.G, sizeof(float) * Jc, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(d.A1, s.A1, sizeof(float) * w.I1 * w.J1, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(d.A2, s.A2, sizeof(float) * w.I2 * w.J2, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(d.A3p, s.A3p, sizeof(float) * w.I3 * w.RP, cudaMemcpyDeviceToDevice, st));
    return NTF_OK;
}

// block update: out = max(pre * (num/den)^gamma, eps), with chi transforms when jcomm
int apply_mu(ntf_ctx *ctx, TuckerWs &w, const float *pre, float *out, int64_t n, float beta, float eps,
             const float *ref, float *c1, float *c2, cudaStream_t st) {
    mu_plain_kernel<<<nblk(n), 256, 0, st>>>(pre, w.num, w.den, n, mu_gamma(beta), eps, out);
    TK(cudaGetLastError());
    if (c1) {
        chi_kernel<<<nblk(n), 256, 0, st>>>(out, ref, n, beta, c1, c2);
        TK(cudaGetLastError());
    }
    return NTF_OK;
}

int mode3_pass(ntf_ctx *ctx, TuckerWs &w, const ntf_tensor *X, const ntf_opts &o, float beta, const float *rrow,
               const float *a3rec, const float *nrow, const float *drow, bool obj, cudaStream_t st) {
    if (w.coo) {
        // Num3[k][c] = sum over the stored entries of P nrow[(i, j)][c]; Q = 1: Den3[k][c] = the
        // column sums of drow over all (i, j), the same for every k
        const float *rec[2] = {rrow, a3rec}, *num[2] = {nrow, a3rec};
        int rc = coo_num_rows(ctx, &w.X2, 1, w.RP, rec, num, beta, (float)o.eps, w.pn3, nullptr, nullptr, st);
        if (rc) return rc;
        if (beta_kind(beta) == BK_KL) {
            if ((rc = colsum_rows(ctx, w, drow, (int64_t)w.I1 * w.I2, st))) return rc;
            const int64_t n = (int64_t)w.I3 * w.RP;
            bcast_rows_kernel<<<nblk(n), 256, 0, st>>>(w.cs, w.I3, w.RP, 1, w.pd3);
            TK(cudaGetLastError());
            return NTF_OK;
        }
        // Den3 over the whole index space: the X-free FP32 pass in mode 3 with explicit rows, its
        // partials then summed (in part order) into the single part the update reads
        Cp3Args a = base_args(X, w, o, beta);
        a.X = nullptr;
        a.vec16 = 0;
        a.rrow = rrow;
        a.nrow = drow;
        a.drow = drow;
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = a3rec;
        a.n_jt = w.plan3.n_jt;
        a.n_kb = w.plan3.n_kb;
        a.n_is = w.plan3.n_is;
        a.p3n = w.pd3x;  // not written by the X-free pass
        a.p3d = w.pd3x;
        TK(cp3_launch(w.plan3, a, PM_M3 | PM_NOX, 1, st));
        const int64_t n = (int64_t)w.I3 * w.RP;
        sum_parts_kernel<<<nblk(n), 256, 0, st>>>(w.pd3x, w.plan3.parts3, n, w.pd3);
        TK(cudaGetLastError());
        return NTF_OK;
    }
    Cp3Args a = base_args(X, w, o, beta);
    a.rrow = rrow;
    a.nrow = nrow;
    a.drow = drow;
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = a3rec;
    if (w.tc) {
        a.I = w.tI;
        a.J = w.tJ;
        a.n_jt = w.tplan3.n_jt;
        a.n_kb = w.tplan3.n_kb;
        a.n_is = w.tplan3.n_is;
        a.p3n = w.pn3;
        a.p3d = w.pd3;
        ctx_wait_opts(ctx, a);
        const bool kl = beta_kind(beta) == BK_KL;
        TK(cp3_tc_launch(w.tplan3, a, PM_M3, kl ? 0 : 1, st));
        if (kl) {
            // Q = 1: Den3[k][c] = sum over the rows of drow, the same for every k (first part;
            // the other parts zero)
            int rc = colsum_rows(ctx, w, drow, (int64_t)w.I1 * w.I2, st);
            if (rc) return rc;
            const int64_t n = (int64_t)w.parts3 * w.I3 * w.RP;
            bcast_rows_kernel<<<nblk(n), 256, 0, st>>>(w.cs, w.I3, w.RP, w.parts3, w.pd3);
            TK(cudaGetLastError());
        }
        return NTF_OK;
    }
    a.n_jt = w.plan3.n_jt;
    a.n_kb = w.plan3.n_kb;
    a.n_is = w.plan3.n_is;
    a.p3n = w.pn3;
    a.p3d = w.pd3;
    TK(cp3_launch(w.plan3, a, PM_M3 | (obj ? 0 : 0), 1, st));
    return NTF_OK;
}

}  // namespace

// core extents 1..64 and at most the tensor's (order 3: each one is a 3-way block; order N >= 4:
// the last run's product must also stay <= 64, checked when the cut is chosen)
static int check_core(ntf_ctx *ctx, const ntf_tensor *X, const int64_t *core_dims, const float *const *factors) {
    for (int n = 0; n < X->order; ++n) {
        if (!factors[n]) return ctx_fail(ctx, NTF_ERR_ARG, "factor is NULL");
        if (core_dims[n] < 1 || core_dims[n] > 64)
            return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "core dimensions must lie in 1..64");
        if (core_dims[n] > X->dims[n]) return ctx_fail(ctx, NTF_ERR_SHAPE, "core dimension exceeds tensor dimension");
    }
    return NTF_OK;
}

int tucker_nway_run(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                    float *const *factors, const ntf_opts &o, double *objective_dev, cudaStream_t st, bool jcomm);
int tucker_nway_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, const float *core,
                         const float *const *factors, const ntf_opts &o, double *out_dev, cudaStream_t st);

int tucker_run(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
               float *const *factors, const ntf_opts &o, double *objective_dev, cudaStream_t st, bool jcomm,
               const TuckerExtrap *xe) {
    if (!core_dims || !core || !factors) return ctx_fail(ctx, NTF_ERR_ARG, "core_dims, core and factors are required");
    if (X->order < 3 || (X->order > 3 && xe)) return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker kernels implement order 3");
    if (int rc0 = check_core(ctx, X, core_dims, factors)) return rc0;
    if (X->order > 3) return tucker_nway_run(ctx, X, beta, core_dims, core, factors, o, objective_dev, st, jcomm);
    TuckerWs w{};
    int rc = setup(ctx, X, core_dims, jcomm, w, o, beta, st);
    if (rc) return rc;
    const float eps = (float)o.eps;
    const int64_t Jc = (int64_t)w.J1 * w.J2 * w.J3;
    const int64_t n1 = (int64_t)w.I1 * w.J1, n2 = (int64_t)w.I2 * w.J2, n3p = (int64_t)w.I3 * w.RP;
    rc = load_blocks(ctx, w, core, factors, w.cur, st);
    if (rc) return rc;
    if (xe && jcomm) {
        // outer-reference extrapolation (Section "Going beyond: Majorization-Minimization with
        // Extrapolation", item (iii)): the objective of the incoming iterate first, then every
        // block moved in place to its extrapolated point, which becomes the reference
        if (objective_dev) {
            if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
            if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, true, st))) return rc;
            TK(reduce_objective(w.obj, w.obj_n, 0.0, objective_dev, st));
            objective_dev = nullptr;
        }
        const int64_t n3 = (int64_t)w.I3 * w.J3;
        bool ok = true;
        float *E3 = wsf(ctx, "tkXE3", n3, ok);
        float *D = wsf(ctx, "tkXD", std::max(std::max(Jc, n1), std::max(n2, n3)), ok);
        double *part = (double *)ctx_ws(ctx, "tkXpart", sizeof(double) * XB);
        if (!ok || !part) return ctx_fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
        auto extrap = [&](const float *A, float *Aprev, int64_t n, float *E) -> int {
            extrap_flat_prep_kernel<<<XB, 256, 0, st>>>(A, Aprev, D, n, part);
            TK(cudaGetLastError());
            extrap_flat_apply_kernel<<<XB, 256, 0, st>>>(A, D, n, part, xe->alpha, xe->cap, xe->delta, eps, E);
            TK(cudaGetLastError());
            return NTF_OK;
        };
        if ((rc = extrap(w.cur.G, xe->core_prev, Jc, w.cur.G))) return rc;
        if ((rc = extrap(w.cur.A1, xe->factors_prev[0], n1, w.cur.A1))) return rc;
        if ((rc = extrap(w.cur.A2, xe->factors_prev[1], n2, w.cur.A2))) return rc;
        if ((rc = extrap(factors[2], xe->factors_prev[2], n3, E3))) return rc;
        pad_cols_kernel<<<nblk(n3p), 256, 0, st>>>(E3, w.I3, w.J3, w.RP, w.cur.A3p);
        TK(cudaGetLastError());
    }

    if (!jcomm) {
        // ---- core block (the pass also yields D_beta of the incoming iterate) ----
        if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
        if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, objective_dev != nullptr, st)))
            return rc;
        if (objective_dev) TK(reduce_objective(w.obj, w.obj_n, 0.0, objective_dev, st));
        if ((rc = contract_from_w(ctx, w, 0, w.cur, w.Wn, w.num, st))) return rc;
        if ((rc = contract_from_w(ctx, w, 0, w.cur, w.Wd, w.den, st))) return rc;
        if ((rc = apply_mu(ctx, w, w.cur.G, w.cur.G, Jc, beta, eps, nullptr, nullptr, nullptr, st))) return rc;
        // ---- modes 1 and 2 (block 2's GA1 = A1 x_1 G is the one the B3 build just made) ----
        for (int blk = 1; blk <= 2; ++blk) {
            if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
            if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, false, st))) return rc;
            if ((rc = contract_from_w(ctx, w, blk, w.cur, w.Wn, w.num, st, /*same_blocks=*/blk == 2))) return rc;
            if ((rc = contract_from_w(ctx, w, blk, w.cur, w.Wd, w.den, st, /*same_blocks=*/true))) return rc;
            float *A = blk == 1 ? w.cur.A1 : w.cur.A2;
            if ((rc = apply_mu(ctx, w, A, A, blk == 1 ? n1 : n2, beta, eps, nullptr, nullptr, nullptr, st))) return rc;
        }
        // ---- mode 3 (A1 and G unchanged since block 2: GA1 still holds their product) ----
        if ((rc = build_b3(ctx, w, w.cur, w.Brec, st, /*ga1_ready=*/true))) return rc;
        if ((rc = mode3_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.Brec, w.Brec, false, st))) return rc;
        MuEpiArgs e{};
        e.pn = w.pn3; e.pd = w.pd3; e.n_parts = w.parts3; e.rows = w.I3; e.RP = w.RP; e.R = w.J3;
        e.pre = w.cur.A3p; e.out = w.cur.A3p; e.beta = beta; e.gamma = mu_gamma(beta); e.eps = eps;
        TK(mu_epilogue(e, st));
    } else {
        if ((rc = copy_blocks(ctx, w, w.cur, w.ref, st))) return rc;
        if ((rc = copy_blocks(ctx, w, w.cur, w.t1, st))) return rc;
        if ((rc = copy_blocks(ctx, w, w.cur, w.t2, st))) return rc;
        // Xtilde rows from the reference, fixed for the whole outer iteration
        if ((rc = build_b3(ctx, w, w.ref, w.Brec, st))) return rc;
        for (int l = 0; l < o.inner_L; ++l) {
            // W from Ptilde with chi1(A3), Wd from Qtilde with chi2(A3): A3 changes only at the
            // end of the sweep, so one pass serves the core and modes 1 and 2
            const bool obj = (l == 0) && objective_dev;
            if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.ref.A3p, w.t1.A3p, w.t2.A3p, obj, st))) return rc;
            if (obj) TK(reduce_objective(w.obj, w.obj_n, 0.0, objective_dev, st));
            // core: Num with A_(1) of modes 1, 2 (and W), Den with A_(2)
            if ((rc = contract_from_w(ctx, w, 0, w.t1, w.Wn, w.num, st))) return rc;
            if ((rc = contract_from_w(ctx, w, 0, w.t2, w.Wd, w.den, st))) return rc;
            if ((rc = apply_mu(ctx, w, w.ref.G, w.cur.G, Jc, beta, eps, w.ref.G, w.t1.G, w.t2.G, st))) return rc;
            for (int blk = 1; blk <= 2; ++blk) {
                if ((rc = contract_from_w(ctx, w, blk, w.t1, w.Wn, w.num, st))) return rc;
                if ((rc = contract_from_w(ctx, w, blk, w.t2, w.Wd, w.den, st))) return rc;
                float *A = blk == 1 ? w.cur.A1 : w.cur.A2;
                const float *At = blk == 1 ? w.ref.A1 : w.ref.A2;
                float *c1 = blk == 1 ? w.t1.A1 : w.t1.A2;
                float *c2 = blk == 1 ? w.t2.A1 : w.t2.A2;
                if ((rc = apply_mu(ctx, w, At, A, blk == 1 ? n1 : n2, beta, eps, At, c1, c2, st))) return rc;
            }
            // mode 3: rows of the transformed partial tensors (the chi2 side first: GA1 still holds
            // A1 x_1 G of the chi2 blocks from block 2, whose update changed only A2)
            if ((rc = build_b3(ctx, w, w.t2, w.Bd, st, /*ga1_ready=*/true))) return rc;
            if ((rc = build_b3(ctx, w, w.t1, w.Bn, st))) return rc;
            if ((rc = mode3_pass(ctx, w, X, o, beta, w.Brec, w.ref.A3p, w.Bn, w.Bd, false, st))) return rc;
            MuEpiArgs e{};
            e.pn = w.pn3; e.pd = w.pd3; e.n_parts = w.parts3; e.rows = w.I3; e.RP = w.RP; e.R = w.J3;
            e.pre = w.ref.A3p; e.out = w.cur.A3p; e.ref = w.ref.A3p; e.chi1_out = w.t1.A3p; e.chi2_out = w.t2.A3p;
            e.beta = beta; e.gamma = mu_gamma(beta); e.eps = eps;
            TK(mu_epilogue(e, st));
        }
    }
    // write back
    TK(cudaMemcpyAsync(core, w.cur.G, sizeof(float) * Jc, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(factors[0], w.cur.A1, sizeof(float) * n1, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(factors[1], w.cur.A2, sizeof(float) * n2, cudaMemcpyDeviceToDevice, st));
    unpad_cols_kernel<<<nblk((int64_t)w.I3 * w.J3), 256, 0, st>>>(w.cur.A3p, w.I3, w.J3, w.RP, factors[2]);
    TK(cudaGetLastError());
    (void)n3p;
    return NTF_OK;
}

int tucker_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, const float *core,
                    const float *const *factors, const ntf_opts &o, double *out_dev, cudaStream_t st) {
    if (!core_dims || !core || !factors) return ctx_fail(ctx, NTF_ERR_ARG, "core_dims, core and factors are required");
    if (X->order < 3) return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker kernels implement orders 3..8");
    if (int rc0 = check_core(ctx, X, core_dims, factors)) return rc0;
    if (X->order > 3) return tucker_nway_beta_div(ctx, X, beta, core_dims, core, factors, o, out_dev, st);
    TuckerWs w{};
    int rc = setup(ctx, X, core_dims, false, w, o, beta, st);
    if (rc) return rc;
    if ((rc = load_blocks(ctx, w, core, factors, w.cur, st))) return rc;
    if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
    if (w.coo) {  // stored-entry part from the 2-way view's pass; the dense part in closed form (KL)
        const float *rec[2] = {w.Brec, w.cur.A3p};  // or from an X-free objective pass (other beta)
        double *objp = nullptr;
        int nobj = 0;
        if ((rc = coo_num_rows(ctx, &w.X2, 0, w.RP, rec, rec, beta, (float)o.eps, nullptr, &objp, &nobj, st))) return rc;
        if (beta_kind(beta) == BK_KL) return coo_kl_objective_total(ctx, &w.X2, rec, w.J3, w.RP, objp, nobj, out_dev, st);
        Cp3Args a = base_args(X, w, o, beta);
        a.X = nullptr;
        a.vec16 = 0;
        a.rrow = w.Brec;
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = w.cur.A3p;
        a.n_jt = w.plan3.n_jt;
        a.n_kb = w.plan3.n_kb;
        a.n_is = w.plan3.n_is;
        TK(cp3_launch(w.plan3, a, PM_OBJ | PM_NOX, 0, st));
        TK(reduce_objective2(objp, nobj, w.obj, w.plan3.grid, out_dev, st));
        return NTF_OK;
    }
    Cp3Args a = base_args(X, w, o, beta);
    a.rrow = w.Brec;
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = w.cur.A3p;
    a.n_jt = w.plan3.n_jt;
    a.n_kb = w.plan3.n_kb;
    a.n_is = w.plan3.n_is;
    TK(cp3_launch(w.plan3, a, PM_OBJ, 0, st));
    TK(reduce_objective(w.obj, w.plan3.grid, 0.0, out_dev, st));
    return NTF_OK;
}

// Extrapolated block-MM sweep for Tucker (Section "Going beyond: Majorization-Minimization
// with Extrapolation", item (ii)): the core, then modes 1..3; each block is moved to its
// extrapolated point just before its update (it depends only on the incoming iterate and the
// previous one), B3 / the mode-3 reconstruction use that block and the current others, and it
// is the multiplicative pre-factor.  The objective of the incoming iterate (when asked for)
// comes from a rows pass over the unextrapolated blocks.
int tucker_run_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                      float *const *factors, float *core_prev, float *const *factors_prev, float alpha, float cap,
                      float delta, const ntf_opts &o, double *objective_dev, cudaStream_t st) {
    if (!core_dims || !core || !factors || !core_prev || !factors_prev)
        return ctx_fail(ctx, NTF_ERR_ARG, "core_dims, core, factors and their previous iterates are required");
    if (X->order != 3) return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker kernels implement order 3");
    for (int n = 0; n < 3; ++n) {
        if (!factors[n] || !factors_prev[n]) return ctx_fail(ctx, NTF_ERR_ARG, "factor is NULL");
        if (core_dims[n] < 1 || core_dims[n] > 64)
            return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "core dimensions must lie in 1..64");
        if (core_dims[n] > X->dims[n]) return ctx_fail(ctx, NTF_ERR_SHAPE, "core dimension exceeds tensor dimension");
    }
    TuckerWs w{};
    int rc = setup(ctx, X, core_dims, false, w, o, beta, st);
    if (rc) return rc;
    const float eps = (float)o.eps;
    const int64_t Jc = (int64_t)w.J1 * w.J2 * w.J3;
    const int64_t n1 = (int64_t)w.I1 * w.J1, n2 = (int64_t)w.I2 * w.J2, n3 = (int64_t)w.I3 * w.J3;
    bool ok = true;
    Blocks hat{};
    hat.G = wsf(ctx, "tkXG", Jc, ok);
    hat.A1 = wsf(ctx, "tkXA1", n1, ok);
    hat.A2 = wsf(ctx, "tkXA2", n2, ok);
    hat.A3p = wsf(ctx, "tkXA3", (int64_t)w.I3 * w.RP, ok);
    float *E3 = wsf(ctx, "tkXE3", n3, ok);
    float *D = wsf(ctx, "tkXD", std::max(std::max(Jc, n1), std::max(n2, n3)), ok);
    double *part = (double *)ctx_ws(ctx, "tkXpart", sizeof(double) * XB);
    if (!ok || !part) return ctx_fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    auto extrap = [&](const float *A, float *Aprev, int64_t n, float *E) -> int {
        extrap_flat_prep_kernel<<<XB, 256, 0, st>>>(A, Aprev, D, n, part);
        TK(cudaGetLastError());
        extrap_flat_apply_kernel<<<XB, 256, 0, st>>>(A, D, n, part, alpha, cap, delta, eps, E);
        TK(cudaGetLastError());
        return NTF_OK;
    };
    if ((rc = load_blocks(ctx, w, core, factors, w.cur, st))) return rc;
    if (objective_dev) {
        if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
        if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, true, st))) return rc;
        TK(reduce_objective(w.obj, w.obj_n, 0.0, objective_dev, st));
    }
    // core block at its extrapolated point
    if ((rc = extrap(w.cur.G, core_prev, Jc, hat.G))) return rc;
    Blocks b = w.cur;
    b.G = hat.G;
    if ((rc = build_b3(ctx, w, b, w.Brec, st))) return rc;
    if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, false, st))) return rc;
    if ((rc = contract_from_w(ctx, w, 0, w.cur, w.Wn, w.num, st))) return rc;
    if ((rc = contract_from_w(ctx, w, 0, w.cur, w.Wd, w.den, st))) return rc;
    if ((rc = apply_mu(ctx, w, hat.G, w.cur.G, Jc, beta, eps, nullptr, nullptr, nullptr, st))) return rc;
    // modes 1 and 2
    for (int blk = 1; blk <= 2; ++blk) {
        float *A = blk == 1 ? w.cur.A1 : w.cur.A2;
        float *Ah = blk == 1 ? hat.A1 : hat.A2;
        if ((rc = extrap(A, factors_prev[blk - 1], blk == 1 ? n1 : n2, Ah))) return rc;
        b = w.cur;
        if (blk == 1) b.A1 = Ah; else b.A2 = Ah;
        if ((rc = build_b3(ctx, w, b, w.Brec, st))) return rc;
        if ((rc = rows_pass(ctx, w, X, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, false, st))) return rc;
        if ((rc = contract_from_w(ctx, w, blk, w.cur, w.Wn, w.num, st))) return rc;
        if ((rc = contract_from_w(ctx, w, blk, w.cur, w.Wd, w.den, st, /*same_blocks=*/true))) return rc;
        if ((rc = apply_mu(ctx, w, Ah, A, blk == 1 ? n1 : n2, beta, eps, nullptr, nullptr, nullptr, st))) return rc;
    }
    // mode 3: extrapolated on the unpadded block, then padded
    if ((rc = extrap(factors[2], factors_prev[2], n3, E3))) return rc;
    pad_cols_kernel<<<nblk((int64_t)w.I3 * w.RP), 256, 0, st>>>(E3, w.I3, w.J3, w.RP, hat.A3p);
    TK(cudaGetLastError());
    if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
    if ((rc = mode3_pass(ctx, w, X, o, beta, w.Brec, hat.A3p, w.Brec, w.Brec, false, st))) return rc;
    MuEpiArgs e{};
    e.pn = w.pn3; e.pd = w.pd3; e.n_parts = w.parts3; e.rows = w.I3; e.RP = w.RP; e.R = w.J3;
    e.pre = hat.A3p; e.out = w.cur.A3p; e.beta = beta; e.gamma = mu_gamma(beta); e.eps = eps;
    TK(mu_epilogue(e, st));
    TK(cudaMemcpyAsync(core, w.cur.G, sizeof(float) * Jc, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(factors[0], w.cur.A1, sizeof(float) * n1, cudaMemcpyDeviceToDevice, st));
    TK(cudaMemcpyAsync(factors[1], w.cur.A2, sizeof(float) * n2, cudaMemcpyDeviceToDevice, st));
    unpad_cols_kernel<<<nblk(n3), 256, 0, st>>>(w.cur.A3p, w.I3, w.J3, w.RP, factors[2]);
    TK(cudaGetLastError());
    return NTF_OK;
}

// ------------------------------------------------------------------ order N >= 4
// The N modes are cut into three runs of consecutive modes [0, a), [a, b), [b, N); X and the
// core (both row-major) are then 3-way with the runs' products as extents, and a run of several
// modes has the Kronecker product of its factors as its 3-way factor.  The core block and
// every mode alone in its run are the 3-way blocks (same passes, GEMMs and updates); a mode
// inside a longer run takes the run's 3-way contraction (Num, Den over the merged row and column
// indices) and folds it against the run's other factors -- the Tucker factor contraction of
// Section 6.2 over the merged indices -- then the run's Kronecker factor is rebuilt.
namespace {

struct TNWay {
    int N;
    int gb[3], ge[3], view[8];
    int64_t dims3[3], cdims3[3];
    int I[8], J[8];
    ntf_tensor X3;
    float *A[8], *At[8], *C1[8], *C2[8];  // own blocks of the modes in runs of several modes
    float *numn, *denn, *S, *Sd;
};

bool tn_single(const TNWay &t, int v) { return t.ge[v] - t.gb[v] == 1; }

float *slot(Blocks &b, int v) { return v == 0 ? b.A1 : v == 1 ? b.A2 : b.A3p; }

int tn_split(ntf_ctx *ctx, const ntf_tensor *X, const int64_t *cd, const ntf_opts &o, float beta, int &a, int &b) {
    const int N = X->order;
    auto fits = [&](int ca, int cb, double *cost) {
        double e[3] = {1, 1, 1}, c[3] = {1, 1, 1};
        for (int m = 0; m < N; ++m) {
            const int v = m < ca ? 0 : m < cb ? 1 : 2;
            e[v] *= (double)X->dims[m];
            c[v] *= (double)cd[m];
        }
        if (c[2] > 64 || e[0] * e[1] >= 2147483648.0 || e[2] >= 2147483648.0 || c[0] * c[1] * c[2] >= 2147483648.0)
            return false;
        const bool tc = o.precision != NTF_PREC_FP32 && c[2] <= 32 && cp3_tc_eligible(32, (int)e[2], X->values);
        const int rp = tc ? 32 : rank_pad((int)c[2]);
        const double tj = rp == 64 ? 64.0 : 128.0;
        const double pass = e[0] * std::ceil(e[1] / tj) * tj * std::ceil(e[2] / 64.0) * 64.0 * rp * 6.0;
        const double gemms = 2.0 * e[0] * e[1] * c[2] * (c[0] + 3.0 * c[1]);
        *cost = pass / (tc ? 8.0 : 1.0) + gemms;
        return true;
    };
    double cost = 0.0, best = -1.0;
    if (o.merge) {
        a = o.merge / 16;
        b = o.merge % 16;
        if (!(1 <= a && a < b && b <= N - 1))
            return ctx_fail(ctx, NTF_ERR_ARG, "merge does not split the modes into three runs");
        if (!fits(a, b, &cost))
            return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "the requested cut needs a last-run core extent <= 64");
        return NTF_OK;
    }
    for (int ca = 1; ca <= N - 2; ++ca)
        for (int cb = ca + 1; cb <= N - 1; ++cb)
            if (fits(ca, cb, &cost) && (best < 0.0 || cost < best)) {
                best = cost;
                a = ca;
                b = cb;
            }
    if (best < 0.0)
        return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "no cut of the modes has a last-run core extent <= 64");
    return NTF_OK;
}

KronArgs tn_kron(const TNWay &t, int v, float *const *B, float *out, int ld) {
    KronArgs k{};
    k.M = t.ge[v] - t.gb[v];
    for (int j = 0; j < k.M; ++j) {
        k.L[j] = B[t.gb[v] + j];
        k.I[j] = t.I[t.gb[v] + j];
        k.J[j] = t.J[t.gb[v] + j];
    }
    k.rows = (int)t.dims3[v];
    k.cols = (int)t.cdims3[v];
    k.ld = ld;
    k.out = out;
    return k;
}

int tn_build(ntf_ctx *ctx, const TNWay &t, int v, float *const *B, float *out, int ld, cudaStream_t st) {
    const KronArgs k = tn_kron(t, v, B, out, ld);
    kron_build_kernel<<<nblk((int64_t)k.rows * ld), 256, 0, st>>>(k);
    TK(cudaGetLastError());
    return NTF_OK;
}

int tn_fold(ntf_ctx *ctx, const TNWay &t, int n, const float *S, int ld, float *const *B, float *out,
            cudaStream_t st) {
    const int v = t.view[n];
    const KronArgs k = tn_kron(t, v, B, nullptr, ld);
    KronFoldArgs f{};
    f.S = S;
    f.ld = ld;
    for (int j = 0; j < k.M; ++j) {
        f.L[j] = k.L[j];
        f.I[j] = k.I[j];
        f.J[j] = k.J[j];
    }
    f.M = k.M;
    f.n = n - t.gb[v];
    f.out = out;
    kron_fold_kernel<<<(unsigned)((int64_t)t.I[n] * t.J[n]), 256, 0, st>>>(f);
    TK(cudaGetLastError());
    return NTF_OK;
}

int tn_setup(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *cd, bool jcomm, const ntf_opts &o,
             TNWay &t, TuckerWs &w) {
    t.N = X->order;
    int a = 0, b = 0;
    int rc = tn_split(ctx, X, cd, o, beta, a, b);
    if (rc) return rc;
    t.gb[0] = 0, t.ge[0] = a, t.gb[1] = a, t.ge[1] = b, t.gb[2] = b, t.ge[2] = t.N;
    for (int v = 0; v < 3; ++v) {
        t.dims3[v] = t.cdims3[v] = 1;
        for (int m = t.gb[v]; m < t.ge[v]; ++m) {
            t.view[m] = v;
            t.I[m] = (int)X->dims[m];
            t.J[m] = (int)cd[m];
            t.dims3[v] *= X->dims[m];
            t.cdims3[v] *= cd[m];
        }
    }
    t.X3 = *X;
    t.X3.order = 3;
    t.X3.dims = t.dims3;
    if ((rc = setup(ctx, &t.X3, t.cdims3, jcomm, w, o, beta))) return rc;
    bool ok = true;
    int64_t mx = 1;
    static const char *nm[4] = {"tnA", "tnAt", "tnC1", "tnC2"};
    for (int m = 0; m < t.N; ++m) {
        t.A[m] = t.At[m] = t.C1[m] = t.C2[m] = nullptr;
        if (tn_single(t, t.view[m])) continue;
        const int64_t n = (int64_t)t.I[m] * t.J[m];
        mx = std::max(mx, n);
        float **dst[4] = {&t.A[m], &t.At[m], &t.C1[m], &t.C2[m]};
        for (int q = 0; q < (jcomm ? 4 : 1); ++q) {
            const std::string name = std::string(nm[q]) + std::to_string(m);
            *dst[q] = wsf(ctx, name.c_str(), n, ok);
        }
    }
    t.numn = wsf(ctx, "tnNum", mx, ok);
    t.denn = wsf(ctx, "tnDen", mx, ok);
    t.S = wsf(ctx, "tnS", t.dims3[2] * w.RP, ok);
    t.Sd = wsf(ctx, "tnSd", t.dims3[2] * w.RP, ok);
    if (!ok) return ctx_fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    return NTF_OK;
}

// the user's core and factors into the view blocks (and the runs' own blocks)
int tn_load(ntf_ctx *ctx, TNWay &t, TuckerWs &w, const float *core, const float *const *factors, cudaStream_t st) {
    TK(cudaMemcpyAsync(w.cur.G, core, sizeof(float) * t.cdims3[0] * t.cdims3[1] * t.cdims3[2],
                       cudaMemcpyDeviceToDevice, st));
    for (int v = 0; v < 3; ++v) {
        const int ld = v == 2 ? w.RP : (int)t.cdims3[v];
        if (tn_single(t, v)) {
            const int m = t.gb[v];
            if (v < 2) {
                TK(cudaMemcpyAsync(slot(w.cur, v), factors[m], sizeof(float) * t.I[m] * t.J[m],
                                   cudaMemcpyDeviceToDevice, st));
            } else {
                pad_cols_kernel<<<nblk((int64_t)t.I[m] * w.RP), 256, 0, st>>>(factors[m], t.I[m], t.J[m], w.RP,
                                                                            w.cur.A3p);
                TK(cudaGetLastError());
            }
            continue;
        }
        for (int m = t.gb[v]; m < t.ge[v]; ++m)
            TK(cudaMemcpyAsync(t.A[m], factors[m], sizeof(float) * t.I[m] * t.J[m], cudaMemcpyDeviceToDevice, st));
        int rc = tn_build(ctx, t, v, t.A, slot(w.cur, v), ld, st);
        if (rc) return rc;
    }
    return NTF_OK;
}

int tn_store(ntf_ctx *ctx, TNWay &t, TuckerWs &w, float *core, float *const *factors, cudaStream_t st) {
    TK(cudaMemcpyAsync(core, w.cur.G, sizeof(float) * t.cdims3[0] * t.cdims3[1] * t.cdims3[2],
                       cudaMemcpyDeviceToDevice, st));
    for (int m = 0; m < t.N; ++m) {
        const int v = t.view[m];
        const int64_t n = (int64_t)t.I[m] * t.J[m];
        if (!tn_single(t, v)) {
            TK(cudaMemcpyAsync(factors[m], t.A[m], sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        } else if (v < 2) {
            TK(cudaMemcpyAsync(factors[m], slot(w.cur, v), sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            unpad_cols_kernel<<<nblk(n), 256, 0, st>>>(w.cur.A3p, t.I[m], t.J[m], w.RP, factors[m]);
            TK(cudaGetLastError());
        }
    }
    return NTF_OK;
}

// mode n inside a run of several modes: Num / Den folded from the run's contraction (S, Sd with
// row stride ld) against fold blocks Bn / Bd, MU from pre into out, chi copies when c1 is given
int tn_run_update(ntf_ctx *ctx, TNWay &t, int n, const float *S, const float *Sd, int ld, float *const *Bn,
                  float *const *Bd, const float *pre, float *out, float *c1, float *c2, float beta, float eps,
                  cudaStream_t st) {
    int rc = tn_fold(ctx, t, n, S, ld, Bn, t.numn, st);
    if (rc) return rc;
    if ((rc = tn_fold(ctx, t, n, Sd, ld, Bd, t.denn, st))) return rc;
    const int64_t cnt = (int64_t)t.I[n] * t.J[n];
    mu_plain_kernel<<<nblk(cnt), 256, 0, st>>>(pre, t.numn, t.denn, cnt, mu_gamma(beta), eps, out);
    TK(cudaGetLastError());
    if (c1) {
        chi_kernel<<<nblk(cnt), 256, 0, st>>>(out, pre, cnt, beta, c1, c2);
        TK(cudaGetLastError());
    }
    return NTF_OK;
}

}  // namespace

int tucker_nway_run(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                    float *const *factors, const ntf_opts &o, double *objective_dev, cudaStream_t st, bool jcomm) {
    TNWay t{};
    TuckerWs w{};
    int rc = tn_setup(ctx, X, beta, core_dims, jcomm, o, t, w);
    if (rc) return rc;
    if ((rc = tn_load(ctx, t, w, core, factors, st))) return rc;
    const float eps = (float)o.eps;
    const int64_t Jc = t.cdims3[0] * t.cdims3[1] * t.cdims3[2];
    const int64_t n3p = t.dims3[2] * w.RP;
    if (!jcomm) {
        // core block (the pass also yields D_beta of the incoming iterate)
        if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
        if ((rc = rows_pass(ctx, w, &t.X3, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, objective_dev != nullptr,
                            st)))
            return rc;
        if (objective_dev) TK(reduce_objective(w.obj, w.obj_n, 0.0, objective_dev, st));
        if ((rc = contract_from_w(ctx, w, 0, w.cur, w.Wn, w.num, st))) return rc;
        if ((rc = contract_from_w(ctx, w, 0, w.cur, w.Wd, w.den, st))) return rc;
        if ((rc = apply_mu(ctx, w, w.cur.G, w.cur.G, Jc, beta, eps, nullptr, nullptr, nullptr, st))) return rc;
        for (int n = 0; n < t.N; ++n) {
            const int v = t.view[n];
            const bool single = tn_single(t, v);
            if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
            if (v < 2) {
                if ((rc = rows_pass(ctx, w, &t.X3, o, beta, w.Brec, w.cur.A3p, w.cur.A3p, w.cur.A3p, false, st)))
                    return rc;
                if ((rc = contract_from_w(ctx, w, v + 1, w.cur, w.Wn, w.num, st))) return rc;
                if ((rc = contract_from_w(ctx, w, v + 1, w.cur, w.Wd, w.den, st, /*same_blocks=*/true))) return rc;
                if (single) {
                    float *A = slot(w.cur, v);
                    if ((rc = apply_mu(ctx, w, A, A, (int64_t)t.I[n] * t.J[n], beta, eps, nullptr, nullptr, nullptr,
                                       st)))
                        return rc;
                    continue;
                }
                const int ld = (int)t.cdims3[v];
                if ((rc = tn_run_update(ctx, t, n, w.num, w.den, ld, t.A, t.A, t.A[n], t.A[n], nullptr, nullptr,
                                        beta, eps, st)))
                    return rc;
                if ((rc = tn_build(ctx, t, v, t.A, slot(w.cur, v), ld, st))) return rc;
                continue;
            }
            if ((rc = mode3_pass(ctx, w, &t.X3, o, beta, w.Brec, w.cur.A3p, w.Brec, w.Brec, false, st))) return rc;
            if (single) {
                MuEpiArgs e{};
                e.pn = w.pn3; e.pd = w.pd3; e.n_parts = w.parts3; e.rows = w.I3; e.RP = w.RP; e.R = w.J3;
                e.pre = w.cur.A3p; e.out = w.cur.A3p; e.beta = beta; e.gamma = mu_gamma(beta); e.eps = eps;
                TK(mu_epilogue(e, st));
                continue;
            }
            sum_parts_kernel<<<nblk(n3p), 256, 0, st>>>(w.pn3, w.parts3, n3p, t.S);
            TK(cudaGetLastError());
            sum_parts_kernel<<<nblk(n3p), 256, 0, st>>>(w.pd3, w.parts3, n3p, t.Sd);
            TK(cudaGetLastError());
            if ((rc = tn_run_update(ctx, t, n, t.S, t.Sd, w.RP, t.A, t.A, t.A[n], t.A[n], nullptr, nullptr, beta, eps,
                                    st)))
                return rc;
            if ((rc = tn_build(ctx, t, 2, t.A, w.cur.A3p, w.RP, st))) return rc;
        }
        return tn_store(ctx, t, w, core, factors, st);
    }
    // J-CoMM (Algorithm 2): reference, chi1 and chi2 copies of every block
    if ((rc = copy_blocks(ctx, w, w.cur, w.ref, st))) return rc;
    if ((rc = copy_blocks(ctx, w, w.cur, w.t1, st))) return rc;
    if ((rc = copy_blocks(ctx, w, w.cur, w.t2, st))) return rc;
    for (int m = 0; m < t.N; ++m) {
        if (tn_single(t, t.view[m])) continue;
        const size_t bytes = sizeof(float) * t.I[m] * t.J[m];
        TK(cudaMemcpyAsync(t.At[m], t.A[m], bytes, cudaMemcpyDeviceToDevice, st));
        TK(cudaMemcpyAsync(t.C1[m], t.A[m], bytes, cudaMemcpyDeviceToDevice, st));
        TK(cudaMemcpyAsync(t.C2[m], t.A[m], bytes, cudaMemcpyDeviceToDevice, st));
    }
    if ((rc = build_b3(ctx, w, w.ref, w.Brec, st))) return rc;
    for (int l = 0; l < o.inner_L; ++l) {
        const bool obj = (l == 0) && objective_dev;
        if ((rc = rows_pass(ctx, w, &t.X3, o, beta, w.Brec, w.ref.A3p, w.t1.A3p, w.t2.A3p, obj, st))) return rc;
        if (obj) TK(reduce_objective(w.obj, w.obj_n, 0.0, objective_dev, st));
        if ((rc = contract_from_w(ctx, w, 0, w.t1, w.Wn, w.num, st))) return rc;
        if ((rc = contract_from_w(ctx, w, 0, w.t2, w.Wd, w.den, st))) return rc;
        if ((rc = apply_mu(ctx, w, w.ref.G, w.cur.G, Jc, beta, eps, w.ref.G, w.t1.G, w.t2.G, st))) return rc;
        bool m3_done = false;
        for (int n = 0; n < t.N; ++n) {
            const int v = t.view[n];
            const bool single = tn_single(t, v);
            if (v < 2) {
                if ((rc = contract_from_w(ctx, w, v + 1, w.t1, w.Wn, w.num, st))) return rc;
                if ((rc = contract_from_w(ctx, w, v + 1, w.t2, w.Wd, w.den, st))) return rc;
                if (single) {
                    float *At = slot(w.ref, v);
                    if ((rc = apply_mu(ctx, w, At, slot(w.cur, v), (int64_t)t.I[n] * t.J[n], beta, eps, At,
                                       slot(w.t1, v), slot(w.t2, v), st)))
                        return rc;
                    continue;
                }
                const int ld = (int)t.cdims3[v];
                if ((rc = tn_run_update(ctx, t, n, w.num, w.den, ld, t.C1, t.C2, t.At[n], t.A[n], t.C1[n], t.C2[n],
                                        beta, eps, st)))
                    return rc;
                if ((rc = tn_build(ctx, t, v, t.C1, slot(w.t1, v), ld, st))) return rc;
                if ((rc = tn_build(ctx, t, v, t.C2, slot(w.t2, v), ld, st))) return rc;
                continue;
            }
            if (!m3_done) {
                // the mode-3 contraction depends on the core and the first two runs only, which
                // are final for this sweep: one pass serves every mode of the last run
                if ((rc = build_b3(ctx, w, w.t1, w.Bn, st))) return rc;
                if ((rc = build_b3(ctx, w, w.t2, w.Bd, st))) return rc;
                if ((rc = mode3_pass(ctx, w, &t.X3, o, beta, w.Brec, w.ref.A3p, w.Bn, w.Bd, false, st))) return rc;
                m3_done = true;
                if (!single) {
                    sum_parts_kernel<<<nblk(n3p), 256, 0, st>>>(w.pn3, w.parts3, n3p, t.S);
                    TK(cudaGetLastError());
                    sum_parts_kernel<<<nblk(n3p), 256, 0, st>>>(w.pd3, w.parts3, n3p, t.Sd);
                    TK(cudaGetLastError());
                }
            }
            if (single) {
                MuEpiArgs e{};
                e.pn = w.pn3; e.pd = w.pd3; e.n_parts = w.parts3; e.rows = w.I3; e.RP = w.RP; e.R = w.J3;
                e.pre = w.ref.A3p; e.out = w.cur.A3p; e.ref = w.ref.A3p; e.chi1_out = w.t1.A3p; e.chi2_out = w.t2.A3p;
                e.beta = beta; e.gamma = mu_gamma(beta); e.eps = eps;
                TK(mu_epilogue(e, st));
                continue;
            }
            if ((rc = tn_run_update(ctx, t, n, t.S, t.Sd, w.RP, t.C1, t.C2, t.At[n], t.A[n], t.C1[n], t.C2[n], beta,
                                    eps, st)))
                return rc;
            if (n == t.ge[2] - 1) {
                if ((rc = tn_build(ctx, t, 2, t.C1, w.t1.A3p, w.RP, st))) return rc;
                if ((rc = tn_build(ctx, t, 2, t.C2, w.t2.A3p, w.RP, st))) return rc;
            }
        }
    }
    return tn_store(ctx, t, w, core, factors, st);
}

int tucker_plan_cut(const ntf_tensor *X, const int64_t *core_dims, const ntf_opts &o, float beta, int &a, int &b) {
    for (int n = 0; n < X->order; ++n)
        if (core_dims[n] < 1 || core_dims[n] > 64 || core_dims[n] > X->dims[n]) return NTF_ERR_UNSUPPORTED;
    return tn_split(nullptr, X, core_dims, o, beta, a, b);
}

int tucker_nway_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, const float *core,
                         const float *const *factors, const ntf_opts &o, double *out_dev, cudaStream_t st) {
    TNWay t{};
    TuckerWs w{};
    ntf_opts o32 = o;
    o32.precision = NTF_PREC_FP32;
    int rc = tn_setup(ctx, X, beta, core_dims, false, o32, t, w);
    if (rc) return rc;
    if ((rc = tn_load(ctx, t, w, core, factors, st))) return rc;
    if ((rc = build_b3(ctx, w, w.cur, w.Brec, st))) return rc;
    Cp3Args a = base_args(&t.X3, w, o, beta);
    a.rrow = w.Brec;
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = w.cur.A3p;
    a.n_jt = w.plan3.n_jt;
    a.n_kb = w.plan3.n_kb;
    a.n_is = w.plan3.n_is;
    TK(cp3_launch(w.plan3, a, PM_OBJ, 0, st));
    TK(reduce_objective(w.obj, w.plan3.grid, 0.0, out_dev, st));
    return NTF_OK;
}

void tucker_release(ntf_ctx *) {}

}  // namespace ntf
