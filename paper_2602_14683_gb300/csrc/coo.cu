// Sparse COO tensors, Section 6.3 ("For sparse tensors"): numerators are sums over the
// stored entries only.  Under KL (beta = 1), Q == 1 makes every denominator the product of
// column sums of the other factors; at other beta the denominators come from a dense pass
// that reads no X (ntf_api.cu), and this file supplies the stored-entry numerators.
//
// Preprocessing (once per tensor, cached by coordinate pointers and sizes):
//   * per mode n a stable permutation pi_n ordering the entries by i_n (LSD radix sort
//     with 11-bit digits; each digit pass is a stable counting sort), bit-identical to a
//     stable sort;
//   * per mode a copy of all coordinates and values in pi_n order (coalesced streams);
//   * per mode a table of work units: each unit is a run of at most UNIT consecutive
//     sorted entries that share the same i_n, so heavy (Zipf) rows are split evenly.
// Pass for mode n (one warp per unit, lane = rank component r, r + 32):
//   Xhat_e = sum_r prod_m A^(m)[i_m(e), r]  (warp shuffle sum),  p_e = x_e / max(Xhat_e, eps)
//   partial[unit][r] = sum_{e in unit} p_e prod_{m != n} B^(m)[i_m(e), r]
// and a fixed-order per-row sum of the unit partials gives Num^(n) deterministically.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ntf_coo.h"
#include "ntf_tucker.h"

namespace ntf {

constexpr int UNIT = 128;
constexpr int DIGIT_BITS = 11;
constexpr int BUCKETS = 1 << DIGIT_BITS;
constexpr int SORT_CHUNK = 2048;

// ---------------------------------------------------------------- stable counting sort
__global__ void digit_hist_kernel(const int32_t *key, const int32_t *perm, int64_t nnz, int shift, int nchunks,
                                  int *hist) {
    __shared__ int cnt[BUCKETS];
    for (int b = threadIdx.x; b < BUCKETS; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int t = threadIdx.x; t < SORT_CHUNK; t += blockDim.x) {
        const int64_t pos = c0 + t;
        if (pos < nnz) {
            const int32_t e = perm ? perm[pos] : (int32_t)pos;
            atomicAdd(&cnt[(key[e] >> shift) & (BUCKETS - 1)], 1);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < BUCKETS; b += blockDim.x) hist[(int64_t)b * nchunks + blockIdx.x] = cnt[b];
}

// exclusive scan of n ints, one CTA of 1024 threads (contiguous segments, then a block scan)
__global__ void scan_kernel(const int *in, int64_t n, int *out) {
    __shared__ int sums[1024];
    const int t = threadIdx.x;
    const int64_t seg = (n + 1023) / 1024;
    const int64_t b = t * seg, e = b + seg < n ? b + seg : n;
    int s = 0;
    for (int64_t q = b; q < e; ++q) s += in[q];
    sums[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int run = t ? sums[t - 1] : 0;
    for (int64_t q = b; q < e; ++q) {
        const int v = in[q];
        out[q] = run;
        run += v;
    }
}

// stable placement: one warp walks its chunk in order; equal digits within a batch of 32
// get their rank from __match_any_sync, and a shared running count carries across batches
__global__ void digit_place_kernel(const int32_t *key, const int32_t *perm_in, int64_t nnz, int shift, int nchunks,
                                   const int *base, int32_t *perm_out) {
    __shared__ int run[BUCKETS];
    const int lane = threadIdx.x;
    for (int b = lane; b < BUCKETS; b += 32) run[b] = 0;
    __syncwarp();
    const int64_t c0 = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int t = 0; t < SORT_CHUNK; t += 32) {
        const int64_t pos = c0 + t + lane;
        const bool valid = pos < nnz;
        int32_t e = 0;
        int d = -1 - lane;  // distinct dummy digits for invalid lanes
        if (valid) {
            e = perm_in ? perm_in[pos] : (int32_t)pos;
            d = (key[e] >> shift) & (BUCKETS - 1);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int r0 = 0;
        if (valid) r0 = run[d];
        __syncwarp();
        if (valid) {
            perm_out[base[(int64_t)d * nchunks + blockIdx.x] + r0 + rank] = e;
            if (rank == 0) run[d] = r0 + __popc(peers);
        }
        __syncwarp();
    }
}

__global__ void count_rows_kernel(const int32_t *key, int64_t nnz, int *cnt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) atomicAdd(&cnt[key[t]], 1);
}

__global__ void gather_i32_kernel(const int32_t *src, const int32_t *perm, int64_t n, int32_t *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[perm[t]];
}
__global__ void gather_f32_kernel(const float *src, const int32_t *perm, int64_t n, float *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[perm[t]];
}

static unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// perm_out = stable order of keys (values in [0, range)); tmp: nnz ints; hist/scan scratch
static cudaError_t stable_sort(const int32_t *keys, int64_t nnz, int64_t range, int32_t *perm_out, int32_t *tmp,
                               int *hist, int *scan, cudaStream_t st, int *launches) {
    int bits = 1;
    while (((int64_t)1 << bits) < range) ++bits;
    const int passes = (bits + DIGIT_BITS - 1) / DIGIT_BITS;
    const int nchunks = (int)((nnz + SORT_CHUNK - 1) / SORT_CHUNK);
    const int32_t *cur = nullptr;  // identity
    // ping-pong so that the last pass writes perm_out
    int32_t *bufs[2] = {(passes % 2) ? perm_out : tmp, (passes % 2) ? tmp : perm_out};
    for (int p = 0; p < passes; ++p) {
        const int shift = p * DIGIT_BITS;
        int32_t *out = bufs[p % 2];
        digit_hist_kernel<<<nchunks, 256, 0, st>>>(keys, cur, nnz, shift, nchunks, hist);
        scan_kernel<<<1, 1024, 0, st>>>(hist, (int64_t)BUCKETS * nchunks, scan);
        digit_place_kernel<<<nchunks, 32, 0, st>>>(keys, cur, nnz, shift, nchunks, scan, out);
        *launches += 3;
        cur = out;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------------- the pass
struct CooPassArgs {
    const int32_t *sidx;  // [N][nnz] coordinates in this mode's order
    const float *sval;    // [nnz]
    int64_t nnz;
    int N, n, RP;
    const float *rec[8];  // factors that rebuild Xhat, [I_m][RP]
    const float *num[8];  // factors of the numerator contraction
    const int32_t *unit_beg, *unit_end;
    int n_units;
    float eps;
    int bkind;     // beta class (BK_KL: p = x / Xhat)
    float beta;
    float *part;   // [n_units][RP]
    double *obj;   // per-warp objective partials or null
};

template <int RG>  // rank registers per lane: RP = 32 * RG
__global__ void __launch_bounds__(256) coo_pass_kernel(const CooPassArgs a) {
    const int lane = threadIdx.x & 31;
    const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= a.n_units) return;
    const int beg = a.unit_beg[u], end = a.unit_end[u];
    float acc[RG];
#pragma unroll
    for (int g = 0; g < RG; ++g) acc[g] = 0.0f;
    float objf = 0.0f;
    for (int t = beg; t < end; ++t) {
        float zall[RG], zex[RG];
#pragma unroll
        for (int g = 0; g < RG; ++g) zall[g] = 1.0f, zex[g] = 1.0f;
        for (int m = 0; m < a.N; ++m) {
            const int64_t row = (int64_t)__ldg(a.sidx + (int64_t)m * a.nnz + t) * a.RP;
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                zall[g] *= __ldg(a.rec[m] + row + lane + 32 * g);
                if (m != a.n) zex[g] *= __ldg(a.num[m] + row + lane + 32 * g);
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int g = 0; g < RG; ++g) s += zall[g];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float x = __ldg(a.sval + t);
        const float y = fmaxf(s, a.eps);
        float p;
        if (a.bkind == BK_KL) {
            p = __fdiv_rn(x, y);
        } else {  // P = x Xhat^(beta - 2) (Section 4.1); Q is the dense pass's
            float q;
            pq_powers(a.bkind, a.beta, x, y, p, q);
        }
#pragma unroll
        for (int g = 0; g < RG; ++g) acc[g] = fmaf(p, zex[g], acc[g]);
        if (a.obj && lane == 0 && x > 0.0f) {
            float d;
            if (a.bkind == BK_KL) {
                // x log(x / y) - x, the stored-entry part of d_1 (the + y part is summed in closed form)
                const float r = __fdiv_rn(y, x);
                if (r > 1e-4f && r < 1e4f) {
                    const float tt = r - 1.0f;
                    d = x * (tt - log1pf(tt)) - y;
                } else {
                    d = x * (logf(x) - logf(y)) - x;
                }
            } else {
                // d_beta(x | y) - d_beta(0 | y): the dense pass adds d_beta(0 | y) = y^beta / beta
                // over every entry, stored or not
                d = dbeta_stable(a.bkind, a.beta, x, y) - dbeta_stable(a.bkind, a.beta, 0.0f, y);
            }
            objf += d;
        }
    }
#pragma unroll
    for (int g = 0; g < RG; ++g) a.part[(int64_t)u * a.RP + lane + 32 * g] = acc[g];
    if (a.obj && lane == 0) a.obj[u] = (double)objf;
}

// Rank 32: one warp per unit; eight lanes per stored entry, four entries of the unit at a
// time (lane group g = lane / 8 takes entries g, g + 4, ...), lane l holding ranks
// 4 (l % 8) .. 4 (l % 8) + 3.  Each factor row other than mode n's is then one 128-byte
// gather per entry (eight 16-byte loads that share a line), the unit's own mode-n row is
// read once, Xhat = sum_r z[r] A^(n)[i_n, r] is a three-step shuffle within the group,
// p = x / max(Xhat, eps) and the lane adds p z[r] for its ranks.  At the end of the unit
// the four groups are added (two shuffle steps, a fixed order).  The reconstruction and
// the numerator use the same factors (beta = 1: block MM, and J-CoMM at the reference).
template <int NMAX>  // order N <= NMAX
__global__ void __launch_bounds__(256) coo_pass32_kernel(const CooPassArgs a) {
    const int lane = threadIdx.x & 31, grp = lane >> 3, sub = lane & 7;
    const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= a.n_units) return;  // warp-uniform
    const int beg = a.unit_beg[u], end = a.unit_end[u];
    const int64_t in = (int64_t)__ldg(a.sidx + (int64_t)a.n * a.nnz + beg) * 32;
    const float4 an = __ldg(reinterpret_cast<const float4 *>(a.rec[a.n] + in) + sub);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float objf = 0.0f;
    // coordinates and value of this group's entry in the next round, loaded one round ahead
    int nid[NMAX];
    float nx = 0.0f;
    auto load_round = [&](int t0) {
        const int t = t0 + grp;
        const bool v = t < end;
#pragma unroll
        for (int m = 0; m < NMAX; ++m) nid[m] = (v && m < a.N && m != a.n) ? __ldg(a.sidx + (int64_t)m * a.nnz + t) : 0;
        nx = v ? __ldg(a.sval + t) : 0.0f;
    };
    load_round(beg);
    for (int t0 = beg; t0 < end; t0 += 4) {
        const bool v = t0 + grp < end;
        int id[NMAX];
#pragma unroll
        for (int m = 0; m < NMAX; ++m) id[m] = nid[m];
        const float x = nx;
        if (t0 + 4 < end) load_round(t0 + 4);
        float4 z = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
#pragma unroll
        for (int m = 0; m < NMAX; ++m) {
            if (m >= a.N || m == a.n) continue;
            const float4 f = __ldg(reinterpret_cast<const float4 *>(a.rec[m] + (int64_t)id[m] * 32) + sub);
            z.x *= f.x; z.y *= f.y; z.z *= f.z; z.w *= f.w;
        }
        float s = fmaf(z.x, an.x, fmaf(z.y, an.y, fmaf(z.z, an.z, z.w * an.w)));
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        const float y = fmaxf(s, a.eps);
        const float p = v ? __fdiv_rn(x, y) : 0.0f;
        acc.x = fmaf(p, z.x, acc.x); acc.y = fmaf(p, z.y, acc.y);
        acc.z = fmaf(p, z.z, acc.z); acc.w = fmaf(p, z.w, acc.w);
        if (a.obj && v && sub == 0 && x > 0.0f) {
            // x log(x / y) - x, the stored-entry part of d_1 (the + y part is summed in closed form)
            const float rr = __fdiv_rn(y, x);
            float d;
            if (rr > 1e-4f && rr < 1e4f) {
                const float tt = rr - 1.0f;
                d = x * (tt - log1pf(tt)) - y;
            } else {
                d = x * (logf(x) - logf(y)) - x;
            }
            objf += d;
        }
    }
#pragma unroll
    for (int k = 8; k <= 16; k <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, k);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, k);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, k);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, k);
    }
    if (lane < 8) reinterpret_cast<float4 *>(a.part + (int64_t)u * 32)[sub] = acc;
    if (a.obj) {
        double o = (double)objf;
#pragma unroll
        for (int k = 16; k >= 1; k >>= 1) o += __shfl_xor_sync(0xffffffffu, o, k);
        if (lane == 0) a.obj[u] = o;
    }
}

// Num[i][r] = sum of the unit partials of row i (units of a row are consecutive), in two
// fixed-order levels: groups of up to GROUP consecutive units of one row, then the groups of
// a row.  Loads are issued sixteen at a time before their adds.
constexpr int GROUP = 32;

template <typename T>
__device__ __forceinline__ T ordered_sum16(const T *src, int64_t stride, int n) {
    T acc = 0;
    for (int p0 = 0; p0 < n; p0 += 16) {
        T v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = p0 + k < n ? src[(int64_t)(p0 + k) * stride] : T(0);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (p0 + k < n) acc += v[k];
    }
    return acc;
}

__global__ void coo_group_reduce_kernel(const float *part, const int32_t *group_beg, int n_groups, int RP, float *gpart) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_groups * RP) return;
    const int g = (int)(t / RP), r = (int)(t % RP);
    const int b = group_beg[g];
    gpart[t] = ordered_sum16(part + (int64_t)b * RP + r, RP, group_beg[g + 1] - b);
}

__global__ void coo_row_reduce_kernel(const float *gpart, const int32_t *row_groups, int rows, int RP, float *num) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * RP) return;
    const int i = (int)(t / RP), r = (int)(t % RP);
    const int g = row_groups[i];
    num[t] = ordered_sum16(gpart + (int64_t)g * RP + r, RP, row_groups[i + 1] - g);
}

// objective: sum of stored-entry terms + sum_r prod_n colsum(A^(n))_r (Section 6.3), one
// CTA of 1024 threads in a fixed order: thread (s, r) sums the rows i = s mod 32 of rank r
// for each factor, the 32 slices are added in order, and the products over ranks r < R
// are added in rank order after the stored-entry partials.
// the padded factors and their row counts, passed by value (no host-to-device copy per call)
struct CooFactorSet {
    const float *f[8];
    int rows[8];
};

__global__ void __launch_bounds__(1024) coo_obj_finish_kernel(const double *parts, int n, const CooFactorSet fs,
                                                              int N, int R, int RP, double *out) {
    __shared__ double sh[1024];
    __shared__ double prod[64];
    const int t = threadIdx.x, r = t % 32, sl = t / 32;
    // stored-entry partials
    double s = 0.0;
    for (int k0 = t; k0 < n; k0 += 8 * 1024) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = k0 + 1024 * k < n ? parts[k0 + 1024 * k] : 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += v[k];
    }
    sh[t] = s;
    __syncthreads();
    for (int w = 512; w >= 1; w >>= 1) {
        if (t < w) sh[t] += sh[t + w];
        __syncthreads();
    }
    const double stored = sh[0];
    __syncthreads();
    // dense part, 32 ranks at a time
    for (int rb = 0; rb < RP; rb += 32) {
        double pr = 1.0;
        for (int m = 0; m < N; ++m) {
            double c = 0.0;
            const float *f = fs.f[m] + rb + r;
            const int rows = fs.rows[m];
            for (int i0 = sl; i0 < rows; i0 += 8 * 32) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = i0 + 32 * k < rows ? f[(int64_t)(i0 + 32 * k) * RP] : 0.0f;
#pragma unroll
                for (int k = 0; k < 8; ++k) c += (double)v[k];
            }
            sh[t] = c;
            __syncthreads();
            if (sl == 0) {
                double cs = 0.0;
                for (int q = 0; q < 32; ++q) cs += sh[q * 32 + r];
                pr *= cs;
            }
            __syncthreads();
        }
        if (sl == 0) prod[rb + r] = pr;
    }
    __syncthreads();
    if (t == 0) {
        double tot = stored;
        for (int q = 0; q < R; ++q) tot += prod[q];
        *out = tot;
    }
}

// the fixed-order objective total: stored-entry partials plus the dense part from the factors
static cudaError_t obj_finish(const double *parts, int n, const float *const *F, const int64_t *dims, int N, int R,
                              int RP, double *out, cudaStream_t st) {
    CooFactorSet fs{};
    for (int m = 0; m < N; ++m) {
        fs.f[m] = F[m];
        fs.rows[m] = (int)dims[m];
    }
    coo_obj_finish_kernel<<<1, 1024, 0, st>>>(parts, n, fs, N, R, RP, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- cache & driver
namespace {

struct ModeData {
    int32_t *perm = nullptr, *sidx = nullptr, *unit_beg = nullptr, *unit_end = nullptr, *row_units = nullptr;
    int32_t *group_beg = nullptr, *row_groups = nullptr;  // unit groups of one row, GROUP units at most
    float *sval = nullptr;
    int n_units = 0, n_groups = 0;
};

struct CooCache {
    bool valid = false;
    int N = 0;
    int64_t nnz = 0;
    int64_t dims[8] = {0};
    const void *idx[8] = {nullptr};
    const void *vals = nullptr;
    ModeData md[8];
    int max_units = 0, max_groups = 0;
};

std::mutex g_mu;
std::map<const ntf_ctx *, CooCache> g_cache;

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return ctx_fail(ctx, NTF_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

int build_cache(ntf_ctx *ctx, const ntf_tensor *X, CooCache &c, cudaStream_t st) {
    const int N = X->order;
    const int64_t nnz = X->nnz;
    c = CooCache{};
    c.N = N;
    c.nnz = nnz;
    c.vals = X->values;
    for (int m = 0; m < N; ++m) { c.dims[m] = X->dims[m]; c.idx[m] = X->idx[m]; }
    const int nchunks = (int)((nnz + SORT_CHUNK - 1) / SORT_CHUNK) + 1;
    int64_t maxdim = 1;
    for (int m = 0; m < N; ++m) maxdim = X->dims[m] > maxdim ? X->dims[m] : maxdim;
    int *hist = (int *)ctx_ws(ctx, "cooHist", sizeof(int) * (size_t)BUCKETS * nchunks);
    int *scan = (int *)ctx_ws(ctx, "cooScan", sizeof(int) * (size_t)BUCKETS * nchunks);
    int32_t *tmp = (int32_t *)ctx_ws(ctx, "cooTmp", sizeof(int32_t) * (size_t)(nnz + 1));
    int *cnt = (int *)ctx_ws(ctx, "cooCnt", sizeof(int) * (size_t)(maxdim + 1));
    int *off = (int *)ctx_ws(ctx, "cooOff", sizeof(int) * (size_t)(maxdim + 1));
    if (!hist || !scan || !tmp || !cnt || !off) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
    std::vector<int> hoff;
    for (int n = 0; n < N; ++n) {
        ModeData &d = c.md[n];
        std::string tag = std::to_string(n);
        d.perm = (int32_t *)ctx_ws(ctx, ("cooPerm" + tag).c_str(), sizeof(int32_t) * (size_t)(nnz + 1));
        d.sidx = (int32_t *)ctx_ws(ctx, ("cooSidx" + tag).c_str(), sizeof(int32_t) * (size_t)N * (nnz + 1));
        d.sval = (float *)ctx_ws(ctx, ("cooSval" + tag).c_str(), sizeof(float) * (size_t)(nnz + 1));
        if (!d.perm || !d.sidx || !d.sval) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
        int launches = 0;
        if (nnz > 0) {
            CK(stable_sort(X->idx[n], nnz, X->dims[n], d.perm, tmp, hist, scan, st, &launches));
            for (int m = 0; m < N; ++m) {
                gather_i32_kernel<<<nb(nnz), 256, 0, st>>>(X->idx[m], d.perm, nnz, d.sidx + (int64_t)m * nnz);
                ++launches;
            }
            gather_f32_kernel<<<nb(nnz), 256, 0, st>>>(X->values, d.perm, nnz, d.sval);
            ++launches;
        }
        // row offsets in sorted order -> unit table (host side, once per tensor)
        CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(X->dims[n] + 1), st));
        if (nnz > 0) {
            count_rows_kernel<<<nb(nnz), 256, 0, st>>>(X->idx[n], nnz, cnt);
            ++launches;
        }
        scan_kernel<<<1, 1024, 0, st>>>(cnt, X->dims[n] + 1, off);
        ++launches;
        CK(cudaGetLastError());
        ctx_count(ctx, launches);
        hoff.resize((size_t)X->dims[n] + 1);
        CK(cudaMemcpyAsync(hoff.data(), off, sizeof(int) * hoff.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<int32_t> ub, ue, ru(hoff.size());
        for (int64_t i = 0; i < X->dims[n]; ++i) {
            ru[i] = (int32_t)ub.size();
            for (int b = hoff[i]; b < hoff[i + 1]; b += UNIT) {
                ub.push_back(b);
                ue.push_back(b + UNIT < hoff[i + 1] ? b + UNIT : hoff[i + 1]);
            }
        }
        ru[X->dims[n]] = (int32_t)ub.size();
        std::vector<int32_t> gb, rg(ru.size());
        for (int64_t i = 0; i < X->dims[n]; ++i) {
            rg[i] = (int32_t)gb.size();
            for (int u = ru[i]; u < ru[i + 1]; u += GROUP) gb.push_back(u);
        }
        rg[X->dims[n]] = (int32_t)gb.size();
        gb.push_back((int32_t)ub.size());
        d.n_groups = (int)gb.size() - 1;
        c.max_groups = d.n_groups > c.max_groups ? d.n_groups : c.max_groups;
        d.n_units = (int)ub.size();
        c.max_units = d.n_units > c.max_units ? d.n_units : c.max_units;
        d.unit_beg = (int32_t *)ctx_ws(ctx, ("cooUb" + tag).c_str(), sizeof(int32_t) * (ub.size() + 1));
        d.unit_end = (int32_t *)ctx_ws(ctx, ("cooUe" + tag).c_str(), sizeof(int32_t) * (ub.size() + 1));
        d.row_units = (int32_t *)ctx_ws(ctx, ("cooRu" + tag).c_str(), sizeof(int32_t) * ru.size());
        d.group_beg = (int32_t *)ctx_ws(ctx, ("cooGb" + tag).c_str(), sizeof(int32_t) * gb.size());
        d.row_groups = (int32_t *)ctx_ws(ctx, ("cooRg" + tag).c_str(), sizeof(int32_t) * rg.size());
        if (!d.unit_beg || !d.unit_end || !d.row_units || !d.group_beg || !d.row_groups)
            return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
        CK(cudaMemcpyAsync(d.group_beg, gb.data(), sizeof(int32_t) * gb.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d.row_groups, rg.data(), sizeof(int32_t) * rg.size(), cudaMemcpyHostToDevice, st));
        if (!ub.empty()) {
            CK(cudaMemcpyAsync(d.unit_beg, ub.data(), sizeof(int32_t) * ub.size(), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d.unit_end, ue.data(), sizeof(int32_t) * ue.size(), cudaMemcpyHostToDevice, st));
        }
        CK(cudaMemcpyAsync(d.row_units, ru.data(), sizeof(int32_t) * ru.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // host vectors go out of scope
    }
    c.valid = true;
    return NTF_OK;
}

int get_cache(ntf_ctx *ctx, const ntf_tensor *X, CooCache *&out, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_mu);
    CooCache &c = g_cache[ctx];
    bool same = c.valid && c.N == X->order && c.nnz == X->nnz && c.vals == (const void *)X->values;
    for (int m = 0; same && m < X->order; ++m) same = c.dims[m] == X->dims[m] && c.idx[m] == (const void *)X->idx[m];
    if (!same) {
        int rc = build_cache(ctx, X, c, st);
        if (rc) { c.valid = false; return rc; }
    }
    out = &c;
    return NTF_OK;
}

int launch_coo_pass(ntf_ctx *ctx, const CooCache &c, int n, int RP, const float *const *rec, const float *const *num,
                    float eps, float *part, double *obj, cudaStream_t st, int bkind = BK_KL, float beta = 1.0f) {
    const ModeData &d = c.md[n];
    if (d.n_units == 0) return NTF_OK;
    CooPassArgs a{};
    a.sidx = d.sidx;
    a.sval = d.sval;
    a.nnz = c.nnz;
    a.N = c.N;
    a.n = n;
    a.RP = RP;
    for (int m = 0; m < c.N; ++m) { a.rec[m] = rec[m]; a.num[m] = num[m]; }
    a.unit_beg = d.unit_beg;
    a.unit_end = d.unit_end;
    a.n_units = d.n_units;
    a.eps = eps;
    a.bkind = bkind;
    a.beta = beta;
    a.part = part;
    a.obj = obj;
    const unsigned grid = (unsigned)((d.n_units + 7) / 8);
    bool same = true;  // the rank-32 kernel reads one set of factors for both roles
    for (int m = 0; m < c.N; ++m) same = same && rec[m] == num[m];
    same = same && bkind == BK_KL;  // the rank-32 kernel computes p = x / Xhat
    if (RP == 32 && same && c.N <= 4) coo_pass32_kernel<4><<<grid, 256, 0, st>>>(a);
    else if (RP == 32 && same) coo_pass32_kernel<8><<<grid, 256, 0, st>>>(a);
    else if (RP == 32) coo_pass_kernel<1><<<grid, 256, 0, st>>>(a);
    else coo_pass_kernel<2><<<grid, 256, 0, st>>>(a);
    CK(cudaGetLastError());
    ctx_count(ctx, 1);
    return NTF_OK;
}

// Num^(n) rows from the unit partials: group sums, then row sums (both in a fixed order)
int row_sums(ntf_ctx *ctx, const CooCache &c, int n, int RP, const float *part, float *gpart, float *out,
             cudaStream_t st) {
    const ModeData &d = c.md[n];
    if (d.n_groups > 0) {
        coo_group_reduce_kernel<<<nb((int64_t)d.n_groups * RP), 256, 0, st>>>(part, d.group_beg, d.n_groups, RP, gpart);
        CK(cudaGetLastError());
    }
    coo_row_reduce_kernel<<<nb(c.dims[n] * RP), 256, 0, st>>>(gpart, d.row_groups, (int)c.dims[n], RP, out);
    CK(cudaGetLastError());
    ctx_count(ctx, d.n_groups > 0 ? 2 : 1);
    return NTF_OK;
}

}  // namespace

int coo_kl_sweep(ntf_ctx *ctx, const ntf_tensor *X, int R, float *const *factors, const ntf_opts &o,
                 double *objective_dev, cudaStream_t st, bool jcomm) {
    CooCache *c = nullptr;
    int rc = get_cache(ctx, X, c, st);
    if (rc) return rc;
    const int N = X->order;
    const int RP = R <= 32 ? 32 : 64;
    float *F[8], *Ft[8];
    for (int m = 0; m < N; ++m) {
        std::string tag = std::to_string(m);
        F[m] = (float *)ctx_ws(ctx, ("cooF" + tag).c_str(), sizeof(float) * (size_t)X->dims[m] * RP);
        Ft[m] = jcomm ? (float *)ctx_ws(ctx, ("cooFt" + tag).c_str(), sizeof(float) * (size_t)X->dims[m] * RP) : F[m];
        if (!F[m] || !Ft[m]) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
        CK(pad_factor(factors[m], (int)X->dims[m], R, F[m], RP, st));
        if (jcomm) CK(copy_f32(F[m], Ft[m], X->dims[m] * RP, st));
        ctx_count(ctx, jcomm ? 2 : 1);
    }
    float *part = (float *)ctx_ws(ctx, "cooPart", sizeof(float) * (size_t)(c->max_units + 1) * RP);
    float *gpart = (float *)ctx_ws(ctx, "cooGpart", sizeof(float) * (size_t)(c->max_groups + 1) * RP);
    double *objp = (double *)ctx_ws(ctx, "cooObjP", sizeof(double) * (size_t)(c->max_units + 1));
    if (!gpart) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
    int64_t maxdim = 1;
    for (int m = 0; m < N; ++m) maxdim = X->dims[m] > maxdim ? X->dims[m] : maxdim;
    float *num = (float *)ctx_ws(ctx, "cooNum", sizeof(float) * (size_t)maxdim * RP);
    float *denc = (float *)ctx_ws(ctx, "cooDenc", sizeof(float) * 64);
    if (!part || !objp || !num || !denc) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");

    // objective of the incoming (= reference) iterate, from the mode-1 pass
    const bool want_obj = objective_dev != nullptr;
    const int L = jcomm ? o.inner_L : 1;
    // at beta = 1, chi1(Z, Zt) = Zt: the J-CoMM numerators depend on the reference only, so
    // they are computed once per outer iteration, before any block changes
    std::vector<float *> jnum;
    if (jcomm) {
        for (int n = 0; n < N; ++n) {
            float *buf = (float *)ctx_ws(ctx, ("cooJnum" + std::to_string(n)).c_str(), sizeof(float) * (size_t)X->dims[n] * RP);
            if (!buf) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
            rc = launch_coo_pass(ctx, *c, n, RP, Ft, Ft, (float)o.eps, part, (n == 0 && want_obj) ? objp : nullptr, st);
            if (rc) return rc;
            if (n == 0 && want_obj) {
                CK(obj_finish(objp, c->md[0].n_units, Ft, X->dims, N, R, RP, objective_dev, st));
                ctx_count(ctx, 1);
            }
            rc = row_sums(ctx, *c, n, RP, part, gpart, buf, st);
            if (rc) return rc;
            jnum.push_back(buf);
        }
    }
    for (int l = 0; l < L; ++l) {
        for (int n = 0; n < N; ++n) {
            const float *nrows = nullptr;
            if (jcomm) {
                nrows = jnum[n];
            } else {
                const bool obj = (n == 0) && want_obj;
                rc = launch_coo_pass(ctx, *c, n, RP, F, F, (float)o.eps, part, obj ? objp : nullptr, st);
                if (rc) return rc;
                if (obj) {
                    CK(obj_finish(objp, c->md[0].n_units, F, X->dims, N, R, RP, objective_dev, st));
                    ctx_count(ctx, 1);
                }
                rc = row_sums(ctx, *c, n, RP, part, gpart, num, st);
                if (rc) return rc;
                nrows = num;
            }
            // Den^(n)_{i r} = prod_{m != n} colsum(A^(m))_r (current blocks; chi2(Z, Zt) = Z)
            const float *f[8];
            int rows[8], q = 0;
            for (int m = 0; m < N; ++m)
                if (m != n) { f[q] = F[m]; rows[q] = (int)X->dims[m]; ++q; }
            CK(colsum_prod(q, f, rows, RP, denc, st));
            MuEpiArgs e{};
            e.pn = nrows;
            e.n_parts = 1;
            e.rows = (int)X->dims[n];
            e.RP = RP;
            e.R = R;
            e.den_closed = denc;
            e.pre = jcomm ? Ft[n] : F[n];
            e.out = F[n];
            e.beta = 1.0f;
            e.gamma = 1.0f;
            e.eps = (float)o.eps;
            CK(mu_epilogue(e, st));
            ctx_count(ctx, 2);
        }
    }
    for (int m = 0; m < N; ++m) {
        CK(unpad_factor(F[m], (int)X->dims[m], R, RP, factors[m], st));
        ctx_count(ctx, 1);
    }
    // the pointer/row tables above are read by kernels in flight; they live in the
    // context's workspace, so later calls may overwrite them only after this stream work
    return NTF_OK;
}

int coo_num_rows(ntf_ctx *ctx, const ntf_tensor *X, int n, int RP, const float *const *rec, const float *const *num,
                 float beta, float eps, float *out, double **obj_parts, int *n_obj, cudaStream_t st) {
    CooCache *c = nullptr;
    int rc = get_cache(ctx, X, c, st);
    if (rc) return rc;
    if (RP != 32 && RP != 64) return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "COO passes pad the rank to 32 or 64");
    float *part = (float *)ctx_ws(ctx, "cooPart", sizeof(float) * (size_t)(c->max_units + 1) * RP);
    float *gpart = (float *)ctx_ws(ctx, "cooGpart", sizeof(float) * (size_t)(c->max_groups + 1) * RP);
    double *objp = (double *)ctx_ws(ctx, "cooObjP", sizeof(double) * (size_t)(c->max_units + 1));
    if (!part || !gpart || !objp) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
    const bool want_obj = obj_parts != nullptr;
    if (want_obj && c->md[n].n_units == 0) CK(cudaMemsetAsync(objp, 0, sizeof(double), st));
    rc = launch_coo_pass(ctx, *c, n, RP, rec, num, eps, part, want_obj ? objp : nullptr, st, beta_kind(beta), beta);
    if (rc) return rc;
    if (want_obj) {
        *obj_parts = objp;
        *n_obj = c->md[n].n_units > 0 ? c->md[n].n_units : 1;
    }
    if (out) return row_sums(ctx, *c, n, RP, part, gpart, out, st);
    return NTF_OK;
}

int coo_kl_objective_total(ntf_ctx *ctx, const ntf_tensor *X, const float *const *F, int R, int RP,
                           const double *parts, int n_parts, double *out_dev, cudaStream_t st) {
    const int N = X->order;
    CK(obj_finish(parts, n_parts, F, X->dims, N, R, RP, out_dev, st));
    ctx_count(ctx, 1);
    return NTF_OK;
}

int coo_kl_objective(ntf_ctx *ctx, const ntf_tensor *X, int R, const float *const *factors, const ntf_opts &o,
                     double *out_dev, cudaStream_t st) {
    CooCache *c = nullptr;
    int rc = get_cache(ctx, X, c, st);
    if (rc) return rc;
    const int N = X->order;
    const int RP = R <= 32 ? 32 : 64;
    float *F[8];
    for (int m = 0; m < N; ++m) {
        F[m] = (float *)ctx_ws(ctx, ("cooF" + std::to_string(m)).c_str(), sizeof(float) * (size_t)X->dims[m] * RP);
        if (!F[m]) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
        CK(pad_factor(factors[m], (int)X->dims[m], R, F[m], RP, st));
        ctx_count(ctx, 1);
    }
    float *part = (float *)ctx_ws(ctx, "cooPart", sizeof(float) * (size_t)(c->max_units + 1) * RP);
    double *objp = (double *)ctx_ws(ctx, "cooObjP", sizeof(double) * (size_t)(c->max_units + 1));
    if (!part || !objp) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
    rc = launch_coo_pass(ctx, *c, 0, RP, F, F, (float)o.eps, part, objp, st);
    if (rc) return rc;
    CK(obj_finish(objp, c->md[0].n_units, F, X->dims, N, R, RP, out_dev, st));
    ctx_count(ctx, 1);
    return NTF_OK;
}

int coo_stable_perm(ntf_ctx *ctx, const int32_t *keys, int64_t nnz, int64_t key_range, int32_t *perm_out,
                    cudaStream_t st) {
    if (nnz == 0) return NTF_OK;
    const int nchunks = (int)((nnz + SORT_CHUNK - 1) / SORT_CHUNK) + 1;
    int *hist = (int *)ctx_ws(ctx, "cooHist", sizeof(int) * (size_t)BUCKETS * nchunks);
    int *scan = (int *)ctx_ws(ctx, "cooScan", sizeof(int) * (size_t)BUCKETS * nchunks);
    int32_t *tmp = (int32_t *)ctx_ws(ctx, "cooTmp", sizeof(int32_t) * (size_t)(nnz + 1));
    if (!hist || !scan || !tmp) return ctx_fail(ctx, NTF_ERR_OOM, "COO workspace allocation failed");
    int launches = 0;
    CK(stable_sort(keys, nnz, key_range, perm_out, tmp, hist, scan, st, &launches));
    ctx_count(ctx, launches);
    return NTF_OK;
}

void coo_release(ntf_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.erase(ctx);
}

}  // namespace ntf
