// Small kernels around the fused passes: factor padding, closed-form KL denominators,
// the partial-sum reduction fused with the multiplicative update (and the chi
// transforms of the new block), and the FP64 objective reduction.
#include "ntf_internal.h"

namespace ntf {

__global__ void pad_kernel(const float *src, int rows, int R, float *dst, int RP) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * RP) return;
    int i = (int)(t / RP), r = (int)(t % RP);
    dst[t] = r < R ? src[(int64_t)i * R + r] : 0.0f;
}

__global__ void unpad_kernel(const float *src, int rows, int R, int RP, float *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * R) return;
    int i = (int)(t / R), r = (int)(t % R);
    dst[t] = src[(int64_t)i * RP + r];
}

cudaError_t pad_factor(const float *src, int rows, int R, float *dst, int RP, cudaStream_t s) {
    int64_t n = (int64_t)rows * RP;
    pad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, rows, R, dst, RP);
    return cudaGetLastError();
}

cudaError_t unpad_factor(const float *src, int rows, int R, int RP, float *dst, cudaStream_t s) {
    int64_t n = (int64_t)rows * R;
    unpad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, rows, R, RP, dst);
    return cudaGetLastError();
}

__global__ void copy_kernel(const float *src, float *dst, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[t];
}

cudaError_t copy_f32(const float *src, float *dst, int64_t n, cudaStream_t s) {
    copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

// Den^(n)_{i r} at beta = 1 (Q == 1, Section 6.3): prod_{m != n} colsum(F^(m))_r.
// One CTA per rank column; FP64 sums in a fixed thread/stride order and tree.
struct ColsumArgs {
    const float *f[8];
    int rows[8];
    int nf, RP;
    float *out;
};

__global__ void colsum_prod_kernel(ColsumArgs c) {
    __shared__ double sh[8];
    const int r = blockIdx.x, t = threadIdx.x;
    double prod = 1.0;
    for (int m = 0; m < c.nf; ++m) {
        double s = 0.0;
        for (int i = t; i < c.rows[m]; i += blockDim.x) s += (double)c.f[m][(int64_t)i * c.RP + r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((t & 31) == 0) sh[t >> 5] = s;
        __syncthreads();
        if (t == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
            prod *= tot;
        }
        __syncthreads();
    }
    if (t == 0) c.out[r] = (float)prod;
}

cudaError_t colsum_prod(int nf, const float *const *f, const int *rows, int RP, float *out,
                        cudaStream_t s) {
    ColsumArgs c{};
    if (nf > 8) return cudaErrorInvalidValue;
    for (int m = 0; m < nf; ++m) {
        c.f[m] = f[m];
        c.rows[m] = rows[m];
    }
    c.nf = nf;
    c.RP = RP;
    c.out = out;
    colsum_prod_kernel<<<RP, 256, 0, s>>>(c);
    return cudaGetLastError();
}

// Multiplicative update with the eps-constrained minimiser (Theorem "CP block
// multiplicative update"; Section 5.3 "CP inner update" with pre = reference block):
//   out = max(pre * (Num / Den)^gamma, eps)
__global__ void mu_epilogue_kernel(MuEpiArgs e) {
    // four consecutive threads per output: each adds a quarter of the parts in part order, and the
    // quarter sums are added in quarter order (lane 0 of the four then applies the update)
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t t = gt >> 2;
    const int q = (int)(gt & 3);
    const int64_t n = (int64_t)e.rows * e.RP;
    const bool live = t < n;
    const int r = live ? (int)(t % e.RP) : 0;
    const bool used = live && r < e.R;
    const int per = (e.n_parts + 3) / 4, p0 = q * per, p1 = min(e.n_parts, p0 + per);
    auto psum = [&](const float *src) {
        float acc = 0.0f;
        if (used) {
            for (int pb = p0; pb < p1; pb += 8) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = pb + k < p1 ? src[(int64_t)(pb + k) * n + t] : 0.0f;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (pb + k < p1) acc += v[k];
            }
        }
        const float a1 = __shfl_down_sync(0xffffffffu, acc, 1), a2 = __shfl_down_sync(0xffffffffu, acc, 2),
                    a3 = __shfl_down_sync(0xffffffffu, acc, 3);
        return ((acc + a1) + a2) + a3;
    };
    const float num = psum(e.pn);
    const float den = e.den_closed ? (used ? e.den_closed[r] : 1.0f) : psum(e.pd);
    if (q != 0 || !live) return;
    if (r >= e.R) {
        e.out[t] = 0.0f;
        if (e.chi1_out) e.chi1_out[t] = 0.0f;
        if (e.chi2_out) e.chi2_out[t] = 0.0f;
        return;
    }
    const float ratio = __fdiv_rn(num, den);
    float m;
    if (e.gamma == 1.0f) m = ratio;
    else if (e.gamma == 0.5f) m = sqrtf(ratio);
    else m = powf(ratio, e.gamma);
    const float v = fmaxf(e.pre[t] * m, e.eps);
    e.out[t] = v;
    if (e.chi1_out) e.chi1_out[t] = chi1_f(e.beta, v, e.ref[t]);
    if (e.chi2_out) e.chi2_out[t] = chi2_f(e.beta, v, e.ref[t]);
}

cudaError_t mu_epilogue(const MuEpiArgs &e, cudaStream_t s) {
    int64_t n = (int64_t)e.rows * e.RP;
    mu_epilogue_kernel<<<(unsigned)((4 * n + 255) / 256), 256, 0, s>>>(e);
    return cudaGetLastError();
}

// Fixed-order FP64 sum over the G row groups of a [G][RP] block of per-thread partials.
__device__ __forceinline__ double group_sum(double *sh, double v, int RP, int t) {
    sh[t] = v;
    __syncthreads();
    double tot = 0.0;
    if (t < RP)
        for (int g = 0; g < (int)blockDim.x / RP; ++g) tot += sh[g * RP + t];
    __syncthreads();
    return tot;
}

__device__ __forceinline__ void prep_body(const PrepArgs &p, const int blk) {
    __shared__ double sh[256];
    int b = blk, m = 0;
    while (m < 2 && b >= row_blocks(p.rows[m], p.RP)) {
        b -= row_blocks(p.rows[m], p.RP);
        ++m;
    }
    const int RP = p.RP, G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    const int rows = p.rows[m], rpb = rows_per_block(rows, RP);
    const int ibeg = b * rpb, iend = min(rows, ibeg + rpb);
    double cs = 0.0;
    for (int i = ibeg + g; i < iend; i += G) {
        const float v = r < p.R ? p.src[m][(int64_t)i * p.R + r] : 0.0f;
        const int64_t o = (int64_t)i * RP + r;
        p.F[m][o] = v;
        if (p.Ft[m]) p.Ft[m][o] = v;
        if (p.C1[m]) p.C1[m][o] = v;
        if (p.C2[m]) p.C2[m][o] = v;
        cs += (double)v;
    }
    if (p.cs[m]) {
        const double tot = group_sum(sh, cs, RP, t);
        if (t < RP) p.cs[m][(int64_t)b * RP + t] = tot;
    }
}

__global__ void prep_kernel(PrepArgs p) { prep_body(p, blockIdx.x); }

// Extrapolation (Section "Going beyond: Majorization-Minimization with Extrapolation"):
// for each factor, D = pad([A - Aprev]_+) and FP64 partial sums of D^2 per row block (the
// row blocking of prep_kernel); then Aprev <- A, the incoming iterate kept for the next call.
__global__ void extrap_prep_kernel(ExtrapArgs x) {
    __shared__ double sh[256];
    int b = blockIdx.x, m = 0;
    while (m < 2 && b >= row_blocks(x.rows[m], x.RP)) {
        b -= row_blocks(x.rows[m], x.RP);
        ++m;
    }
    const int RP = x.RP, G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    const int rows = x.rows[m], rpb = rows_per_block(rows, RP);
    const int ibeg = b * rpb, iend = min(rows, ibeg + rpb);
    double s2 = 0.0;
    for (int i = ibeg + g; i < iend; i += G) {
        float d = 0.0f;
        if (r < x.R) {
            const int64_t o = (int64_t)i * x.R + r;
            const float a = x.A[m][o];
            d = fmaxf(a - x.Aprev[m][o], 0.0f);
            x.Aprev[m][o] = a;
        }
        x.D[m][(int64_t)i * RP + r] = d;
        s2 += (double)d * (double)d;
    }
    const double tot = group_sum(sh, s2, RP, t);
    if (t < RP) x.nrm[m][(int64_t)b * RP + t] = tot;
}

// E = max(F + alpha_n D, eps), alpha_n = min(alpha, cap / (||D||_F + delta)); every block
// sums the norm partials of its factor in the same order, so alpha_n is the same everywhere.
__global__ void extrap_apply_kernel(ExtrapArgs x) {
    __shared__ double sh[256];
    __shared__ double alpha_s;
    int b = blockIdx.x, m = 0;
    while (m < 2 && b >= row_blocks(x.rows[m], x.RP)) {
        b -= row_blocks(x.rows[m], x.RP);
        ++m;
    }
    const int RP = x.RP, t = threadIdx.x;
    {
        // ||D||^2: thread t adds partials t, t + 256, ... in order, then a fixed tree
        const int n = row_blocks(x.rows[m], RP) * RP;
        double s2 = 0.0;
        for (int k = t; k < n; k += blockDim.x) s2 += x.nrm[m][k];
        sh[t] = s2;
        __syncthreads();
        for (int w = 128; w >= 1; w >>= 1) {
            if (t < w) sh[t] += sh[t + w];
            __syncthreads();
        }
        if (t == 0) {
            const double cap = (double)x.cap / (sqrt(sh[0]) + (double)x.delta);
            alpha_s = (double)x.alpha < cap ? (double)x.alpha : cap;
        }
        __syncthreads();
    }
    const float alpha = (float)alpha_s;
    const int G = blockDim.x / RP, r = t % RP, g = t / RP;
    const int rows = x.rows[m], rpb = rows_per_block(rows, RP);
    const int ibeg = b * rpb, iend = min(rows, ibeg + rpb);
    double cs = 0.0;
    for (int i = ibeg + g; i < iend; i += G) {
        const int64_t e = (int64_t)i * RP + r;
        const float v = r < x.R ? fmaxf(fmaf(alpha, x.D[m][e], x.F[m][e]), x.eps) : 0.0f;
        x.E[m][e] = v;
        if (x.E2[m]) x.E2[m][e] = v;
        if (x.E3[m]) x.E3[m][e] = v;
        cs += (double)v;
    }
    if (x.cs[m]) {
        const double tot = group_sum(sh, cs, RP, t);
        if (t < RP) x.cs[m][(int64_t)b * RP + t] = tot;
    }
}

cudaError_t extrapolate(const ExtrapArgs &x, cudaStream_t s) {
    int blocks = 0;
    for (int m = 0; m < 3; ++m) blocks += row_blocks(x.rows[m], x.RP);
    extrap_prep_kernel<<<blocks, 256, 0, s>>>(x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    extrap_apply_kernel<<<blocks, 256, 0, s>>>(x);
    return cudaGetLastError();
}

// Order N >= 4 on the 3-way kernels: a run of consecutive modes is merged into one mode whose
// index is the row-major multi-index (last mode of the run fastest -- the memory order of X),
// with the Khatri-Rao factor KR[(i_0..i_{M-1})][r] = prod_m L_m[i_m][r].
__global__ void kr_merge_kernel(KrArgs k) {
    __shared__ double sh[256];
    const int RP = k.RP, G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    const int rpb = rows_per_block(k.rows, RP);
    const int ibeg = blockIdx.x * rpb, iend = min(k.rows, ibeg + rpb);
    double cs = 0.0;
    for (int i = ibeg + g; i < iend; i += G) {
        int rem = i;
        float v = 1.0f;
        for (int m = k.M - 1; m >= 0; --m) {
            const int im = rem % k.dims[m];
            rem /= k.dims[m];
            v *= k.L[m][(int64_t)im * RP + r];
        }
        if (k.out) k.out[(int64_t)i * RP + r] = v;
        cs += (double)v;
    }
    if (k.cs) {
        const double tot = group_sum(sh, cs, RP, t);
        if (t < RP) k.cs[(int64_t)blockIdx.x * RP + t] = tot;
    }
}

cudaError_t kr_merge(const KrArgs &k, cudaStream_t s) {
    kr_merge_kernel<<<row_blocks(k.rows, k.RP), 256, 0, s>>>(k);
    return cudaGetLastError();
}

// One block per row i_n of the mode; RP-lane group g of the block takes the other-index
// positions q = g, g + G, ... of the fold and the rows g, g + G, ... of the column sums.
__global__ void run_update_kernel(RunUpdArgs u) {
    __shared__ double sh[256];
    __shared__ float num_s[64], den_s[64];
    const int RP = u.RP, G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    const int in = blockIdx.x;
    if (!u.pd) {
        double prod = 1.0;
        for (int k = 0; k < u.ncf; ++k) {
            // rows i = g, g + G, ... added in order, eight loads issued before their adds
            const int nr = u.cf_rows[k];
            double cs = 0.0;
            for (int i0 = g; i0 < nr; i0 += 8 * G) {
                float x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = i0 + j * G < nr ? u.cf[k][(int64_t)(i0 + j * G) * RP + r] : 0.0f;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (i0 + j * G < nr) cs += (double)x[j];
            }
            prod *= group_sum(sh, cs, RP, t);
        }
        if (t < RP) den_s[t] = (float)prod;
    }
    int64_t other = 1;
    for (int m = 0; m < u.M; ++m)
        if (m != u.n) other *= u.dims[m];
    const int64_t stride = (int64_t)u.rows * RP;
    for (int side = 0; side < (u.pd ? 2 : 1); ++side) {
        if (side == 0 && u.num_rows) {  // the numerator is given (uniform over the block)
            if (t < RP) num_s[t] = u.num_rows[(int64_t)in * RP + t];
            continue;
        }
        const float *parts = side ? u.pd : u.pn;
        const float *const *L = side ? u.Ld : u.Ln;
        double acc = 0.0;
        // the thread's rows q = g, g + G, ... of the other merged modes, four per step: their merged
        // row, Khatri-Rao weight and partials are all loaded before any of them is added; each
        // partial sum and acc keep the order of one row at a time, parts in order (the merged
        // run has fewer than 2^31 rows: 32-bit index arithmetic)
        const int oth = (int)other;
        for (int q0 = g; q0 < oth; q0 += 4 * G) {
            int rowq[4];
            float wq[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = q0 + j * G;
                int rem = q < oth ? q : 0, row = 0, mul = 1;
                float w = 1.0f;
                for (int m = u.M - 1; m >= 0; --m) {
                    int im;
                    if (m == u.n) {
                        im = in;
                    } else {
                        const int d = u.dims[m], nx = rem / d;
                        im = rem - nx * d;
                        rem = nx;
                        w *= L[m][(int64_t)im * RP + r];
                    }
                    row += im * mul;
                    mul *= u.dims[m];
                }
                rowq[j] = row;
                wq[j] = w;
            }
            float sv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int p0 = 0; p0 < u.n_parts; p0 += 8) {
                float x[4][8];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        x[j][k] = (q0 + j * G < oth && p0 + k < u.n_parts)
                                      ? parts[(int64_t)(p0 + k) * stride + (int64_t)rowq[j] * RP + r]
                                      : 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (p0 + k < u.n_parts) sv[j] += x[j][k];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (q0 + j * G < oth) acc += (double)sv[j] * (double)wq[j];
        }
        const double tot = group_sum(sh, acc, RP, t);
        if (t < RP) (side ? den_s : num_s)[t] = (float)tot;
    }
    __syncthreads();
    if (t >= RP) return;
    const int64_t o = (int64_t)in * RP + t;
    float v = 0.0f, c1 = 0.0f, c2 = 0.0f;
    if (t < u.R) {
        const float ratio = __fdiv_rn(num_s[t], den_s[t]);
        float m;
        if (u.gamma == 1.0f) m = ratio;
        else if (u.gamma == 0.5f) m = sqrtf(ratio);
        else m = powf(ratio, u.gamma);
        v = fmaxf(u.pre[o] * m, u.eps);
        if (u.chi1) c1 = chi1_f(u.beta, v, u.ref[o]);
        if (u.chi2) c2 = chi2_f(u.beta, v, u.ref[o]);
        if (u.user) u.user[(int64_t)in * u.R + t] = v;
    }
    u.out[o] = v;
    if (u.chi1) u.chi1[o] = c1;
    if (u.chi2) u.chi2[o] = c2;
}

cudaError_t run_update(const RunUpdArgs &u, cudaStream_t s) {
    run_update_kernel<<<u.dims[u.n], 256, 0, s>>>(u);
    return cudaGetLastError();
}

int prep_items(const PrepArgs &p) {
    int blocks = 0;
    for (int m = 0; m < 3; ++m) blocks += row_blocks(p.rows[m], p.RP);
    return blocks;
}

cudaError_t prep_factors(const PrepArgs &p, cudaStream_t s) {
    const int blocks = prep_items(p);
    if (blocks == 0) return cudaSuccess;
    prep_kernel<<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// One block per row block of the mode, plus (when the objective is wanted) one more block
// that only sums the objective partials, so that this reduction is off the critical path.
// A thread's loads of the column-sum partials and of its first row's partial sums are all
// issued before the first barrier.
__device__ __forceinline__ void mode_update_body(const UpdArgs &u, const int blk) {
    __shared__ double sh[256];
    __shared__ float den_s[64];
    const MuEpiArgs &e = u.e;
    const int RP = e.RP, G = blockDim.x / RP, t = threadIdx.x, r = t % RP, g = t / RP;
    const int nrb = row_blocks(e.rows, RP);
    if (blk == nrb) {  // the objective block: same order as reduce_obj_kernel
        double v = 0.0;
        for (int k = t; k < u.obj_n; k += blockDim.x) v += u.obj_parts[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) sh[t >> 5] = v;
        __syncthreads();
        if (t == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
            *u.obj_out = tot;
        }
        return;
    }
    const int rpb = rows_per_block(e.rows, RP);
    const int ibeg = blk * rpb, iend = min(e.rows, ibeg + rpb);
    const int64_t stride = (int64_t)e.rows * RP;
    // partials in batches of 16, each batch added as a fixed tree and the batch sums in order
    // (a fixed order for every run); 32 loads are in flight at once
    auto load32 = [&](const float *src, int64_t o, int p0, float *v) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = p0 + k < e.n_parts ? src[(int64_t)(p0 + k) * stride + o] : 0.0f;
    };
    auto add32 = [&](int p0, float *v, float acc) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (p0 + 16 * b >= e.n_parts) break;
            float *w16 = v + 16 * b;
#pragma unroll
            for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
                for (int k = 0; k < w; ++k) w16[k] += w16[k + w];
            acc += w16[0];
        }
        return acc;
    };
    auto psum = [&](const float *src, int64_t o, float *first) {  // first: loaded batch 0 or null
        float acc = 0.0f;
        for (int p0 = 0; p0 < e.n_parts; p0 += 32) {
            float v[32];
            if (p0 == 0 && first) {
#pragma unroll
                for (int k = 0; k < 32; ++k) v[k] = first[k];
            } else {
                load32(src, o, p0, v);
            }
            acc = add32(p0, v, acc);
        }
        return acc;
    };
    // the first row's numerator partials, loaded ahead of the column-sum phase
    const int i_first = ibeg + g;
    const bool pre = i_first < iend && r < e.R;
    float first[32];
    if (pre) load32(e.pn, (int64_t)i_first * RP + r, 0, first);
    if (u.n_cs > 0) {
        // each factor's column sums: thread (g, r) adds blocks g, g + G, ..., then the G
        // group sums are added in order (fixed order, the same in every block); the loads of
        // both factors' first eight blocks are issued together
        double sum[2] = {0.0, 0.0};
        for (int b0 = g; b0 < u.cs_nb[0] || (u.n_cs > 1 && b0 < u.cs_nb[1]); b0 += 8 * G) {
            double v[2][8];
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int b = b0 + q * G;
                    v[k][q] = (k < u.n_cs && b < u.cs_nb[k]) ? u.cs_in[k][(int64_t)b * RP + r] : 0.0;
                }
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int q = 0; q < 8; ++q) sum[k] += v[k][q];
        }
        double prod = 1.0;
        for (int k = 0; k < u.n_cs; ++k) prod *= group_sum(sh, sum[k], RP, t);
        if (t < RP) den_s[t] = (float)prod;
        __syncthreads();
    }
    double cs = 0.0;
    for (int i = ibeg + g; i < iend; i += G) {
        const int64_t o = (int64_t)i * RP + r;
        float v = 0.0f, c1 = 0.0f, c2 = 0.0f;
        if (r < e.R) {
            const float num = psum(e.pn, o, (pre && i == i_first) ? first : nullptr);
            float den;
            if (u.n_cs > 0) den = den_s[r];
            else if (e.den_closed) den = e.den_closed[r];
            else den = psum(e.pd, o, nullptr);
            const float ratio = __fdiv_rn(num, den);
            float m;
            if (e.gamma == 1.0f) m = ratio;
            else if (e.gamma == 0.5f) m = sqrtf(ratio);
            else m = powf(ratio, e.gamma);
            v = fmaxf(e.pre[o] * m, e.eps);
            if (e.chi1_out) c1 = chi1_f(e.beta, v, e.ref[o]);
            if (e.chi2_out) c2 = chi2_f(e.beta, v, e.ref[o]);
            if (u.user_out) u.user_out[(int64_t)i * e.R + r] = v;
        }
        e.out[o] = v;
        if (e.chi1_out) e.chi1_out[o] = c1;
        if (e.chi2_out) e.chi2_out[o] = c2;
        cs += (double)v;
    }
    if (u.cs_out) {
        const double tot = group_sum(sh, cs, RP, t);
        if (t < RP) u.cs_out[(int64_t)blk * RP + t] = tot;
    }
}

__global__ void mode_update_kernel(UpdArgs u) { mode_update_body(u, blockIdx.x); }

int mode_update_items(const UpdArgs &u) { return row_blocks(u.e.rows, u.e.RP) + (u.obj_out ? 1 : 0); }

cudaError_t mode_update(const UpdArgs &u, cudaStream_t s) {
    mode_update_kernel<<<mode_update_items(u), 256, 0, s>>>(u);
    return cudaGetLastError();
}

// Batched forms: a persistent grid walks the work items of every resident job that has not
// stopped; each item is the block of the single-job launch with the same index.
__global__ void prep_batched_kernel(const BatchTable<PrepArgs> t) {
    const int n = *t.n;
    const int total = n > 0 ? t.pfx[n] : 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = batch_job_of(t.pfx, n, item);
        if (t.state[j].done) continue;
        const PrepArgs p = t.args[j];
        prep_body(p, item - t.pfx[j]);
        __syncthreads();
    }
}

__global__ void mode_update_batched_kernel(const BatchTable<UpdArgs> t) {
    const int n = *t.n;
    const int total = n > 0 ? t.pfx[n] : 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = batch_job_of(t.pfx, n, item);
        if (t.state[j].done) continue;
        const UpdArgs u = t.args[j];
        mode_update_body(u, item - t.pfx[j]);
        __syncthreads();
    }
}

cudaError_t prep_batched(const BatchTable<PrepArgs> &t, int grid, cudaStream_t s) {
    prep_batched_kernel<<<grid, 256, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t mode_update_batched(const BatchTable<UpdArgs> &t, int grid, cudaStream_t s) {
    mode_update_batched_kernel<<<grid, 256, 0, s>>>(t);
    return cudaGetLastError();
}

// Fixed-order FP64 sum of per-CTA objective partials (one CTA; lane-strided then tree).
__global__ void reduce_obj_kernel(const double *parts, int n, double *out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) s += parts[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

cudaError_t reduce_objective(const double *parts, int n, double, double *out, cudaStream_t s) {
    reduce_obj_kernel<<<1, 256, 0, s>>>(parts, n, out);
    return cudaGetLastError();
}

// Two partial-sum arrays, each summed as reduce_obj_kernel does, then added (a first).
__global__ void reduce_obj2_kernel(const double *a, int na, const double *b, int nb, double *out) {
    __shared__ double sh[32];
    double tot[2];
    for (int k = 0; k < 2; ++k) {
        const double *p = k ? b : a;
        const int n = k ? nb : na;
        double s = 0.0;
        for (int t = threadIdx.x; t < n; t += blockDim.x) s += p[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        tot[k] = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot[k] += sh[w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = tot[0] + tot[1];
}

cudaError_t reduce_objective2(const double *a, int na, const double *b, int nb, double *out, cudaStream_t s) {
    reduce_obj2_kernel<<<1, 256, 0, s>>>(a, na, b, nb, out);
    return cudaGetLastError();
}

}  // namespace ntf
