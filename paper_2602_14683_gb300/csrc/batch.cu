// Launches shared by many small dense 3-way CP jobs.
//
// A batch holds resident jobs in classes keyed by rank padding RP (8, 16, 32, 64) and the
// shape of one iteration:
//   KL1 : J-CoMM at beta = 1 -- one pass with every numerator and the objective, then the
//         three mode updates with closed-form denominators (Algorithm 2 at beta = 1);
//   P3  : block MM at beta = 1 -- three passes (mode 1 with the objective, 2, 3), each
//         followed by its mode update with the closed-form denominator (Algorithm 1);
//   P3D : beta != 1 -- three passes with numerators and denominators, each followed by its
//         mode update; J-CoMM (reference pre-factor, chi_1 / chi_2 of the current blocks,
//         Section 5.3) and block MM jobs share the class, since they differ only in the
//         arguments of the same launches.
// Every step of an iteration (padding the factors, each pass, each mode update, the stopping
// test) is ONE launch for all jobs of the class: a persistent grid walks a device-resident
// work table in which job j owns the items of its own single-job launch (its own plan and
// row blocking), so each job does exactly the arithmetic of the single-job FP32 path and its
// result does not depend on the other jobs.  A class's iteration is captured once as the body
// of a conditional WHILE graph node; one graph launch runs up to `iters` iterations, and the
// stopping-test kernel (the FP64 objective's relative change, or the iteration cap) marks
// finished jobs, which later launches skip, and ends the loop when none is left.  Between
// graph launches the host retires finished jobs (their workspaces return to the arena),
// admits new ones and rewrites the tables: continuous batching at iteration granularity.
// Workspaces come from one device arena sized at creation, so admission is by memory.
#include <chrono>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/ntf.h"
#include "ntf_batch.h"
#include "ntf_internal.h"

namespace {

using ntf::BatchTable;
using ntf::Cp3Args;
using ntf::JobState;
using ntf::PrepArgs;
using ntf::UpdArgs;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int rank_pad(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : 64; }

enum Kind : int { KIND_KL1 = 0, KIND_P3 = 1, KIND_P3D = 2, NKIND = 3 };
constexpr int NRP = 4;
int rp_index(int RP) { return RP == 8 ? 0 : RP == 16 ? 1 : RP == 32 ? 2 : 3; }

// First-fit allocator over one device buffer (offsets in 256-byte units).
struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    void init(char *b, size_t n) {
        base = b;
        bytes = n & ~(size_t)255;
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t n, size_t &off) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            off = it->first;
            const size_t rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// One resident job: its request, plan and the workspace pointers inside its arena block.
struct Entry {
    ntf_job job{};
    int64_t id = -1;
    double t_submit = 0.0, t_admit = 0.0;
    int RP = 0, kind = 0;
    bool jcomm = false, den = false;
    ntf::Cp3Plan plan{};
    size_t off = 0, bytes = 0;
    float *F[3]{}, *Ft[3]{}, *C1[3]{}, *C2[3]{}, *pn[3]{}, *pd[3]{};
    double *obj = nullptr, *cs[3]{};
    JobState st{};
};

// Steps whose work tables a class keeps: the padding, the pass (one Cp3Args for all passes of
// an iteration: the pointers are the same), and the three mode updates.
enum Step : int { ST_PREP = 0, ST_PASS = 1, ST_UPD0 = 2, NSTEP = 5 };

struct Class {
    int RP = 0, kind = 0, cap = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    // device tables
    int *d_n = nullptr, *d_pfx = nullptr, *d_ctl = nullptr;  // d_pfx: [NSTEP][cap + 1]; d_ctl: {iters, done}
    Cp3Args *d_pass = nullptr;
    PrepArgs *d_prep = nullptr;
    UpdArgs *d_upd = nullptr;  // [3][cap]
    JobState *d_state = nullptr;
    double *d_F = nullptr;     // [cap] objective of each job's incoming iterate
    // pinned host mirrors
    int *h_n = nullptr, *h_pfx = nullptr, *h_ctl = nullptr;
    Cp3Args *h_pass = nullptr;
    PrepArgs *h_prep = nullptr;
    UpdArgs *h_upd = nullptr;
    JobState *h_state = nullptr;
    std::vector<Entry> jobs;  // jobs added while a launch runs are appended after launched_n
    int launched_n = 0;       // jobs covered by the launch in flight
    bool dirty = false, in_flight = false;
};

__global__ void batch_stop_kernel(const int *n_ptr, JobState *S, const double *F, int *ctl,
                                  cudaGraphConditionalHandle h) {
    __shared__ int alive;
    if (threadIdx.x == 0) alive = 0;
    __syncthreads();
    const int n = *n_ptr;
    int mine = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (S[j].done) continue;
        ntf::job_step(S + j, F + j);
        if (!S[j].done) mine = 1;
    }
    if (mine) atomicOr(&alive, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int it = ++ctl[1];
        cudaGraphSetConditional(h, (alive && it < ctl[0]) ? 1u : 0u);
    }
}

}  // namespace

struct ntf_batch {
    int device = 0, sms = 1, capacity = 0, resident = 0;
    int upd_grid = 0;
    char *arena_mem = nullptr;
    Arena arena;
    Class cls[NRP][NKIND];
    std::vector<ntf_result> done;
    int64_t next_id = 0;
};

namespace {

#define BCUDA(x)                                        \
    do {                                                \
        if ((x) != cudaSuccess) {                       \
            cudaGetLastError();                         \
            return NTF_ERR_CUDA;                        \
        }                                               \
    } while (0)

int class_alloc(Class &c, int RP, int kind, int cap) {
    c.RP = RP;
    c.kind = kind;
    c.cap = cap;
    BCUDA(cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking));
    BCUDA(cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming));
    BCUDA(cudaMalloc(&c.d_n, sizeof(int)));
    BCUDA(cudaMalloc(&c.d_ctl, 2 * sizeof(int)));
    BCUDA(cudaMalloc(&c.d_pfx, sizeof(int) * NSTEP * (size_t)(cap + 1)));
    BCUDA(cudaMalloc(&c.d_pass, sizeof(Cp3Args) * (size_t)cap));
    BCUDA(cudaMalloc(&c.d_prep, sizeof(PrepArgs) * (size_t)cap));
    BCUDA(cudaMalloc(&c.d_upd, sizeof(UpdArgs) * 3 * (size_t)cap));
    BCUDA(cudaMalloc(&c.d_state, sizeof(JobState) * (size_t)cap));
    BCUDA(cudaMalloc(&c.d_F, sizeof(double) * (size_t)cap));
    BCUDA(cudaMallocHost(&c.h_n, sizeof(int)));
    BCUDA(cudaMallocHost(&c.h_ctl, 2 * sizeof(int)));
    BCUDA(cudaMallocHost(&c.h_pfx, sizeof(int) * NSTEP * (size_t)(cap + 1)));
    BCUDA(cudaMallocHost(&c.h_pass, sizeof(Cp3Args) * (size_t)cap));
    BCUDA(cudaMallocHost(&c.h_prep, sizeof(PrepArgs) * (size_t)cap));
    BCUDA(cudaMallocHost(&c.h_upd, sizeof(UpdArgs) * 3 * (size_t)cap));
    BCUDA(cudaMallocHost(&c.h_state, sizeof(JobState) * (size_t)cap));
    *c.h_n = 0;
    BCUDA(cudaMemcpyAsync(c.d_n, c.h_n, sizeof(int), cudaMemcpyHostToDevice, c.st));
    BCUDA(cudaStreamSynchronize(c.st));
    return NTF_OK;
}

void class_free(Class &c) {
    if (c.st) cudaStreamSynchronize(c.st);
    if (c.exec) cudaGraphExecDestroy(c.exec);
    if (c.ev) cudaEventDestroy(c.ev);
    if (c.st) cudaStreamDestroy(c.st);
    for (void *p : {(void *)c.d_n, (void *)c.d_ctl, (void *)c.d_pfx, (void *)c.d_pass, (void *)c.d_prep,
                    (void *)c.d_upd, (void *)c.d_state, (void *)c.d_F})
        if (p) cudaFree(p);
    for (void *p : {(void *)c.h_n, (void *)c.h_ctl, (void *)c.h_pfx, (void *)c.h_pass, (void *)c.h_prep,
                    (void *)c.h_upd, (void *)c.h_state})
        if (p) cudaFreeHost(p);
    c = Class{};
}

BatchTable<Cp3Args> pass_table(const Class &c) {
    return {c.d_n, c.d_pfx + ST_PASS * (c.cap + 1), c.d_pass, c.d_state};
}
BatchTable<PrepArgs> prep_table(const Class &c) {
    return {c.d_n, c.d_pfx + ST_PREP * (c.cap + 1), c.d_prep, c.d_state};
}
BatchTable<UpdArgs> upd_table(const Class &c, int n) {
    return {c.d_n, c.d_pfx + (ST_UPD0 + n) * (c.cap + 1), c.d_upd + (size_t)n * c.cap, c.d_state};
}

// One iteration of the class, launched on its stream (captured into the WHILE body).
int class_iteration(const ntf_batch *b, Class &c, cudaGraphConditionalHandle h) {
    const int pgrid = 0;  // persistent grid of the pass kernel: every CTA that fits
    const bool den = c.kind == KIND_P3D;
    BCUDA(ntf::prep_batched(prep_table(c), b->upd_grid, c.st));
    if (c.kind == KIND_KL1) {
        BCUDA(ntf::cp3_batched_launch(c.RP, pass_table(c), ntf::PM_M1 | ntf::PM_M2 | ntf::PM_M3 | ntf::PM_OBJ, 0,
                                      pgrid, c.st));
        for (int n = 0; n < 3; ++n) BCUDA(ntf::mode_update_batched(upd_table(c, n), b->upd_grid, c.st));
    } else {
        for (int n = 0; n < 3; ++n) {
            const int ms = n == 0 ? (ntf::PM_M1 | ntf::PM_OBJ) : n == 1 ? ntf::PM_M2 : ntf::PM_M3;
            BCUDA(ntf::cp3_batched_launch(c.RP, pass_table(c), ms, den ? 1 : 0, pgrid, c.st));
            BCUDA(ntf::mode_update_batched(upd_table(c, n), b->upd_grid, c.st));
        }
    }
    batch_stop_kernel<<<1, 256, 0, c.st>>>(c.d_n, c.d_state, c.d_F, c.d_ctl, h);
    BCUDA(cudaGetLastError());
    return NTF_OK;
}

// Graph of one launch: a WHILE node whose body is one captured iteration.
int class_capture(const ntf_batch *b, Class &c) {
    cudaGraph_t g = nullptr;
    BCUDA(cudaGraphCreate(&g, 0));
    auto bail = [&](int code) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return code;
    };
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return bail(NTF_ERR_CUDA);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) return bail(NTF_ERR_CUDA);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return bail(NTF_ERR_CUDA);
    const int rc = class_iteration(b, c, h);
    cudaGraph_t captured = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c.st, &captured);
    if (rc) return bail(rc);
    if (e != cudaSuccess) return bail(NTF_ERR_CUDA);
    const cudaError_t ei = cudaGraphInstantiate(&c.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return NTF_ERR_CUDA;
    }
    return NTF_OK;
}

// Workspace of one job inside its arena block (sizes as the single-job FP32 path's).
size_t entry_layout(Entry &e, char *base) {
    const int dims[3] = {(int)e.job.dims[0], (int)e.job.dims[1], (int)e.job.dims[2]};
    const int parts[3] = {e.plan.parts1, e.plan.parts2, e.plan.parts3};
    size_t o = 0;
    auto take = [&](size_t n) {
        char *p = base ? base + o : nullptr;
        o += (n + 255) & ~(size_t)255;
        return p;
    };
    for (int n = 0; n < 3; ++n) {
        const size_t fb = sizeof(float) * (size_t)dims[n] * e.RP;
        e.F[n] = (float *)take(fb);
        e.Ft[n] = e.jcomm ? (float *)take(fb) : nullptr;
        e.C1[n] = (e.jcomm && e.den) ? (float *)take(fb) : nullptr;
        e.C2[n] = (e.jcomm && e.den) ? (float *)take(fb) : nullptr;
        const size_t pb = sizeof(float) * (size_t)parts[n] * dims[n] * e.RP;
        e.pn[n] = (float *)take(pb);
        e.pd[n] = e.den ? (float *)take(pb) : nullptr;
        e.cs[n] = e.den ? nullptr : (double *)take(sizeof(double) * (size_t)ntf::row_blocks(dims[n], e.RP) * e.RP);
    }
    e.obj = (double *)take(sizeof(double) * (size_t)e.plan.grid);
    return o;
}

// Arguments of the class steps for the job in table row j (the single-job FP32 path's).
void entry_args(const Entry &e, int j, const Class &c, Cp3Args &a, PrepArgs &p, UpdArgs *u) {
    const int dims[3] = {(int)e.job.dims[0], (int)e.job.dims[1], (int)e.job.dims[2]};
    const int parts[3] = {e.plan.parts1, e.plan.parts2, e.plan.parts3};
    const float eps = (float)(e.job.eps > 0 ? e.job.eps : 1e-12);
    const float beta = e.job.beta;
    a = Cp3Args{};
    a.X = e.job.X;
    a.I = dims[0];
    a.J = dims[1];
    a.K = dims[2];
    for (int m = 0; m < 3; ++m) {
        a.rec[m] = e.jcomm ? e.Ft[m] : e.F[m];
        a.num[m] = (e.jcomm && e.den) ? e.C1[m] : a.rec[m];
        a.den[m] = (e.jcomm && e.den) ? e.C2[m] : a.rec[m];
    }
    a.bkind = ntf::beta_kind(beta);
    a.beta = beta;
    a.eps = eps;
    a.eps_x = 1e-12f;
    a.n_jt = e.plan.n_jt;
    a.n_kb = e.plan.n_kb;
    a.n_is = e.plan.n_is;
    a.vec16 = (a.K % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
    a.p1n = e.pn[0];
    a.p1d = e.pd[0];
    a.p2n = e.pn[1];
    a.p2d = e.pd[1];
    a.p3n = e.pn[2];
    a.p3d = e.pd[2];
    a.obj = e.obj;
    p = PrepArgs{};
    for (int m = 0; m < 3; ++m) {
        p.src[m] = e.job.factors[m];
        p.rows[m] = dims[m];
        p.F[m] = e.F[m];
        p.Ft[m] = e.jcomm ? e.Ft[m] : nullptr;
        p.C1[m] = e.C1[m];
        p.C2[m] = e.C2[m];
        p.cs[m] = e.den ? nullptr : e.cs[m];
    }
    p.R = e.job.rank;
    p.RP = e.RP;
    for (int n = 0; n < 3; ++n) {
        UpdArgs &v = u[n];
        v = UpdArgs{};
        ntf::MuEpiArgs &m = v.e;
        m.pn = e.pn[n];
        m.pd = e.den ? e.pd[n] : nullptr;
        m.n_parts = parts[n];
        m.rows = dims[n];
        m.RP = e.RP;
        m.R = e.job.rank;
        m.pre = e.jcomm ? e.Ft[n] : e.F[n];
        m.out = e.F[n];
        m.beta = beta;
        m.gamma = ntf::mu_gamma(beta);
        m.eps = eps;
        if (e.jcomm && e.den) {
            m.ref = e.Ft[n];
            m.chi1_out = e.C1[n];
            m.chi2_out = e.C2[n];
        }
        if (!e.den) {
            for (int q = 0; q < 3; ++q)
                if (q != n) {
                    v.cs_in[v.n_cs] = e.cs[q];
                    v.cs_nb[v.n_cs] = ntf::row_blocks(dims[q], e.RP);
                    ++v.n_cs;
                }
            v.cs_out = e.cs[n];
        }
        v.user_out = e.job.factors[n];
        if (n == 0) {
            v.obj_parts = e.obj;
            v.obj_n = e.plan.grid;
            v.obj_out = c.d_F + j;
        }
    }
}

// Host mirrors of the class tables from its resident jobs, copied to the device on its stream.
int class_upload(Class &c) {
    const int n = (int)c.jobs.size();
    int *pfx[NSTEP];
    for (int s = 0; s < NSTEP; ++s) {
        pfx[s] = c.h_pfx + s * (c.cap + 1);
        pfx[s][0] = 0;
    }
    for (int j = 0; j < n; ++j) {
        const Entry &e = c.jobs[j];
        UpdArgs *u = c.h_upd;
        UpdArgs uj[3];
        entry_args(e, j, c, c.h_pass[j], c.h_prep[j], uj);
        for (int q = 0; q < 3; ++q) u[(size_t)q * c.cap + j] = uj[q];
        c.h_state[j] = e.st;
        pfx[ST_PREP][j + 1] = pfx[ST_PREP][j] + ntf::prep_items(c.h_prep[j]);
        pfx[ST_PASS][j + 1] = pfx[ST_PASS][j] + e.plan.grid;
        for (int q = 0; q < 3; ++q) pfx[ST_UPD0 + q][j + 1] = pfx[ST_UPD0 + q][j] + ntf::mode_update_items(uj[q]);
    }
    *c.h_n = n;
    BCUDA(cudaMemcpyAsync(c.d_n, c.h_n, sizeof(int), cudaMemcpyHostToDevice, c.st));
    BCUDA(cudaMemcpyAsync(c.d_pfx, c.h_pfx, sizeof(int) * NSTEP * (size_t)(c.cap + 1), cudaMemcpyHostToDevice, c.st));
    if (n > 0) {
        BCUDA(cudaMemcpyAsync(c.d_pass, c.h_pass, sizeof(Cp3Args) * n, cudaMemcpyHostToDevice, c.st));
        BCUDA(cudaMemcpyAsync(c.d_prep, c.h_prep, sizeof(PrepArgs) * n, cudaMemcpyHostToDevice, c.st));
        for (int q = 0; q < 3; ++q)
            BCUDA(cudaMemcpyAsync(c.d_upd + (size_t)q * c.cap, c.h_upd + (size_t)q * c.cap, sizeof(UpdArgs) * n,
                                  cudaMemcpyHostToDevice, c.st));
        BCUDA(cudaMemcpyAsync(c.d_state, c.h_state, sizeof(JobState) * n, cudaMemcpyHostToDevice, c.st));
    }
    c.dirty = false;
    return NTF_OK;
}

void retire(ntf_batch *b, Class &c, size_t j, int status) {
    Entry &e = c.jobs[j];
    ntf_result r{};
    r.id = e.id;
    r.status = status;
    r.iterations = status == NTF_OK ? e.st.iters : 0;
    r.objective = status == NTF_OK ? e.st.F_last : 0.0;
    r.t_submit = e.t_submit;
    r.t_admit = e.t_admit;
    r.t_done = now_s();
    b->done.push_back(r);
    b->arena.release(e.off, e.bytes);
    --b->resident;
    c.jobs.erase(c.jobs.begin() + (std::ptrdiff_t)j);
    c.dirty = true;
}

// A class whose launch has finished: read the job states, retire the stopped jobs.
int class_collect(ntf_batch *b, Class &c, bool wait) {
    if (!c.in_flight) return NTF_OK;
    cudaError_t q = wait ? cudaEventSynchronize(c.ev) : cudaEventQuery(c.ev);
    if (q == cudaErrorNotReady) return 1;
    c.in_flight = false;
    if (q != cudaSuccess) {
        cudaGetLastError();
        for (int j = c.launched_n; j-- > 0;) retire(b, c, (size_t)j, NTF_ERR_CUDA);
        return NTF_OK;
    }
    // the launch covered the first launched_n jobs; later additions keep their initial state
    for (int j = 0; j < c.launched_n; ++j) c.jobs[j].st = c.h_state[j];
    for (int j = c.launched_n; j-- > 0;)
        if (c.jobs[j].st.done) retire(b, c, (size_t)j, NTF_OK);
    return NTF_OK;
}

// Up to `iters` iterations of every resident job of the class: one graph launch.
int class_launch(Class &c, int iters) {
    if (c.jobs.empty()) return NTF_OK;
    if (c.dirty) {
        const int rc = class_upload(c);
        if (rc) return rc;
    }
    c.h_ctl[0] = iters;
    c.h_ctl[1] = 0;
    BCUDA(cudaMemcpyAsync(c.d_ctl, c.h_ctl, 2 * sizeof(int), cudaMemcpyHostToDevice, c.st));
    BCUDA(cudaGraphLaunch(c.exec, c.st));
    BCUDA(cudaMemcpyAsync(c.h_state, c.d_state, sizeof(JobState) * c.jobs.size(), cudaMemcpyDeviceToHost, c.st));
    BCUDA(cudaEventRecord(c.ev, c.st));
    c.launched_n = (int)c.jobs.size();
    c.in_flight = true;
    return NTF_OK;
}

}  // namespace

namespace ntf {

int batch_add(ntf_batch *b, const ntf_job *job, int64_t id, double t_submit) {
    if (!b || !job) return NTF_ERR_ARG;
    if (job->model != NTF_CP || job->precision != NTF_PREC_FP32) return NTF_ERR_UNSUPPORTED;
    if (!job->X || !job->factors[0] || !job->factors[1] || !job->factors[2]) return NTF_ERR_ARG;
    if (!(job->beta >= 0.0f && job->beta < 2.0f)) return NTF_ERR_BETA;
    if (job->max_iters < 1 || job->method < 0 || job->method > 1) return NTF_ERR_ARG;
    if (job->rank < 1 || job->rank > 64) return NTF_ERR_UNSUPPORTED;
    for (int n = 0; n < 3; ++n)
        if (job->dims[n] < 1 || job->dims[n] > (1 << 30)) return NTF_ERR_SHAPE;
    if (b->resident >= b->capacity) return NTF_ERR_OOM;
    Entry e;
    e.job = *job;
    e.id = id;
    e.t_submit = t_submit;
    e.RP = rank_pad(job->rank);
    e.jcomm = job->method == 0;
    e.den = ntf::beta_kind(job->beta) != ntf::BK_KL;
    e.kind = e.den ? KIND_P3D : e.jcomm ? KIND_KL1 : KIND_P3;
    e.plan = ntf::cp3_plan((int)job->dims[0], (int)job->dims[1], (int)job->dims[2], e.RP, b->sms, 64);
    e.bytes = entry_layout(e, nullptr);
    if (!b->arena.alloc(e.bytes, e.off)) return NTF_ERR_OOM;
    entry_layout(e, b->arena.base + e.off);
    e.st = JobState{};
    e.st.rtol = job->rtol;
    e.st.max_iters = job->max_iters;
    e.t_admit = now_s();
    Class &c = b->cls[rp_index(e.RP)][e.kind];
    c.jobs.push_back(e);
    c.dirty = true;
    ++b->resident;
    return NTF_OK;
}

int batch_tick(ntf_batch *b, int iters, int wait) {
    if (!b || iters < 1) return NTF_ERR_ARG;
    cudaSetDevice(b->device);
    for (auto &row : b->cls)
        for (auto &c : row) {
            const int q = class_collect(b, c, wait != 0);
            if (q == 1) continue;  // still running
            const int rc = class_launch(c, iters);
            if (rc)  // the class's jobs end with the launch's error
                for (size_t j = c.jobs.size(); j-- > 0;) retire(b, c, j, rc);
        }
    return b->resident;
}

size_t batch_job_bytes(const ntf_batch *b, const ntf_job *job) {
    Entry e;
    e.job = *job;
    e.RP = rank_pad(job->rank);
    e.jcomm = job->method == 0;
    e.den = ntf::beta_kind(job->beta) != ntf::BK_KL;
    e.plan = ntf::cp3_plan((int)job->dims[0], (int)job->dims[1], (int)job->dims[2], e.RP, b->sms, 64);
    return entry_layout(e, nullptr);
}

}  // namespace ntf

extern "C" {

int ntf_batch_create(ntf_batch **out, int device, int capacity, size_t mem_budget_bytes) {
    if (!out || capacity < 1 || capacity > 65536) return NTF_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return NTF_ERR_CUDA;
    }
    ntf_batch *b = new ntf_batch();
    b->device = device;
    b->capacity = capacity;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
    if (b->sms < 1) b->sms = 1;
    b->upd_grid = 4 * b->sms;
    if (mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        mem_budget_bytes = fr / 4;
    }
    int rc = NTF_OK;
    if (cudaMalloc(&b->arena_mem, mem_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        rc = NTF_ERR_OOM;
    } else {
        b->arena.init(b->arena_mem, mem_budget_bytes);
    }
    static const int rps[NRP] = {8, 16, 32, 64};
    for (int r = 0; r < NRP && !rc; ++r)
        for (int k = 0; k < NKIND && !rc; ++k) {
            rc = class_alloc(b->cls[r][k], rps[r], k, capacity);
            if (!rc) rc = class_capture(b, b->cls[r][k]);
        }
    if (rc) {
        ntf_batch_destroy(b);
        return rc;
    }
    *out = b;
    return NTF_OK;
}

int ntf_batch_add(ntf_batch *b, const ntf_job *job, int64_t *id_out) {
    if (!b) return NTF_ERR_ARG;
    const int64_t id = b->next_id;
    const int rc = ntf::batch_add(b, job, id, now_s());
    if (rc) return rc;
    ++b->next_id;
    if (id_out) *id_out = id;
    return NTF_OK;
}

int ntf_batch_tick(ntf_batch *b, int iters, int wait) { return ntf::batch_tick(b, iters, wait); }

int ntf_batch_results(ntf_batch *b, ntf_result *out, int max_results) {
    if (!b || (!out && max_results > 0)) return NTF_ERR_ARG;
    int n = 0;
    while (n < max_results && n < (int)b->done.size()) {
        out[n] = b->done[n];
        ++n;
    }
    b->done.erase(b->done.begin(), b->done.begin() + n);
    return n;
}

int ntf_batch_resident(const ntf_batch *b) { return b ? b->resident : NTF_ERR_ARG; }

void ntf_batch_destroy(ntf_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    for (auto &row : b->cls)
        for (auto &c : row) class_free(c);
    if (b->arena_mem) cudaFree(b->arena_mem);
    delete b;
}

}  // extern "C"
