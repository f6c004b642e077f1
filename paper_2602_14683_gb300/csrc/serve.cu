// Continuous-batching server for many small factorization jobs.
//
// Dense CP jobs on the FP32 path go to a batch (batch.cu): resident jobs of a class share
// every launch of an iteration, the batch runs a few iterations per graph launch, and jobs
// join and leave it between launches, admitted by the memory of the batch's arena.  Every
// other job (Tucker, tensor-core precisions, a CP job larger than the arena) runs in a slot:
// A server owns `slots` execution slots, each an ntf context (its own workspaces) and a
// CUDA stream.  Jobs wait in a FIFO queue; a scheduler thread admits the head of the queue
// into a free slot when the slot's estimated workspace fits the device-memory budget, runs
// one eager iteration (which sizes the workspaces) followed by a one-thread kernel that
// applies the stopping test to its objective, and then launches the rest of the job as ONE
// CUDA graph: a conditional WHILE node whose body is one captured iteration of the job's
// method plus the same stopping-test kernel, which clears the loop condition when
// |F_{t-1} - F_t| / F_{t-1} <= rtol or the iteration cap is reached.  The whole solve thus
// runs on the device without a host round trip per iteration; the host only sees the job's
// final state (iterations, last objective), copied to pinned memory behind an event.  Jobs
// in different slots overlap on the device through their streams.  A job's kernels, launch
// shapes and reduction orders depend only on its own shapes, so its result is the same
// whether it runs alone or among others.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ntf.h"
#include "ntf_batch.h"
#include "ntf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

using ntf::JobState;
using ntf::job_step;

// iterations of every batched job per graph launch of its class (the admission granularity)
constexpr int kBatchIters = 4;

struct Slot {
    ntf_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    double *F_dev = nullptr;
    JobState *S_dev = nullptr;
    JobState *S_host = nullptr;  // pinned
    cudaGraphExec_t exec = nullptr;
    bool busy = false;
    ntf_job job{};
    int64_t id = -1;
    double t_submit = 0.0, t_admit = 0.0;
    size_t bytes = 0;
};

__global__ void job_check_kernel(JobState *s, const double *F) { job_step(s, F); }
__global__ void job_check_loop_kernel(JobState *s, const double *F, cudaGraphConditionalHandle h) {
    job_step(s, F);
    cudaGraphSetConditional(h, s->done ? 0u : 1u);
}

struct Pending {
    ntf_job job;
    int64_t id;
    double t_submit;
    bool slot_lane;  // a batch-lane job that does not fit the batch's empty arena
};

int rank_pad(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : 64; }

// workspace bytes a job's context grows to (padded blocks, partial sums, Tucker partial
// tensors); an estimate used for admission, not an allocation
size_t estimate_bytes(const ntf_job &j, int sms) {
    const int64_t I = j.dims[0], J = j.dims[1], K = j.dims[2];
    size_t b = 0;
    if (j.model == NTF_CP) {
        // tensor-core passes pad the rank to 32
        const int RP = (j.precision != NTF_PREC_FP32 && j.rank <= 32) ? 32 : rank_pad(j.rank);
        // the tensor-core plan (128-column blocks, four mode-1 partials per row tile) where
        // the job asks for it, else the FP32 plan; the larger of the two when either may run
        const ntf::Cp3Plan p32 = ntf::cp3_plan((int)I, (int)J, (int)K, RP, sms, 64);
        size_t parts = (size_t)p32.parts1 * I + (size_t)p32.parts2 * J + (size_t)p32.parts3 * K;
        int grid = p32.grid;
        if (j.precision != NTF_PREC_FP32 && RP == 32) {
            for (int kb = 128; kb <= 256; kb *= 2) {
                const ntf::Cp3Plan ptc = ntf::cp3_plan((int)I, (int)J, (int)K, RP, sms, kb);
                const size_t pt = (size_t)ptc.parts1 * I + (size_t)ptc.parts2 * J + (size_t)ptc.parts3 * K;
                parts = pt > parts ? pt : parts;
                grid = ptc.grid > grid ? ptc.grid : grid;
            }
        }
        b += 4 * sizeof(float) * (size_t)(I + J + K) * RP;
        b += 2 * sizeof(float) * parts * RP;
        b += sizeof(double) * (size_t)grid;
        b += sizeof(double) * (size_t)(ntf::row_blocks((int)I, RP) + ntf::row_blocks((int)J, RP) +
                                       ntf::row_blocks((int)K, RP)) * RP;
    } else {
        const int RP = (j.precision != NTF_PREC_FP32 && j.core_dims[2] <= 32) ? 32 : rank_pad((int)j.core_dims[2]);
        const int64_t Jc = j.core_dims[0] * j.core_dims[1] * j.core_dims[2];
        b += 5 * sizeof(float) * (size_t)(I * J) * RP;  // B3 rec / num / den, W, Wd
        b += 4 * sizeof(float) * (size_t)(4 * Jc + I * j.core_dims[0] + J * j.core_dims[1] + K * RP);
        b += 3 * sizeof(float) * (size_t)(I * j.core_dims[1] * j.core_dims[2]);
        const ntf::Cp3Plan p = ntf::cp3_plan((int)I, (int)J, (int)K, RP, sms, 64);
        b += 2 * sizeof(float) * (size_t)p.parts3 * K * RP + sizeof(double) * (size_t)p.grid * 4;
    }
    return b + (1u << 20);
}

}  // namespace

struct ntf_server {
    int device = 0, sms = 1;
    size_t budget = 0, used = 0;  // slot lane: budget and estimated use
    ntf_batch *batch = nullptr;   // batched lane (dense CP, FP32)
    std::vector<Slot> slots;
    std::deque<Pending> pending;
    std::vector<ntf_result> done;
    int64_t next_id = 0;
    int active = 0;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::thread worker;
    bool stop = false;
};

namespace {

int run_step(Slot &s, cudaStream_t st) {
    const ntf_job &j = s.job;
    ntf_opts o;
    ntf_opts_default(&o);
    o.precision = j.precision;
    o.eps = j.eps > 0 ? j.eps : o.eps;
    ntf_tensor X{};
    X.order = 3;
    X.dims = j.dims;
    X.kind = NTF_DENSE;
    X.values = j.X;
    float *const *f = j.factors;
    if (j.method == 1) {
        if (j.model == NTF_CP) return ntf_cp_mu_sweep(s.ctx, &X, j.beta, j.rank, f, &o, s.F_dev, st);
        return ntf_tucker_mu_sweep(s.ctx, &X, j.beta, j.core_dims, j.core, f, &o, s.F_dev, st);
    }
    if (j.model == NTF_CP) return ntf_jcomm_outer(s.ctx, NTF_CP, &X, j.beta, j.rank, nullptr, nullptr, f, &o, s.F_dev, st);
    return ntf_jcomm_outer(s.ctx, NTF_TUCKER, &X, j.beta, 0, j.core_dims, j.core, f, &o, s.F_dev, st);
}

void finish(ntf_server *sv, Slot &s, int status) {
    ntf_result r{};
    r.id = s.id;
    r.status = status;
    r.iterations = status == NTF_OK ? s.S_host->iters : 0;
    r.objective = status == NTF_OK ? s.S_host->F_last : 0.0;
    r.t_submit = s.t_submit;
    r.t_admit = s.t_admit;
    r.t_done = now_s();
    if (s.exec) {
        cudaGraphExecDestroy(s.exec);
        s.exec = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->done.push_back(r);
        sv->used -= s.bytes;
        --sv->active;
    }
    s.busy = false;
    sv->cv_done.notify_all();
}

// First (eager) iteration and its stopping test, then the remaining iterations as one
// graph launch (WHILE node over one captured iteration + the stopping test), then the
// job's final state to pinned memory and the slot's event.
int admit(Slot &s) {
    JobState init{};
    init.rtol = s.job.rtol;
    init.max_iters = s.job.max_iters;
    *s.S_host = init;
    if (cudaMemcpyAsync(s.S_dev, s.S_host, sizeof(JobState), cudaMemcpyHostToDevice, s.st) != cudaSuccess)
        return NTF_ERR_CUDA;
    int rc = run_step(s, s.st);
    if (rc) return rc;
    job_check_kernel<<<1, 1, 0, s.st>>>(s.S_dev, s.F_dev);
    if (cudaGetLastError() != cudaSuccess) return NTF_ERR_CUDA;
    if (s.job.max_iters > 1) {
        cudaGraph_t g = nullptr;
        if (cudaGraphCreate(&g, 0) != cudaSuccess) return NTF_ERR_CUDA;
        auto bail = [&](int code) {
            cudaGraphDestroy(g);
            return code;
        };
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
            return bail(NTF_ERR_CUDA);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) return bail(NTF_ERR_CUDA);
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(s.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return bail(NTF_ERR_CUDA);
        rc = run_step(s, s.st);
        if (!rc) {
            job_check_loop_kernel<<<1, 1, 0, s.st>>>(s.S_dev, s.F_dev, h);
            if (cudaGetLastError() != cudaSuccess) rc = NTF_ERR_CUDA;
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s.st, &captured);
        if (rc) return bail(rc);
        if (e != cudaSuccess) return bail(NTF_ERR_CUDA);
        const cudaError_t ei = cudaGraphInstantiate(&s.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return NTF_ERR_CUDA;
        if (cudaGraphLaunch(s.exec, s.st) != cudaSuccess) return NTF_ERR_CUDA;
    }
    if (cudaMemcpyAsync(s.S_host, s.S_dev, sizeof(JobState), cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
        return NTF_ERR_CUDA;
    if (cudaEventRecord(s.ev, s.st) != cudaSuccess) return NTF_ERR_CUDA;
    return NTF_OK;
}

bool batch_lane(const ntf_server *sv, const Pending &p) {
    return sv->batch && !p.slot_lane && p.job.model == NTF_CP && p.job.precision == NTF_PREC_FP32;
}

// Batched-lane admissions, in queue order: each CP job joins the batch if its workspace fits
// the arena now (a job that does not fit an empty arena goes to the slot lane instead); the
// first one that does not fit stops the lane's admissions until jobs retire.
void admit_batched(ntf_server *sv) {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        if (!batch_lane(sv, *it)) {
            ++it;
            continue;
        }
        const int rc = ntf::batch_add(sv->batch, &it->job, it->id, it->t_submit);
        if (rc == NTF_ERR_OOM) {
            if (ntf_batch_resident(sv->batch) == 0) {
                it->slot_lane = true;
                ++it;
                continue;
            }
            break;
        }
        if (rc) {
            ntf_result r{};
            r.id = it->id;
            r.status = rc;
            r.t_submit = it->t_submit;
            r.t_admit = r.t_done = now_s();
            sv->done.push_back(r);
            sv->cv_done.notify_all();
        } else {
            ++sv->active;
        }
        it = sv->pending.erase(it);
    }
}

// Launches the batch's next iterations where the previous launch has finished and moves
// the finished jobs' results to the server's list.  Returns the number of resident jobs.
int drive_batch(ntf_server *sv) {
    if (!sv->batch) return 0;
    const int res = ntf::batch_tick(sv->batch, kBatchIters, 0);
    ntf_result buf[256];
    for (;;) {
        const int n = ntf_batch_results(sv->batch, buf, 256);
        if (n <= 0) break;
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int q = 0; q < n; ++q) sv->done.push_back(buf[q]);
        sv->active -= n;
        sv->cv_done.notify_all();
    }
    return res > 0 ? res : 0;
}

void worker_loop(ntf_server *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        admit_batched(sv);
        // slot-lane admissions (FIFO over the slot lane's jobs: the first waits until a slot
        // and the memory budget allow it)
        for (;;) {
            Pending p;
            int slot = -1;
            {
                std::unique_lock<std::mutex> lk(sv->mu);
                if (sv->stop) return;
                auto head = sv->pending.begin();
                while (head != sv->pending.end() && batch_lane(sv, *head)) ++head;
                if (head == sv->pending.end()) break;
                const size_t need = estimate_bytes(head->job, sv->sms);
                for (size_t q = 0; q < sv->slots.size(); ++q)
                    if (!sv->slots[q].busy) { slot = (int)q; break; }
                if (slot < 0 || (sv->used + need > sv->budget && sv->active > 0)) break;
                p = *head;
                sv->pending.erase(head);
                sv->used += need;
                ++sv->active;
                sv->slots[slot].bytes = need;
            }
            Slot &s = sv->slots[slot];
            s.busy = true;
            s.job = p.job;
            s.id = p.id;
            s.t_submit = p.t_submit;
            s.t_admit = now_s();
            const int rc = admit(s);
            if (rc) finish(sv, s, rc);
        }
        // the batch's next launches and its finished jobs
        bool any = drive_batch(sv) > 0;
        // completion of active slots (each runs its whole job as one graph launch)
        for (auto &s : sv->slots) {
            if (!s.busy) continue;
            any = true;
            const cudaError_t q = cudaEventQuery(s.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                finish(sv, s, NTF_ERR_CUDA);
                continue;
            }
            finish(sv, s, NTF_OK);
        }
        if (!any) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return sv->stop || !sv->pending.empty(); });
            if (sv->stop) return;
        } else {
            std::this_thread::yield();
        }
    }
}

}  // namespace

extern "C" {

int ntf_server_create(ntf_server **out, int device, int slots, size_t mem_budget_bytes) {
    if (!out || slots < 1 || slots > 256) return NTF_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return NTF_ERR_CUDA;
    }
    ntf_server *sv = new ntf_server();
    sv->device = device;
    cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, device);
    if (sv->sms < 1) sv->sms = 1;
    if (mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        mem_budget_bytes = fr / 2;
    }
    // half of the budget is the batch's arena (allocated now), half the slots' estimate
    const size_t arena = mem_budget_bytes / 2;
    sv->budget = mem_budget_bytes - arena;
    if (ntf_batch_create(&sv->batch, device, 4096, arena) != NTF_OK) {
        sv->batch = nullptr;
        delete sv;
        return NTF_ERR_CUDA;
    }
    sv->slots.resize(slots);
    for (auto &s : sv->slots) {
        if (ntf_ctx_create(&s.ctx, device) != NTF_OK || cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&s.F_dev, sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s.S_dev, sizeof(JobState)) != cudaSuccess ||
            cudaMallocHost(&s.S_host, sizeof(JobState)) != cudaSuccess) {
            cudaGetLastError();
            ntf_server_destroy(sv);
            return NTF_ERR_CUDA;
        }
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return NTF_OK;
}

int ntf_server_submit(ntf_server *sv, const ntf_job *job, int64_t *id_out) {
    if (!sv || !job) return NTF_ERR_ARG;
    if (job->model != NTF_CP && job->model != NTF_TUCKER) return NTF_ERR_ARG;
    if (!job->X || !job->factors[0] || !job->factors[1] || !job->factors[2]) return NTF_ERR_ARG;
    if (job->model == NTF_TUCKER && !job->core) return NTF_ERR_ARG;
    if (!(job->beta >= 0.0f && job->beta < 2.0f)) return NTF_ERR_BETA;
    if (job->max_iters < 1 || job->method < 0 || job->method > 1) return NTF_ERR_ARG;
    for (int n = 0; n < 3; ++n)
        if (job->dims[n] < 1) return NTF_ERR_SHAPE;
    std::lock_guard<std::mutex> lk(sv->mu);
    const int64_t id = sv->next_id++;
    sv->pending.push_back({*job, id, now_s(), false});
    if (id_out) *id_out = id;
    sv->cv.notify_all();
    return NTF_OK;
}

int ntf_server_poll(ntf_server *sv, ntf_result *out, int max_results, int wait_all) {
    if (!sv || (!out && max_results > 0)) return NTF_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (wait_all) sv->cv_done.wait(lk, [&] { return sv->pending.empty() && sv->active == 0; });
    int n = 0;
    while (n < max_results && !sv->done.empty()) {
        out[n++] = sv->done.front();
        sv->done.erase(sv->done.begin());
    }
    return n;
}

void ntf_server_destroy(ntf_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    if (sv->batch) ntf_batch_destroy(sv->batch);
    for (auto &s : sv->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.exec) cudaGraphExecDestroy(s.exec);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.st) cudaStreamDestroy(s.st);
        if (s.F_dev) cudaFree(s.F_dev);
        if (s.S_dev) cudaFree(s.S_dev);
        if (s.S_host) cudaFreeHost(s.S_host);
        if (s.ctx) ntf_ctx_destroy(s.ctx);
    }
    delete sv;
}

}  // extern "C"
