// Allocation-free variant of the dense CP objective (D_beta of a CP model).
//
// The regular entry points keep their scratch (padded factor copies, per-CTA partial
// sums) in workspaces that a context grows with cudaMalloc.  Some callers cannot allocate
// device memory at call time: a serving process whose device memory is carved out up
// front by another framework's allocator, or an embedded caller held to a fixed memory
// budget, where a cudaMalloc inside the library would fail or take memory already given out.  For them this file keeps
// the scratch in one file-scope __device__ array of fixed size, which the driver creates
// when the library's module is loaded on a device and keeps until the process exits.
#include <mutex>

#include "../../include/ntf.h"
#include "ntf_internal.h"

namespace {

constexpr size_t kScratchBytes = NTF_NOALLOC_SCRATCH_BYTES;

// Scratch of every call on a device: padded factor copies, then per-CTA FP64 partials.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device.  In host code the symbol is only a
// host-side handle; the address is looked up once per device, with that device current.
int scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return NTF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NTF_ERR_CUDA;
        }
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return NTF_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" int ntf_cp_beta_div_noalloc(const ntf_tensor *X, float beta, int rank, const float *const *factors,
                                       double eps, double eps_x, double *out_dev, void *stream) {
    if (!X || !X->dims || !X->values || !factors || !out_dev) return NTF_ERR_ARG;
    if (X->kind != NTF_DENSE) return NTF_ERR_UNSUPPORTED;
    if (X->order != 3) return NTF_ERR_UNSUPPORTED;
    if (!(beta >= 0.0f && beta < 2.0f)) return NTF_ERR_BETA;
    if (!(eps > 0.0) || !(eps_x > 0.0)) return NTF_ERR_ARG;
    if (rank < 1 || rank > 64) return NTF_ERR_UNSUPPORTED;
    for (int n = 0; n < 3; ++n) {
        if (!factors[n]) return NTF_ERR_ARG;
        if (X->dims[n] < 1 || X->dims[n] > (int64_t)0x7fffffff) return NTF_ERR_SHAPE;
    }
    const int I = (int)X->dims[0], J = (int)X->dims[1], K = (int)X->dims[2];
    const int RP = rank <= 8 ? 8 : rank <= 16 ? 16 : rank <= 32 ? 32 : 64;
    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return NTF_ERR_CUDA;
    }
    const ntf::Cp3Plan plan = ntf::cp3_plan(I, J, K, RP, sms > 0 ? sms : 1, 64);
    const int dims[3] = {I, J, K};
    size_t off[3], need = 0;
    for (int n = 0; n < 3; ++n) {
        off[n] = need;
        need += align256(sizeof(float) * (size_t)dims[n] * RP);
    }
    const size_t obj_off = need;
    need += align256(sizeof(double) * (size_t)plan.grid);
    if (need > kScratchBytes) return NTF_ERR_UNSUPPORTED;  // beyond the fixed scratch size

    void *base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc) return rc;
    unsigned char *sc = (unsigned char *)base;
    cudaStream_t st = (cudaStream_t)stream;
    float *F[3];
    for (int n = 0; n < 3; ++n) {
        F[n] = (float *)(sc + off[n]);
        // every element of the padded copy is written, so nothing of a previous call leaks in
        if (ntf::pad_factor(factors[n], dims[n], rank, F[n], RP, st) != cudaSuccess) return NTF_ERR_CUDA;
    }
    ntf::Cp3Args a{};
    a.X = X->values;
    a.I = I;
    a.J = J;
    a.K = K;
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = F[m];
    a.bkind = ntf::beta_kind(beta);
    a.beta = beta;
    a.eps = (float)eps;
    a.eps_x = (float)eps_x;
    a.n_jt = plan.n_jt;
    a.n_kb = plan.n_kb;
    a.n_is = plan.n_is;
    a.vec16 = (K % 4 == 0) && ((reinterpret_cast<uintptr_t>(X->values) & 15) == 0);
    a.obj = (double *)(sc + obj_off);  // every CTA writes its own slot
    if (ntf::cp3_launch(plan, a, ntf::PM_OBJ, 0, st) != cudaSuccess) return NTF_ERR_CUDA;
    if (ntf::reduce_objective(a.obj, plan.grid, 0.0, out_dev, st) != cudaSuccess) return NTF_ERR_CUDA;
    return NTF_OK;
}
