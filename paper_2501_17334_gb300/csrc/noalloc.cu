// qst_loglik_noalloc: log-likelihood of a batch of latent vectors that allocates no device
// memory.  It runs the same kernels as qst_evaluate with the plain FP32 contraction (the
// proposal kernel in evaluation mode, the FP32 projection, the log-likelihood combine),
// but every intermediate buffer lives in one file-scope device array, g_noalloc_scratch,
// instead of a workspace.
//
// Who needs it: callers that cannot call cudaMalloc on their call path -- code inside a
// host application whose device memory belongs to another allocator (a framework's memory
// pool), or a pipeline that must stay asynchronous (cudaMalloc and cudaFree can synchronise
// the whole device and stall every stream).  They pass their own inputs and outputs; the
// library supplies the scratch.
//
// Scratch layout (bytes, all offsets 256-aligned): the padded projector matrix, the
// per-column weights and per-setting shot totals, the packed rho of every row, its trace, and the per-column-group
// partial sums, for at most QST_NOALLOC_MAX_ROWS rows of at most 4 qubits.
//
// The per-column weights are formed on the host from the caller's host counts and reach the
// scratch as the launch parameters of a small kernel, not through a copy from host memory:
// launch parameters are taken by value when the launch is enqueued, so nothing on the call
// path waits for the device and no host buffer has to outlive the call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/qst.h"
#include "qst_internal.cuh"

namespace {

constexpr int kMaxD = 16;
constexpr int kMaxDPad = 256;        // D^2 rounded up to 64
constexpr int kMaxKDPad = 1408;      // 81 settings x 16 outcomes rounded up to 128
constexpr int kMaxGroups = kMaxKDPad / 128;
constexpr int64_t kMaxRows = QST_NOALLOC_MAX_ROWS;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffP = 0;
constexpr size_t kOffCnt = align256(kOffP + sizeof(float) * kMaxDPad * kMaxKDPad);
constexpr size_t kOffInvf = align256(kOffCnt + sizeof(float) * kMaxKDPad);
constexpr size_t kOffPtot = align256(kOffInvf + sizeof(float) * kMaxKDPad);
constexpr size_t kOffRho = align256(kOffPtot + sizeof(float) * (kMaxKDPad / 2));
constexpr size_t kOffTrace = align256(kOffRho + sizeof(float) * kMaxRows * kMaxDPad);
constexpr size_t kOffPart = align256(kOffTrace + sizeof(double) * kMaxRows);
constexpr size_t kScratchBytes = align256(kOffPart + sizeof(double) * kMaxGroups * kMaxRows);
static_assert(kScratchBytes == QST_NOALLOC_SCRATCH_BYTES, "qst.h states the scratch size");

// The scratch itself.  In host code this name is only a host-side stand-in for the device
// symbol; kernels get the device address obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

// failures are reported through qst_last_error(), like every other entry point
qst_status noalloc_fail(qst_status s, const char *msg) {
    qst::set_last_error(msg);
    return s;
}

// Returns the current device's scratch address, doing the one-time lookup on first use.
qst_status scratch_for_current_device(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(QST_ERR_CUDA, "qst_loglik_noalloc: no usable current CUDA device");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return noalloc_fail(QST_ERR_CUDA, "qst_loglik_noalloc: cudaGetSymbolAddress of the scratch failed");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return QST_OK;
}

// The deviance weights of every padded column, passed by value (14 KB of launch parameters,
// within the 32 KB that kernels may take).
struct NoallocWeights {
    float cnt[kMaxKDPad];
    float invf[kMaxKDPad];
    float ptot[kMaxKDPad / 2];   // shots P_k of each setting (at most 704 settings of 2 outcomes)
    int n;                       // padded columns to write
    int nk;                      // settings to write
};

__global__ void noalloc_weights_kernel(const __grid_constant__ NoallocWeights w, float *cnt, float *invf,
                                       float *ptot) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < w.n; m += gridDim.x * blockDim.x) {
        cnt[m] = w.cnt[m];
        invf[m] = w.invf[m];
        if (m < w.nk) ptot[m] = w.ptot[m];
    }
}

}  // namespace

extern "C" qst_status qst_loglik_noalloc(int32_t num_qubits, int32_t num_povms, const float *P, const int32_t *counts,
                                         const float *x, int64_t n, double *logl, void *cuda_stream) {
    using namespace qst;
    if (num_qubits < 1 || num_qubits > 4)
        return noalloc_fail(QST_ERR_INVALID_ARG, "qst_loglik_noalloc: num_qubits must be 1..4");
    const int D = 1 << num_qubits, d = D * D;
    // bound num_povms before forming K D, so that no product can wrap
    if (num_povms < 1 || num_povms > kMaxKDPad / D)
        return noalloc_fail(QST_ERR_INVALID_ARG,
                            "qst_loglik_noalloc: at most 1408 POVM elements (81 settings of 16 outcomes)");
    const int KD = num_povms * D;
    const int d_pad = (d + 63) / 64 * 64;
    const int KD_pad = (KD + 127) / 128 * 128;
    if (KD_pad > kMaxKDPad || d_pad > kMaxDPad || D > kMaxD)
        return noalloc_fail(QST_ERR_INVALID_ARG,
                            "qst_loglik_noalloc: at most 1408 POVM elements (81 settings of 16 outcomes)");
    if (n < 0 || n > kMaxRows)
        return noalloc_fail(QST_ERR_INVALID_ARG, "qst_loglik_noalloc: n must be in [0, QST_NOALLOC_MAX_ROWS]");
    if (n == 0) return QST_OK;
    if (!P || !counts || !x || !logl) return noalloc_fail(QST_ERR_INVALID_ARG, "qst_loglik_noalloc: NULL argument");
    for (int m = 0; m < KD; ++m)
        if (counts[m] < 0) return noalloc_fail(QST_ERR_INVALID_ARG, "qst_loglik_noalloc: negative count");

    unsigned char *scratch = nullptr;
    qst_status st = scratch_for_current_device(&scratch);
    if (st != QST_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

    // deviance weights (as qst_create computes them), straight into the launch parameters
    NoallocWeights w;
    float *cnt = w.cnt, *invf = w.invf;
    w.n = KD_pad;
    w.nk = num_povms;
    double C0 = 0.0, Ntot = 0.0;
    for (int m = 0; m < KD_pad; ++m) {
        cnt[m] = 0.0f;
        invf[m] = 1.0f;
    }
    for (int k = 0; k < num_povms; ++k) {
        int64_t Pk = 0;
        for (int l = 0; l < D; ++l) Pk += counts[k * D + l];
        w.ptot[k] = (float)Pk;
        for (int l = 0; l < D; ++l) {
            const int m = k * D + l;
            if (counts[m] == 0) continue;
            cnt[m] = (float)counts[m];
            invf[m] = (float)((double)Pk / (double)counts[m]);
            C0 -= (double)counts[m] * std::log((double)invf[m]);
            Ntot += (double)counts[m];
        }
    }

    ProblemView v{};
    v.D = D;
    v.d = d;
    v.nx = 4 * d;
    v.KD = KD;
    v.KD_pad = KD_pad;
    v.d_pad = d_pad;
    v.R = n;
    v.C0 = C0;
    v.Ntot = Ntot;
    v.P32 = reinterpret_cast<const float *>(scratch + kOffP);
    v.cnt = reinterpret_cast<const float *>(scratch + kOffCnt);
    v.invf = reinterpret_cast<const float *>(scratch + kOffInvf);
    v.ptot = reinterpret_cast<const float *>(scratch + kOffPtot);
    v.rho_prop = reinterpret_cast<float *>(scratch + kOffRho);
    v.trace_prop = reinterpret_cast<double *>(scratch + kOffTrace);
    v.logl_part = reinterpret_cast<double *>(scratch + kOffPart);
    v.qr_passes = 3;   // the default configuration's assembly
    v.ngroups = fp32_ngroups(v, n);

    // The scratch keeps the previous call's contents: rewrite everything this call reads.
    float *P32 = reinterpret_cast<float *>(scratch + kOffP);
    cudaError_t e = cudaMemsetAsync(P32, 0, sizeof(float) * (size_t)d_pad * KD_pad, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(P32, sizeof(float) * KD_pad, P, sizeof(float) * KD, sizeof(float) * KD, d,
                              cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        noalloc_weights_kernel<<<(KD_pad + 255) / 256, 256, 0, s>>>(w, reinterpret_cast<float *>(scratch + kOffCnt),
                                                                   reinterpret_cast<float *>(scratch + kOffInvf),
                                                                   reinterpret_cast<float *>(scratch + kOffPtot));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d < d_pad)   // padding columns of the operand must be zero
        e = cudaMemsetAsync(scratch + kOffRho, 0, sizeof(float) * (size_t)n * d_pad, s);
    if (e == cudaSuccess) e = launch_propose(v, MODE_EVAL, 0u, nullptr, x, n, false, nullptr, nullptr, s);
    if (e == cudaSuccess) e = launch_project_fp32(v, v.rho_prop, n, v.logl_part, nullptr, s);
    if (e == cudaSuccess) e = launch_logl_combine(v, n, logl, s);
    if (e != cudaSuccess) return noalloc_fail(QST_ERR_CUDA, cudaGetErrorString(e));
    return QST_OK;
}
