// ctfmnmf_cost_noalloc: the negative log-likelihood of a demixed state computed without
// allocating device memory. The per-bin partial sums live in a fixed file-scope device
// array instead of a buffer that a handle allocates.
//
// Why: some callers cannot call cudaMalloc at the point where they need the cost - a
// real-time audio thread (an allocation may synchronise the device and has no latency
// bound), code inside an allocator or memory-pool callback (it would re-enter the
// allocator), or a host application whose device memory is owned and budgeted by another
// framework. They pass their own inputs and output; the scratch is ours.
#include <stdio.h>

#include <mutex>

#include <cuda.h>   // CUresult and the context id type only: the function itself comes from
                    // the runtime's driver entry-point query, so no link to libcuda

#include "internal.cuh"

namespace ctf {

constexpr int kNoAllocMaxBins = 16384;   // most frequency bins per call (128 KiB of scratch)

// Scratch shared by every call on a device: one FP64 partial per bin. Each call writes
// slots [0, F) before reading them, so nothing has to start at zero; two calls whose
// kernels overlap on the GPU race on these slots.
static __device__ __align__(256) double g_cost_scratch[kNoAllocMaxBins];

struct NoAllocShape {
    int M, N, B, F, J;
    int row_n[CTFMNMF_MAX_M], row_l[CTFMNMF_MAX_M];
};

// Per bin i: sum over rows r = (n,l) and frames j >= l of log lambda + |y|^2 / lambda with
// lambda_{n,i,j-l} = max(sum_k T[n][i][k] V[n][k][j-l], floor), then minus 2 J log|det W_i|.
__global__ void noalloc_cost_bins(const NoAllocShape s, const float2* __restrict__ Y,
                                  const float* __restrict__ T, const float* __restrict__ V,
                                  const double* __restrict__ logdet, double* __restrict__ scratch)
{
    __shared__ double part[32];
    const int i = blockIdx.x;
    const int M = s.M, B = s.B, F = s.F, J = s.J;
    double acc = 0.0;
    for (int r = 0; r < M; ++r) {
        const int n = s.row_n[r], l = s.row_l[r];
        const float2* yr = Y + ((size_t)r * F + i) * J;
        const float* Ti = T + ((size_t)n * F + i) * B;
        float a = 0.f;
        for (int j = l + threadIdx.x; j < J; j += blockDim.x) {
            float lam = 0.f;
            for (int k = 0; k < B; ++k) lam = fmaf(Ti[k], V[((size_t)n * B + k) * J + j - l], lam);
            lam = fmaxf(lam, kFloorPsd);
            a += logf(lam) + abs2(yr[j]) / lam;
        }
        acc += (double)a;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        scratch[i] = t - 2.0 * (double)J * logdet[i];
    }
}

__global__ void noalloc_cost_sum(const int F, const double* __restrict__ scratch, double* __restrict__ out)
{
    __shared__ double part[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < F; i += blockDim.x) acc += scratch[i];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = t;
    }
}

// Id of the context current on this thread (cuCtxGetId of the current context), 0 when none
// is current or the query is unavailable. The id is unique for the life of the process, so
// a device reset (a new primary context) shows up as a new id.
static unsigned long long current_context_id()
{
    typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
    static CtxGetIdFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (CtxGetIdFn) nullptr;
        }
        return reinterpret_cast<CtxGetIdFn>(p);
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device (the array's name in host code
// is only a host-side stand-in, not a device address). Looked up with cudaGetSymbolAddress
// once per device and context: after a device reset the library's module is loaded again
// and the array may move, so a new context id triggers a fresh lookup.
static double* scratch_address(int* err)
{
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    static unsigned long long ctx_of[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *err = e != cudaSuccess ? (int)e : (int)cudaErrorInvalidDevice;
        return nullptr;
    }
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || ctx == 0 || ctx != ctx_of[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cost_scratch);     // makes the device's context current
        if (e != cudaSuccess) {
            *err = (int)e;
            return nullptr;
        }
        addr[dev] = static_cast<double*>(p);
        ctx_of[dev] = current_context_id();
    }
    return addr[dev];
}

}  // namespace ctf

extern "C" int ctfmnmf_cost_noalloc(int M, int N, const int* Ln, int B, int F, int J, const void* Y,
                                    const float* T, const float* V, const double* logdet, double* out,
                                    void* stream)
{
    using namespace ctf;
    char msg[256];
    set_thread_error("");
    if (M <= 0 || N <= 0 || B <= 0 || F <= 0 || J <= 0 || N > M || M > CTFMNMF_MAX_M) {
        snprintf(msg, sizeof(msg), "invalid dimensions");
        set_thread_error(msg);
        return CTFMNMF_EINVAL;
    }
    if (F > kNoAllocMaxBins) {
        snprintf(msg, sizeof(msg), "F=%d exceeds the %d bins of the static scratch", F,
                 kNoAllocMaxBins);
        set_thread_error(msg);
        return CTFMNMF_EINVAL;
    }
    if (!Ln || !Y || !T || !V || !logdet || !out) {
        snprintf(msg, sizeof(msg), "null pointer argument");
        set_thread_error(msg);
        return CTFMNMF_EINVAL;
    }
    NoAllocShape s;
    s.M = M; s.N = N; s.B = B; s.F = F; s.J = J;
    int total = 0, lmax = 0;
    for (int n = 0; n < N; ++n) {
        if (Ln[n] <= 0 || total + Ln[n] > M) {
            snprintf(msg, sizeof(msg), "taps must be positive and sum to M");
            set_thread_error(msg);
            return CTFMNMF_EINVAL;
        }
        for (int l = 0; l < Ln[n]; ++l) {
            s.row_n[total + l] = n;
            s.row_l[total + l] = l;
        }
        total += Ln[n];
        if (Ln[n] > lmax) lmax = Ln[n];
    }
    if (total != M || J <= lmax) {
        snprintf(msg, sizeof(msg), "taps must sum to M and J must exceed every tap count");
        set_thread_error(msg);
        return CTFMNMF_EINVAL;
    }
    int err = 0;
    double* scratch = scratch_address(&err);
    if (!scratch) {
        snprintf(msg, sizeof(msg), "cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString((cudaError_t)err));
        set_thread_error(msg);
        return CTFMNMF_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    noalloc_cost_bins<<<F, 256, 0, st>>>(s, (const float2*)Y, T, V, logdet, scratch);
    noalloc_cost_sum<<<1, 256, 0, st>>>(F, scratch, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "launch failed: %s", cudaGetErrorString(e));
        set_thread_error(msg);
        return CTFMNMF_ECUDA;
    }
    return CTFMNMF_OK;
}
