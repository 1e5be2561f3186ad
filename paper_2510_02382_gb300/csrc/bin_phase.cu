// Bin phase of the two-kernel path: one CTA per frequency bin runs the ISS sweep (or, for
// handles created with the IP update, the IP sweep of Eqs. 9-10) and the basis update of
// Sec. III for its bin (device code in phases.cuh).
#include "phases.cuh"

namespace ctf {

template <int M, int FPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
bin_phase_kernel(const Shape s, const State d, const int v_tap0)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ float s_scale[CTFMNMF_MAX_M];
    const int i = blockIdx.x;
    const Grp g{(int)threadIdx.x, (int)blockDim.x, 0};
    if (threadIdx.x < CTFMNMF_MAX_M) s_scale[threadIdx.x] = (int)threadIdx.x < M ? d.scale[threadIdx.x] : 1.f;
    __syncthreads();

    float2 y[M][FPT];
    float2 wcol[M];
    float2* Yb = d.Y + (size_t)i * M * s.Jp;
    float2* Wb = d.W + (size_t)i * M * M;
    load_bin<M, FPT, true>(s.Jp, Yb, Wb, g, s_scale, y, wcol);
    const float detf = bin_body<M, FPT, true>(s, d, i, g, smem, y, wcol, Yb, Wb, s_scale, v_tap0);
    if (g.tid == 0) {
        double f = (double)detf;
#pragma unroll
        for (int r = 0; r < M; ++r) f *= (double)s_scale[r];
        logdet_mul(d, i, f);
    }
}

// IP update (Eqs. 9-10) in place of the ISS sweep: same tail (rows, P, basis MU).
template <int M, int FPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
ip_bin_kernel(const Shape s, const State d, const int v_tap0)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ float s_scale[CTFMNMF_MAX_M];
    const int i = blockIdx.x;
    const Grp g{(int)threadIdx.x, (int)blockDim.x, 0};
    if (threadIdx.x < CTFMNMF_MAX_M) s_scale[threadIdx.x] = (int)threadIdx.x < M ? d.scale[threadIdx.x] : 1.f;
    __syncthreads();

    float2 y[M][FPT];
    float2 wcol[M];
    float2* Yb = d.Y + (size_t)i * M * s.Jp;
    float2* Wb = d.W + (size_t)i * M * M;
    load_bin<M, FPT, true>(s.Jp, Yb, Wb, g, s_scale, y, wcol);
    const float detf = bin_body<M, FPT, true, 16, true>(s, d, i, g, smem, y, wcol, Yb, Wb, s_scale, v_tap0);
    if (g.tid == 0) {
        double f = (double)detf;
#pragma unroll
        for (int r = 0; r < M; ++r) f *= (double)s_scale[r];
        logdet_mul(d, i, f);
    }
}

bool bin_phase_config(int M, int J, int* fpt, int* threads)
{
    // frames per thread 1, 2, 4 with at most 256 threads; 8 (M <= 4) with up to 512
    static const int cands[4] = {1, 2, 4, 8};
    for (int c = 0; c < 4; ++c) {
        const int f = cands[c];
        if (M * f > 32) break;
        const int cap = f == 8 ? 512 : 256;
        const int nt = (J + f - 1) / f;
        if (nt <= cap) {
            *fpt = f;
            *threads = ((nt + 31) / 32) * 32;
            if (*threads < 64) *threads = 64;
            return true;
        }
    }
    return false;
}

size_t bin_phase_smem(const Shape& s)
{
    int fpt = 0, nt = 0;
    bin_phase_config(s.M, s.J, &fpt, &nt);
    return sizeof(float) * (size_t)bin_smem_layout(s.M, s.N, s.Jp, nt).total;
}

// Every (frames per thread, threads) the bin phase can run this shape with: for each of
// 1, 2, 4 (up to 256 threads) and 8 (M <= 4, up to 512 threads) the threads that cover J.
int bin_phase_candidates(int M, int J, int* fpts, int* nts)
{
    static const int cands[4] = {1, 2, 4, 8};
    int k = 0;
    for (int c = 0; c < 4; ++c) {
        const int f = cands[c];
        if (M * f > 32) break;
        const int cap = f == 8 ? 512 : 256;
        const int nt = (J + f - 1) / f;
        if (nt > cap) continue;
        fpts[k] = f;
        nts[k] = nt < 64 ? 64 : ((nt + 31) / 32) * 32;
        ++k;
    }
    return k;
}

int bin_smem_floats(const Shape& s, int nt) { return bin_smem_layout(s.M, s.N, s.Jp, nt).total; }

template <int M, int FPT>
static cudaError_t launch_mf(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st,
                             bool configure_only)
{
    // 8 frames per thread: up to 512 threads, 128 registers; otherwise 256 threads and
    // 4 CTAs per SM (64 registers) for 4 frames per thread and M <= 3, else 2 CTAs per SM
    constexpr int kMaxT = FPT == 8 ? 512 : 256;
    constexpr int kMinB = FPT == 8 ? 1 : ((FPT == 4 && M * FPT < 16) ? 4 : 2);
    if (configure_only) {
        // the device's opt-in maximum, so that handles of different J share the setting
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, bin_phase_kernel<M, FPT, kMaxT, kMinB>);
        if (e != cudaSuccess) return e;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;      // static shared memory counts too
        if (dyn_max < (int)(sizeof(float) * (size_t)bin_smem_layout(s.M, s.N, s.Jp, nt).total))
            return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(bin_phase_kernel<M, FPT, kMaxT, kMinB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    }
    // float4 views of the staged rows need 16-byte aligned row starts
    if (s.Jp % 8 != 0 || nt > kMaxT) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)bin_smem_layout(s.M, s.N, s.Jp, nt).total;
    bin_phase_kernel<M, FPT, kMaxT, kMinB><<<s.F, nt, smem, st>>>(s, d, v_tap0);
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_m(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st,
                            bool cfg)
{
    switch (fpt) {
        case 1: return launch_mf<M, 1>(s, d, v_tap0, nt, st, cfg);
        case 2: return launch_mf<M, 2>(s, d, v_tap0, nt, st, cfg);
        case 4: return launch_mf<M, 4>(s, d, v_tap0, nt, st, cfg);
        case 8: if constexpr (M <= 4) return launch_mf<M, 8>(s, d, v_tap0, nt, st, cfg);
                return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dispatch(const Shape& s, const State& d, int v_tap0, cudaStream_t st, bool cfg, int fpt = 0,
                            int nt = 0)
{
    if (fpt == 0 && !bin_phase_config(s.M, s.J, &fpt, &nt)) return cudaErrorInvalidValue;
    switch (s.M) {
        case 2: return launch_m<2>(s, d, v_tap0, fpt, nt, st, cfg);
        case 3: return launch_m<3>(s, d, v_tap0, fpt, nt, st, cfg);
        case 4: return launch_m<4>(s, d, v_tap0, fpt, nt, st, cfg);
        case 5: return launch_m<5>(s, d, v_tap0, fpt, nt, st, cfg);
        case 6: return launch_m<6>(s, d, v_tap0, fpt, nt, st, cfg);
        case 7: return launch_m<7>(s, d, v_tap0, fpt, nt, st, cfg);
        case 8: return launch_m<8>(s, d, v_tap0, fpt, nt, st, cfg);
    }
    return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of the instantiation this shape uses (once per
// handle, outside any stream capture).
cudaError_t configure_bin_phase(const Shape& s)
{
    State none = {};
    return dispatch(s, none, 0, nullptr, true);
}

cudaError_t launch_bin_phase(const Shape& s, const State& d, int v_tap0, cudaStream_t st)
{
    return dispatch(s, d, v_tap0, st, false);
}

cudaError_t configure_bin_phase_as(const Shape& s, int fpt, int nt)
{
    State none = {};
    return dispatch(s, none, 0, nullptr, true, fpt, nt);
}

cudaError_t launch_bin_phase_as(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st)
{
    return dispatch(s, d, v_tap0, st, false, fpt, nt);
}

template <int M, int FPT>
static cudaError_t launch_ip_mf(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st, bool cfg)
{
    // one block per SM guaranteed: the covariance sums and the FP64 solve need registers
    constexpr int kMaxT = FPT == 8 ? 512 : 256;
    constexpr int kMinB = 1;
    if (cfg) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, ip_bin_kernel<M, FPT, kMaxT, kMinB>);
        if (e != cudaSuccess) return e;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;
        if (dyn_max < (int)bin_phase_smem(s)) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(ip_bin_kernel<M, FPT, kMaxT, kMinB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    dyn_max);
    }
    if (s.Jp % 8 != 0 || nt > kMaxT || !d.X) return cudaErrorInvalidValue;
    ip_bin_kernel<M, FPT, kMaxT, kMinB><<<s.F, nt, bin_phase_smem(s), st>>>(s, d, v_tap0);
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_ip_m(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg)
{
    switch (fpt) {
        case 1: return launch_ip_mf<M, 1>(s, d, v_tap0, nt, st, cfg);
        case 2: return launch_ip_mf<M, 2>(s, d, v_tap0, nt, st, cfg);
        case 4: return launch_ip_mf<M, 4>(s, d, v_tap0, nt, st, cfg);
        case 8: return launch_ip_mf<M, 8>(s, d, v_tap0, nt, st, cfg);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dispatch_ip(const Shape& s, const State& d, int v_tap0, cudaStream_t st, bool cfg)
{
    int fpt = 0, nt = 0;
    if (!bin_phase_config(s.M, s.J, &fpt, &nt)) return cudaErrorInvalidValue;
    switch (s.M) {
        case 2: return launch_ip_m<2>(s, d, v_tap0, fpt, nt, st, cfg);
        case 3: return launch_ip_m<3>(s, d, v_tap0, fpt, nt, st, cfg);
        case 4: return launch_ip_m<4>(s, d, v_tap0, fpt, nt, st, cfg);
    }
    return cudaErrorInvalidValue;
}

cudaError_t configure_ip_bin_phase(const Shape& s)
{
    State none = {};
    return dispatch_ip(s, none, 0, nullptr, true);
}

cudaError_t launch_ip_bin_phase(const Shape& s, const State& d, int v_tap0, cudaStream_t st)
{
    return dispatch_ip(s, d, v_tap0, st, false);
}

}  // namespace ctf
