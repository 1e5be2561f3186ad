// Bin-phase kernels of the two-kernel path and their launch templates, instantiated once
// per M in bin_phase_m<M>.cu so that the translation units compile in parallel.
#pragma once

#include "phases.cuh"

namespace ctf {

// KB: bases per basis-MU pass (4, 8, 10 or 16: the smallest class holding B, 16 above).
template <int M, int FPT, int MAXT, int MINB, int KB>
__global__ void __launch_bounds__(MAXT, MINB)
bin_phase_kernel(const Shape s, const State d, const int v_tap0)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ float s_scale[CTFMNMF_MAX_M];
    const int i = blockIdx.x;
#ifdef CTFMNMF_DEBUG
    if (i >= s.F || (int)blockDim.x * FPT < s.J) {     // a bin or a frame outside the launch
        if (threadIdx.x == 0) atomicOr(d.flag + 3, 1);
        return;
    }
#endif
    const Grp g{(int)threadIdx.x, (int)blockDim.x, 0};
    float2 y[M][FPT];
    float2 wcol[M];
    float2* Yb = d.Y + (size_t)i * M * s.Jp;
    float2* Wb = d.W + (size_t)i * M * M;
    load_bin_unscaled<M, FPT>(s.Jp, Yb, Wb, g, y, wcol);     // in flight while the scale arrives
    if (threadIdx.x < CTFMNMF_MAX_M) s_scale[threadIdx.x] = (int)threadIdx.x < M ? d.scale[threadIdx.x] : 1.f;
    __syncthreads();
    apply_bin_scale<M, FPT>(g, s_scale, y, wcol);
    const float detf = bin_body<M, FPT, true, KB, false, true, true>(s, d, i, g, smem, y, wcol, Yb, Wb, s_scale, v_tap0);
    if (g.tid == 0) d.detb[i] = det_factor<M>(detf, s_scale);   // folded by the frame phase
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
    float2 y[M][FPT];
    float2 wcol[M];
    float2* Yb = d.Y + (size_t)i * M * s.Jp;
    float2* Wb = d.W + (size_t)i * M * M;
    load_bin_unscaled<M, FPT>(s.Jp, Yb, Wb, g, y, wcol);     // in flight while the scale arrives
    if (threadIdx.x < CTFMNMF_MAX_M) s_scale[threadIdx.x] = (int)threadIdx.x < M ? d.scale[threadIdx.x] : 1.f;
    __syncthreads();
    apply_bin_scale<M, FPT>(g, s_scale, y, wcol);
    const float detf = bin_body<M, FPT, true, 16, true, false, true>(s, d, i, g, smem, y, wcol, Yb, Wb, s_scale, v_tap0);
    if (g.tid == 0) d.detb[i] = det_factor<M>(detf, s_scale);   // folded by the frame phase
}

template <int M, int FPT, int KB>
inline cudaError_t launch_mfk(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st,
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
        e = cudaFuncGetAttributes(&fa, bin_phase_kernel<M, FPT, kMaxT, kMinB, KB>);
        if (e != cudaSuccess) return e;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;      // static shared memory counts too
        if (dyn_max < (int)(sizeof(float) * (size_t)bin_smem_layout(s.M, s.N, s.Jp, nt).total))
            return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(bin_phase_kernel<M, FPT, kMaxT, kMinB, KB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    }
    // float4 views of the staged rows need 16-byte aligned row starts
    if (s.Jp % 8 != 0 || nt > kMaxT) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)bin_smem_layout(s.M, s.N, s.Jp, nt).total;
    bin_phase_kernel<M, FPT, kMaxT, kMinB, KB><<<s.F, nt, smem, st>>>(s, d, v_tap0);
    return cudaGetLastError();
}

template <int M, int FPT>
inline cudaError_t launch_mf(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st,
                             bool configure_only)
{
    switch (bases_class(s.B)) {
        case 4: return launch_mfk<M, FPT, 4>(s, d, v_tap0, nt, st, configure_only);
        case 8: return launch_mfk<M, FPT, 8>(s, d, v_tap0, nt, st, configure_only);
        case 10: return launch_mfk<M, FPT, 10>(s, d, v_tap0, nt, st, configure_only);
    }
    return launch_mfk<M, FPT, 16>(s, d, v_tap0, nt, st, configure_only);
}

template <int M>
inline cudaError_t launch_m(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st,
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

template <int M, int FPT>
inline cudaError_t launch_ip_mf(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st, bool cfg)
{
    // the covariance sums hold M (M + 1) / 2 complex partials per frame and the FP64 solve
    // runs on warp 0 with a few doubles per lane: 64 registers (four 256-thread blocks per
    // SM, so that 4 x 152 blocks cover 513 bins in one wave) below 8 frames per thread
    constexpr int kMaxT = FPT == 8 ? 512 : 256;
    constexpr int kMinB = FPT == 8 ? 1 : 4;
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
inline cudaError_t launch_ip_m(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg)
{
    switch (fpt) {
        case 1: return launch_ip_mf<M, 1>(s, d, v_tap0, nt, st, cfg);
        case 2: return launch_ip_mf<M, 2>(s, d, v_tap0, nt, st, cfg);
        case 4: return launch_ip_mf<M, 4>(s, d, v_tap0, nt, st, cfg);
        case 8: return launch_ip_mf<M, 8>(s, d, v_tap0, nt, st, cfg);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ctf
