// Batched bin-phase kernel and its launch templates, instantiated once per M in
// batch_m<M>.cu so that the translation units compile in parallel.
#pragma once

#include "phases.cuh"

namespace ctf {

// ---------------------------------------------------------------- bin phase (batched)
template <int M, int FPT, int MAXT, int MINB, int KB>
__global__ void __launch_bounds__(MAXT, MINB)
batch_bin_kernel(const MixDesc* __restrict__ mixes, const int2* __restrict__ work, const int v_tap0)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ MixDesc md;
    __shared__ float s_scale[CTFMNMF_MAX_M];
    const int2 w = work[blockIdx.x];                   // (mixture, bin)
    {
        const int* src = reinterpret_cast<const int*>(mixes + w.x);
        int* dst = reinterpret_cast<int*>(&md);
        for (int e = threadIdx.x; e < (int)(sizeof(MixDesc) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
    }
    __syncthreads();
    const Shape& s = md.s;
    const State& d = md.d;
#ifdef CTFMNMF_DEBUG
    if (w.y < 0 || w.y >= s.F) {                       // a bin outside the mixture: report, touch nothing
        if (threadIdx.x == 0) atomicOr(d.flag + 3, 1);
        return;
    }
#endif
    const int i = w.y;
    const Grp g{(int)threadIdx.x, (int)blockDim.x, 0};
    float2 y[M][FPT];
    float2 wcol[M];
    float2* Yb = d.Y + (size_t)i * M * s.Jp;
    float2* Wb = d.W + (size_t)i * M * M;
    load_bin_unscaled<M, FPT>(s.Jp, Yb, Wb, g, y, wcol);     // in flight while the scale arrives
    if (threadIdx.x < CTFMNMF_MAX_M) s_scale[threadIdx.x] = (int)threadIdx.x < M ? d.scale[threadIdx.x] : 1.f;
    __syncthreads();
    apply_bin_scale<M, FPT>(g, s_scale, y, wcol);
    const float detf = bin_body<M, FPT, true, KB, false, false, true>(s, d, i, g, smem, y, wcol, Yb, Wb, s_scale, v_tap0);
    if (g.tid == 0) d.detb[i] = det_factor<M>(detf, s_scale);   // folded by the frame phase
}

template <int M, int FPT, int KB>
inline cudaError_t bin_mfk(const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem, int v_tap0,
                           cudaStream_t st, bool configure)
{
    constexpr int kMaxT = FPT == 8 ? 512 : 256;
    constexpr int kMinB = FPT == 8 ? 1 : ((FPT == 4 && M * FPT < 16) ? 4 : 2);
    if (configure) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, batch_bin_kernel<M, FPT, kMaxT, kMinB, KB>);
        if (e != cudaSuccess) return e;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;
        if (dyn_max < (int)smem) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(batch_bin_kernel<M, FPT, kMaxT, kMinB, KB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    }
    if (nt > kMaxT || nt % 32 != 0) return cudaErrorInvalidValue;
    batch_bin_kernel<M, FPT, kMaxT, kMinB, KB><<<blocks, nt, smem, st>>>(mixes, work, v_tap0);
    return cudaGetLastError();
}

template <int M, int FPT>
inline cudaError_t bin_mf(int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool configure)
{
    switch (kb) {
        case 4: return bin_mfk<M, FPT, 4>(mixes, work, blocks, nt, smem, v_tap0, st, configure);
        case 8: return bin_mfk<M, FPT, 8>(mixes, work, blocks, nt, smem, v_tap0, st, configure);
        case 10: return bin_mfk<M, FPT, 10>(mixes, work, blocks, nt, smem, v_tap0, st, configure);
    }
    return bin_mfk<M, FPT, 16>(mixes, work, blocks, nt, smem, v_tap0, st, configure);
}

template <int M>
inline cudaError_t bin_m(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                         int v_tap0, cudaStream_t st, bool cfg)
{
    switch (fpt) {
        case 1: return bin_mf<M, 1>(kb, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 2: return bin_mf<M, 2>(kb, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 4: return bin_mf<M, 4>(kb, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 8: if constexpr (M <= 4) return bin_mf<M, 8>(kb, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
                return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

}  // namespace ctf
