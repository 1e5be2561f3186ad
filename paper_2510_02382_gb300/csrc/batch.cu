// Batched path: many mixtures (each a ctfmnmf handle with its own shape and state)
// advanced together. Per iteration every launch class runs one bin-phase kernel whose
// blocks each take one (mixture, bin) pair, then every frame class runs one frame-phase
// kernel whose blocks each take one (mixture, 8-frame tile, source) item; the device code
// is bin_body / frame_item of phases.cuh, reading the mixture's shape and buffers from a
// descriptor table in device memory.
#include "phases.cuh"

namespace ctf {

// ---------------------------------------------------------------- bin phase (batched)
template <int M, int FPT, int MAXT, int MINB>
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
    const int i = w.y;
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

// ---------------------------------------------------------------- frame phase (batched)
constexpr int kBatchFrameThreads = 256;
constexpr int kBatchFrameSmemBytes = 48 * 1024;

template <int BB>
__global__ void __launch_bounds__(kBatchFrameThreads)
batch_frame_kernel(const MixDesc* __restrict__ mixes, const int2* __restrict__ work, const int v_tap0,
                   const int normalize)
{
    extern __shared__ float4 fsm4[];
    __shared__ MixDesc md;
    __shared__ float s_scale[CTFMNMF_MAX_M];
    __shared__ float red_cta[(kBatchFrameThreads / 32) * CTFMNMF_MAX_M];
    const int2 w = work[blockIdx.x];                   // (mixture, item)
    {
        const int* src = reinterpret_cast<const int*>(mixes + w.x);
        int* dst = reinterpret_cast<int*>(&md);
        for (int e = threadIdx.x; e < (int)(sizeof(MixDesc) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
    }
    __syncthreads();
    const Shape& s = md.s;
    const State& d = md.d;
    const Grp g{(int)threadIdx.x, kBatchFrameThreads, 0};
    const int fixed = frame_smem_fixed<BB>(kBatchFrameThreads);
    const int FC = frame_chunk(kBatchFrameSmemBytes / 4, s.B, fixed);
    const ScaleJob job{s_scale, red_cta, normalize};
    if constexpr (BB <= 16) frame_item<BB>(s, d, w.y, g, reinterpret_cast<float*>(fsm4), FC, s_scale, v_tap0, &job);
    else frame_item_wide<BB>(s, d, w.y, g, reinterpret_cast<float*>(fsm4), FC, s_scale, v_tap0, &job);
    if (w.y == 0 && threadIdx.x < s.M) d.scale[threadIdx.x] = s_scale[threadIdx.x];
}

// ---------------------------------------------------------------- dispatch
template <int M, int FPT>
static cudaError_t bin_mf(const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem, int v_tap0,
                          cudaStream_t st, bool configure)
{
    constexpr int kMaxT = FPT == 8 ? 512 : 256;
    constexpr int kMinB = FPT == 8 ? 1 : ((FPT == 4 && M * FPT < 16) ? 4 : 2);
    if (configure) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, batch_bin_kernel<M, FPT, kMaxT, kMinB>);
        if (e != cudaSuccess) return e;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;
        if (dyn_max < (int)smem) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(batch_bin_kernel<M, FPT, kMaxT, kMinB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    }
    if (nt > kMaxT || nt % 32 != 0) return cudaErrorInvalidValue;
    batch_bin_kernel<M, FPT, kMaxT, kMinB><<<blocks, nt, smem, st>>>(mixes, work, v_tap0);
    return cudaGetLastError();
}

template <int M>
static cudaError_t bin_m(int fpt, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                         int v_tap0, cudaStream_t st, bool cfg)
{
    switch (fpt) {
        case 1: return bin_mf<M, 1>(mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 2: return bin_mf<M, 2>(mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 4: return bin_mf<M, 4>(mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 8: if constexpr (M <= 4) return bin_mf<M, 8>(mixes, work, blocks, nt, smem, v_tap0, st, cfg);
                return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_bin(const BatchClass& c, const MixDesc* mixes, int v_tap0, cudaStream_t st, bool configure)
{
    switch (c.M) {
        case 2: return bin_m<2>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 3: return bin_m<3>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 4: return bin_m<4>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 5: return bin_m<5>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 6: return bin_m<6>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 7: return bin_m<7>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 8: return bin_m<8>(c.fpt, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
    }
    return cudaErrorInvalidValue;
}

static int batch_frame_bb(int B) { return B <= 4 ? 4 : B <= 8 ? 8 : B <= 10 ? 10 : B <= 16 ? 16 : 32; }

cudaError_t configure_batch_frame()
{
    const int bytes = kBatchFrameSmemBytes;
    cudaError_t e = cudaFuncSetAttribute(batch_frame_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_frame_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_frame_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_frame_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_frame_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

int batch_frame_class(int B) { return batch_frame_bb(B); }

// Frame chunk of a mixture with B bases in a frame class of width BB (host check).
int batch_frame_chunk(int B, int BB)
{
    const int fixed = BB == 4 ? frame_smem_fixed<4>(kBatchFrameThreads)
                    : BB == 8 ? frame_smem_fixed<8>(kBatchFrameThreads)
                    : BB == 10 ? frame_smem_fixed<10>(kBatchFrameThreads)
                    : BB == 16 ? frame_smem_fixed<16>(kBatchFrameThreads) : frame_smem_fixed<32>(kBatchFrameThreads);
    return frame_chunk(kBatchFrameSmemBytes / 4, B, fixed);
}

cudaError_t launch_batch_frame(int BB, const MixDesc* mixes, const int2* work, int blocks, int v_tap0,
                               int normalize, cudaStream_t st)
{
    const size_t smem = kBatchFrameSmemBytes;
    switch (BB) {
        case 4: batch_frame_kernel<4><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize); break;
        case 8: batch_frame_kernel<8><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize); break;
        case 10: batch_frame_kernel<10><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize); break;
        case 16: batch_frame_kernel<16><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize); break;
        case 32: batch_frame_kernel<32><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ctf
