// Batched path: many mixtures (each a ctfmnmf handle with its own shape and state)
// advanced together. Per iteration every launch class runs one bin-phase kernel whose
// blocks each take one (mixture, bin) pair, then every frame class runs one frame-phase
// kernel whose blocks each take one (mixture, 8-frame tile, source) item; the device code
// is bin_body / frame_item of phases.cuh, reading the mixture's shape and buffers from a
// descriptor table in device memory.
#include "phases.cuh"

namespace ctf {

// bin-phase instantiations in batch_m<M>.cu (kernel: batch_kernels.cuh)
cudaError_t batch_bin_m2(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);
cudaError_t batch_bin_m3(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);
cudaError_t batch_bin_m4(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);
cudaError_t batch_bin_m5(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);
cudaError_t batch_bin_m6(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);
cudaError_t batch_bin_m7(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);
cudaError_t batch_bin_m8(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg);

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
cudaError_t launch_batch_bin(const BatchClass& c, const MixDesc* mixes, int v_tap0, cudaStream_t st, bool configure)
{
    switch (c.M) {
        case 2: return batch_bin_m2(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 3: return batch_bin_m3(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 4: return batch_bin_m4(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 5: return batch_bin_m5(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 6: return batch_bin_m6(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 7: return batch_bin_m7(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
        case 8: return batch_bin_m8(c.fpt, c.kb, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st, configure);
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
