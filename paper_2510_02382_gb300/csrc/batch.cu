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

// EXACT: every mixture of the launch has B equal to the class width BB. A work item
// (mixture, -1) forms that mixture's normalisation scale of this iteration (FP64, Eq. 19)
// and stores it as its pending scale; every other item is one (8-frame tile, source).
template <int BB, bool EXACT>
__global__ void __launch_bounds__(kBatchFrameThreads, frame_min_blocks<BB>())
batch_frame_kernel(const MixDesc* __restrict__ mixes, const int2* __restrict__ work, const int v_tap0,
                   const int normalize)
{
    extern __shared__ float4 fsm4[];
    __shared__ MixDesc md;
    const int2 w = work[blockIdx.x];                   // (mixture, item)
    {
        const int* src = reinterpret_cast<const int*>(mixes + w.x);
        int* dst = reinterpret_cast<int*>(&md);
        for (int e = threadIdx.x; e < (int)(sizeof(MixDesc) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
    }
    __syncthreads();
    const Shape& s = md.s;
    const State& d = md.d;
#ifdef CTFMNMF_DEBUG
    if (w.y < -1 || w.y >= (s.Jp / kFrameTile) * s.N) {   // an item outside the mixture
        if (threadIdx.x == 0) atomicOr(d.flag + 3, 1);
        return;
    }
#endif
    if (w.y < 0) {
        scales_fp64<true>(s, d, normalize, reinterpret_cast<double*>(fsm4));
        return;
    }
    const Grp g{(int)threadIdx.x, kBatchFrameThreads, 0};
    const int fixed = frame_smem_fixed<BB>(kBatchFrameThreads);
    const int FC = frame_chunk(kBatchFrameSmemBytes / 4, s.B, fixed);
    if constexpr (BB <= 16)
        frame_item<BB, EXACT, true>(s, d, w.y, g, reinterpret_cast<float*>(fsm4), FC, v_tap0);
    else
        frame_item_wide<BB, EXACT, true>(s, d, w.y, g, reinterpret_cast<float*>(fsm4), FC, v_tap0);
}

// ---------------------------------------------------------------- dispatch
cudaError_t launch_batch_bin(const BatchClass& c, const MixDesc* mixes, int v_tap0, cudaStream_t st, bool configure)
{
    if (c.fpt == kBinContig) {
        const Shape none_s = {};
        const State none_d = {};
        return contig_dispatch(c.M, c.N, c.kb, none_s, none_d, mixes, c.work, c.blocks, c.nt, c.smem, v_tap0, st,
                               configure);
    }
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

template <int BB>
static cudaError_t batch_frame_set(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(batch_frame_kernel<BB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_frame_kernel<BB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t configure_batch_frame()
{
    const int bytes = kBatchFrameSmemBytes;
    cudaError_t e = batch_frame_set<4>(bytes);
    if (e == cudaSuccess) e = batch_frame_set<8>(bytes);
    if (e == cudaSuccess) e = batch_frame_set<10>(bytes);
    if (e == cudaSuccess) e = batch_frame_set<16>(bytes);
    if (e == cudaSuccess) e = batch_frame_set<32>(bytes);
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

template <int BB>
static void batch_frame_launch(bool exact, const MixDesc* mixes, const int2* work, int blocks, int v_tap0,
                               int normalize, size_t smem, cudaStream_t st)
{
    if (exact) batch_frame_kernel<BB, true><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize);
    else batch_frame_kernel<BB, false><<<blocks, kBatchFrameThreads, smem, st>>>(mixes, work, v_tap0, normalize);
}

cudaError_t launch_batch_frame(int BB, int exact, const MixDesc* mixes, const int2* work, int blocks, int v_tap0,
                               int normalize, cudaStream_t st)
{
    const size_t smem = kBatchFrameSmemBytes;
    const bool ex = exact != 0;
    switch (BB) {
        case 4: batch_frame_launch<4>(ex, mixes, work, blocks, v_tap0, normalize, smem, st); break;
        case 8: batch_frame_launch<8>(ex, mixes, work, blocks, v_tap0, normalize, smem, st); break;
        case 10: batch_frame_launch<10>(ex, mixes, work, blocks, v_tap0, normalize, smem, st); break;
        case 16: batch_frame_launch<16>(ex, mixes, work, blocks, v_tap0, normalize, smem, st); break;
        case 32: batch_frame_launch<32>(ex, mixes, work, blocks, v_tap0, normalize, smem, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ctf
