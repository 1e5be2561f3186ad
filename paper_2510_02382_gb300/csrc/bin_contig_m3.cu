// Contiguous-frame bin-phase instantiations for M = 3 extended rows (every source count N <= M
// with the default taps, each bases-group count), the two-kernel and the batched kernels.
#include "bin_contig.cuh"

namespace ctf {

template <int N, int GB>
static cudaError_t contig_launch_n(const Shape& s, const State& d, const MixDesc* mixes, const int2* work,
                                   int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg)
{
    if (cfg) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mixes ? (const void*)batch_contig_bin_kernel<3, N, GB>
                                                                   : (const void*)contig_bin_kernel<3, N, GB>);
        if (e != cudaSuccess) return e;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;
        if (dyn_max < (int)smem) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(mixes ? (const void*)batch_contig_bin_kernel<3, N, GB> : (const void*)contig_bin_kernel<3, N, GB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    }
    if (nt % 32 != 0 || nt > kContigMaxThreads) return cudaErrorInvalidValue;
    if (mixes) batch_contig_bin_kernel<3, N, GB><<<blocks, nt, smem, st>>>(mixes, work, v_tap0);
    else contig_bin_kernel<3, N, GB><<<s.F, nt, smem, st>>>(s, d, v_tap0);
    return cudaGetLastError();
}

template <int N>
static cudaError_t contig_launch_g(int GB, const Shape& s, const State& d, const MixDesc* mixes, const int2* work,
                              int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg)
{
    switch (GB) {
        case 1: return contig_launch_n<N, 1>(s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 3: return contig_launch_n<N, 3>(s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 4: return contig_launch_n<N, 4>(s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 8: return contig_launch_n<N, 8>(s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
    }
    return cudaErrorInvalidValue;
}

cudaError_t contig_launch_m3(int N, int GB, const Shape& s, const State& d, const MixDesc* mixes, const int2* work,
                              int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg)
{
    switch (N) {
        case 1: return contig_launch_g<1>(GB, s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 2: return contig_launch_g<2>(GB, s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 3: return contig_launch_g<3>(GB, s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ctf
