// Batched bin-phase instantiations for M = 6 extended rows.
#include "batch_kernels.cuh"

namespace ctf {

cudaError_t batch_bin_m6(int fpt, int kb, const MixDesc* mixes, const int2* work, int blocks, int nt, size_t smem,
                          int v_tap0, cudaStream_t st, bool cfg)
{
    return bin_m<6>(fpt, kb, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
}

}  // namespace ctf
