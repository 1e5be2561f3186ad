// Bin-phase instantiations for M = 6 extended rows.
#include "bin_phase_kernels.cuh"

namespace ctf {

cudaError_t bin_phase_m6(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg)
{
    return launch_m<6>(s, d, v_tap0, fpt, nt, st, cfg);
}

}  // namespace ctf
