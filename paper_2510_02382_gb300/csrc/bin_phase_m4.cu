// Bin-phase instantiations for M = 4 extended rows.
#include "bin_phase_kernels.cuh"

namespace ctf {

cudaError_t bin_phase_m4(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg)
{
    return launch_m<4>(s, d, v_tap0, fpt, nt, st, cfg);
}

cudaError_t ip_bin_phase_m4(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg)
{
    return launch_ip_m<4>(s, d, v_tap0, fpt, nt, st, cfg);
}

}  // namespace ctf
