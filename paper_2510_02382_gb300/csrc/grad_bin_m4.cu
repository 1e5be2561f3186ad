// Per-bin adjoint instantiations for M = 4 extended rows.
#include "grad_bin.cuh"

namespace ctf {

cudaError_t grad_bin_m4(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                         cudaStream_t st, bool configure)
{
    return bin_m<4>(s, S, cur, nxt, g, st, configure);
}

}  // namespace ctf
