// Per-bin adjoint instantiations for M = 2 extended rows.
#include "grad_bin.cuh"

namespace ctf {

cudaError_t grad_bin_m2(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                         cudaStream_t st, bool configure)
{
    return bin_m<2>(s, S, cur, nxt, g, st, configure);
}

}  // namespace ctf
