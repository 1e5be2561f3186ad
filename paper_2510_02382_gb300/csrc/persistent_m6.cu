// Persistent kernel instantiations for M = 6 microphones (4 frames per thread).
#include "persistent_kernel.cuh"

namespace ctf {

const void* persistent_ptr_m6(int BB)
{
    switch (BB) {
        case 4: return reinterpret_cast<const void*>(persistent_kernel<6, 4, 4>);
        case 8: return reinterpret_cast<const void*>(persistent_kernel<6, 4, 8>);
        case 10: return reinterpret_cast<const void*>(persistent_kernel<6, 4, 10>);
        case 16: return reinterpret_cast<const void*>(persistent_kernel<6, 4, 16>);
    }
    return nullptr;
}

}  // namespace ctf
