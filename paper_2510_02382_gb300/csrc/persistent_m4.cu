// Persistent kernel instantiations for M = 4 microphones (8 frames per thread).
#include "persistent_kernel.cuh"

namespace ctf {

const void* persistent_ptr_m4(int BB)
{
    switch (BB) {
        case 4: return reinterpret_cast<const void*>(persistent_kernel<4, 8, 4>);
        case 8: return reinterpret_cast<const void*>(persistent_kernel<4, 8, 8>);
        case 10: return reinterpret_cast<const void*>(persistent_kernel<4, 8, 10>);
        case 16: return reinterpret_cast<const void*>(persistent_kernel<4, 8, 16>);
    }
    return nullptr;
}

}  // namespace ctf
