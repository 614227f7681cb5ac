// labs_walk16.cu -- instantiations of the walk kernel with two walkers per warp (16 lanes each).
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn16(int rmax)
{
    switch (rmax) {
        case 1: return walk_chunk_kernel<16, 1>;
        case 2: return walk_chunk_kernel<16, 2>;
        case 3: return walk_chunk_kernel<16, 3>;
        case 4: return walk_chunk_kernel<16, 4>;
        case 5: return walk_chunk_kernel<16, 5>;
        case 6: return walk_chunk_kernel<16, 6>;
        case 7: return walk_chunk_kernel<16, 7>;
        default: return walk_chunk_kernel<16, 8>;
    }
}

}  // namespace labsgpu
