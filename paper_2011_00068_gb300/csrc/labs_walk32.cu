// labs_walk32.cu -- instantiations of the walk kernel with one walker per warp: the plain walk.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn32(int rmax)
{
    switch (rmax) {  // block_R(n, 32) is odd
        case 1: return walk_chunk_kernel<32, 1, 0>;
        case 3: return walk_chunk_kernel<32, 3, 0>;
        case 5: return walk_chunk_kernel<32, 5, 0>;
        case 7: return walk_chunk_kernel<32, 7, 0>;
        default: return walk_chunk_kernel<32, 9, 0>;
    }
}

}  // namespace labsgpu
