// labs_walk32b.cu -- instantiations of the walk kernel with one walker per warp: the best-first search.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn32b(int rmax)
{
    switch (rmax) {  // block_R(n, 32) is odd
        case 1: return walk_chunk_kernel<32, 1, 2>;
        case 3: return walk_chunk_kernel<32, 3, 2>;
        case 5: return walk_chunk_kernel<32, 5, 2>;
        case 7: return walk_chunk_kernel<32, 7, 2>;
        default: return walk_chunk_kernel<32, 9, 2>;
    }
}

}  // namespace labsgpu
