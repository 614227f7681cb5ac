// labs_walk32l.cu -- instantiations of the walk kernel with one walker per warp: the learned mode.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn32l(int rmax)
{
    switch (rmax) {  // block_R(n, 32) is odd
        case 1: return walk_chunk_kernel<32, 1, 1>;
        case 3: return walk_chunk_kernel<32, 3, 1>;
        case 5: return walk_chunk_kernel<32, 5, 1>;
        case 7: return walk_chunk_kernel<32, 7, 1>;
        default: return walk_chunk_kernel<32, 9, 1>;
    }
}

}  // namespace labsgpu
