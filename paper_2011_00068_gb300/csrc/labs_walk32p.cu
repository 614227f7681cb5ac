// labs_walk32p.cu -- instantiations of the walk kernel with one walker per warp: the walk under the PSL objective.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn32p(int rmax)
{
    switch (rmax) {  // block_R(n, 32) is odd
        case 1: return walk_chunk_kernel<32, 1, 3>;
        case 3: return walk_chunk_kernel<32, 3, 3>;
        case 5: return walk_chunk_kernel<32, 5, 3>;
        case 7: return walk_chunk_kernel<32, 7, 3>;
        default: return walk_chunk_kernel<32, 9, 3>;
    }
}

}  // namespace labsgpu
