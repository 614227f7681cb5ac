// labs_walk8b.cu -- instantiations of the walk kernel with four walkers per warp, lane blocks 7-10.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn8b(int rmax)
{
    switch (rmax) {  // block_R(n, 8) is never a multiple of 8
        case 7: return walk_quad_kernel<7>;
        case 9: return walk_quad_kernel<9>;
        default: return walk_quad_kernel<10>;
    }
}

}  // namespace labsgpu
