// labs_walk8a.cu -- instantiations of the walk kernel with four walkers per warp, lane blocks 1-6.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn8a(int rmax)
{
    switch (rmax) {
        case 1: return walk_quad_kernel<1>;
        case 2: return walk_quad_kernel<2>;
        case 3: return walk_quad_kernel<3>;
        case 4: return walk_quad_kernel<4>;
        case 5: return walk_quad_kernel<5>;
        default: return walk_quad_kernel<6>;
    }
}

}  // namespace labsgpu
