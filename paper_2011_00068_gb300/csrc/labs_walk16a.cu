// labs_walk16a.cu -- instantiations of the walk kernel with two walkers per warp, lane blocks 1-5.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn16a(int rmax)
{
    switch (rmax) {
        case 1: return walk_pair_kernel<1>;
        case 2: return walk_pair_kernel<2>;
        case 3: return walk_pair_kernel<3>;
        case 4: return walk_pair_kernel<4>;
        case 5: return walk_pair_kernel<5>;
        default: return walk_pair_kernel<5>;
    }
}

}  // namespace labsgpu
