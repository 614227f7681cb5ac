// labs_walk16b.cu -- instantiations of the walk kernel with two walkers per warp, lane blocks 6-10.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn16b(int rmax)
{
    switch (rmax) {
        case 6: return walk_pair_kernel<6>;
        case 7: return walk_pair_kernel<7>;
        case 8: return walk_pair_kernel<8>;
        case 9: return walk_pair_kernel<9>;
        default: return walk_pair_kernel<10>;
    }
}

}  // namespace labsgpu
