// labs_walk16q.cu -- instantiations of the walk kernel with two walkers per warp under the PSL objective, lane
// blocks 6-9.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn16q(int rmax)
{
    switch (rmax) {  // block_R(n, 16) for n <= 128: 1, 2, 3, 5, 6, 7, 9
        case 6: return walk_psl_pair_kernel<6>;
        case 7: return walk_psl_pair_kernel<7>;
        default: return walk_psl_pair_kernel<9>;
    }
}

}  // namespace labsgpu
