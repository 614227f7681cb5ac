// labs_walk16p.cu -- instantiations of the walk kernel with two walkers per warp under the PSL objective, lane
// blocks 1-5.
#include "labs_device.cuh"

namespace labsgpu {

WalkFn walk_fn16p(int rmax)
{
    switch (rmax) {  // block_R(n, 16) for n <= 128: 1, 2, 3, 5, 6, 7, 9
        case 1: return walk_psl_pair_kernel<1>;
        case 2: return walk_psl_pair_kernel<2>;
        case 3: return walk_psl_pair_kernel<3>;
        default: return walk_psl_pair_kernel<5>;
    }
}

}  // namespace labsgpu
