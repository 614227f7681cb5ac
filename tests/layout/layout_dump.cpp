// Prints the shared-memory layouts the kernels use (labs_internal.cuh, compiled for the
// host): one line per (kind, tile, n_max): apad alen gpad glen bvec xoff words R xp hoff hlen hpad roff (the
// walk, and as "warpp" the PSL walk with two walkers per warp; the
// row layout: apad alen gpad glen bvec boff poff words R roff xp hoff hlen hpad; the long
// layout: apad alen gpad glen bvec xoff words R limit psl xp hoff hlen hpad roff).
#define __host__
#define __device__
#include <cstdio>

#include "labs_internal.cuh"

using namespace labsgpu;

int main()
{
    const int tiles[3] = {8, 16, 32};
    for (int ti = 0; ti < 3; ++ti)
        for (int n = 2; n <= kMaxN; ++n) {
            const WarpSmem w = warp_smem(n, tiles[ti]);
            std::printf("warp %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", tiles[ti], n, w.apad, w.alen, w.gpad,
                        w.glen, w.bvec, w.xoff, w.words, block_R(n, tiles[ti]), w.xp, w.hoff, w.hlen, w.hpad, w.roff);
        }
    for (int n = 2; n <= 128; ++n) {  // the PSL walk with two walkers per warp
        const WarpSmem w = warp_smem(n, 16, true);
        std::printf("warpp 16 %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", n, w.apad, w.alen, w.gpad, w.glen, w.bvec,
                    w.xoff, w.words, block_R(n, 16), w.xp, w.hoff, w.hlen, w.hpad, w.roff);
    }
    for (int n = 2; n <= kMaxN; ++n) {  // the row kernels: two rows per warp up to n = 160
        const int tile = n <= 160 ? 16 : 32;
        const WarpSmem w = row_smem(n, tile);
        std::printf("row %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", tile, n, w.apad, w.alen, w.gpad, w.glen,
                    w.bvec, w.boff, w.poff, w.words, block_R(n, tile), w.roff, w.xp, w.hoff, w.hlen, w.hpad);
    }
    for (int n = kMaxN + 1; n <= kMaxNLong; ++n)
        for (int psl = 0; psl < 2; ++psl) {  // the CTA width of the walk and of the PSL walk
            const int nt = long_threads(n, psl != 0);
            if (psl && nt == long_threads(n, false)) continue;
            const WarpSmem w = long_smem(n, nt);
            std::printf("long %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", nt, n, w.apad, w.alen, w.gpad,
                        w.glen, w.bvec, w.xoff, w.words, long_R(n, nt), long_isl_limit(2 * n - 1, n), psl, w.xp,
                        w.hoff, w.hlen, w.hpad, w.roff);
        }
    return 0;
}
