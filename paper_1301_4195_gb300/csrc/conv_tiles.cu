// K2 with other tile shapes (the autotuner's xi-tile and ring-depth choices,
// CS_TUNE_TILE): the strip kernel of conv_strip.cu at N = 16 and 32 with
// blocks of U = 4 uniform rows instead of 8, or a ring of 2 or 4 stages
// instead of 3, in a translation unit of its own so these instantiations
// compile in parallel with the others.  Every output still adds its terms
// row by row in increasing m3 (the block size only groups the unrolled rows)
// and the ring depth moves no arithmetic, so each choice gives the same
// result bit for bit; only the time differs.
#include <algorithm>

#include "strip.cuh"

namespace cs {

namespace {

template <int U, int NST>
int launch_tile_shape(const Handle &hd, int ncells, cudaStream_t s)
{
    switch (hd.g.N) {
    case 16:
        return conv_split(hd) == 2 ? launch_n<16, 8, U, NST, NST, 2, false>(hd, ncells, s)
                                   : launch_n<16, 8, U, NST, NST, 4, false>(hd, ncells, s);
    case 32: return launch_n<32, 8, U, NST, NST, 1, false>(hd, ncells, s);
    default: return set_error(CS_ENOTSUP, "tile shapes other than the default: N = 16 and 32 only");
    }
}

}  // namespace

int launch_strip_tiles(const Handle &hd, int ncells, cudaStream_t s)
{
    switch (hd.tune_tile) {
    case 2: return launch_tile_shape<4, 3>(hd, ncells, s);
    case 3: return launch_tile_shape<8, 4>(hd, ncells, s);
    case 4: return launch_tile_shape<8, 2>(hd, ncells, s);
    default: return set_error(CS_EINVAL, "unknown tile shape");
    }
}

}  // namespace cs
