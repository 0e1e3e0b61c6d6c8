// K2 at N = 32 with the tile split (CS_TUNE_SPLIT = 2 or 4): the strip
// kernel of conv_strip.cu (stored tiles) and conv_radius.cu (tiles rebuilt
// from the radius tables) with each pencil's tiles cut into S consecutive
// ranges, in a translation unit of its own so these instantiations compile
// in parallel with the others.  A range's partial sum goes to its own
// buffer and the last range to finish adds them in range order, as at
// N = 16; the few-cell kernel cuts and adds the same way, so a handle's
// results do not depend on which kernel served a call.  The split changes
// the rounding of each output's sum, not its terms; whole pencils (S = 1)
// remain the default at N = 32.
#include "strip.cuh"

namespace cs {

int launch_strip_split32(const Handle &hd, int ncells, cudaStream_t s, bool rad)
{
    const int S = conv_split(hd);
    if (rad)
        return S == 4 ? launch_n<32, 8, 8, 3, 3, 4, true>(hd, ncells, s) : launch_n<32, 8, 8, 3, 3, 2, true>(hd, ncells, s);
    return S == 4 ? launch_n<32, 8, 8, 3, 2, 4, false>(hd, ncells, s) : launch_n<32, 8, 8, 3, 2, 2, false>(hd, ncells, s);
}

}  // namespace cs
