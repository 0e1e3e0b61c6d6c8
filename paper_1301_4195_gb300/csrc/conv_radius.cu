// K2 with the weights rebuilt from the radius tables (weights.cu): the strip
// kernel of conv_strip.cu with RAD = true, in a translation unit of its own
// so the two sets of instantiations compile in parallel.  Each warp rebuilds
// its strip's weight segment of every tile in shared memory (three float
// gathers per entry: A(|k'|^2, |2m'-k'|^2), B(|m'|^2), B(|k'-m'|^2)) while
// the tile's f-hat rows are in flight; the rest of the kernel is unchanged.
#include <algorithm>

#include "strip.cuh"

namespace cs {

int launch_strip_radius(const Handle &hd, int ncells, cudaStream_t s)
{
    if (!hd.radA) return set_error(CS_ENOTSUP, "strip kernel: the handle has no radius tables");
    return launch_strip_mode<true>(hd, ncells, s);
}

}  // namespace cs
