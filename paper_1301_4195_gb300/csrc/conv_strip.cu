// K2, strip kernel (float; N in {8, 16, 24, 32, 48, 64}): the weighted convolution of
// Sec. 3.2 (the kernel and its launchers are templates in strip.cuh; this
// translation unit instantiates them with stored weight tiles, conv_radius.cu
// with tiles rebuilt from the radius tables, conv_mixed.cu for uneven batches),
//   Qhat(zeta_k) = dzeta^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m),
// over the symmetrised half-tiles of the weight table (weights.cu).
//
// Work decomposition.  A work item is one output pencil (k1, k2, all k3) of
// GPC groups of 32 cells (one cell per lane), or, with S parts, one of S
// consecutive ranges of that pencil's tiles: part p sums tiles
// ceil(pT/S) .. ceil((p+1)T/S)-1 into its own partial sum (Qh, Qh2, Qh3,
// Qh4); the last range of a (pencil, block) to finish adds the partial sums
// into Qh in that fixed order.  At N = 16 S is 4 or 2, a handle's tuning
// choice (CS_TUNE_SPLIT): smaller items shorten the tail of a launch over
// few cells (128 cells: 3 % less time with 4), fewer save the combining at
// many (2048 cells: 5 % less with 2).  At N = 32 S is 1 (default), 2 or 4
// (conv_split32.cu); the few-cell kernel splits the same way.  The split belongs to the handle, not
// to a call, so a cell's result never depends on how many cells share the
// launch.  The pencil's k3 range is cut
// into N/K strips of K outputs; warp (group g, strip w) keeps only its K
// complex accumulators (plus a compensation pair) in registers.  CTAs are
// persistent and take items from an atomic counter, heaviest pencils first.
//
// Data movement.  Per (m1, m2) tile the CTA needs the partner rows
// fhat(m1, m2, :) and fhat(s1, s2, :) of its 32 cells and the tile's weights.
// One elected thread stages the three (two rows of N*256 bytes and the weight
// tile) into shared memory with cp.async.bulk (TMA bulk copies) on a ring of
// NST stages guarded by mbarriers ("full": bytes landed; "empty": every warp is
// done with the stage), so the warps never wait on global memory and each tile
// crosses L2 once per CTA.
//
// Inner loop.  For strip [k0, k0+K) the valid m3 form a run of "uniform" rows
// where all K outputs are valid and a triangle where they are not (see the
// STRIP layout in cs_internal.cuh).  Uniform rows are processed in blocks of U:
// U values fhat(m1,m2,m3), the U+K-1 partner values of the sliding window
// fhat(s1,s2,k3-m3+N/2) and U*K weights (float4 broadcasts) are read from
// shared memory and combined in U*K fully unrolled complex multiply-adds; the
// block loop itself is a runtime loop, so the code stays small.  The triangle
// rows are unrolled at compile time.  No pair is computed that the method
// drops, and no index arithmetic sits in the multiply-add stream.
//
// Precision.  Each m1 slab is accumulated in float and folded into a (hi, lo)
// pair by an error-free two-sum (compensated sum over xi).
//
// Waits.  Every mbarrier wait is bounded by %globaltimer (2 s); on expiry the
// kernel sets bit 0 of *err, tells the other warps through shared memory,
// waits (bounded) for the copies it issued, and returns; cs_status() reports it.
#include <algorithm>

#include "strip.cuh"

namespace cs {

int conv_split_max(const Handle &hd)
{
    return (hd.precision == CS_FP32 && hd.g.layout == LAYOUT_STRIP && (hd.g.N == 16 || hd.g.N == 32)) ? 4 : 1;
}

int conv_split(const Handle &hd)
{
    if (conv_split_max(hd) == 1) return 1;
    if (hd.g.N == 32) return hd.tune_split == 4 ? 4 : hd.tune_split == 2 ? 2 : 1;  // default: whole pencils
    return hd.tune_split == 4 ? 4 : 2;
}

bool strip_uses_radius(const Handle &hd)
{
    return hd.radA && (!hd.has_table || hd.tune_weights == 2);
}

bool tile_shapes_available(const Handle &hd)
{
    return hd.precision == CS_FP32 && hd.g.layout == LAYOUT_STRIP &&
           (hd.g.N == 16 || (hd.g.N == 32 && conv_split(hd) == 1)) && !strip_uses_radius(hd);
}

int launch_strip(const Handle &hd, int ncells, cudaStream_t s)
{
    if (lane_conv_applies(hd, ncells)) return launch_strip_lane(hd, ncells, s);
    if (strip_uses_radius(hd)) return launch_strip_radius(hd, ncells, s);
    if (hd.tune_tile >= 2 && tile_shapes_available(hd)) return launch_strip_tiles(hd, ncells, s);
    return launch_strip_mode<false>(hd, ncells, s);
}

}  // namespace cs
