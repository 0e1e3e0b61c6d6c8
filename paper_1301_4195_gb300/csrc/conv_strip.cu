// K2, strip kernel (float; N in {8, 16, 24, 32, 48, 64}): the weighted convolution of
// Sec. 3.2,
//   Qhat(zeta_k) = dzeta^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m),
// over the symmetrised half-tiles of the weight table (weights.cu).
//
// Work decomposition.  A work item is one output pencil (k1, k2, all k3) of
// GPC groups of 32 cells (one cell per lane), or, with S = 2 parts, one half
// of that pencil's tiles: part 0 sums the first ceil(T/2) tiles into Qh,
// part 1 the rest into Qh2, and the consumer adds the two partial sums in
// that fixed order.  Halving the items lets more, smaller CTAs share an SM
// without a long tail; the split depends only on N and the precision, so a
// cell's result never depends on how many cells share the launch.  The pencil's k3 range is cut
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

namespace {

// Persistent kernel: CTAs take (pencil, group block) items from an atomic
// counter, heaviest pencils first, so the tail of the launch holds only the
// smallest items.
// Resident CTAs per SM the register allocation must allow: at N = 16 the
// kernel is latency-bound and 128 registers (8 one-group or 4 two-group CTAs
// per SM) measured faster than the ~134 the compiler picks on its own; for
// the other N one CTA (no cap) measured best.
template <int N, int GPC>
constexpr int strip_min_ctas() { return N == 16 ? (GPC == 1 ? 8 : 4) : 1; }

template <int N, int K, int U, int NST, int GPC, int S>
__global__ void __launch_bounds__(32 * (N / K) * GPC, strip_min_ctas<N, GPC>())
    conv_strip_kernel(StripJob jb, int *counter)
{
    using C = StripCfg<N, K, U, NST, GPC>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    Ring rg = ring_init<NST, C::WARPS>(smem, jb.err);
    const int nitems = N * N * jb.nblocks * S;
    bool ok = true;
    for (;;) {
        // thread 0 decides for the whole CTA, so every thread leaves the loop together
        if (threadIdx.x == 0) s_item = *rg.abort_flag ? nitems : atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        if (!strip_item<N, K, U, NST, GPC, S>(jb, item, rg)) {
            ok = false;
            break;
        }
    }
    ring_drain<NST>(rg, ok);
}

template <int N, int K, int U, int NST, int GPC, int S>
int launch_cfg(const Handle &hd, int ncells, cudaStream_t s)
{
    using C = StripCfg<N, K, U, NST, GPC>;
    static_assert(K % 4 == 0 && (N / 2) % K == 0, "strip width must divide N/2 and be a multiple of 4");
    static_assert(C::STAGE % 16 == 0 && C::ROWB % 16 == 0 && C::GB % 16 == 0, "bulk copies need 16-byte units");
    auto kern = conv_strip_kernel<N, K, U, NST, GPC, S>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_error(e, "strip kernel shared-memory attribute");
    }
    const int ng = ngroups_of(ncells);
    const int nblocks = ng / GPC;  // callers pick GPC dividing ng
    const int nitems = N * N * nblocks * S;
    static int per_sm[2] = {0, 0};  // resident CTAs per SM, per GPC variant
    int &occ = per_sm[GPC - 1];
    if (occ == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 32 * C::WARPS, C::SMEM) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        occ = v;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hd.device);
    // automatic: about two items per resident CTA, so the queue can balance
    // pencils of unequal size (measured best at N = 16, 128 cells)
    const int autoper = std::max(1, std::min(occ, (int)((nitems + 2 * sms - 1) / (2 * std::max(1, sms)))));
    const int per = hd.tune_ctas > 0 ? std::min(hd.tune_ctas, occ) : autoper;
    const int grid = std::min(nitems, std::max(1, sms) * per);
    const float omega = (float)(hd.g.dz * hd.g.dz * hd.g.dz);
    cudaError_t e = cudaMemsetAsync(hd.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_error(e, "strip kernel work counter");
    const StripJob jb{(const float *)hd.ghat, hd.pencil_tile0, hd.pencil_order, (const float2 *)hd.F,
                      (float2 *)hd.Qh, (float2 *)hd.Qh2, hd.err, omega, nblocks, N, 0};
    kern<<<grid, 32 * C::WARPS, C::SMEM, s>>>(jb, hd.counter);
    CS_LAUNCHED(1, s, "convolution (strip kernel)");
    return CS_OK;
}

template <int N, int K, int U, int NST1, int NST2, int S>
int launch_n(const Handle &hd, int ncells, cudaStream_t s)
{
    const bool even = ngroups_of(ncells) % 2 == 0;
    const bool two = hd.tune_gpc == 2 || (hd.tune_gpc == 0 && N <= 16);  // measured: 1 group per CTA wins at N = 32
    if (even && two) return launch_cfg<N, K, U, NST2, 2, S>(hd, ncells, s);
    return launch_cfg<N, K, U, NST1, 1, S>(hd, ncells, s);
}

}  // namespace

int conv_parts(const Handle &hd)
{
    return (hd.precision == CS_FP32 && hd.g.layout == LAYOUT_STRIP && hd.g.N == 16) ? 2 : 1;
}

int launch_strip(const Handle &hd, int ncells, cudaStream_t s)
{
    switch (hd.g.N) {
    case 8: return launch_n<8, 4, 4, 4, 4, 1>(hd, ncells, s);
    case 16: return launch_n<16, 8, 8, 3, 3, 2>(hd, ncells, s);
    case 24: return launch_n<24, 12, 4, 3, 2, 1>(hd, ncells, s);
    case 32: return launch_n<32, 8, 8, 3, 3, 1>(hd, ncells, s);
    case 48: return launch_n<48, 8, 8, 3, 2, 1>(hd, ncells, s);
    case 64: return launch_n<64, 8, 8, 3, 2, 1>(hd, ncells, s);
    default: return set_error(CS_ENOTSUP, "strip kernel: unsupported N");
    }
}

}  // namespace cs
