// K2 for uneven batches: the strip convolutions (Sec. 3.2) of several float
// handles — any mix of N in {8, 16, 24, 32} and of lambda — in one persistent
// launch.  Each handle is a job with its own weights, tile tables and
// workspace; the launch numbers the jobs' items one after the other, the
// jobs of larger N (heavier items) first, and CTAs take items from one atomic
// counter, so the light items of the small grids fill the tail left by the
// heavy ones instead of every grid having a tail of its own.
//
// One CTA shape serves every N: 4 warps, i.e. two strips for each of two
// 32-cell groups at N = 8, 16, 24 (the strip widths of conv_strip.cu) and
// four strips of one group at N = 32.  Each item runs the same strip body,
// with the same strip width, split and summation order as the handle's own
// launch, so a cell's result is bit-identical to cs_collide on its own.  The
// stage ring has one depth for the launch and a stage size per item (the
// ring is empty between items).  Pairing groups needs an even group count:
// the caller pads those jobs' cells to a multiple of 64 (workspace and
// forward transform), and the padded lanes' outputs are never read.
#include <algorithm>

#include "strip.cuh"

namespace cs {

namespace {

constexpr int kMixedWarps = 4;
constexpr int kMixedNST = 2;  // ring depth of a mixed launch

// item shape per N: strip width K, uniform block U, groups per CTA, parts S
// (S = conv_split: the split at N = 16 must match the handle's own launch)
template <int N>
struct MixedShape;
template <>
struct MixedShape<8> {
    static constexpr int K = 4, U = 4, GPC = 2, S = 1;
};
template <>
struct MixedShape<16> {
    static constexpr int K = 8, U = 8, GPC = 2, S = 2;  // handles split 4 ways run outside the shared launch
};
template <>
struct MixedShape<24> {
    static constexpr int K = 12, U = 4, GPC = 2, S = 1;
};
template <>
struct MixedShape<32> {
    static constexpr int K = 8, U = 8, GPC = 1, S = 1;
};

template <int N>
using MixedCfg = StripCfg<N, MixedShape<N>::K, MixedShape<N>::U, kMixedNST, MixedShape<N>::GPC>;

constexpr size_t kMixedSmem =
    std::max(std::max(MixedCfg<8>::SMEM, MixedCfg<16>::SMEM), std::max(MixedCfg<24>::SMEM, MixedCfg<32>::SMEM));

constexpr int kMaxJobs = 16;

struct StripJobs {
    StripJob j[kMaxJobs];
    int n, nitems;
};

template <int N>
__device__ __forceinline__ bool mixed_item(const StripJob &jb, int item, Ring &rg)
{
    using S = MixedShape<N>;
    static_assert(MixedCfg<N>::WARPS == kMixedWarps, "one CTA shape for every N");
    return strip_item<N, S::K, S::U, kMixedNST, S::GPC, S::S>(jb, item, rg);
}

__global__ void __launch_bounds__(32 * kMixedWarps) conv_mixed_kernel(StripJobs js, int *counter)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    Ring rg = ring_init<kMixedNST, kMixedWarps>(smem, js.j[0].err);
    bool ok = true;
    for (;;) {
        // thread 0 decides for the whole CTA, so every thread leaves the loop together
        if (threadIdx.x == 0) s_item = *rg.abort_flag ? js.nitems : atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= js.nitems) break;
        int q = 0;
        while (q + 1 < js.n && item >= js.j[q + 1].first) ++q;
        const StripJob jb = js.j[q];
        const int it = item - jb.first;
        bool r = false;
        switch (jb.N) {  // CTA-uniform
        case 8: r = mixed_item<8>(jb, it, rg); break;
        case 16: r = mixed_item<16>(jb, it, rg); break;
        case 24: r = mixed_item<24>(jb, it, rg); break;
        case 32: r = mixed_item<32>(jb, it, rg); break;
        default: break;
        }
        if (!r) {
            ok = false;
            break;
        }
    }
    ring_drain<kMixedNST>(rg, ok);
}

int groups_per_cta(int N) { return N == 32 ? 1 : 2; }

}  // namespace

bool strip_mixable(const Handle &hd)
{
    const int N = hd.g.N;
    // one body per N keeps the kernel's code small: a handle at N = 16 split
    // four ways (a second body measured 5 % slower for the whole launch) or
    // rebuilding its weights runs on its own
    return hd.precision == CS_FP32 && hd.g.layout == LAYOUT_STRIP && (N == 8 || N == 16 || N == 24 || N == 32) &&
           hd.has_table && !strip_uses_radius(hd) && conv_split(hd) == (N == 16 ? MixedShape<16>::S : 1);
}

int strip_mixed_cells(const Handle &hd, int ncells)
{
    const int per = kGroup * groups_per_cta(hd.g.N);
    return (ncells + per - 1) / per * per;
}

int launch_strip_mixed(const Handle *const *hds, const int *ncells, int n, cudaStream_t s)
{
    if (n < 1 || n > kMaxJobs) return set_error(CS_EINVAL, "mixed convolution: 1 to 16 jobs");
    int idx[kMaxJobs];
    for (int i = 0; i < n; ++i) {
        if (!strip_mixable(*hds[i])) return set_error(CS_ENOTSUP, "mixed convolution: float strip handles only");
        if (hds[i]->ws_cells < strip_mixed_cells(*hds[i], ncells[i]))
            return set_error(CS_EINVAL, "mixed convolution: workspace not padded to whole CTA groups");
        idx[i] = i;
    }
    // heaviest items first: larger N before smaller, in the callers' order otherwise
    std::stable_sort(idx, idx + n, [&](int a, int b) { return hds[a]->g.N > hds[b]->g.N; });
    StripJobs js{};
    long long first = 0;
    for (int k = 0; k < n; ++k) {
        const Handle &hd = *hds[idx[k]];
        const int N = hd.g.N, gpc = groups_per_cta(N);
        const int parts = conv_split(hd);  // 2 at N = 16 (strip_mixable), else 1
        const int nblocks = strip_mixed_cells(hd, ncells[idx[k]]) / kGroup / gpc;
        js.j[k] = StripJob{(const float *)hd.ghat, hd.pencil_tile0, hd.pencil_order, (const float2 *)hd.F,
                           (float2 *)hd.Qh, (float2 *)hd.Qh2, (float2 *)hd.Qh3, (float2 *)hd.Qh4, hd.done, hd.err,
                           (float)(hd.g.dz * hd.g.dz * hd.g.dz),
                           nblocks, N, (int)first};
        js.j[k].S = parts;
        js.j[k].wait_us = hd.wait_us ? hd.wait_us : kWaitUs;
        js.j[k].stall = hd.test_stall;
        js.j[k].l2hint = l2_hint_bits(hd.tune_l2);
        first += (long long)N * N * nblocks * parts;
    }
    if (first > 0x7fffffff) return set_error(CS_EINVAL, "mixed convolution: too many items");
    js.n = n;
    js.nitems = (int)first;
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(conv_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMixedSmem);
        if (e != cudaSuccess) return cuda_error(e, "mixed convolution: shared-memory attribute");
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, conv_mixed_kernel, 32 * kMixedWarps, kMixedSmem) !=
                cudaSuccess ||
            v < 1) {
            cudaGetLastError();
            v = 1;
        }
        occ = v;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hds[0]->device);
    const int grid = std::min(js.nitems, std::max(1, sms) * occ);
    // the work counter: a word of the first job's handle that its own launches never use
    int *counter = hds[idx[0]]->err + 48;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    for (int k = 0; k < n && e == cudaSuccess; ++k)  // finished-range counters of the split jobs
        if (js.j[k].N == 16) e = cudaMemsetAsync(js.j[k].done, 0, sizeof(int) * 16 * 16 * js.j[k].nblocks, s);
    if (e != cudaSuccess) return cuda_error(e, "mixed convolution: work counters");
    conv_mixed_kernel<<<grid, 32 * kMixedWarps, kMixedSmem, s>>>(js, counter);
    CS_LAUNCHED(1, s, "convolution (mixed strip kernel)");
    return CS_OK;
}

}  // namespace cs
