// K2, strip kernel (float; N in {8, 16, 24, 32}): the weighted convolution of
// Sec. 3.2,
//   Qhat(zeta_k) = dzeta^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m),
// over the symmetrised half-tiles of the weight table (weights.cu).
//
// Work decomposition.  One CTA owns one output pencil (k1, k2, all k3) of one
// group of 32 cells (one cell per lane).  The pencil's k3 range is cut into
// N/K strips of K outputs; warp w owns strip w and keeps only its K complex
// accumulators (plus a compensation pair) in registers.
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
#include <cstdint>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bulk copy global -> shared, completion counted on bar (bytes and addresses 16-byte multiples)
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// wait for the phase of parity `parity`; false if the CTA aborted or the wait
// exceeded its time limit (then the CTA is told to abort and *err is set)
__device__ bool wait_phase(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err, unsigned long long limit)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > limit) {
                *abort_flag = 1;
                atomicOr(err, 1);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void two_sum(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ void cmad(float2 &acc, float g, float2 a, float2 b)
{
    const float tr = fmaf(a.x, b.x, -a.y * b.y);
    const float ti = fmaf(a.x, b.y, a.y * b.x);
    acc.x = fmaf(g, tr, acc.x);
    acc.y = fmaf(g, ti, acc.y);
}

// UB uniform rows starting at row m3 = m3b: window value t is the partner at
// s3 = smin + t; entry (u, j) uses t = j - u + UB - 1.  Weights: UB rows of K.
template <int K, int UB>
__device__ __forceinline__ void uniform_block(const float2 *__restrict__ arow, const float2 *__restrict__ brow,
                                              const float *__restrict__ g, int m3b, int smin, int lane,
                                              float2 (&acc)[K])
{
    float2 a[UB], bw[UB + K - 1];
#pragma unroll
    for (int u = 0; u < UB; ++u) a[u] = arow[(m3b + u) * kGroup + lane];
#pragma unroll
    for (int t = 0; t < UB + K - 1; ++t) bw[t] = brow[(smin + t) * kGroup + lane];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 g4 = reinterpret_cast<const float4 *>(g + u * K)[q];
            cmad(acc[4 * q + 0], g4.x, a[u], bw[4 * q + 0 - u + UB - 1]);
            cmad(acc[4 * q + 1], g4.y, a[u], bw[4 * q + 1 - u + UB - 1]);
            cmad(acc[4 * q + 2], g4.z, a[u], bw[4 * q + 2 - u + UB - 1]);
            cmad(acc[4 * q + 3], g4.w, a[u], bw[4 * q + 3 - u + UB - 1]);
        }
    }
}

// the uniform run: nrows rows from m3 = m3s, partner s3 = C - r + j for row r
template <int K, int U, int R>
__device__ __forceinline__ void uniform_run(const float2 *arow, const float2 *brow, const float *g, int m3s, int C,
                                            int nrows, int lane, float2 (&acc)[K])
{
    const int nblk = nrows / U;
    int r = 0;
#pragma unroll 1
    for (int b = 0; b < nblk; ++b, r += U) uniform_block<K, U>(arow, brow, g + r * K, m3s + r, C - r - (U - 1), lane, acc);
    if constexpr (R > 0) uniform_block<K, R>(arow, brow, g + r * K, m3s + r, C - r - (R - 1), lane, acc);
}

// strip of kind A: uniform rows m3 = 0 .. k0+H, then triangle rows m3 = k0+H+t,
// t = 1..K-1, outputs j = t..K-1, partner s3 = j - t
template <int N, int K, int U>
__device__ __forceinline__ void strip_a(const float2 *arow, const float2 *brow, const float *g, int k0, int lane,
                                        float2 (&acc)[K])
{
    constexpr int H = N / 2;
    constexpr int R = (H + 1) % U;
    const int lu = k0 + H + 1;
    uniform_run<K, U, R>(arow, brow, g, 0, k0 + H, lu, lane, acc);
    const float *gt = g + lu * K;
    float2 b[K - 1];
#pragma unroll
    for (int i = 0; i < K - 1; ++i) b[i] = brow[i * kGroup + lane];
#pragma unroll
    for (int t = 1; t < K; ++t) {
        const float2 a = arow[(k0 + H + t) * kGroup + lane];
#pragma unroll
        for (int j = t; j < K; ++j) cmad(acc[j], gt[strip_tri_a_off(K, t) + j - t], a, b[j - t]);
    }
}

// strip of kind B: triangle rows m3 = k0-H+1+t, t = 0..K-2, outputs j = 0..t,
// partner s3 = N-1+j-t; then uniform rows m3 = k0+K-H .. N-1 (s3 = N-K-r+j)
template <int N, int K, int U>
__device__ __forceinline__ void strip_b(const float2 *arow, const float2 *brow, const float *g, int k0, int lane,
                                        float2 (&acc)[K])
{
    constexpr int H = N / 2;
    constexpr int R = (N + H - K) % U;
    float2 b[K - 1];
#pragma unroll
    for (int i = 0; i < K - 1; ++i) b[i] = brow[(N - K + 1 + i) * kGroup + lane];
#pragma unroll
    for (int t = 0; t < K - 1; ++t) {
        const float2 a = arow[(k0 - H + 1 + t) * kGroup + lane];
#pragma unroll
        for (int j = 0; j <= t; ++j) cmad(acc[j], g[strip_tri_b_off(t) + j], a, b[K - 2 + j - t]);
    }
    const int lu = N + H - k0 - K;
    uniform_run<K, U, R>(arow, brow, g + strip_round4(strip_tri(K)), k0 + K - H, N - K, lu, lane, acc);
}

// GPC cell groups per CTA share each stage's weight tile (each group has its
// own two rows); warp = (group g_local, strip w)
template <int N, int K, int U, int NST, int GPC>
struct StripCfg {
    static constexpr int W = N / K;
    static constexpr int WARPS = W * GPC;
    static constexpr int M = N * N * N;
    static constexpr int TSV = strip_stride(N, K);
    static constexpr uint32_t ROWB = N * kGroup * sizeof(float2);
    static constexpr uint32_t GB = TSV * sizeof(float);
    static constexpr uint32_t STAGE = (2 * GPC * ROWB + GB + 127) / 128 * 128;
    static constexpr size_t SMEM = (size_t)NST * STAGE + 2 * NST * sizeof(uint64_t) + 16;
};

template <int N, int K, int U, int NST, int GPC>
__global__ void __launch_bounds__(32 * (N / K) * GPC) conv_strip_kernel(const float *__restrict__ ghat,
                                                                        const int *__restrict__ tile0,
                                                                        const int *__restrict__ order, int nblocks,
                                                                        const float2 *__restrict__ F,
                                                                        float2 *__restrict__ Qh, float omega,
                                                                        int *err)
{
    using C = StripCfg<N, K, U, NST, GPC>;
    constexpr int H = N / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NST * C::STAGE);
    uint64_t *empty = full + NST;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NST);

    const int warp_id = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gl = warp_id / C::W, warp = warp_id % C::W;  // group within the CTA, strip
    const int item = blockIdx.x;
    const int pencil = order[item / nblocks];
    const int gblk = item % nblocks;
    const int grp = gblk * GPC + gl;
    const int k1 = pencil / N, k2 = pencil % N;
    const int K1 = k1 + H, K2 = k2 + H;
    const int lo1 = max(0, K1 - N + 1), hi1 = min(N - 1, K1);
    const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
    const int v2 = hi2 - lo2 + 1;
    const int nfull = ((hi1 - lo1 + 1) / 2) * v2;
    const int T = tile0[pencil + 1] - tile0[pencil];
    const float2 *Fb0 = F + (size_t)gblk * GPC * C::M * kGroup;  // first group of this CTA
    const float *Gp = ghat + (size_t)tile0[pencil] * C::TSV;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], C::WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    auto rows_of = [&](int t, int &m1, int &m2) {
        if (t < nfull) {
            m1 = lo1 + t / v2;
            m2 = lo2 + t % v2;
        } else {
            m1 = K1 / 2;
            m2 = lo2 + (t - nfull);
        }
    };
    auto issue = [&](int t) {
        const int s = t % NST;
        int m1, m2;
        rows_of(t, m1, m2);
        unsigned char *st = smem + s * C::STAGE;
        mbar_arrive_expect_tx(&full[s], 2 * GPC * C::ROWB + C::GB);
#pragma unroll
        for (int q = 0; q < GPC; ++q) {
            const float2 *Fq = Fb0 + (size_t)q * C::M * kGroup;
            bulk_copy(st + q * C::ROWB, Fq + (size_t)(m1 * N + m2) * N * kGroup, C::ROWB, &full[s]);
            bulk_copy(st + (GPC + q) * C::ROWB, Fq + (size_t)((K1 - m1) * N + (K2 - m2)) * N * kGroup, C::ROWB,
                      &full[s]);
        }
        bulk_copy(st + 2 * GPC * C::ROWB, Gp + (size_t)t * C::TSV, C::GB, &full[s]);
    };

    int issued = 0;
    if (threadIdx.x == 0)
        for (; issued < NST && issued < T; ++issued) issue(issued);

    const int k0 = warp * K;
    const bool kind_a = k0 < H;
    const int seg = strip_seg_off(N, K, warp);
    float2 acc[K], hi[K], lo[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        acc[j] = make_float2(0.f, 0.f);
        hi[j] = make_float2(0.f, 0.f);
        lo[j] = make_float2(0.f, 0.f);
    }
    int cur_m1 = lo1;
    bool ok = true;
    int t = 0;
    for (; t < T; ++t) {
        const int s = t % NST;
        const uint32_t par = (uint32_t)(t / NST) & 1u;
        if (!wait_phase(&full[s], par, abort_flag, err, kWaitNs)) {
            ok = false;
            break;
        }
        int m1, m2;
        rows_of(t, m1, m2);
        if (m1 != cur_m1) {  // new slab: fold the finished one
#pragma unroll
            for (int j = 0; j < K; ++j) {
                two_sum(hi[j].x, lo[j].x, acc[j].x);
                two_sum(hi[j].y, lo[j].y, acc[j].y);
                acc[j] = make_float2(0.f, 0.f);
            }
            cur_m1 = m1;
        }
        const unsigned char *st = smem + s * C::STAGE;
        const float2 *arow = reinterpret_cast<const float2 *>(st + gl * C::ROWB);
        const float2 *brow = reinterpret_cast<const float2 *>(st + (GPC + gl) * C::ROWB);
        const float *gt = reinterpret_cast<const float *>(st + 2 * GPC * C::ROWB) + seg;
        if (kind_a)
            strip_a<N, K, U>(arow, brow, gt, k0, lane, acc);
        else
            strip_b<N, K, U>(arow, brow, gt, k0, lane, acc);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (threadIdx.x == 0 && issued < T) {
            // stage s is refilled with tile t + NST once every warp released tile t
            if (!wait_phase(&empty[s], par, abort_flag, err, kWaitNs)) {
                ok = false;
            } else {
                issue(issued);
                ++issued;
            }
        }
        __syncwarp();
        if (!ok) break;
    }
    if (ok && !*abort_flag) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            two_sum(hi[j].x, lo[j].x, acc[j].x);
            two_sum(hi[j].y, lo[j].y, acc[j].y);
            Qh[((size_t)grp * C::M + (size_t)pencil * N + k0 + j) * kGroup + lane] =
                make_float2(omega * (hi[j].x + lo[j].x), omega * (hi[j].y + lo[j].y));
        }
    }
    if (threadIdx.x == 0 && !ok) {
        // give the copies this thread issued a bounded time to land before the CTA exits
        for (int u = t; u < issued; ++u) {
            volatile int dummy = 0;
            wait_phase(&full[u % NST], (uint32_t)(u / NST) & 1u, &dummy, err, kWaitNs / 20);
        }
    }
}

template <int N, int K, int U, int NST, int GPC>
int launch_cfg(const Handle &hd, int ncells, cudaStream_t s)
{
    using C = StripCfg<N, K, U, NST, GPC>;
    static_assert(K % 4 == 0 && (N / 2) % K == 0, "strip width must divide N/2 and be a multiple of 4");
    static_assert(C::STAGE % 16 == 0 && C::ROWB % 16 == 0 && C::GB % 16 == 0, "bulk copies need 16-byte units");
    auto kern = conv_strip_kernel<N, K, U, NST, GPC>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_error(e, "strip kernel shared-memory attribute");
    }
    const int ng = ngroups_of(ncells);
    const int nblocks = ng / GPC;  // callers pick GPC dividing ng
    const unsigned blocks = (unsigned)(N * N * nblocks);
    const float omega = (float)(hd.g.dz * hd.g.dz * hd.g.dz);
    kern<<<blocks, 32 * C::WARPS, C::SMEM, s>>>((const float *)hd.ghat, hd.pencil_tile0, hd.pencil_order, nblocks,
                                                (const float2 *)hd.F, (float2 *)hd.Qh, omega, hd.err);
    CS_CHECK_LAUNCH("convolution (strip kernel)");
    return CS_OK;
}

template <int N, int K, int U, int NST1, int NST2>
int launch_n(const Handle &hd, int ncells, cudaStream_t s)
{
    if (ngroups_of(ncells) % 2 == 0) return launch_cfg<N, K, U, NST2, 2>(hd, ncells, s);
    return launch_cfg<N, K, U, NST1, 1>(hd, ncells, s);
}

}  // namespace

int launch_strip(const Handle &hd, int ncells, cudaStream_t s)
{
    switch (hd.g.N) {
    case 8: return launch_n<8, 4, 4, 4, 4>(hd, ncells, s);
    case 16: return launch_n<16, 8, 8, 4, 3>(hd, ncells, s);
    case 24: return launch_n<24, 12, 4, 3, 2>(hd, ncells, s);
    case 32: return launch_n<32, 8, 8, 3, 3>(hd, ncells, s);
    default: return set_error(CS_ENOTSUP, "strip kernel: unsupported N");
    }
}

}  // namespace cs
