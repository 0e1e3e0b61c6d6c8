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

// Complex multiply-add acc += g a b on packed float pairs (f32x2 instructions,
// half the issue slots of the scalar form): axx = (a.x, a.x), ayy = (a.y, a.y),
// bs = (-b.y, b.x), gg = (g, g);
//   t = axx * b = (a.x b.x, a.x b.y);  t += ayy * bs  ->  t = a b;  acc += gg * t.
__device__ __forceinline__ void cmad2(float2 &acc, float2 gg, float2 axx, float2 ayy, float2 b, float2 bs)
{
    float2 t = __fmul2_rn(axx, b);
    t = __ffma2_rn(ayy, bs, t);
    acc = __ffma2_rn(gg, t, acc);
}

__device__ __forceinline__ float2 dup_x(float2 a) { return make_float2(a.x, a.x); }
__device__ __forceinline__ float2 dup_y(float2 a) { return make_float2(a.y, a.y); }
__device__ __forceinline__ float2 rot_i(float2 b) { return make_float2(-b.y, b.x); }  // i b

// K consecutive weights from entry e0 (a multiple of 4), read with 128-bit
// loads, each as the packed pair (w, w) cmad2 takes.  (Storing every weight
// twice in the table instead measured slower: it doubles the shared-memory
// reads of the weights.)
template <int K>
__device__ __forceinline__ void wrow(const float *g, int e0, float2 (&w)[K])
{
    const float4 *p = reinterpret_cast<const float4 *>(g + e0);
#pragma unroll
    for (int q = 0; q < K / 4; ++q) {
        const float4 v = p[q];
        w[4 * q] = make_float2(v.x, v.x);
        w[4 * q + 1] = make_float2(v.y, v.y);
        w[4 * q + 2] = make_float2(v.z, v.z);
        w[4 * q + 3] = make_float2(v.w, v.w);
    }
}

__device__ __forceinline__ float2 wpair(const float *g, int e) { return make_float2(g[e], g[e]); }

// UB uniform rows starting at row m3 = m3b: window value t is the partner at
// s3 = smin + t; entry (u, j) uses t = j - u + UB - 1.  Weights: UB rows of K.
template <int K, int UB>
__device__ __forceinline__ void uniform_block(const float2 *__restrict__ arow, const float2 *__restrict__ brow,
                                              const float *__restrict__ g, int m3b, int smin, int lane,
                                              float2 (&acc)[K])
{
    float2 axx[UB], ayy[UB], bw[UB + K - 1], bs[UB + K - 1];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const float2 a = arow[(m3b + u) * kGroup + lane];
        axx[u] = dup_x(a);
        ayy[u] = dup_y(a);
    }
#pragma unroll
    for (int t = 0; t < UB + K - 1; ++t) {
        bw[t] = brow[(smin + t) * kGroup + lane];
        bs[t] = rot_i(bw[t]);
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        float2 w[K];
        wrow<K>(g, u * K, w);
#pragma unroll
        for (int j = 0; j < K; ++j) cmad2(acc[j], w[j], axx[u], ayy[u], bw[j - u + UB - 1], bs[j - u + UB - 1]);
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
    for (int b = 0; b < nblk; ++b, r += U)
        uniform_block<K, U>(arow, brow, g + r * K, m3s + r, C - r - (U - 1), lane, acc);
    if constexpr (R > 0) uniform_block<K, R>(arow, brow, g + r * K, m3s + r, C - r - (R - 1), lane, acc);
}

// Strip of kind A: uniform rows m3 = 0 .. k0+H (partner s3 = k0+H-m3+j),
// then the triangle m3 = k0+H+t, t = 1..K-1, outputs j = t..K-1 (s3 = j-t).
// The last R = (H+1) mod U uniform rows join the triangle in a compile-time
// tail (partners s3 = 0 .. R+K-2).
template <int N, int K, int U>
__device__ __forceinline__ void strip_a(const float2 *arow, const float2 *brow, const float *g, int k0, int lane,
                                        float2 (&acc)[K])
{
    constexpr int H = N / 2;
    constexpr int R = (H + 1) % U;
    const int lu = k0 + H + 1;
    uniform_run<K, U, 0>(arow, brow, g, 0, k0 + H, lu - R, lane, acc);
    const float *gt = g + (lu - R) * K;
    float2 b[R + K - 1], bs[R + K - 1];
#pragma unroll
    for (int i = 0; i < R + K - 1; ++i) {
        b[i] = brow[i * kGroup + lane];
        bs[i] = rot_i(b[i]);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {  // full rows m3 = lu - R + i, s3 = R - 1 - i + j
        const float2 a = arow[(lu - R + i) * kGroup + lane];
        float2 w[K];
        wrow<K>(gt, i * K, w);
#pragma unroll
        for (int j = 0; j < K; ++j) cmad2(acc[j], w[j], dup_x(a), dup_y(a), b[R - 1 - i + j], bs[R - 1 - i + j]);
    }
#pragma unroll
    for (int t = 1; t < K; ++t) {  // triangle
        const float2 a = arow[(k0 + H + t) * kGroup + lane];
#pragma unroll
        for (int j = t; j < K; ++j)
            cmad2(acc[j], wpair(gt, R * K + strip_tri_a_off(K, t) + j - t), dup_x(a), dup_y(a), b[j - t],
                  bs[j - t]);
    }
}

// Strip of kind B: triangle m3 = k0-H+1+t, t = 0..K-2, outputs j = 0..t
// (s3 = N-1+j-t), then uniform rows m3 = k0+K-H+r (s3 = N-K-r+j).  The first
// R = (N+H-K) mod U uniform rows join the triangle in a compile-time head.
template <int N, int K, int U>
__device__ __forceinline__ void strip_b(const float2 *arow, const float2 *brow, const float *g, int k0, int lane,
                                        float2 (&acc)[K])
{
    constexpr int H = N / 2;
    constexpr int R = (N + H - K) % U;
    constexpr int TRI4 = strip_round4(strip_tri(K));
    constexpr int HEADG = TRI4 + R * K;
    constexpr int B0 = N - K - R + 1;  // lowest partner index of the head
    float2 b[K + R - 1], bs[K + R - 1];
#pragma unroll
    for (int i = 0; i < K + R - 1; ++i) {
        b[i] = brow[(B0 + i) * kGroup + lane];
        bs[i] = rot_i(b[i]);
    }
#pragma unroll
    for (int t = 0; t < K - 1; ++t) {  // triangle
        const float2 a = arow[(k0 - H + 1 + t) * kGroup + lane];
#pragma unroll
        for (int j = 0; j <= t; ++j)
            cmad2(acc[j], wpair(g, strip_tri_b_off(t) + j), dup_x(a), dup_y(a), b[N - 1 + j - t - B0],
                  bs[N - 1 + j - t - B0]);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {  // first R uniform rows
        const float2 a = arow[(k0 + K - H + i) * kGroup + lane];
        float2 w[K];
        wrow<K>(g, TRI4 + i * K, w);
#pragma unroll
        for (int j = 0; j < K; ++j)
            cmad2(acc[j], w[j], dup_x(a), dup_y(a), b[N - K - i + j - B0], bs[N - K - i + j - B0]);
    }
    const int lu = N + H - k0 - K;
    uniform_run<K, U, 0>(arow, brow, g + HEADG, k0 + K - H + R, N - K - R, lu - R, lane, acc);
}

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

// Tile coordinates of one pencil, advanced in the order of the weight table:
// m1 = lo1 .. K1/2; m2 = lo2 .. hi2, except m2 = lo2 .. K2/2 when 2 m1 = K1.
struct TileWalk {
    int m1, m2, m2end, lo2, hi2, K1, K2;
    __device__ void start(int lo1, int lo2_, int hi2_, int K1_, int K2_)
    {
        lo2 = lo2_;
        hi2 = hi2_;
        K1 = K1_;
        K2 = K2_;
        m1 = lo1;
        m2 = lo2;
        m2end = (2 * m1 < K1) ? hi2 : K2 / 2;
    }
    __device__ void next()
    {
        if (++m2 > m2end) {
            ++m1;
            m2 = lo2;
            m2end = (2 * m1 < K1) ? hi2 : K2 / 2;
        }
    }
};

// Persistent kernel: CTAs take (pencil, group block) items from an atomic
// counter, heaviest pencils first, so the tail of the launch holds only the
// smallest items.  The stage ring runs across items: ring use u sits in
// slot u % NST, phase u / NST.
// Resident CTAs per SM the register allocation must allow: at N = 16 the
// kernel is latency-bound and 128 registers (8 one-group or 4 two-group CTAs
// per SM) measured faster than the ~134 the compiler picks on its own; for
// the other N one CTA (no cap) measured best.
template <int N, int GPC>
constexpr int strip_min_ctas() { return N == 16 ? (GPC == 1 ? 8 : 4) : 1; }

template <int N, int K, int U, int NST, int GPC, int S>
__global__ void __launch_bounds__(32 * (N / K) * GPC, strip_min_ctas<N, GPC>()) conv_strip_kernel(const float *__restrict__ ghat,
                                                                        const int *__restrict__ tile0,
                                                                        const int *__restrict__ order, int nblocks,
                                                                        const float2 *__restrict__ F,
                                                                        float2 *__restrict__ Qh,
                                                                        float2 *__restrict__ Qh2, float omega,
                                                                        int *err, int *counter)
{
    using C = StripCfg<N, K, U, NST, GPC>;
    constexpr int H = N / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NST * C::STAGE);
    uint64_t *empty = full + NST;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NST);
    __shared__ int s_item;

    const int warp_id = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gl = warp_id / C::W, warp = warp_id % C::W;  // group within the CTA, strip
    const int k0 = warp * K;
    const bool kind_a = k0 < H;
    const int seg = strip_seg_off(N, K, warp);
    const int nitems = N * N * nblocks * S;

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

    uint32_t tt = 0;  // ring uses consumed by this CTA before the current item
    uint32_t issued = 0;
    bool ok = true;
    for (;;) {
        // thread 0 decides for the whole CTA, so every thread leaves the loop together
        if (threadIdx.x == 0) s_item = *abort_flag ? nitems : atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        const int part = item % S, rest = item / S;
        const int pencil = order[rest / nblocks];
        const int gblk = rest % nblocks;
        const int grp = gblk * GPC + gl;
        const int k1 = pencil / N, k2 = pencil % N;
        const int K1 = k1 + H, K2 = k2 + H;
        const int lo1 = max(0, K1 - N + 1);
        const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
        const int Tall = tile0[pencil + 1] - tile0[pencil];
        const int tb = part == 0 ? 0 : (Tall + 1) / 2;  // this part's tiles: tb .. te-1
        const int te = (S == 1 || part == 1) ? Tall : (Tall + 1) / 2;
        const int T = te - tb;
        const float2 *Fb0 = F + (size_t)gblk * GPC * C::M * kGroup;
        const float *Gp = ghat + (size_t)(tile0[pencil] + tb) * C::TSV;
        float2 *Qout = part == 0 ? Qh : Qh2;

        TileWalk pw;  // producer's walk (thread 0), NST tiles ahead of the consumers
        int pt = 0;
        auto issue_next = [&]() -> bool {
            const uint32_t u = tt + pt;
            const int s = u % NST;
            if (u >= NST && !wait_phase(&empty[s], ((u / NST) + 1) & 1u, abort_flag, err, kWaitNs)) return false;
            unsigned char *st = smem + s * C::STAGE;
            mbar_arrive_expect_tx(&full[s], 2 * GPC * C::ROWB + C::GB);
#pragma unroll
            for (int q = 0; q < GPC; ++q) {
                const float2 *Fq = Fb0 + (size_t)q * C::M * kGroup;
                bulk_copy(st + q * C::ROWB, Fq + (size_t)(pw.m1 * N + pw.m2) * N * kGroup, C::ROWB, &full[s]);
                bulk_copy(st + (GPC + q) * C::ROWB, Fq + (size_t)((K1 - pw.m1) * N + (K2 - pw.m2)) * N * kGroup,
                          C::ROWB, &full[s]);
            }
            bulk_copy(st + 2 * GPC * C::ROWB, Gp + (size_t)pt * C::TSV, C::GB, &full[s]);
            ++pt;
            ++issued;
            pw.next();
            return true;
        };
        if (threadIdx.x == 0) {
            pw.start(lo1, lo2, hi2, K1, K2);
            for (int i = 0; i < tb; ++i) pw.next();
            while (pt < NST && pt < T)
                if (!issue_next()) {
                    ok = false;
                    break;
                }
        }

        float2 acc[K], hi[K], lo[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            acc[j] = make_float2(0.f, 0.f);
            hi[j] = make_float2(0.f, 0.f);
            lo[j] = make_float2(0.f, 0.f);
        }
        TileWalk cw;
        cw.start(lo1, lo2, hi2, K1, K2);
        for (int i = 0; i < tb; ++i) cw.next();
        int cur_m1 = cw.m1;
        for (int t = 0; t < T && ok; ++t) {
            const uint32_t u = tt + t;
            const int s = u % NST;
            if (!wait_phase(&full[s], (u / NST) & 1u, abort_flag, err, kWaitNs)) {
                ok = false;
                break;
            }
            if (cw.m1 != cur_m1) {  // new m1 slab: fold the finished one
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    two_sum(hi[j].x, lo[j].x, acc[j].x);
                    two_sum(hi[j].y, lo[j].y, acc[j].y);
                    acc[j] = make_float2(0.f, 0.f);
                }
                cur_m1 = cw.m1;
            }
            const unsigned char *st = smem + s * C::STAGE;
            const float2 *arow = reinterpret_cast<const float2 *>(st + gl * C::ROWB);
            const float2 *brow = reinterpret_cast<const float2 *>(st + (GPC + gl) * C::ROWB);
            const float *gt = reinterpret_cast<const float *>(st + 2 * GPC * C::ROWB) + seg;
            if (kind_a)
                strip_a<N, K, U>(arow, brow, gt, k0, lane, acc);
            else
                strip_b<N, K, U>(arow, brow, gt, k0, lane, acc);
            cw.next();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (threadIdx.x == 0 && pt < T)
                if (!issue_next()) ok = false;
            __syncwarp();
        }
        if (__syncthreads_or(!ok || *abort_flag)) {  // CTA-uniform
            ok = false;
            break;
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
            two_sum(hi[j].x, lo[j].x, acc[j].x);
            two_sum(hi[j].y, lo[j].y, acc[j].y);
            Qout[((size_t)grp * C::M + (size_t)pencil * N + k0 + j) * kGroup + lane] =
                make_float2(omega * (hi[j].x + lo[j].x), omega * (hi[j].y + lo[j].y));
        }
        tt += T;
    }
    if (threadIdx.x == 0 && (!ok || *abort_flag)) {
        // give the copies this thread issued a bounded time to land before the CTA exits
        for (uint32_t u = tt; u < issued; ++u) {
            volatile int dummy = 0;
            wait_phase(&full[u % NST], (u / NST) & 1u, &dummy, err, kWaitNs / 20);
        }
    }
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
    kern<<<grid, 32 * C::WARPS, C::SMEM, s>>>((const float *)hd.ghat, hd.pencil_tile0, hd.pencil_order, nblocks,
                                              (const float2 *)hd.F, (float2 *)hd.Qh, (float2 *)hd.Qh2, omega,
                                              hd.err, hd.counter);
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
