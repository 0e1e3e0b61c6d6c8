// Device building blocks of the strip convolution (conv_strip.cu: one
// handle per launch; conv_mixed.cu: several handles of different N in one
// persistent launch): mbarrier and bulk-copy wrappers with bounded waits,
// the packed complex multiply-add, the strip bodies of kinds A and B, the
// tile walk of a pencil, and one work item on a CTA's stage ring.
#pragma once

#include <cstdint>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr unsigned kWaitUs = 2000000u;  // default limit of a bounded wait: 2 s

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

// the same with an L2 eviction priority for the source lines (a policy from
// createpolicy): the weight tiles stream through L2 once per launch (evict
// first) while the f-hat rows are read again by every pencil that needs them
// (evict last)
__device__ __forceinline__ void bulk_copy_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                               uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// wait for the phase of parity `parity`; false if the CTA aborted or the wait
// exceeded its time limit (then the CTA is told to abort and *err is set)
__device__ bool wait_phase(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err, unsigned limit_us)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > 1000ull * limit_us) {
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

// The compensated sums (hi, lo) of a strip's K outputs, folded once per m1
// slab: in registers (WHERE 0), in local memory (1), where the volatile
// array keeps them out of the register file, or in shared memory (2), value
// i of thread t at i * stride + t (no bank conflicts).  At N = 24 local
// memory frees 48 registers a thread and lets three CTAs share an SM instead
// of two; at N = 32 with two groups per CTA shared memory frees 53 and lets
// two 8-warp CTAs share one, where local memory would spill to L2 and DRAM
// once two rings fill the SM's shared memory.  All forms run the same
// operations in the same order.
template <int K, int WHERE>
struct CompSum;

template <int K>
struct CompSum<K, 0> {
    float2 hi[K], lo[K];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            hi[j] = make_float2(0.f, 0.f);
            lo[j] = make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void add(int j, float2 p)
    {
        two_sum(hi[j].x, lo[j].x, p.x);
        two_sum(hi[j].y, lo[j].y, p.y);
    }
    __device__ __forceinline__ float2 value(int j) const { return make_float2(hi[j].x + lo[j].x, hi[j].y + lo[j].y); }
};

template <int K>
struct CompSum<K, 1> {
    volatile float v[4 * K];  // (hi.x, hi.y, lo.x, lo.y) per output
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 4 * K; ++i) v[i] = 0.f;
    }
    __device__ __forceinline__ void add(int j, float2 p)
    {
        float hx = v[4 * j], hy = v[4 * j + 1], lx = v[4 * j + 2], ly = v[4 * j + 3];
        two_sum(hx, lx, p.x);
        two_sum(hy, ly, p.y);
        v[4 * j] = hx;
        v[4 * j + 1] = hy;
        v[4 * j + 2] = lx;
        v[4 * j + 3] = ly;
    }
    __device__ __forceinline__ float2 value(int j) const
    {
        return make_float2(v[4 * j] + v[4 * j + 2], v[4 * j + 1] + v[4 * j + 3]);
    }
};

template <int K>
struct CompSum<K, 2> {
    float *v;    // this thread's first value
    int stride;  // threads of the CTA
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 4 * K; ++i) v[i * stride] = 0.f;
    }
    __device__ __forceinline__ void add(int j, float2 p)
    {
        float hx = v[(4 * j) * stride], hy = v[(4 * j + 1) * stride], lx = v[(4 * j + 2) * stride],
              ly = v[(4 * j + 3) * stride];
        two_sum(hx, lx, p.x);
        two_sum(hy, ly, p.y);
        v[(4 * j) * stride] = hx;
        v[(4 * j + 1) * stride] = hy;
        v[(4 * j + 2) * stride] = lx;
        v[(4 * j + 3) * stride] = ly;
    }
    __device__ __forceinline__ float2 value(int j) const
    {
        return make_float2(v[(4 * j) * stride] + v[(4 * j + 2) * stride],
                           v[(4 * j + 1) * stride] + v[(4 * j + 3) * stride]);
    }
};

// where a strip keeps its compensated sums (measured: local memory wins at
// N = 24; at N = 32 with two groups per CTA shared memory, whose freed
// registers (166 -> ~113) let two 8-warp CTAs share an SM; at N = 16, and at
// N = 32 with one group, leaving the registers measured 1-2 % slower)
template <int N, int GPC = 1, bool RAD = false>
constexpr int strip_comp_where() { return N == 24 ? 1 : (N == 32 && GPC >= 2 && !RAD) ? 2 : 0; }

// One problem of a strip launch: a handle's weights, tile tables and
// workspace.  A mixed launch carries several (of different N), each owning
// the items first .. first + N^2 nblocks S - 1 of the launch's item space.
struct StripJob {
    const float *ghat;
    const int *tile0, *order;
    const float2 *F;
    float2 *Qh, *Qh2, *Qh3, *Qh4;  // partial sums of tile ranges 0, 1, 2, 3 (Qh: their sum at the end)
    int *done;                     // S > 1: finished ranges per (pencil, block), zero at the launch
    int *err;                      // the handle's status word
    float omega;
    int nblocks, N, first;
    int S = 1;  // tile ranges per pencil (the mixed kernel dispatches on it at N = 16)
    // radius tables (launches that rebuild the weight tiles): A, B, the tile
    // entry map and the row length of A
    const float *radA = nullptr, *radB = nullptr;
    const int *emap = nullptr;
    int bbn = 0;
    // limit of the item's bounded waits, and the test stall (the launch's
    // first CTA issues no copy for its first item, so its waits run out)
    unsigned wait_us = kWaitUs;
    int stall = 0;
    int l2hint = 0;  // L2 eviction priorities: bit 0 weight tiles evict first, bit 1 f-hat rows evict last
};

// A persistent CTA's stage ring: barriers and the abort word at the front of
// the dynamic shared memory, then the stages.  The use counters run across
// items: ring use u sits in slot u % NST, phase u / NST.  Between items every
// use has landed and been consumed, so the stage size may change from one
// item to the next (a mixed launch); the slot and phase arithmetic may not,
// so one launch has one NST.
constexpr int kRingHead = 128;

struct Ring {
    unsigned char *stages;
    uint64_t *full, *empty;
    volatile int *abort_flag;
    int *err;         // status word of the item in flight
    uint32_t tt;      // ring uses consumed by this CTA before the current item
    uint32_t issued;  // ring uses issued (thread 0)
};

__host__ __device__ constexpr int strip_seg_max(int N, int K)
{
    int m = 0;
    for (int w = 0; w < N / K; ++w) m = strip_seg_size(N, K, w) > m ? strip_seg_size(N, K, w) : m;
    return m;
}

// the L2 eviction priorities of a handle's setting (CS_TUNE_L2_HINT): 1 none,
// 0 or 2 both, 3 the weight tiles only, 4 the f-hat rows only
__host__ __device__ inline int l2_hint_bits(int tune) { return tune == 1 ? 0 : tune == 3 ? 1 : tune == 4 ? 2 : 3; }

// Shared memory of a strip CTA: the ring head, NST stages (two f-hat rows per
// group, plus the weight tile unless RAD), and with RAD one weight segment
// per warp rebuilt from the radius tables, the tile entry map and the table
// B (both copied in once per CTA).
// HS = 2 (few cells): a warp sums two strips of the same kind for 16 cells
// of one group, lanes 0-15 the first strip, lanes 16-31 the second; every
// (cell, output) runs the same operations in the same order as with HS = 1,
// so results are the same bit for bit.
template <int N, int K, int U, int NST, int GPC, bool RAD = false, int HS = 1>
struct StripCfg {
    static constexpr int W = N / K;
    static constexpr int WARPS = W * GPC / HS;
    static constexpr int M = N * N * N;
    static constexpr int TSV = strip_stride(N, K);
    static constexpr uint32_t ROWB = N * kGroup * sizeof(float2);
    static constexpr uint32_t GB = TSV * sizeof(float);
    static constexpr uint32_t STAGE = (2 * GPC * ROWB + (RAD ? 0 : GB) + 127) / 128 * 128;
    static constexpr int WBUF = RAD ? strip_round4(strip_seg_max(N, K)) : 0;  // floats per warp
    static constexpr int NB = RAD ? 3 * (N / 2) * (N / 2) + 1 : 0;              // entries of B
    static constexpr int COMPF = strip_comp_where<N, GPC, RAD>() == 2 ? 4 * K * 32 * WARPS : 0;  // compensated sums
    static constexpr size_t SMEM = kRingHead + (size_t)NST * STAGE +
                                   sizeof(float) * ((size_t)WARPS * WBUF + (RAD ? TSV : 0) + strip_round4(NB) + COMPF);
};

// RAD: the per-CTA copies of the tile entry map and of B, after the warps'
// weight segments


// The weight segment of strip w (entries seg .. seg+nseg-1 of the tile
// layout) of tile (m1, m2) of pencil (k1, k2), rebuilt from the radius
// tables: entry (m3, k3) gets (A - B(|m'|^2)) + (A - B(|s'|^2)), the centre
// tile A - B(|m'|^2), zero where k' = 0 and in the padding.  Lane l takes
// entries l, l + 32, ...  In two steps, so the loads from A (the only ones
// from global memory; the entry map and B are in shared memory) can be
// issued a tile ahead: radius_gather loads A into registers, radius_combine
// forms the weights into the warp's buffer.
struct RadiusTile {
    int kk12, bb12, mm12, ss12;
    bool centre;
};

template <int N>
__device__ __forceinline__ RadiusTile radius_tile(int k1, int k2, int m1, int m2)
{
    constexpr int h = N / 2;
    const int k1p = k1 - h, k2p = k2 - h, m1p = m1 - h, m2p = m2 - h;
    const int s1p = k1p - m1p, s2p = k2p - m2p, d1 = 2 * m1p - k1p, d2 = 2 * m2p - k2p;
    RadiusTile r;
    r.centre = s1p == m1p && s2p == m2p;
    r.kk12 = k1p * k1p + k2p * k2p;
    r.bb12 = d1 * d1 + d2 * d2;
    r.mm12 = m1p * m1p + m2p * m2p;
    r.ss12 = s1p * s1p + s2p * s2p;
    return r;
}

template <int N, int EPL>
__device__ __forceinline__ void radius_gather(const StripJob &jb, const int *emap, int seg, int nseg,
                                              const RadiusTile &rt, int lane, float (&pa)[EPL])
{
    constexpr int h = N / 2;
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
        const int p = lane + 32 * i;
        pa[i] = 0.f;
        if (p < nseg) {
            const int e = emap[seg + p];
            if (e >= 0) {
                const int m3p = (e >> 8) - h, k3p = (e & 255) - h;
                const int kk = rt.kk12 + k3p * k3p, d3 = 2 * m3p - k3p;
                if (kk != 0) pa[i] = __ldg(jb.radA + (size_t)kk * jb.bbn + rt.bb12 + d3 * d3);
            }
        }
    }
}

template <int N, int EPL>
__device__ __forceinline__ void radius_combine(const int *emap, const float *radB, int seg, int nseg,
                                               const RadiusTile &rt, int lane, const float (&pa)[EPL], float *wb)
{
    constexpr int h = N / 2;
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
        const int p = lane + 32 * i;
        if (p < nseg) {
            const int e = emap[seg + p];
            float w = 0.f;
            if (e >= 0) {
                const int m3p = (e >> 8) - h, k3p = (e & 255) - h;
                if (rt.kk12 + k3p * k3p != 0) {
                    const int s3p = k3p - m3p;
                    w = pa[i] - radB[rt.mm12 + m3p * m3p];
                    if (!rt.centre) w += pa[i] - radB[rt.ss12 + s3p * s3p];
                }
            }
            wb[p] = w;
        }
    }
}

template <int NST, int WARPS>
__device__ __forceinline__ Ring ring_init(unsigned char *smem, int *err)
{
    static_assert(2 * NST * sizeof(uint64_t) + sizeof(int) <= kRingHead, "ring head");
    Ring r;
    r.full = reinterpret_cast<uint64_t *>(smem);
    r.empty = r.full + NST;
    r.abort_flag = reinterpret_cast<volatile int *>(r.empty + NST);
    r.stages = smem + kRingHead;
    r.err = err;
    r.tt = 0;
    r.issued = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&r.full[s], 1);
            mbar_init(&r.empty[s], WARPS);
        }
        *r.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    return r;
}

// after an abort: give the copies thread 0 issued a bounded time to land
// before the CTA exits.  Only the last NST uses can be in flight (thread 0
// issues use u after every warp released use u - NST, i.e. after it landed),
// and those sit in distinct slots, each in its slot's latest phase.  The
// limit is fixed (0.1 s), whatever the handle's wait limit.
template <int NST>
__device__ __forceinline__ void ring_drain(const Ring &r, bool ok)
{
    if (threadIdx.x == 0 && (!ok || *r.abort_flag)) {
        const uint32_t from = r.issued > r.tt + NST ? r.issued - NST : r.tt;
        for (uint32_t u = from; u < r.issued; ++u) {
            volatile int dummy = 0;
            wait_phase(&r.full[u % NST], (u / NST) & 1u, &dummy, r.err, kWaitUs / 20);
        }
    }
}

// One work item of job jb (item numbered within the job): a (pencil, group
// block) pair, or the part-th of S ranges of its tiles.  Thread 0 produces the
// pencil's tiles into the ring, NST ahead of the warps; every warp sums its
// strip.  Returns false (CTA-uniform) if a wait expired or the CTA aborted.
template <int N, int K, int U, int NST, int GPC, int S, bool RAD = false, int HS = 1>
__device__ __forceinline__ bool strip_item(const StripJob &jb, int item, Ring &rg)
{
    using C = StripCfg<N, K, U, NST, GPC, RAD, HS>;
    constexpr int H = N / 2;
    static_assert(HS == 1 || (HS == 2 && GPC == 1 && !RAD && (C::W / 2) % 2 == 0),
                  "two strips per warp: one group, stored tiles, pairs of strips of one kind");
    const int warp_id = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // group within the CTA, strip, and the cell's lane in the group.
    // Warps issue from the SM's four sub-partitions by warp slot mod 4, and
    // the strips of a tile carry unequal work (N = 32: 164, 228, 220 and 156
    // pairs for strips 0 .. 3), so with two groups the second takes the
    // strips shifted by W/2: the two warps of a CTA that share a
    // sub-partition then hold a light and a heavy strip (164 + 220 and
    // 228 + 156 at N = 32) instead of the same one twice.  Which warp sums
    // which strip moves no arithmetic.
    const int gl = HS == 1 ? warp_id / C::W : 0;
    // (with four groups the shifts are 0, W/2, W/4, 3W/4: every sub-partition
    // holds each of four strips once)
    static_assert(GPC != 4 || C::W % 4 == 0, "four groups per CTA need a multiple of four strips");
    const int warp = HS == 1 ? (GPC == 2   ? (warp_id % C::W + gl * (C::W / 2)) % C::W
                                : GPC == 4 ? (warp_id % C::W + ((gl & 1) * 2 + (gl >> 1)) * (C::W / 4)) % C::W
                                           : warp_id % C::W)
                             : 2 * warp_id + (lane >> 4);
    const int cl = HS == 1 ? lane : (lane & 15);
    const int k0 = warp * K;
    const bool kind_a = k0 < H;
    const int seg = strip_seg_off(N, K, warp);
    const int nblocks = jb.nblocks;
    rg.err = jb.err;

    const int part = item % S, rest = item / S;
    const int pencil = jb.order[rest / nblocks];
    const int gblk = rest % nblocks;
    const int grp = gblk * GPC + gl;
    const int k1 = pencil / N, k2 = pencil % N;
    const int K1 = k1 + H, K2 = k2 + H;
    const int lo1 = max(0, K1 - N + 1);
    const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
    const int Tall = jb.tile0[pencil + 1] - jb.tile0[pencil];
    const int tb = (part * Tall + S - 1) / S;  // this part's tiles: tb .. te-1
    const int te = ((part + 1) * Tall + S - 1) / S;
    const int T = te - tb;
    const float2 *Fb0 = jb.F + (size_t)gblk * GPC * C::M * kGroup;
    const float *Gp = jb.ghat + (size_t)(jb.tile0[pencil] + tb) * C::TSV;
    float2 *Qout = part == 0 ? jb.Qh : part == 1 ? jb.Qh2 : part == 2 ? jb.Qh3 : jb.Qh4;
    bool ok = true;

    TileWalk pw;  // producer's walk (thread 0), NST tiles ahead of the consumers
    int pt = 0;
    auto issue_next = [&]() -> bool {
        const uint32_t u = rg.tt + pt;
        const int s = u % NST;
        if (u >= NST && !wait_phase(&rg.empty[s], ((u / NST) + 1) & 1u, rg.abort_flag, rg.err, jb.wait_us))
            return false;
        unsigned char *st = rg.stages + s * C::STAGE;
        mbar_arrive_expect_tx(&rg.full[s], 2 * GPC * C::ROWB + (RAD ? 0 : C::GB));
        const size_t ra = (size_t)(pw.m1 * N + pw.m2) * N * kGroup;
        const size_t rb = (size_t)((K1 - pw.m1) * N + (K2 - pw.m2)) * N * kGroup;
        // policies made here (one instruction each), so no thread holds them in registers
        if (jb.l2hint & 2) {
            const uint64_t pol_f = l2_policy_evict_last();
#pragma unroll
            for (int q = 0; q < GPC; ++q) {
                const float2 *Fq = Fb0 + (size_t)q * C::M * kGroup;
                bulk_copy_hint(st + q * C::ROWB, Fq + ra, C::ROWB, &rg.full[s], pol_f);
                bulk_copy_hint(st + (GPC + q) * C::ROWB, Fq + rb, C::ROWB, &rg.full[s], pol_f);
            }
        } else {
#pragma unroll
            for (int q = 0; q < GPC; ++q) {
                const float2 *Fq = Fb0 + (size_t)q * C::M * kGroup;
                bulk_copy(st + q * C::ROWB, Fq + ra, C::ROWB, &rg.full[s]);
                bulk_copy(st + (GPC + q) * C::ROWB, Fq + rb, C::ROWB, &rg.full[s]);
            }
        }
        if constexpr (!RAD) {
            if (jb.l2hint & 1)
                bulk_copy_hint(st + 2 * GPC * C::ROWB, Gp + (size_t)pt * C::TSV, C::GB, &rg.full[s],
                               l2_policy_evict_first());
            else
                bulk_copy(st + 2 * GPC * C::ROWB, Gp + (size_t)pt * C::TSV, C::GB, &rg.full[s]);
        }
        ++pt;
        ++rg.issued;
        pw.next();
        return true;
    };
    // the test stall: the first CTA issues nothing for its first item
    const bool stalled = jb.stall && blockIdx.x == 0 && rg.tt == 0;
    if (threadIdx.x == 0 && !stalled) {
        pw.start(lo1, lo2, hi2, K1, K2);
        for (int i = 0; i < tb; ++i) pw.next();
        while (pt < NST && pt < T)
            if (!issue_next()) {
                ok = false;
                break;
            }
    }

    float2 acc[K];
    CompSum<K, strip_comp_where<N, GPC, RAD>()> cs;
    if constexpr (strip_comp_where<N, GPC, RAD>() == 2) {
        cs.v = reinterpret_cast<float *>(rg.stages + NST * C::STAGE) + C::WARPS * C::WBUF + (RAD ? C::TSV : 0) +
               strip_round4(C::NB) + threadIdx.x;
        cs.stride = 32 * C::WARPS;
    }
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = make_float2(0.f, 0.f);
    cs.zero();
    TileWalk cw;
    cw.start(lo1, lo2, hi2, K1, K2);
    for (int i = 0; i < tb; ++i) cw.next();
    int cur_m1 = cw.m1;
    float *wb = nullptr;  // RAD: this warp's weight segment, the entry map and B
    const int *s_emap = nullptr;
    const float *s_radB = nullptr;
    constexpr int EPL = RAD ? (C::WBUF + 31) / 32 : 1;  // segment entries per lane
    float pa[EPL];                                      // A of the next tile's entries, loaded a tile ahead
    const int nseg = strip_seg_size(N, K, warp);
    if constexpr (RAD) {
        float *r = reinterpret_cast<float *>(rg.stages + NST * C::STAGE);
        wb = r + warp_id * C::WBUF;
        s_emap = reinterpret_cast<const int *>(r + C::WARPS * C::WBUF);
        s_radB = r + C::WARPS * C::WBUF + C::TSV;
        if (T > 0) radius_gather<N, EPL>(jb, s_emap, seg, nseg, radius_tile<N>(k1, k2, cw.m1, cw.m2), lane, pa);
    }
    for (int t = 0; t < T && ok; ++t) {
        const uint32_t u = rg.tt + t;
        const int s = u % NST;
        if constexpr (RAD) {  // this tile's weights from the loads issued a tile ago, then the next tile's loads
            radius_combine<N, EPL>(s_emap, s_radB, seg, nseg, radius_tile<N>(k1, k2, cw.m1, cw.m2), lane, pa, wb);
            __syncwarp();
            if (t + 1 < T) {
                TileWalk nw = cw;
                nw.next();
                radius_gather<N, EPL>(jb, s_emap, seg, nseg, radius_tile<N>(k1, k2, nw.m1, nw.m2), lane, pa);
            }
        }
        if (!wait_phase(&rg.full[s], (u / NST) & 1u, rg.abort_flag, rg.err, jb.wait_us)) {
            ok = false;
            break;
        }
        if (cw.m1 != cur_m1) {  // new m1 slab: fold the finished one
#pragma unroll
            for (int j = 0; j < K; ++j) {
                cs.add(j, acc[j]);
                acc[j] = make_float2(0.f, 0.f);
            }
            cur_m1 = cw.m1;
        }
        const unsigned char *st = rg.stages + s * C::STAGE;
        const float2 *arow = reinterpret_cast<const float2 *>(st + gl * C::ROWB);
        const float2 *brow = reinterpret_cast<const float2 *>(st + (GPC + gl) * C::ROWB);
        const float *gt = RAD ? wb : reinterpret_cast<const float *>(st + 2 * GPC * C::ROWB) + seg;
        if (kind_a)
            strip_a<N, K, U>(arow, brow, gt, k0, cl, acc);
        else
            strip_b<N, K, U>(arow, brow, gt, k0, cl, acc);
        cw.next();
        __syncwarp();
        if (lane == 0) mbar_arrive(&rg.empty[s]);
        if (threadIdx.x == 0 && pt < T && !stalled)
            if (!issue_next()) ok = false;
        __syncwarp();
    }
    if (__syncthreads_or(!ok || *rg.abort_flag)) return false;  // CTA-uniform
#pragma unroll
    for (int j = 0; j < K; ++j) {
        cs.add(j, acc[j]);
        const float2 v = cs.value(j);
        Qout[((size_t)grp * C::M + (size_t)pencil * N + k0 + j) * kGroup + cl] =
            make_float2(jb.omega * v.x, jb.omega * v.y);
    }
    rg.tt += T;
    if constexpr (S > 1) {
        // the last of a (pencil, block)'s S ranges adds the partial sums into
        // Qh, in range order: every consumer reads one buffer, and the sum
        // does not depend on which range finished last.  The CTA's stores
        // are ordered before thread 0's count by the barrier and the count's
        // release; the last CTA's reads after it by the count's acquire and
        // the barrier, and they bypass L1
        __shared__ int s_last;
        __syncthreads();
        if (threadIdx.x == 0) {
            int old;
            asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], 1;" : "=r"(old) : "l"(jb.done + rest) : "memory");
            s_last = old == S - 1;
        }
        __syncthreads();
        if (s_last) {
            const float2 *more[3] = {jb.Qh2, jb.Qh3, jb.Qh4};
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const size_t idx = ((size_t)grp * C::M + (size_t)pencil * N + k0 + j) * kGroup + cl;
                float2 v = __ldcg(jb.Qh + idx);
#pragma unroll
                for (int m = 0; m < S - 1; ++m) {
                    const float2 w = __ldcg(more[m] + idx);
                    v = make_float2(v.x + w.x, v.y + w.y);
                }
                jb.Qh[idx] = v;
            }
        }
    }
    return true;
}


// Persistent kernel: CTAs take (pencil, group block) items from an atomic
// counter, heaviest pencils first, so the tail of the launch holds only the
// smallest items.
// Resident CTAs per SM the register allocation must allow: at N = 16 the
// kernel is latency-bound and 128 registers (8 one-group or 4 two-group CTAs
// per SM) measured faster than the ~134 the compiler picks on its own; for
// the other N one CTA (no cap) measured best, except N = 32 with two groups
// per CTA (compensated sums in local memory, 113 registers, two CTAs of 8
// warps per SM).  At N = 32 with one group per CTA three CTAs share an SM
// only while a thread needs at most 168 registers (they are allocated in
// steps of 8): 170 rounded up to 176 and left two, 7 % slower, and a cap of
// three CTAs made the compiler settle at 163, 2 % slower than its own 166.
template <int N, int GPC, bool RAD = false>
constexpr int strip_min_ctas() { return N == 16 ? (GPC == 1 ? 8 : 4) : (N == 32 && GPC == 2 && !RAD) ? 2 : 1; }

template <int N, int K, int U, int NST, int GPC, int S, bool RAD, int HS = 1>
__global__ void __launch_bounds__(32 * (N / K) * GPC / HS, strip_min_ctas<N, GPC, RAD>())
    conv_strip_kernel(StripJob jb, int *counter)
{
    using C = StripCfg<N, K, U, NST, GPC, RAD, HS>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    Ring rg = ring_init<NST, C::WARPS>(smem, jb.err);
    if constexpr (RAD) {  // the entry map and B into shared memory, once per CTA
        float *r = reinterpret_cast<float *>(rg.stages + NST * C::STAGE) + C::WARPS * C::WBUF;
        int *se = reinterpret_cast<int *>(r);
        for (int i = threadIdx.x; i < C::TSV; i += blockDim.x) se[i] = jb.emap[i];
        for (int i = threadIdx.x; i < C::NB; i += blockDim.x) r[C::TSV + i] = jb.radB[i];
        __syncthreads();
    }
    const int nitems = N * N * jb.nblocks * S;
    bool ok = true;
    for (;;) {
        // thread 0 decides for the whole CTA, so every thread leaves the loop together
        if (threadIdx.x == 0) s_item = *rg.abort_flag ? nitems : atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        if (!strip_item<N, K, U, NST, GPC, S, RAD, HS>(jb, item, rg)) {
            ok = false;
            break;
        }
    }
    ring_drain<NST>(rg, ok);
}

template <int N, int K, int U, int NST, int GPC, int S, bool RAD, int HS = 1>
int launch_cfg(const Handle &hd, int ncells, cudaStream_t s)
{
    using C = StripCfg<N, K, U, NST, GPC, RAD, HS>;
    static_assert(K % 4 == 0 && (N / 2) % K == 0, "strip width must divide N/2 and be a multiple of 4");
    static_assert(K % U == 0, "the row block must divide the strip width (the strip bodies' remainders assume it)");
    static_assert(C::STAGE % 16 == 0 && C::ROWB % 16 == 0 && C::GB % 16 == 0, "bulk copies need 16-byte units");
    auto kern = conv_strip_kernel<N, K, U, NST, GPC, S, RAD, HS>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_error(e, "strip kernel shared-memory attribute");
    }
    const int ng = ngroups_of(ncells);
    const int nblocks = ng / GPC;  // callers pick GPC dividing ng
    const int nitems = N * N * nblocks * S;
    static int occ = 0;  // resident CTAs per SM of this instantiation
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
    if (e == cudaSuccess && S > 1) e = cudaMemsetAsync(hd.done, 0, sizeof(int) * N * N * nblocks, s);
    if (e != cudaSuccess) return cuda_error(e, "strip kernel work counters");
    StripJob jb{(const float *)hd.ghat, hd.pencil_tile0, hd.pencil_order, (const float2 *)hd.F,
                (float2 *)hd.Qh, (float2 *)hd.Qh2, (float2 *)hd.Qh3, (float2 *)hd.Qh4, hd.done, hd.err, omega,
                nblocks, N, 0};
    jb.wait_us = hd.wait_us ? hd.wait_us : kWaitUs;
    jb.stall = hd.test_stall;
    jb.l2hint = l2_hint_bits(hd.tune_l2);
    if constexpr (RAD) {
        jb.radA = hd.radA;
        jb.radB = hd.radB;
        jb.emap = hd.emap;
        jb.bbn = hd.rad_bb;
    }
    kern<<<grid, 32 * C::WARPS, C::SMEM, s>>>(jb, hd.counter);
    CS_LAUNCHED(1, s, RAD ? "convolution (strip kernel, radius tables)" : "convolution (strip kernel)");
    return CS_OK;
}

template <int N, int K, int U, int NST1, int NST2, int S, bool RAD>
int launch_n(const Handle &hd, int ncells, cudaStream_t s)
{
    const bool even = ngroups_of(ncells) % 2 == 0;
    // two groups per CTA by default up to N = 32 (N = 32, 256 cells: 13.27 ms against 13.44 ms with one
    // group, and 1.6 GB of DRAM reads instead of 2.2 GB); at N = 48 and 64 one group fills a CTA
    const bool two = hd.tune_gpc == 2 || (hd.tune_gpc == 0 && N <= 32);
    // four groups per CTA (N = 32, stored tiles, a launch choice): one CTA of
    // 16 warps per SM, each weight tile staged once for 128 cells
    if constexpr (!RAD && N == 32 && StripCfg<N, K, U, NST2, 4>::SMEM <= 227 * 1024)
        if (hd.tune_gpc == 4 && ngroups_of(ncells) % 4 == 0) return launch_cfg<N, K, U, NST2, 4, S, RAD>(hd, ncells, s);
    if (even && (two || hd.tune_gpc == 4)) return launch_cfg<N, K, U, NST2, 2, S, RAD>(hd, ncells, s);
    // at most 16 cells: two strips per warp, 16 lanes each, so no lane holds padding
    if constexpr (!RAD && (N == 32 || N == 64))
        if (ncells <= 16 && hd.tune_gpc != 1) return launch_cfg<N, K, U, NST1, 1, S, RAD, 2>(hd, ncells, s);
    return launch_cfg<N, K, U, NST1, 1, S, RAD>(hd, ncells, s);
}

// the strip launch of every N, with stored weight tiles or (RAD) tiles
// rebuilt from the radius tables; conv_strip.cu and conv_radius.cu each
// instantiate one
template <bool RAD>
int launch_strip_mode(const Handle &hd, int ncells, cudaStream_t s)
{
    switch (hd.g.N) {
    case 8: return launch_n<8, 4, 4, 4, 4, 1, RAD>(hd, ncells, s);
    case 16:
        return conv_split(hd) == 2 ? launch_n<16, 8, 8, 3, 3, 2, RAD>(hd, ncells, s)
                                   : launch_n<16, 8, 8, 3, 3, 4, RAD>(hd, ncells, s);
    case 24: return launch_n<24, 12, 4, 3, 2, 1, RAD>(hd, ncells, s);
    case 32:  // tile split (CS_TUNE_SPLIT) in a translation unit of its own
        return conv_split(hd) > 1 ? launch_strip_split32(hd, ncells, s, RAD)
                                  : launch_n<32, 8, 8, 3, RAD ? 3 : 2, 1, RAD>(hd, ncells, s);
    case 48: return launch_n<48, 8, 8, 3, 2, 1, RAD>(hd, ncells, s);
    case 64: return launch_n<64, 8, 8, 3, 2, 1, RAD>(hd, ncells, s);
    default: return set_error(CS_ENOTSUP, "strip kernel: unsupported N");
    }
}

}  // namespace

}  // namespace cs
