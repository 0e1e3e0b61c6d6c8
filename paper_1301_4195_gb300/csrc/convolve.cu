// K2: the weighted convolution of Sec. 3.2 (trapezoid rule, omega = dzeta^3,
// terms with zeta_k - xi_m off the grid dropped):
//   Qhat(zeta_k) = omega sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m).
// With K = k + N/2 the partner index is s = K - m.  The sum runs over the
// symmetrised half-tiles of the weight table (see weights.cu): for each
// (m1, m2) with (m1, m2) <= (s1, s2) lexicographically and each valid m3,
//   Qhat_k += w(m, k) fhat_m fhat_s,
// where w already holds Ghat(m, k) + Ghat(s, k) off the centre tile.
//
// Thread mapping: one warp per output zeta_k of one group of 32 cells, one
// cell per lane.  All lanes share k, hence the loop bounds and the weight
// (a broadcast load); each lane loads its own cell's fhat values, which sit
// in consecutive addresses across the warp (grouped layout).
//
// Precision: double accumulates directly.  float accumulates each (m1, m2)
// tile (at most N terms) into a float partial and adds the partial into a
// (hi, lo) pair by an error-free two-sum, so the long sum over xi is
// compensated.
#include <utility>

#include "cs_internal.cuh"

namespace cs {

namespace {

template <typename T> struct Acc;

template <> struct Acc<double> {
    double re = 0, im = 0;
    __device__ void add(double pr, double pi) { re += pr; im += pi; }
    __device__ double2 value(double omega) const { return make_double2(omega * re, omega * im); }
};

__device__ __forceinline__ void two_sum(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

template <> struct Acc<float> {
    float hr = 0, lr = 0, hi_ = 0, li = 0;
    __device__ void add(float pr, float pi) { two_sum(hr, lr, pr); two_sum(hi_, li, pi); }
    __device__ float2 value(float omega) const { return make_float2(omega * (hr + lr), omega * (hi_ + li)); }
};

template <typename T>
__global__ void __launch_bounds__(128) conv_generic_kernel(Geom g, const T *__restrict__ ghat,
                                                           const int *__restrict__ tile0,
                                                           const c2_t<T> *__restrict__ F,
                                                           c2_t<T> *__restrict__ Qh, T omega)
{
    const int N = g.N, h = g.h, M = g.M;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kf = blockIdx.x * 4 + w;
    if (kf >= M) return;
    const int grp = blockIdx.y;
    const int k1 = kf / (N * N), k2 = (kf / N) % N, k3 = kf % N;
    const int K1 = k1 + h, K2 = k2 + h, K3 = k3 + h;
    const int lo1 = max(0, K1 - N + 1);
    const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
    const int m3lo = max(0, K3 - N + 1), m3hi = min(N - 1, K3);
    const T *Gp = ghat + (size_t)tile0[k1 * N + k2] * g.TSp;
    const c2_t<T> *Fg = F + (size_t)grp * M * kGroup + lane;
    Acc<T> acc;
    int t = 0;
    for (int m1 = lo1; 2 * m1 <= K1; ++m1) {
        const int s1 = K1 - m1;
        const int m2end = (2 * m1 < K1) ? hi2 : (K2 / 2);
        for (int m2 = lo2; m2 <= m2end; ++m2, ++t) {
            const int s2 = K2 - m2;
            const T *Gt = Gp + (size_t)t * g.TSp;
            const c2_t<T> *Fa = Fg + (size_t)((m1 * N + m2) * N) * kGroup;
            const c2_t<T> *Fb = Fg + (size_t)((s1 * N + s2) * N) * kGroup;
            T pr = 0, pi = 0;
            for (int m3 = m3lo; m3 <= m3hi; ++m3) {
                const T wgt = Gt[g.off[m3] + k3 - kmin_of(m3, h)];
                const c2_t<T> a = Fa[(size_t)m3 * kGroup];
                const c2_t<T> b = Fb[(size_t)(K3 - m3) * kGroup];
                pr += wgt * (a.x * b.x - a.y * b.y);
                pi += wgt * (a.x * b.y + a.y * b.x);
            }
            acc.add(pr, pi);
        }
    }
    Qh[((size_t)grp * M + kf) * kGroup + lane] = acc.value(omega);
}

// ---------------------------------------------------------------------------
// Pencil kernel (float, N a multiple of 4).  One warp owns one output pencil
// (k1, k2, all k3) of one 32-cell group, one cell per lane.  Each thread keeps
// the N complex accumulators of its pencil and, per (m1, m2) tile, the partner
// row fhat(s1, s2, :) in registers; the tile's (m3, k3) loops are unrolled at
// compile time, so there is no index arithmetic, no mask and no wasted pair.
// The weights are read as warp-uniform float4 (one broadcast per four pairs).
// The next tile's rows and weights are prefetched into L1 while the current
// one is computed.  Each m1 slab is summed in float and added to a running
// (hi, lo) pair kept in global memory by an error-free two-sum.

__host__ __device__ constexpr int cx_kmin(int m3, int h) { return m3 - h > 0 ? m3 - h : 0; }
__host__ __device__ constexpr int cx_kmax(int m3, int h, int n) { return m3 + h - 1 < n - 1 ? m3 + h - 1 : n - 1; }
__host__ __device__ constexpr int cx_off(int m3, int n)
{
    int o = 0;
    for (int m = 0; m < m3; ++m) o += ((cx_kmax(m, n / 2, n) - cx_kmin(m, n / 2) + 1) + 3) & ~3;
    return o;
}

__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// one row (fixed m3) of a tile: acc[k3] += w(m3, k3) a fhat(s1, s2, k3 - m3 + N/2)
template <int N, int M3>
__device__ __forceinline__ void pencil_row(const float *__restrict__ Gt, const float2 *__restrict__ Fa,
                                           const float2 (&b)[N], float2 (&acc)[N])
{
    constexpr int H = N / 2;
    constexpr int KLO = cx_kmin(M3, H), KHI = cx_kmax(M3, H, N);
    constexpr int NQ = (KHI - KLO + 4) / 4;
    const float2 a = __ldg(Fa + M3 * kGroup);
    const float4 *Gr = reinterpret_cast<const float4 *>(Gt + cx_off(M3, N));
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float4 g4 = __ldg(Gr + q);
        const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k3 = KLO + 4 * q + j;
            if (k3 <= KHI) {
                const float2 bb = b[k3 - M3 + H];
                const float tr = fmaf(a.x, bb.x, -a.y * bb.y);
                const float ti = fmaf(a.x, bb.y, a.y * bb.x);
                acc[k3].x = fmaf(gv[j], tr, acc[k3].x);
                acc[k3].y = fmaf(gv[j], ti, acc[k3].y);
            }
        }
    }
}

template <int N, int... M3s>
__device__ __forceinline__ void pencil_tile(std::integer_sequence<int, M3s...>, const float *__restrict__ Gt,
                                            const float2 *__restrict__ Fa, const float2 (&b)[N], float2 (&acc)[N])
{
    (pencil_row<N, M3s>(Gt, Fa, b, acc), ...);
}

template <int N>
__global__ void __launch_bounds__(128) conv_pencil_kernel(const float *__restrict__ ghat,
                                                          const int *__restrict__ tile0,
                                                          const int *__restrict__ order, int ngroups,
                                                          const float2 *__restrict__ F, float2 *__restrict__ Qh,
                                                          float2 *__restrict__ Lo, float omega)
{
    constexpr int H = N / 2;
    constexpr int M = N * N * N;
    constexpr int TS = cx_off(N, N);
    constexpr int ROW = N * kGroup;  // float2 per (m1, m2) row of one group
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= N * N * ngroups) return;
    const int pencil = order[item / ngroups];
    const int grp = item % ngroups;
    const int k1 = pencil / N, k2 = pencil % N;
    const int K1 = k1 + H, K2 = k2 + H;
    const int lo1 = max(0, K1 - N + 1);
    const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
    const int m1last = K1 / 2;
    const float *G = ghat + (size_t)tile0[pencil] * TS;
    const float2 *Fg = F + (size_t)grp * M * kGroup;
    const size_t obase = ((size_t)grp * M + (size_t)pencil * N) * kGroup + lane;

    float2 acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = make_float2(0.f, 0.f);

    for (int m1 = lo1; m1 <= m1last; ++m1) {
        const int s1 = K1 - m1;
        const int m2end = (2 * m1 < K1) ? hi2 : (K2 / 2);
        for (int m2 = lo2; m2 <= m2end; ++m2) {
            const int s2 = K2 - m2;
            const float2 *Fa = Fg + (size_t)(m1 * N + m2) * ROW + lane;
            const float2 *Fb = Fg + (size_t)(s1 * N + s2) * ROW + lane;
            {   // prefetch the next tile (rows of 256 N bytes, weights of 4 TS bytes)
                int n1 = m1, n2 = m2 + 1;
                if (n2 > m2end) {
                    n1 = m1 + 1;
                    n2 = lo2;
                }
                if (n1 <= m1last) {
                    const char *pa = (const char *)(Fg + (size_t)(n1 * N + n2) * ROW);
                    const char *pb = (const char *)(Fg + (size_t)((K1 - n1) * N + (K2 - n2)) * ROW);
                    for (int l = lane; l < 2 * N; l += 32) {
                        prefetch_l1(pa + 128 * l);
                        prefetch_l1(pb + 128 * l);
                    }
                    for (int l = lane; l * 32 < TS; l += 32) prefetch_l1(G + TS + 32 * l);
                }
            }
            float2 b[N];
#pragma unroll
            for (int s3 = 0; s3 < N; ++s3) b[s3] = __ldg(Fb + s3 * kGroup);
            pencil_tile<N>(std::make_integer_sequence<int, N>{}, G, Fa, b, acc);
            G += TS;
        }
        // fold this m1 slab into the running (hi, lo) sum
        const bool first = (m1 == lo1), last = (m1 == m1last);
#pragma unroll
        for (int k3 = 0; k3 < N; ++k3) {
            const size_t o = obase + (size_t)k3 * kGroup;
            float2 hv = acc[k3], lv = make_float2(0.f, 0.f);
            if (!first) {
                hv = Qh[o];
                lv = Lo[o];
                two_sum(hv.x, lv.x, acc[k3].x);
                two_sum(hv.y, lv.y, acc[k3].y);
            }
            if (last) {
                Qh[o] = make_float2(omega * (hv.x + lv.x), omega * (hv.y + lv.y));
            } else {
                Qh[o] = hv;
                Lo[o] = lv;
            }
            acc[k3] = make_float2(0.f, 0.f);
        }
    }
}

template <int N>
int launch_pencil(const Handle &hd, int ncells, cudaStream_t s)
{
    const int ng = ngroups_of(ncells);
    const long long items = (long long)N * N * ng;
    const unsigned blocks = (unsigned)((items + 3) / 4);
    const float omega = (float)(hd.g.dz * hd.g.dz * hd.g.dz);
    conv_pencil_kernel<N><<<blocks, 128, 0, s>>>((const float *)hd.ghat, hd.pencil_tile0, hd.pencil_order, ng,
                                                 (const float2 *)hd.F, (float2 *)hd.Qh, (float2 *)hd.Y, omega);
    CS_LAUNCHED(1, s, "convolution (pencil kernel)");
    return CS_OK;
}

template <typename T>
int convolve_impl(const Handle &hd, int ncells, cudaStream_t s)
{
    const Geom &g = hd.g;
    if (sizeof(T) == 4) {
        if (g.layout == LAYOUT_STRIP) return launch_strip(hd, ncells, s);
        switch (g.N) {  // float, ROWS layout
        case 12: return launch_pencil<12>(hd, ncells, s);
        case 20: return launch_pencil<20>(hd, ncells, s);
        case 28: return launch_pencil<28>(hd, ncells, s);
        default: break;
        }
    }
    const T omega = (T)(g.dz * g.dz * g.dz);
    dim3 grid((unsigned)((g.M + 3) / 4), (unsigned)ngroups_of(ncells));
    conv_generic_kernel<T><<<grid, 128, 0, s>>>(g, (const T *)hd.ghat, hd.pencil_tile0, (const c2_t<T> *)hd.F,
                                                (c2_t<T> *)hd.Qh, omega);
    CS_LAUNCHED(1, s, "convolution");
    return CS_OK;
}

}  // namespace

int launch_convolve(const Handle &hd, int ncells, cudaStream_t s)
{
    return hd.precision == CS_FP32 ? convolve_impl<float>(hd, ncells, s) : convolve_impl<double>(hd, ncells, s);
}

}  // namespace cs
