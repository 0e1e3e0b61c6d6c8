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

template <typename T>
int convolve_impl(const Handle &hd, int ncells, cudaStream_t s)
{
    const Geom &g = hd.g;
    const T omega = (T)(g.dz * g.dz * g.dz);
    dim3 grid((unsigned)((g.M + 3) / 4), (unsigned)ngroups_of(ncells));
    conv_generic_kernel<T><<<grid, 128, 0, s>>>(g, (const T *)hd.ghat, hd.pencil_tile0, (const c2_t<T> *)hd.F,
                                                (c2_t<T> *)hd.Qh, omega);
    CS_CHECK_LAUNCH("convolution");
    return CS_OK;
}

}  // namespace

int launch_convolve(const Handle &hd, int ncells, cudaStream_t s)
{
    return hd.precision == CS_FP32 ? convolve_impl<float>(hd, ncells, s) : convolve_impl<double>(hd, ncells, s);
}

}  // namespace cs
