// K0: the convolution weights Ghat(xi, zeta) of Sec. 2.2 (eq. GHat_calc),
// isotropic b = 1/(4 pi), beta = 1, radial integral cut at r0 = L:
//   Ghat = sqrt(2/pi) int_0^{r0} r^{lambda+2} [sinc(r a) sinc(r b) - sinc(r c)] dr,
//   a = |zeta|/2, b = |xi - zeta/2|, c = |xi|.
// For lambda = 0, 1 the closed forms of Sec. 2.2 are used with
// p = a - b, q = a + b (so that sinc(ar) sinc(br) = [cos(pr) - cos(qr)] / (2ab r^2));
// other lambda use composite Gauss-Legendre on the radial integral.
//
// Table layout.  Output zeta_k is split into pencils (k1, k2) along k3.  For
// pencil (k1, k2) with K = k + N/2 the valid xi_m satisfy, per axis,
// m_i in [max(0, K_i - N + 1), min(N - 1, K_i)] (Sec. 3.2: terms whose
// zeta_k - xi_m leaves the grid are dropped), and the partner index is
// s = K - m.  The pair (m, s) and (s, m) multiply the same fhat product, so
// the table keeps one "tile" per (m1, m2) in the lower half
//   2 m1 < K1,  or  2 m1 = K1 and 2 m2 <= K2,
// holding for every valid (m3, k3) the weight Ghat(m, k) + Ghat(K - m, k);
// the centre tile (m1, m2) = (s1, s2) keeps the plain weight Ghat(m, k).
// Inside a tile the pairs are ordered by m3, then k3 in
// [max(0, m3 - N/2), min(N - 1, m3 + N/2 - 1)]; a tile holds 3N^2/4 pairs and
// each row (one m3) is padded with zeros to a multiple of 4 entries so rows
// start on 16-byte boundaries.  Tiles of one pencil are consecutive, pencils
// in (k1, k2) order.
//
// Radius tables (the alternative to storing every pair).  Ghat depends on the
// pair only through three integer squared radii, with k' = k - N/2 and
// m' = m - N/2:  a = dz |k'| / 2,  b = dz |2m' - k'| / 2,  c = dz |m'|, and
// splits into two one- and two-index integrals,
//   Ghat(m, k) = A(|k'|^2, |2m' - k'|^2) - B(|m'|^2),
//   A = sqrt(2/pi) int_0^{r0} r^{lambda+2} sinc(r a) sinc(r b) dr,
//   B = sqrt(2/pi) int_0^{r0} r^{lambda+2} sinc(r c) dr,
// (Ghat = 0 when k' = 0).  For the mirror partner s' = k' - m' the middle
// radius is the same, so the symmetrised weight of a tile entry is
// 2 A - B(|m'|^2) - B(|s'|^2).  A holds (3 h^2 + 1) x (3 (N-1)^2 + 1) floats
// (h = N/2: 9 MB at N = 32, 146 MB at N = 64), B 3 h^2 + 1; both are
// evaluated in double (the same closed forms and quadrature as the table) and
// kept in float.  The strip kernel can rebuild each weight tile from them in
// shared memory instead of reading the stored tile (conv_strip.cu).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kQuadNodes = 24;

struct QuadRule {
    double x[kQuadNodes];
    double w[kQuadNodes];
};

// Gauss-Legendre rule on [-1, 1] (Newton iteration on P_n from its recurrence).
QuadRule make_rule()
{
    QuadRule r{};
    const int n = kQuadNodes;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0, pm = 0;
        for (int it = 0; it < 100; ++it) {
            pn = 1.0;
            pm = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double t = pm;
                pm = pn;
                pn = ((2 * j - 1) * z * pm - (j - 1) * t) / j;
            }
            const double d = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / d;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        pn = 1.0;
        pm = 0.0;
        for (int j = 1; j <= n; ++j) {
            const double t = pm;
            pm = pn;
            pn = ((2 * j - 1) * z * pm - (j - 1) * t) / j;
        }
        const double d = n * (z * pn - pm) / (z * z - 1.0);
        r.x[i] = z;
        r.w[i] = 2.0 / ((1.0 - z * z) * d * d);
    }
    return r;
}

__device__ double series_cos_moment(double x, double r0, double lam)
{
    // int_0^r0 r^lam cos(x r) dr = r0^{lam+1} sum_n (-1)^n y^{2n} / ((2n)! (2n + lam + 1))
    const double y2 = (x * r0) * (x * r0);
    double term = 1.0, sum = 0.0;
    for (int n = 0; n < 40; ++n) {
        const double t = term / (2.0 * n + lam + 1.0);
        sum += t;
        if (fabs(t) < 1e-18 * fabs(sum) && n > 2) break;
        term *= -y2 / ((2.0 * n + 1.0) * (2.0 * n + 2.0));
    }
    return pow(r0, lam + 1.0) * sum;
}

__device__ double series_sinc_moment(double x, double r0, double lam)
{
    // int_0^r0 r^{lam+2} sinc(x r) dr = r0^{lam+3} sum_n (-1)^n y^{2n} / ((2n+1)! (2n + lam + 3))
    const double y2 = (x * r0) * (x * r0);
    double term = 1.0, sum = 0.0;
    for (int n = 0; n < 40; ++n) {
        const double t = term / (2.0 * n + lam + 3.0);
        sum += t;
        if (fabs(t) < 1e-18 * fabs(sum) && n > 2) break;
        term *= -y2 / ((2.0 * n + 2.0) * (2.0 * n + 3.0));
    }
    return pow(r0, lam + 3.0) * sum;
}

// Phi(x) = int_0^r0 r^lam cos(x r) dr, lam in {0, 1}
__device__ double cos_moment(double x, double r0, int lam)
{
    const double y = x * r0;
    if (fabs(y) < 0.5) return series_cos_moment(x, r0, lam);
    double s, c;
    sincos(y, &s, &c);
    if (lam == 0) return s / x;
    return (y * s + c - 1.0) / (x * x);
}

// Psi(x) = int_0^r0 r^{lam+2} sinc(x r) dr, lam in {0, 1}
__device__ double sinc_moment(double x, double r0, int lam)
{
    const double y = x * r0;
    if (fabs(y) < 1.0) return series_sinc_moment(x, r0, lam);
    double s, c;
    sincos(y, &s, &c);
    if (lam == 0) return (s - y * c) / (x * x * x);
    return ((2.0 - y * y) * c + 2.0 * y * s - 2.0) / (x * x * x * x);
}

__device__ double dsinc(double x)
{
    if (fabs(x) < 1e-4) return 1.0 - x * x * (1.0 / 6.0) + x * x * x * x * (1.0 / 120.0);
    return sin(x) / x;
}

// radial integral of the bracket by composite Gauss-Legendre, first panel
// graded geometrically toward r = 0 for r^{lambda+2}
__device__ double radial_bracket_quad(double a, double b, double c, double r0, double lam,
                                      const QuadRule &q)
{
    const int np = (int)ceil((a + b + c) * r0 / 3.0) + 2;
    const double hw = r0 / np;
    double total = 0.0;
    for (int p = 0; p < np; ++p) {
        const int nsub = (p == 0) ? 12 : 1;
        for (int sidx = 0; sidx < nsub; ++sidx) {
            double lo, hi;
            if (p == 0) {
                hi = hw * exp2(-(double)(nsub - 1 - sidx));
                lo = (sidx == 0) ? 0.0 : hw * exp2(-(double)(nsub - sidx));
            } else {
                lo = p * hw;
                hi = (p + 1) * hw;
            }
            const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int i = 0; i < kQuadNodes; ++i) {
                const double r = mid + half * q.x[i];
                total += half * q.w[i] * pow(r, lam + 2.0) * (dsinc(a * r) * dsinc(b * r) - dsinc(c * r));
            }
        }
    }
    return total;
}

// Ghat for centred integer indices kp = k - N/2 (zeta), mp = m - N/2 (xi).
__device__ double ghat_centered(const Geom &g, const QuadRule &q, int kp1, int kp2, int kp3,
                                int mp1, int mp2, int mp3)
{
    const long kk = (long)kp1 * kp1 + (long)kp2 * kp2 + (long)kp3 * kp3;
    if (kk == 0) return 0.0;  // G(u, 0) = 0
    const long mm = (long)mp1 * mp1 + (long)mp2 * mp2 + (long)mp3 * mp3;
    const long d1 = 2 * mp1 - kp1, d2 = 2 * mp2 - kp2, d3 = 2 * mp3 - kp3;
    const long bb = d1 * d1 + d2 * d2 + d3 * d3;
    const long mk = (long)mp1 * kp1 + (long)mp2 * kp2 + (long)mp3 * kp3;
    const double dz = g.dz, r0 = g.L;
    const double a = 0.5 * dz * sqrt((double)kk);
    const double b = 0.5 * dz * sqrt((double)bb);
    const double c = dz * sqrt((double)mm);
    const double pref = 0.79788456080286535588;  // sqrt(2 / pi) = 4 pi / (2 pi)^{3/2}
    const double lam = g.lambda;
    if (lam == 0.0 || lam == 1.0) {
        const int il = (int)lam;
        double t1;
        if (bb == 0) {
            t1 = sinc_moment(a, r0, il);
        } else {
            // p = a - b = (a^2 - b^2)/(a + b), a^2 - b^2 = dz^2 (m'.k' - |m'|^2) exactly
            const double qv = a + b;
            const double pv = dz * dz * (double)(mk - mm) / qv;
            t1 = (cos_moment(pv, r0, il) - cos_moment(qv, r0, il)) / (2.0 * a * b);
        }
        const double t2 = (mm == 0) ? sinc_moment(0.0, r0, il) : sinc_moment(c, r0, il);
        return pref * (t1 - t2);
    }
    return pref * radial_bracket_quad(a, b, c, r0, lam, q);
}

// ---- anisotropic scattering (Sec. 2: B = |u|^lambda b(cos theta)).  With the
// Legendre moments bl[l] = int_{S^2} b P_l dsigma, the Funk-Hecke theorem turns
// the sphere integral of G(u, zeta) into a Legendre series in cos(u^, zeta^),
// and the Fourier transform in u keeps one Bessel product per degree:
//   Ghat(xi, zeta) = sqrt(2/pi) [ sum_l (2l+1) (-1)^l bl[l] P_l(cos g) R_l(a, b)
//                                 - bl[0] int_0^r0 r^{lambda+2} sinc(c r) dr ],
//   R_l(a, b) = int_0^r0 r^{lambda+2} j_l(a r) j_l(b r) dr,
// a = |zeta|/2, b = |xi - zeta/2|, c = |xi|, cos g = zeta^ . (xi - zeta/2)^.
// The mirror partner xi' = zeta - xi flips the sign of cos g, so in the
// symmetrised table entry Ghat(xi) + Ghat(zeta - xi) the odd degrees cancel
// exactly (P_l(-t) = (-1)^l P_l(t) holds bit for bit in the recurrence) and
// only the even ones are tabulated.

// spherical Bessel function j_l(x), x >= 0: power series below x = 1/2;
// Miller's downward recurrence up to x = l, normalised by the larger of the
// exact j_0 and j_1; the upward recurrence (stable there) above
__device__ double sph_bessel_j(int l, double x)
{
    if (x < 0.5) {
        double lead = 1.0;
        for (int i = 1; i <= l; ++i) lead *= x / (2.0 * i + 1.0);
        double term = 1.0, sum = 1.0;
        for (int k = 1; k < 30; ++k) {
            term *= -0.5 * x * x / (k * (2.0 * l + 2.0 * k + 1.0));
            sum += term;
            if (fabs(term) < 1e-17 * fabs(sum)) break;
        }
        return lead * sum;
    }
    double sx, cx;
    sincos(x, &sx, &cx);
    const double j0 = sx / x, j1 = sx / (x * x) - cx / x;
    if (l == 0) return j0;
    if (l == 1) return j1;
    if (x > l) {
        double jm = j0, jc = j1;
        for (int n = 1; n < l; ++n) {
            const double jn = (2.0 * n + 1.0) / x * jc - jm;
            jm = jc;
            jc = jn;
        }
        return jc;
    }
    const int top = l + 24 + (int)x;
    double jp = 0.0, jc = 1e-200, jl = 0.0, f0 = 1.0, f1 = 1.0;
    for (int n = top; n >= 1; --n) {  // j_{n-1} from j_n and j_{n+1}
        const double jm = (2.0 * n + 1.0) / x * jc - jp;
        jp = jc;
        jc = jm;
        if (n - 1 == l) jl = jc;
        if (n - 1 == 1) f1 = jc;
    }
    f0 = jc;
    return fabs(j0) > fabs(j1) ? jl * (j0 / f0) : jl * (j1 / f1);
}

__device__ double legendre_poly(int l, double t)
{
    double p0 = 1.0, p1 = t;
    if (l == 0) return 1.0;
    for (int n = 1; n < l; ++n) {
        const double p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// R_l(a, b) by composite Gauss-Legendre, the panels as in radial_bracket_quad
__device__ double aniso_radial(int l, double a, double b, double r0, double lam, const QuadRule &q)
{
    const int np = (int)ceil((a + b) * r0 / 3.0) + 2;
    const double hw = r0 / np;
    double total = 0.0;
    for (int p = 0; p < np; ++p) {
        const int nsub = (p == 0) ? 12 : 1;
        for (int sidx = 0; sidx < nsub; ++sidx) {
            double lo, hi;
            if (p == 0) {
                hi = hw * exp2(-(double)(nsub - 1 - sidx));
                lo = (sidx == 0) ? 0.0 : hw * exp2(-(double)(nsub - sidx));
            } else {
                lo = p * hw;
                hi = (p + 1) * hw;
            }
            const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int i = 0; i < kQuadNodes; ++i) {
                const double r = mid + half * q.x[i];
                total += half * q.w[i] * pow(r, lam + 2.0) * sph_bessel_j(l, a * r) * sph_bessel_j(l, b * r);
            }
        }
    }
    return total;
}

__device__ double radial_pair_quad(double a, double b, double r0, double lam, const QuadRule &q);

// int_0^r0 r^{lambda+2} sinc(c r) dr: closed forms at lambda = 0, 1, else quadrature
__device__ double loss_integral(double c, double r0, double lam, const QuadRule &q)
{
    if (lam == 0.0 || lam == 1.0) return sinc_moment(c, r0, (int)lam);
    return radial_pair_quad(c, 0.0, r0, lam, q);
}

// The tabulated integrals of an anisotropic handle: R_l(kk, bb) for the even
// degrees l = ls[s] of the slots s, and the loss integral of every |xi|^2
struct AnisoTables {
    const double *R;  // [nslot][nkk][nbb]
    const double *B;  // [nkk]
    int nslot, nkk, nbb;
    int ls[kMaxLeg / 2];
};

// Ghat (unsymmetrised) from the tables, even degrees only: the half of the
// weight that survives the symmetrisation
__device__ double ghat_aniso_tab(const Geom &g, const AnisoTables &t, long kk, long bb, long mm, long kd)
{
    if (kk == 0) return 0.0;
    const double cg = bb == 0 ? 0.0 : (double)kd / (sqrt((double)kk) * sqrt((double)bb));
    double gain = 0.0;
    for (int s = 0; s < t.nslot; ++s) {
        const int l = t.ls[s];
        if (l > 0 && bb == 0) continue;
        gain += (2.0 * l + 1.0) * g.bl[l] * legendre_poly(l, cg) * t.R[((size_t)s * t.nkk + kk) * t.nbb + bb];
    }
    return 0.79788456080286535588 * (gain - g.bl[0] * t.B[mm]);
}

// Ghat (unsymmetrised, every degree) computed directly: cs_weights_sample
__device__ double ghat_aniso_direct(const Geom &g, const QuadRule &q, long kk, long bb, long mm, long kd)
{
    if (kk == 0) return 0.0;
    const double a = 0.5 * g.dz * sqrt((double)kk), b = 0.5 * g.dz * sqrt((double)bb), c = g.dz * sqrt((double)mm);
    const double cg = bb == 0 ? 0.0 : (double)kd / (sqrt((double)kk) * sqrt((double)bb));
    double gain = 0.0;
    for (int l = 0; l < g.nleg; ++l) {
        if (g.bl[l] == 0.0 || (l > 0 && bb == 0)) continue;
        const double sgn = (l & 1) ? -1.0 : 1.0;
        gain += (2.0 * l + 1.0) * sgn * g.bl[l] * legendre_poly(l, cg) * aniso_radial(l, a, b, g.L, g.lambda, q);
    }
    return 0.79788456080286535588 * (gain - g.bl[0] * loss_integral(c, g.L, g.lambda, q));
}

__device__ void aniso_radii(int kp1, int kp2, int kp3, int mp1, int mp2, int mp3, long &kk, long &bb, long &mm,
                            long &kd)
{
    const long d1 = 2 * mp1 - kp1, d2 = 2 * mp2 - kp2, d3 = 2 * mp3 - kp3;
    kk = (long)kp1 * kp1 + (long)kp2 * kp2 + (long)kp3 * kp3;
    mm = (long)mp1 * mp1 + (long)mp2 * mp2 + (long)mp3 * mp3;
    bb = d1 * d1 + d2 * d2 + d3 * d3;
    kd = kp1 * d1 + kp2 * d2 + kp3 * d3;
}

__global__ void aniso_radial_kernel(Geom g, QuadRule q, AnisoTables t, double *__restrict__ R, double *__restrict__ B)
{
    const long long n = (long long)t.nslot * t.nkk * t.nbb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n + t.nkk;
         i += (long long)gridDim.x * blockDim.x) {
        if (i >= n) {  // the loss integrals
            const int mm = (int)(i - n);
            B[mm] = loss_integral(g.dz * sqrt((double)mm), g.L, g.lambda, q);
            continue;
        }
        const int s = (int)(i / ((long long)t.nkk * t.nbb));
        const int kk = (int)((i / t.nbb) % t.nkk), bb = (int)(i % t.nbb);
        const int l = t.ls[s];
        double v = 0.0;
        if (kk > 0 && !(l > 0 && bb == 0))
            v = aniso_radial(l, 0.5 * g.dz * sqrt((double)kk), 0.5 * g.dz * sqrt((double)bb), g.L, g.lambda, q);
        R[i] = v;
    }
}

template <typename T>
__global__ void build_table_kernel(Geom g, QuadRule q, const int *__restrict__ tile0, long long total,
                                   const int *__restrict__ emap, T *__restrict__ out, AnisoTables at)
{
    const long long tile = blockIdx.x;
    if (tile >= total) return;
    const int N = g.N, h = g.h;
    // pencil of this tile: largest P with tile0[P] <= tile
    int lo = 0, hi = N * N - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    const int P = lo;
    const int k1 = P / N, k2 = P % N;
    const int K1 = k1 + h, K2 = k2 + h;
    const int lo1 = max(0, K1 - N + 1), hi1 = min(N - 1, K1);
    const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
    const int v1 = hi1 - lo1 + 1, v2 = hi2 - lo2 + 1;
    const long long t = tile - tile0[P];
    const int nfull = (v1 / 2) * v2;
    int m1, m2;
    if (t < nfull) {
        m1 = lo1 + (int)(t / v2);
        m2 = lo2 + (int)(t % v2);
    } else {
        m1 = K1 / 2;
        m2 = lo2 + (int)(t - nfull);
    }
    const bool centre = (2 * m1 == K1) && (2 * m2 == K2);
    const int s1 = K1 - m1, s2 = K2 - m2;
    T *dst = out + tile * g.TSp;
    for (int p = threadIdx.x; p < g.TSp; p += blockDim.x) {
        const int e = emap[p];
        if (e < 0) {  // padding
            dst[p] = T(0);
            continue;
        }
        const int m3 = e >> 8, k3 = e & 255;
        const int s3 = k3 + h - m3;
        double w;
        if (g.nleg > 0) {
            long kk, bb, mm, kd;
            aniso_radii(k1 - h, k2 - h, k3 - h, m1 - h, m2 - h, m3 - h, kk, bb, mm, kd);
            w = ghat_aniso_tab(g, at, kk, bb, mm, kd);
            if (!centre) {
                aniso_radii(k1 - h, k2 - h, k3 - h, s1 - h, s2 - h, s3 - h, kk, bb, mm, kd);
                w += ghat_aniso_tab(g, at, kk, bb, mm, kd);
            }
        } else {
            w = ghat_centered(g, q, k1 - h, k2 - h, k3 - h, m1 - h, m2 - h, m3 - h);
            if (!centre) w += ghat_centered(g, q, k1 - h, k2 - h, k3 - h, s1 - h, s2 - h, s3 - h);
        }
        dst[p] = (T)w;
    }
}

// int_0^r0 r^{lambda+2} sinc(a r) sinc(b r) dr by composite Gauss-Legendre,
// the panels as in radial_bracket_quad (b = 0 gives the one-radius integral)
__device__ double radial_pair_quad(double a, double b, double r0, double lam, const QuadRule &q)
{
    const int np = (int)ceil((a + b) * r0 / 3.0) + 2;
    const double hw = r0 / np;
    double total = 0.0;
    for (int p = 0; p < np; ++p) {
        const int nsub = (p == 0) ? 12 : 1;
        for (int sidx = 0; sidx < nsub; ++sidx) {
            double lo, hi;
            if (p == 0) {
                hi = hw * exp2(-(double)(nsub - 1 - sidx));
                lo = (sidx == 0) ? 0.0 : hw * exp2(-(double)(nsub - sidx));
            } else {
                lo = p * hw;
                hi = (p + 1) * hw;
            }
            const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int i = 0; i < kQuadNodes; ++i) {
                const double r = mid + half * q.x[i];
                total += half * q.w[i] * pow(r, lam + 2.0) * (dsinc(a * r) * dsinc(b * r));
            }
        }
    }
    return total;
}

// A(kk, bb) for kk = 1 .. KK-1, bb = 0 .. BB-1 (row kk = 0 is never read: Ghat(xi, 0) = 0)
__global__ void radius_a_kernel(Geom g, QuadRule q, int KK, int BB, float *__restrict__ A)
{
    const long long n = (long long)KK * BB;
    const double dz = g.dz, r0 = g.L, lam = g.lambda;
    const double pref = 0.79788456080286535588;  // sqrt(2 / pi)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(i / BB), bb = (int)(i % BB);
        double v = 0.0;
        if (kk > 0) {
            const double a = 0.5 * dz * sqrt((double)kk), b = 0.5 * dz * sqrt((double)bb);
            if (lam == 0.0 || lam == 1.0) {
                const int il = (int)lam;
                if (bb == 0) {
                    v = sinc_moment(a, r0, il);
                } else {
                    // a^2 - b^2 = dz^2 (kk - bb) / 4 = dz^2 (m'.k' - |m'|^2), an integer multiple
                    const double qv = a + b;
                    const double pv = dz * dz * (0.25 * (double)(kk - bb)) / qv;
                    v = (cos_moment(pv, r0, il) - cos_moment(qv, r0, il)) / (2.0 * a * b);
                }
            } else {
                v = radial_pair_quad(a, b, r0, lam, q);
            }
        }
        A[i] = (float)(pref * v);
    }
}

// B(mm) for mm = 0 .. MM-1
__global__ void radius_b_kernel(Geom g, QuadRule q, int MM, float *__restrict__ B)
{
    const int mm = blockIdx.x * blockDim.x + threadIdx.x;
    if (mm >= MM) return;
    const double c = g.dz * sqrt((double)mm), r0 = g.L, lam = g.lambda;
    const double pref = 0.79788456080286535588;
    double v;
    if (lam == 0.0 || lam == 1.0)
        v = sinc_moment(mm == 0 ? 0.0 : c, r0, (int)lam);
    else
        v = radial_pair_quad(c, 0.0, r0, lam, q);
    B[mm] = (float)(pref * v);
}

__global__ void sample_kernel(Geom g, QuadRule q, const int *__restrict__ km, int n, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int *e = km + 6 * i;
    const int h = g.h;
    if (g.nleg > 0) {
        long kk, bb, mm, kd;
        aniso_radii(e[0] - h, e[1] - h, e[2] - h, e[3] - h, e[4] - h, e[5] - h, kk, bb, mm, kd);
        out[i] = ghat_aniso_direct(g, q, kk, bb, mm, kd);
        return;
    }
    out[i] = ghat_centered(g, q, e[0] - h, e[1] - h, e[2] - h, e[3] - h, e[4] - h, e[5] - h);
}

}  // namespace

long long count_tiles(int N, int *pencil_tile0)
{
    const int h = N / 2;
    long long total = 0;
    for (int k1 = 0; k1 < N; ++k1)
        for (int k2 = 0; k2 < N; ++k2) {
            const int K1 = k1 + h, K2 = k2 + h;
            const int v1 = (K1 < N - 1 ? K1 : N - 1) - (K1 - N + 1 > 0 ? K1 - N + 1 : 0) + 1;
            const int v2 = (K2 < N - 1 ? K2 : N - 1) - (K2 - N + 1 > 0 ? K2 - N + 1 : 0) + 1;
            if (pencil_tile0) pencil_tile0[k1 * N + k2] = (int)total;
            total += (long long)(v1 * v2 + 1) / 2;
        }
    if (pencil_tile0) pencil_tile0[N * N] = (int)total;
    return total;
}

void radius_dims(int N, int *KK, int *BB, int *MM)
{
    const int h = N / 2;
    *KK = 3 * h * h + 1;            // |k'|^2, k'_i in [-h, h-1]
    *BB = 3 * (N - 1) * (N - 1) + 1;  // |2m' - k'|^2, components in [-(N-1), N-1] for valid pairs
    *MM = 3 * h * h + 1;            // |m'|^2 and |k' - m'|^2
}

size_t radius_bytes(int N)
{
    const int K = strip_width(N);
    if (K == 0) return 0;
    int KK, BB, MM;
    radius_dims(N, &KK, &BB, &MM);
    const int TSp = strip_stride(N, K);
    return sizeof(float) * ((size_t)KK * BB + MM) + sizeof(int) * (size_t)TSp;
}

int build_radius_tables(Handle &hd, cudaStream_t s)
{
    const Geom &g = hd.g;
    if (g.layout != LAYOUT_STRIP) return set_error(CS_ENOTSUP, "radius tables serve the float strip kernel only");
    int KK, BB, MM;
    radius_dims(g.N, &KK, &BB, &MM);
    hd.rad_bb = BB;
    cudaError_t e = cudaMalloc(&hd.radA, sizeof(float) * (size_t)KK * BB);
    if (e == cudaSuccess) e = cudaMalloc(&hd.radB, sizeof(float) * (size_t)MM);
    if (e == cudaSuccess) e = cudaMalloc(&hd.emap, sizeof(int) * (size_t)g.TSp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_ENOMEM, "cudaMalloc of the radius tables failed");
    }
    std::vector<int> emap;
    tile_entry_map(g, emap);
    e = cudaMemcpyAsync(hd.emap, emap.data(), sizeof(int) * emap.size(), cudaMemcpyHostToDevice, s);
    const QuadRule q = make_rule();
    if (e == cudaSuccess) {
        const long long n = (long long)KK * BB;
        const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 65536);
        radius_a_kernel<<<blocks, 256, 0, s>>>(g, q, KK, BB, hd.radA);
        radius_b_kernel<<<(MM + 127) / 128, 128, 0, s>>>(g, q, MM, hd.radB);
        e = cudaGetLastError();
        if (e == cudaSuccess) note_kernels(s, 2);
    }
    // the host map behind the async copy must outlive it
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "radius table build");
    if (e2 != cudaSuccess) return cuda_error(e2, "radius table build");
    hd.rad_bytes = radius_bytes(g.N);
    return CS_OK;
}

int build_weights(Handle &hd, cudaStream_t s)
{
    const Geom &g = hd.g;
    std::vector<int> tile0(g.N * g.N + 1);
    hd.total_tiles = count_tiles(g.N, tile0.data());
    // heaviest pencils first, so the longest work items start earliest
    hd.order_host.resize(g.N * g.N);
    for (int i = 0; i < g.N * g.N; ++i) hd.order_host[i] = i;
    std::stable_sort(hd.order_host.begin(), hd.order_host.end(), [&](int x, int y) {
        return tile0[x + 1] - tile0[x] > tile0[y + 1] - tile0[y];
    });
    cudaError_t e = cudaMalloc(&hd.pencil_tile0, sizeof(int) * tile0.size());
    if (e == cudaSuccess) e = cudaMalloc(&hd.pencil_order, sizeof(int) * hd.order_host.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_ENOMEM, "cudaMalloc of the pencil index failed");
    }
    e = cudaMemcpyAsync(hd.pencil_tile0, tile0.data(), sizeof(int) * tile0.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hd.pencil_order, hd.order_host.data(), sizeof(int) * hd.order_host.size(),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "copy of the pencil index");
    // the host copies above are read asynchronously: keep tile0 alive until the stream passes
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "copy of the pencil index");
    if (!hd.has_table) return CS_OK;  // radius tables only
    hd.ghat_bytes = (size_t)hd.total_tiles * g.TSp * elem_bytes(hd.precision);
    e = cudaMalloc(&hd.ghat, hd.ghat_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_ENOMEM, "cudaMalloc of the weight table failed (" +
                                        std::to_string(hd.ghat_bytes) + " bytes)");
    }
    std::vector<int> emap;
    tile_entry_map(g, emap);
    int *demap = nullptr;
    e = cudaMalloc(&demap, sizeof(int) * emap.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_ENOMEM, "cudaMalloc of the tile entry map failed");
    }
    e = cudaMemcpyAsync(demap, emap.data(), sizeof(int) * emap.size(), cudaMemcpyHostToDevice, s);
    const QuadRule q = make_rule();
    // anisotropic b: the radial integrals of the even degrees and the loss
    // integrals, tabulated over the grid's integer squared radii first
    AnisoTables at{};
    double *aR = nullptr, *aB = nullptr;
    if (e == cudaSuccess && g.nleg > 0) {
        int KK, BB, MM;
        radius_dims(g.N, &KK, &BB, &MM);
        at.nkk = KK;
        at.nbb = BB;
        for (int l = 0; l < g.nleg; l += 2)
            if (l == 0 || g.bl[l] != 0.0) at.ls[at.nslot++] = l;
        e = cudaMalloc(&aR, sizeof(double) * (size_t)at.nslot * KK * BB);
        if (e == cudaSuccess) e = cudaMalloc(&aB, sizeof(double) * (size_t)KK);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(aR);
            cudaFree(demap);
            return set_error(CS_ENOMEM, "cudaMalloc of the anisotropic radial tables failed");
        }
        at.R = aR;
        at.B = aB;
        const long long n = (long long)at.nslot * KK * BB + KK;
        aniso_radial_kernel<<<(unsigned)std::min<long long>((n + 127) / 128, 1 << 20), 128, 0, s>>>(g, q, at, aR, aB);
        e = cudaGetLastError();
        if (e == cudaSuccess) note_kernels(s, 1);
    }
    if (e == cudaSuccess) {
        if (hd.precision == CS_FP32)
            build_table_kernel<float><<<(unsigned)hd.total_tiles, 128, 0, s>>>(g, q, hd.pencil_tile0, hd.total_tiles,
                                                                                demap, (float *)hd.ghat, at);
        else
            build_table_kernel<double><<<(unsigned)hd.total_tiles, 128, 0, s>>>(g, q, hd.pencil_tile0,
                                                                                 hd.total_tiles, demap,
                                                                                 (double *)hd.ghat, at);
        e = cudaGetLastError();
        if (e == cudaSuccess) note_kernels(s, 1);
    }
    // the map (and the host vector behind the async copy) must outlive the kernel
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(demap);
    cudaFree(aR);
    cudaFree(aB);
    if (e != cudaSuccess) return cuda_error(e, "weight table build");
    if (e2 != cudaSuccess) return cuda_error(e2, "weight table build");
    return CS_OK;
}

int sample_weights(Handle &hd, const int *km_host, int n, double *out_host)
{
    int *dkm = nullptr;
    double *dout = nullptr;
    cudaError_t e = cudaMalloc(&dkm, sizeof(int) * 6 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * (size_t)n);
    if (e != cudaSuccess) {
        cudaFree(dkm);
        return set_error(CS_ENOMEM, "cudaMalloc in cs_weights_sample failed");
    }
    e = cudaMemcpy(dkm, km_host, sizeof(int) * 6 * (size_t)n, cudaMemcpyHostToDevice);
    int rc = CS_OK;
    if (e == cudaSuccess) {
        const QuadRule q = make_rule();
        sample_kernel<<<(n + 127) / 128, 128>>>(hd.g, q, dkm, n, dout);
        e = cudaGetLastError();
        if (e == cudaSuccess) note_kernels(nullptr, 1);
        if (e == cudaSuccess) e = cudaMemcpy(out_host, dout, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) rc = cuda_error(e, "cs_weights_sample");
    cudaFree(dkm);
    cudaFree(dout);
    return rc;
}

}  // namespace cs
