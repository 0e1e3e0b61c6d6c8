/*
 * cs_oracle.c -- plain FP64 CPU oracle of the conservative spectral method for
 * the Boltzmann collision operator (J. R. Haack, "A hybrid OpenMP and MPI
 * implementation of a conservative spectral method for the Boltzmann
 * equation", arXiv:1301.4195).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Every routine is written out from the paper's definitions, in the paper's
 * order, without blocking or fusion.  The one liberty is that the
 * forward/inverse discrete transforms are evaluated axis by axis (the 3-D
 * sum of a product of per-axis exponentials factorises exactly).
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes):
 *   - beta = 1 (elastic collisions; the collision law of Sec. 2 gives the
 *     sinc form of G only for beta = 1).
 *   - p = beta|zeta|/2 - |xi - beta zeta/2|, q = beta|zeta|/2 + |xi - beta zeta/2|
 *     in the closed forms of Ghat (Sec. 2.2; p and q are not defined in the
 *     text; this choice reproduces both printed forms).
 *   - sinc(x) = sin(x)/x.
 *   - trapezoid weights omega_m = dzeta^3 on the uniform grid (no endpoint
 *     halving); likewise dv^3 in the integration matrix C.
 *   - a term is dropped iff an axis index k - m + N/2 leaves [0, N-1]
 *     (no periodic wrap, Sec. 3.2).
 *   - Qtilde is the real part of the inverse transform.
 *   - the projection is Q = Qt - C^T (C C^T)^{-1} C Qt (the printed sign and
 *     transpose in Sec. 3.3 are garbled; this is the unique minimiser).
 *   - r0 = L.
 *   - transport: see or_transport_rk2 below.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Grids, Sec. 3.1 ("meshpoints"): v_k = dv (k - N/2), zeta_k = dzeta (k - N/2),
 * dv = 2L/N, dzeta = pi/L, 0 <= k_j <= N-1.                                  */

double or_dv(int N, double L) { return 2.0 * L / N; }
double or_dzeta(double L) { return OR_PI / L; }

static int idx3(int N, int i, int j, int k) { return (i * N + j) * N + k; }

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on the
 * three-term Legendre recurrence.                                           */
void or_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double p0 = 0.0, p1 = 0.0, dp = 0.0;
        for (int it = 0; it < 200; ++it) {
            p0 = 1.0;
            p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double step = p0 / dp;
            z -= step;
            if (fabs(step) < 1e-16) break;
        }
        /* re-evaluate the derivative at the converged node */
        p0 = 1.0;
        p1 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
        }
        dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------------ */
/* Forward transform, Sec. 2.2 and 3.2:
 *   fhat(zeta_k) = (2 pi)^{-3/2} dv^3 sum_j f(v_j) exp(-i zeta_k . v_j).
 * Per axis zeta_k v_j = (2 pi / N)(k - N/2)(j - N/2), so the phase is taken
 * from the exact integer residue ((k - N/2)(j - N/2)) mod N.
 * f: [ncells][N^3] real.  fhat: [ncells][N^3][2] (re, im).                  */

static void twiddle(int N, int k, int j, int sign, double *c, double *s)
{
    long r = (long)(k - N / 2) * (long)(j - N / 2);
    r %= N;
    if (r < 0) r += N;
    double ang = 2.0 * OR_PI * (double)r / (double)N;
    *c = cos(ang);
    *s = sign * sin(ang);
}

/* One axis of a separable transform on complex data x[N^3][2], in place.
 * axis 0,1,2; sign -1 forward, +1 inverse.                                  */
static void axis_dft(int N, double *x, int axis, int sign)
{
    int M = N * N * N;
    double *y = (double *)calloc((size_t)2 * M, sizeof(double));
    for (int i1 = 0; i1 < N; ++i1)
        for (int i2 = 0; i2 < N; ++i2)
            for (int i3 = 0; i3 < N; ++i3) {
                int kout[3] = {i1, i2, i3};
                double re = 0.0, im = 0.0;
                for (int j = 0; j < N; ++j) {
                    int jin[3] = {i1, i2, i3};
                    jin[axis] = j;
                    double c, s;
                    twiddle(N, kout[axis], j, sign, &c, &s);
                    const double *xv = x + 2 * idx3(N, jin[0], jin[1], jin[2]);
                    re += xv[0] * c - xv[1] * s;
                    im += xv[0] * s + xv[1] * c;
                }
                y[2 * idx3(N, i1, i2, i3)] = re;
                y[2 * idx3(N, i1, i2, i3) + 1] = im;
            }
    memcpy(x, y, sizeof(double) * 2 * M);
    free(y);
}

int or_dft_forward(int N, double L, int ncells, const double *f, double *fhat)
{
    int M = N * N * N;
    double dv = or_dv(N, L);
    double cf = pow(2.0 * OR_PI, -1.5) * dv * dv * dv;
    for (int c = 0; c < ncells; ++c) {
        double *x = fhat + (size_t)2 * M * c;
        for (int j = 0; j < M; ++j) {
            x[2 * j] = f[(size_t)M * c + j];
            x[2 * j + 1] = 0.0;
        }
        axis_dft(N, x, 2, -1);
        axis_dft(N, x, 1, -1);
        axis_dft(N, x, 0, -1);
        for (int j = 0; j < 2 * M; ++j) x[j] *= cf;
    }
    return 0;
}

/* Inverse transform, Sec. 3.2:
 *   Qt(v_j) = Re[(2 pi)^{-3/2} dzeta^3 sum_k Qhat(zeta_k) exp(+i zeta_k . v_j)] / eps.
 * qimag (may be NULL) receives the imaginary part, a diagnostic only.       */
int or_dft_inverse(int N, double L, int ncells, const double *qhat, double eps,
                   double *qreal, double *qimag)
{
    int M = N * N * N;
    double dz = or_dzeta(L);
    double ci = pow(2.0 * OR_PI, -1.5) * dz * dz * dz / eps;
    double *x = (double *)malloc(sizeof(double) * 2 * M);
    for (int c = 0; c < ncells; ++c) {
        memcpy(x, qhat + (size_t)2 * M * c, sizeof(double) * 2 * M);
        axis_dft(N, x, 2, +1);
        axis_dft(N, x, 1, +1);
        axis_dft(N, x, 0, +1);
        for (int j = 0; j < M; ++j) {
            qreal[(size_t)M * c + j] = ci * x[2 * j];
            if (qimag) qimag[(size_t)M * c + j] = ci * x[2 * j + 1];
        }
    }
    free(x);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Convolution weights, Sec. 2.2 ("GHat_calc"), isotropic b = 1/(4 pi), d = 3:
 *   Ghat(xi, zeta) = sqrt(2/pi) * int_0^{r0} r^{lambda+2}
 *        [ sinc(r |zeta|/2) sinc(r |xi - zeta/2|) - sinc(r |xi|) ] dr.
 * With a = |zeta|/2, b = |xi - zeta/2|, c = |xi| the first term is
 *   (Phi(a - b) - Phi(a + b)) / (2 a b),  Phi(x) = int_0^{r0} r^lambda cos(x r) dr,
 * and the second is Psi(c),  Psi(x) = int_0^{r0} r^{lambda+2} sinc(x r) dr.
 * The closed forms printed for lambda = 1 and lambda = 0 are these Phi, Psi.
 * Removable singularities: a = 0 gives Ghat = 0 exactly (G(u, 0) = 0);
 * b = 0 gives first term Psi(a); x = 0 limits are the series' first terms.   */

/* Phi by its Taylor series: r0^{l+1} sum_n (-1)^n y^{2n} / ((2n)! (2n+l+1)), y = x r0 */
static double phi_series(double x, double r0, double lam)
{
    double y2 = (x * r0) * (x * r0);
    double term = 1.0, sum = 0.0; /* term = (-1)^n y^{2n} / (2n)! */
    for (int n = 0; n < 60; ++n) {
        double t = term / (2.0 * n + lam + 1.0);
        sum += t;
        if (fabs(t) < 1e-18 * fabs(sum) && n > 2) break;
        term *= -y2 / ((2.0 * n + 1.0) * (2.0 * n + 2.0));
    }
    return pow(r0, lam + 1.0) * sum;
}

/* Psi by its Taylor series: r0^{l+3} sum_n (-1)^n y^{2n} / ((2n+1)! (2n+l+3)) */
static double psi_series(double x, double r0, double lam)
{
    double y2 = (x * r0) * (x * r0);
    double term = 1.0, sum = 0.0; /* term = (-1)^n y^{2n} / (2n+1)! */
    for (int n = 0; n < 60; ++n) {
        double t = term / (2.0 * n + lam + 3.0);
        sum += t;
        if (fabs(t) < 1e-18 * fabs(sum) && n > 2) break;
        term *= -y2 / ((2.0 * n + 2.0) * (2.0 * n + 3.0));
    }
    return pow(r0, lam + 3.0) * sum;
}

/* closed forms (lambda = 0 or 1), Sec. 2.2 */
static double phi_closed(double x, double r0, int lam)
{
    double y = x * r0;
    if (fabs(y) < 0.5) return phi_series(x, r0, (double)lam);
    if (lam == 0) return sin(y) / x;
    return (y * sin(y) + cos(y) - 1.0) / (x * x);
}

static double psi_closed(double x, double r0, int lam)
{
    double y = x * r0;
    if (fabs(y) < 1.0) return psi_series(x, r0, (double)lam);
    if (lam == 0) return (sin(y) - y * cos(y)) / (x * x * x);
    return ((2.0 - y * y) * cos(y) + 2.0 * y * sin(y) - 2.0) / (x * x * x * x);
}

static double sinc(double x)
{
    if (fabs(x) < 1e-4) return 1.0 - x * x / 6.0 + x * x * x * x / 120.0;
    return sin(x) / x;
}

/* Radial integral of the bracket by composite Gauss-Legendre; the first panel
 * is graded geometrically toward r = 0 so that r^{lambda+2} with non-integer
 * lambda is resolved.  This is the general-lambda route (Sec. 2.2: "a
 * one-dimensional integral ... numerical quadrature") and, for integer
 * lambda, an independent check of the closed forms.                        */
double or_ghat_radial_quad(double a, double b, double c, double r0, double lam,
                           int npanel, int nodes)
{
    double *x = (double *)malloc(sizeof(double) * nodes);
    double *w = (double *)malloc(sizeof(double) * nodes);
    or_gauss_legendre(nodes, x, w);
    double h = r0 / npanel;
    double total = 0.0;
    for (int p = 0; p < npanel; ++p) {
        /* sub-intervals: panel 0 is split as [0,h/2^G],[h/2^G,h/2^{G-1}],...,[h/2,h] */
        int nsub = (p == 0) ? 12 : 1;
        for (int sidx = 0; sidx < nsub; ++sidx) {
            double lo, hi;
            if (p == 0) {
                hi = h / pow(2.0, (double)(nsub - 1 - sidx));
                lo = (sidx == 0) ? 0.0 : h / pow(2.0, (double)(nsub - sidx));
            } else {
                lo = p * h;
                hi = (p + 1) * h;
            }
            double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int i = 0; i < nodes; ++i) {
                double r = mid + half * x[i];
                double g = sinc(a * r) * sinc(b * r) - sinc(c * r);
                total += half * w[i] * pow(r, lam + 2.0) * g;
            }
        }
    }
    free(x);
    free(w);
    return total;
}

/* Ghat for grid indices k (zeta) and m (xi), each an int[3] in [0, N-1]. */
double or_ghat(int N, double L, double lambda, const int *k, const int *m)
{
    double dz = or_dzeta(L);
    double r0 = L;
    int kp[3], mp[3];
    long kk = 0, mm = 0, bb = 0;
    for (int d = 0; d < 3; ++d) {
        kp[d] = k[d] - N / 2;
        mp[d] = m[d] - N / 2;
        kk += (long)kp[d] * kp[d];
        mm += (long)mp[d] * mp[d];
        bb += (long)(2 * mp[d] - kp[d]) * (2 * mp[d] - kp[d]);
    }
    if (kk == 0) return 0.0; /* G(u, 0) = 0 */
    double a = 0.5 * dz * sqrt((double)kk);  /* beta |zeta| / 2 */
    double b = 0.5 * dz * sqrt((double)bb);  /* |xi - beta zeta / 2| */
    double c = dz * sqrt((double)mm);        /* |xi| */
    double pref = sqrt(2.0 / OR_PI);         /* 4 pi / (2 pi)^{3/2} */
    int lam = (int)lambda;
    if ((double)lam == lambda && (lam == 0 || lam == 1)) {
        double t1;
        if (bb == 0)
            t1 = psi_closed(a, r0, lam);
        else
            t1 = (phi_closed(a - b, r0, lam) - phi_closed(a + b, r0, lam)) / (2.0 * a * b);
        double t2 = psi_closed(c, r0, lam);
        return pref * (t1 - t2);
    }
    /* other lambda: radial quadrature */
    double fmax = a + b + c;
    int np = (int)ceil(fmax * r0 / 3.0) + 2;
    return pref * or_ghat_radial_quad(a, b, c, r0, lambda, np, 24);
}

/* ------------------------------------------------------------------------ */
/* Anisotropic scattering, Sec. 2 (B = |u|^lambda b(cos theta)) with the
 * weights of Sec. 2.2 left as integrals (the paper computes only b = 1/4pi;
 * Sec. 4.2 notes the same convolution serves anisotropic b).  The sphere
 * integral in G(u, zeta) is reduced with the Funk-Hecke theorem and the
 * angular part of the Fourier transform in u with the addition theorem of
 * Legendre polynomials:
 *   Ghat(xi, zeta) = sqrt(2/pi) [ sum_l (2l+1) (-1)^l beta_l P_l(cos g) R_l
 *                                 - beta_0 int_0^r0 r^{lambda+2} sinc(|xi| r) dr ],
 *   R_l = int_0^r0 r^{lambda+2} j_l(|zeta| r / 2) j_l(|xi - zeta/2| r) dr,
 * cos g the cosine between zeta and xi - zeta/2, j_l the spherical Bessel
 * functions and beta_l = int_{S^2} b(sigma . u^) P_l(sigma . u^) dsigma the
 * Legendre moments of b (beta_0 = 1 under the normalisation of Sec. 2;
 * b(t) = sum_l (2l+1) beta_l P_l(t) / 4pi).  beta_0 = 1 and no other moment
 * is the isotropic case.                                                    */

/* Legendre polynomial P_l(t) by the three-term recurrence */
static double legendre_p(int l, double t)
{
    double p0 = 1.0, p1 = t;
    if (l == 0) return p0;
    for (int n = 1; n < l; ++n) {
        double p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* spherical Bessel function j_l(x), x >= 0: the power series
 *   j_l(x) = x^l / (2l+1)!! sum_k (-x^2/2)^k / (k! (2l+3)(2l+5)...(2l+2k+1))
 * below x = l + 1, the upward recurrence j_{n+1} = (2n+1)/x j_n - j_{n-1}
 * from j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x above (stable there) */
static double sph_bessel(int l, double x)
{
    if (x < l + 1.0) {
        double lead = 1.0;
        for (int i = 1; i <= l; ++i) lead *= x / (2.0 * i + 1.0);
        double term = 1.0, sum = 1.0;
        for (int k = 1; k < 200; ++k) {
            term *= -0.5 * x * x / (k * (2.0 * l + 2.0 * k + 1.0));
            sum += term;
            if (fabs(term) < 1e-18 * fabs(sum)) break;
        }
        return lead * sum;
    }
    double j0 = sin(x) / x;
    if (l == 0) return j0;
    double j1 = sin(x) / (x * x) - cos(x) / x;
    for (int n = 1; n < l; ++n) {
        double j2 = (2.0 * n + 1.0) / x * j1 - j0;
        j0 = j1;
        j1 = j2;
    }
    return j1;
}

/* R_l(a, b) and, with l < 0, the loss integral int r^{lambda+2} j_0(a r) dr,
 * by composite Gauss-Legendre (first panel graded toward r = 0, as above) */
static double radial_l_quad(int l, double a, double b, double r0, double lam)
{
    int nodes = 24;
    double x[24], w[24];
    or_gauss_legendre(nodes, x, w);
    int npanel = (int)ceil((a + b) * r0 / 2.0) + 4;
    double h = r0 / npanel;
    double total = 0.0;
    for (int p = 0; p < npanel; ++p) {
        int nsub = (p == 0) ? 12 : 1;
        for (int sidx = 0; sidx < nsub; ++sidx) {
            double lo, hi;
            if (p == 0) {
                hi = h / pow(2.0, (double)(nsub - 1 - sidx));
                lo = (sidx == 0) ? 0.0 : h / pow(2.0, (double)(nsub - sidx));
            } else {
                lo = p * h;
                hi = (p + 1) * h;
            }
            double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int i = 0; i < nodes; ++i) {
                double r = mid + half * x[i];
                double g = (l < 0) ? sph_bessel(0, a * r) : sph_bessel(l, a * r) * sph_bessel(l, b * r);
                total += half * w[i] * pow(r, lam + 2.0) * g;
            }
        }
    }
    return total;
}

/* the weight of a collision model: isotropic (nl = 0) or given by the
 * Legendre moments of b.  rtab / btab, when set, hold the radial integrals
 * R_l(kk, bb) and the loss integrals of every integer squared radius of the
 * grid (each the same radial_l_quad value the direct route computes), so a
 * convolution evaluates each distinct integral once instead of once per pair. */
struct or_model {
    double lambda;
    int nl;
    const double *beta;
    const double *rtab; /* [nl][nkk][nbb] */
    const double *btab; /* [nkk] */
    int nkk, nbb;
};

static double aniso_weight(const struct or_model *md, int N, double L, const int *k, const int *m)
{
    double dz = or_dzeta(L);
    double r0 = L;
    long kk = 0, mm = 0, bb = 0, kd = 0;
    for (int d = 0; d < 3; ++d) {
        long kp = k[d] - N / 2, mp = m[d] - N / 2, dd = 2 * mp - kp;
        kk += kp * kp;
        mm += mp * mp;
        bb += dd * dd;
        kd += kp * dd; /* zeta . (2 xi - zeta) in units of dzeta^2 */
    }
    if (kk == 0) return 0.0; /* G(u, 0) = 0 */
    double a = 0.5 * dz * sqrt((double)kk); /* |zeta| / 2 */
    double b = 0.5 * dz * sqrt((double)bb); /* |xi - zeta / 2| */
    double c = dz * sqrt((double)mm);       /* |xi| */
    double cg = (bb == 0) ? 0.0 : (double)kd / (sqrt((double)kk) * sqrt((double)bb));
    double gain = 0.0;
    for (int l = 0; l < md->nl; ++l) {
        if (md->beta[l] == 0.0) continue;
        if (l > 0 && bb == 0) continue; /* j_l(0) = 0 for l > 0 */
        double sgn = (l % 2) ? -1.0 : 1.0;
        double R = md->rtab ? md->rtab[((size_t)l * md->nkk + kk) * md->nbb + bb]
                            : radial_l_quad(l, a, b, r0, md->lambda);
        gain += (2.0 * l + 1.0) * sgn * md->beta[l] * legendre_p(l, cg) * R;
    }
    double lossint = md->btab ? md->btab[mm] : radial_l_quad(-1, c, 0.0, r0, md->lambda);
    return sqrt(2.0 / OR_PI) * (gain - md->beta[0] * lossint);
}

double or_ghat_aniso(int N, double L, double lambda, int nl, const double *beta, const int *k, const int *m)
{
    struct or_model md = {lambda, nl, beta, NULL, NULL, 0, 0};
    return aniso_weight(&md, N, L, k, m);
}

/* the radial integrals of every integer squared radius of an N-grid:
 * |zeta|^2 / dzeta^2 = kk <= 3 (N/2)^2, |2 xi - zeta|^2 / dzeta^2 = bb <= 3 (N-1)^2,
 * |xi|^2 / dzeta^2 = mm <= 3 (N/2)^2 */
static void aniso_tables(struct or_model *md, int N, double L, double **rt, double **bt)
{
    double dz = or_dzeta(L);
    int nkk = 3 * (N / 2) * (N / 2) + 1, nbb = 3 * (N - 1) * (N - 1) + 1;
    double *R = (double *)calloc((size_t)md->nl * nkk * nbb, sizeof(double));
    double *B = (double *)calloc((size_t)nkk, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int row = 0; row < md->nl * nkk; ++row) {
        int l = row / nkk, kk = row % nkk;
        if (md->beta[l] == 0.0 || kk == 0) continue;
        double a = 0.5 * dz * sqrt((double)kk);
        for (int bb = 0; bb < nbb; ++bb) {
            if (l > 0 && bb == 0) continue;
            double b = 0.5 * dz * sqrt((double)bb);
            R[((size_t)l * nkk + kk) * nbb + bb] = radial_l_quad(l, a, b, L, md->lambda);
        }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int mm = 0; mm < nkk; ++mm) B[mm] = radial_l_quad(-1, dz * sqrt((double)mm), 0.0, L, md->lambda);
    md->rtab = R;
    md->btab = B;
    md->nkk = nkk;
    md->nbb = nbb;
    *rt = R;
    *bt = B;
}

static double model_ghat(const struct or_model *md, int N, double L, const int *k, const int *m)
{
    if (md->nl > 0) return aniso_weight(md, N, L, k, m);
    return or_ghat(N, L, md->lambda, k, m);
}

/* Same, always through the quadrature route (independent check). */
double or_ghat_quad(int N, double L, double lambda, const int *k, const int *m,
                    int nodes)
{
    double dz = or_dzeta(L);
    double zeta[3], xi[3], w[3];
    for (int d = 0; d < 3; ++d) {
        zeta[d] = dz * (k[d] - N / 2);
        xi[d] = dz * (m[d] - N / 2);
        w[d] = xi[d] - 0.5 * zeta[d];
    }
    double a = 0.5 * sqrt(zeta[0] * zeta[0] + zeta[1] * zeta[1] + zeta[2] * zeta[2]);
    double b = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double c = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    double r0 = L;
    int np = (int)ceil((a + b + c) * r0 / 3.0) + 2;
    return sqrt(2.0 / OR_PI) * or_ghat_radial_quad(a, b, c, r0, lambda, np, nodes);
}

/* Full table Ghat[k][m] for small N (N^6 doubles). */
int or_ghat_table(int N, double L, double lambda, double *out)
{
    int M = N * N * N;
    for (int kf = 0; kf < M; ++kf) {
        int k[3] = {kf / (N * N), (kf / N) % N, kf % N};
        for (int mf = 0; mf < M; ++mf) {
            int m[3] = {mf / (N * N), (mf / N) % N, mf % N};
            out[(size_t)kf * M + mf] = or_ghat(N, L, lambda, k, m);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Weighted convolution, Sec. 3.2:
 *   Qhat(zeta_k) = sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m) omega_m,
 * omega_m = dzeta^3, and fhat(zeta_k - xi_m) = 0 when the index k - m + N/2
 * leaves [0, N-1] on some axis.  m runs in lexicographic order.  The weight
 * of each (k, m) is evaluated once and applied to every cell.  OpenMP splits
 * the zeta_k outputs over threads, as in Sec. 4.1.                          */
/* One output zeta_k of the convolution for ncells cells: acc[2c], acc[2c+1]
 * receive the real and imaginary sums (before the factor omega).            */
static void convolve_one(int N, double L, const struct or_model *md, const int *k, int ncells,
                         const double *fhat, double *acc)
{
    int M = N * N * N;
    int h = N / 2;
    for (int c = 0; c < 2 * ncells; ++c) acc[c] = 0.0;
    for (int m1 = 0; m1 < N; ++m1) {
        int s1 = k[0] - m1 + h;
        if (s1 < 0 || s1 > N - 1) continue;
        for (int m2 = 0; m2 < N; ++m2) {
            int s2 = k[1] - m2 + h;
            if (s2 < 0 || s2 > N - 1) continue;
            for (int m3 = 0; m3 < N; ++m3) {
                int s3 = k[2] - m3 + h;
                if (s3 < 0 || s3 > N - 1) continue;
                int m[3] = {m1, m2, m3};
                double g = model_ghat(md, N, L, k, m);
                int im = idx3(N, m1, m2, m3), is = idx3(N, s1, s2, s3);
                for (int c = 0; c < ncells; ++c) {
                    const double *F = fhat + (size_t)2 * M * c;
                    double ar = F[2 * im], ai = F[2 * im + 1];
                    double br = F[2 * is], bi = F[2 * is + 1];
                    acc[2 * c] += g * (ar * br - ai * bi);
                    acc[2 * c + 1] += g * (ar * bi + ai * br);
                }
            }
        }
    }
}

static int convolve_model(int N, double L, const struct or_model *md, int ncells, const double *fhat,
                          double *qhat, int nthreads)
{
    int M = N * N * N;
    double dz = or_dzeta(L);
    double omega = dz * dz * dz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)ncells);
#pragma omp for schedule(dynamic, 4)
        for (int kf = 0; kf < M; ++kf) {
            int k[3] = {kf / (N * N), (kf / N) % N, kf % N};
            convolve_one(N, L, md, k, ncells, fhat, acc);
            for (int c = 0; c < ncells; ++c) {
                qhat[(size_t)2 * M * c + 2 * kf] = omega * acc[2 * c];
                qhat[(size_t)2 * M * c + 2 * kf + 1] = omega * acc[2 * c + 1];
            }
        }
        free(acc);
    }
    return 0;
}

int or_convolve(int N, double L, double lambda, int ncells, const double *fhat,
                double *qhat, int nthreads)
{
    struct or_model md = {lambda, 0, NULL, NULL, NULL, 0, 0};
    return convolve_model(N, L, &md, ncells, fhat, qhat, nthreads);
}

int or_convolve_b(int N, double L, double lambda, int nl, const double *beta, int ncells, const double *fhat,
                  double *qhat, int nthreads)
{
    struct or_model md = {lambda, nl, beta, NULL, NULL, 0, 0};
    double *rt, *bt;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    aniso_tables(&md, N, L, &rt, &bt);
    int rc = convolve_model(N, L, &md, ncells, fhat, qhat, nthreads);
    free(rt);
    free(bt);
    return rc;
}

/* The convolution at nk selected outputs kf[i] (flat indices) only, for
 * grids too large for the full sum: qhat [ncells][nk][2].  Each output is
 * the same sum as in or_convolve, bit for bit.                              */
int or_convolve_at(int N, double L, double lambda, int ncells, const double *fhat, int nk, const int *kf,
                   double *qhat, int nthreads)
{
    struct or_model md = {lambda, 0, NULL, NULL, NULL, 0, 0};
    double dz = or_dzeta(L);
    double omega = dz * dz * dz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)ncells);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < nk; ++i) {
            int k[3] = {kf[i] / (N * N), (kf[i] / N) % N, kf[i] % N};
            convolve_one(N, L, &md, k, ncells, fhat, acc);
            for (int c = 0; c < ncells; ++c) {
                qhat[(size_t)2 * nk * c + 2 * i] = omega * acc[2 * c];
                qhat[(size_t)2 * nk * c + 2 * i + 1] = omega * acc[2 * c + 1];
            }
        }
        free(acc);
    }
    return 0;
}

/* The rounding scale of the convolution (an error yardstick for a float
 * evaluation; not a step of the method): the same sum as Sec. 3.2 with every
 * term replaced by its magnitude,
 *   Shat_k = omega sum_m |Ghat(xi_m, zeta_k)| |fhat(xi_m)| |fhat(zeta_k - xi_m)|,
 * carried through the inverse transform of Sec. 3.2 as the bound
 *   S = (2 pi)^{-3/2} dzeta^3 sum_k Shat_k / eps  >=  max_j |Qt(v_j)|.
 * A float sum of these terms has an error of order u S (u the unit
 * roundoff), whatever |Qt| is: near equilibrium |Qt| << S.  S[c] per cell. */
int or_rounding_scale(int N, double L, double lambda, int ncells, const double *f, double eps, double *S,
                      int nthreads)
{
    int M = N * N * N;
    int h = N / 2;
    double dz = or_dzeta(L);
    double omega = dz * dz * dz;
    double *fh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    or_dft_forward(N, L, ncells, f, fh);
    for (int c = 0; c < ncells; ++c) S[c] = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int c = 0; c < ncells; ++c) {
        const double *F = fh + (size_t)2 * M * c;
        double total = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total)
        for (int kf = 0; kf < M; ++kf) {
            int k[3] = {kf / (N * N), (kf / N) % N, kf % N};
            double acc = 0.0;
            for (int m1 = 0; m1 < N; ++m1) {
                int s1 = k[0] - m1 + h;
                if (s1 < 0 || s1 > N - 1) continue;
                for (int m2 = 0; m2 < N; ++m2) {
                    int s2 = k[1] - m2 + h;
                    if (s2 < 0 || s2 > N - 1) continue;
                    for (int m3 = 0; m3 < N; ++m3) {
                        int s3 = k[2] - m3 + h;
                        if (s3 < 0 || s3 > N - 1) continue;
                        int m[3] = {m1, m2, m3};
                        int im = idx3(N, m1, m2, m3), is = idx3(N, s1, s2, s3);
                        double a = hypot(F[2 * im], F[2 * im + 1]);
                        double b = hypot(F[2 * is], F[2 * is + 1]);
                        acc += fabs(or_ghat(N, L, lambda, k, m)) * a * b;
                    }
                }
            }
            total += omega * acc;
        }
        S[c] = pow(2.0 * OR_PI, -1.5) * omega * total / eps;
    }
    free(fh);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Moments and conservation, Sec. 2 ("moments") and Sec. 3.3.
 * Integration matrix C (5 x M): rows dv^3 * (1, v^1, v^2, v^3, |v|^2).      */
static void c_row(int N, double L, int j, double *row)
{
    double dv = or_dv(N, L);
    double w = dv * dv * dv;
    double v1 = dv * (j / (N * N) - N / 2);
    double v2 = dv * ((j / N) % N - N / 2);
    double v3 = dv * (j % N - N / 2);
    row[0] = w;
    row[1] = w * v1;
    row[2] = w * v2;
    row[3] = w * v3;
    row[4] = w * (v1 * v1 + v2 * v2 + v3 * v3);
}

int or_moments(int N, double L, int ncells, const double *f, double *out)
{
    int M = N * N * N;
    for (int c = 0; c < ncells; ++c) {
        double s[5] = {0, 0, 0, 0, 0};
        for (int j = 0; j < M; ++j) {
            double row[5];
            c_row(N, L, j, row);
            for (int i = 0; i < 5; ++i) s[i] += row[i] * f[(size_t)M * c + j];
        }
        for (int i = 0; i < 5; ++i) out[5 * c + i] = s[i];
    }
    return 0;
}

/* C C^T, 5 x 5 */
int or_cct(int N, double L, double *A)
{
    int M = N * N * N;
    for (int i = 0; i < 25; ++i) A[i] = 0.0;
    for (int j = 0; j < M; ++j) {
        double row[5];
        c_row(N, L, j, row);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) A[5 * a + b] += row[a] * row[b];
    }
    return 0;
}

/* Solve A y = r for symmetric positive definite 5x5 A by Cholesky. */
static void chol_solve5(const double *A, const double *r, double *y)
{
    double Lm[25] = {0};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[5 * i + j];
            for (int k = 0; k < j; ++k) s -= Lm[5 * i + k] * Lm[5 * j + k];
            if (i == j)
                Lm[5 * i + i] = sqrt(s);
            else
                Lm[5 * i + j] = s / Lm[5 * j + j];
        }
    double z[5];
    for (int i = 0; i < 5; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= Lm[5 * i + k] * z[k];
        z[i] = s / Lm[5 * i + i];
    }
    for (int i = 4; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < 5; ++k) s -= Lm[5 * k + i] * y[k];
        y[i] = s / Lm[5 * i + i];
    }
}

/* Projection P_N, Sec. 3.3: Q = Qt - C^T (C C^T)^{-1} C Qt, in place. */
int or_conserve(int N, double L, int ncells, double *Q)
{
    int M = N * N * N;
    double A[25];
    or_cct(N, L, A);
    for (int c = 0; c < ncells; ++c) {
        double *q = Q + (size_t)M * c;
        double mom[5] = {0, 0, 0, 0, 0}, y[5];
        for (int j = 0; j < M; ++j) {
            double row[5];
            c_row(N, L, j, row);
            for (int i = 0; i < 5; ++i) mom[i] += row[i] * q[j];
        }
        chol_solve5(A, mom, y);
        for (int j = 0; j < M; ++j) {
            double row[5];
            c_row(N, L, j, row);
            double corr = 0.0;
            for (int i = 0; i < 5; ++i) corr += row[i] * y[i];
            q[j] -= corr;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The whole collision evaluation: forward transform, weighted convolution,
 * inverse transform (real part, / eps) and, if conserve != 0, the projection. */
static int collide_model(int N, double L, const struct or_model *md, int ncells, const double *f,
                         double eps, double *Q, int conserve, int nthreads)
{
    int M = N * N * N;
    double *fh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    double *qh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    or_dft_forward(N, L, ncells, f, fh);
    convolve_model(N, L, md, ncells, fh, qh, nthreads);
    or_dft_inverse(N, L, ncells, qh, eps, Q, NULL);
    if (conserve) or_conserve(N, L, ncells, Q);
    free(fh);
    free(qh);
    return 0;
}

int or_collide(int N, double L, double lambda, int ncells, const double *f,
               double eps, double *Q, int conserve, int nthreads)
{
    struct or_model md = {lambda, 0, NULL, NULL, NULL, 0, 0};
    return collide_model(N, L, &md, ncells, f, eps, Q, conserve, nthreads);
}

/* the collision evaluation with an anisotropic b (Legendre moments beta) */
int or_collide_b(int N, double L, double lambda, int nl, const double *beta, int ncells, const double *f,
                 double eps, double *Q, int conserve, int nthreads)
{
    struct or_model md = {lambda, nl, beta, NULL, NULL, 0, 0};
    double *rt, *bt;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    aniso_tables(&md, N, L, &rt, &bt);
    int rc = collide_model(N, L, &md, ncells, f, eps, Q, conserve, nthreads);
    free(rt);
    free(bt);
    return rc;
}

/* Space-homogeneous second-order Runge-Kutta (Heun), Sec. 3.1, on
 *   d f / dt = P_N Qt(f) / eps.                                               */
int or_rk2_homogeneous(int N, double L, double lambda, int ncells, double *f,
                       double dt, int nsteps, double eps, int conserve, int nthreads)
{
    size_t n = (size_t)N * N * N * ncells;
    double *q = (double *)malloc(sizeof(double) * n);
    double *f1 = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < nsteps; ++s) {
        or_collide(N, L, lambda, ncells, f, eps, q, conserve, nthreads);
        for (size_t i = 0; i < n; ++i) f1[i] = f[i] + dt * q[i];
        or_collide(N, L, lambda, ncells, f1, eps, q, conserve, nthreads);
        for (size_t i = 0; i < n; ++i) f[i] = 0.5 * (f[i] + f1[i] + dt * q[i]);
    }
    free(q);
    free(f1);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Transport, Sec. 3.4, 1-D in x on cells of width dx_j (wall face at x = 0,
 * cell j spans [sum_{i<j} dx_i, sum_{i<=j} dx_i], centre x_j).
 *   d f_j / dt = -(F_{j+1/2} - F_{j-1/2}) / dx_j,
 *   F_{j+1/2} = v1 (f_j + dx_j/2 s_j)          if v1 >= 0,
 *             = v1 (f_{j+1} - dx_{j+1}/2 s_{j+1}) otherwise,
 *   s_j = minmod((f_{j+1}-f_j)/(x_{j+1}-x_j), (f_j-f_{j-1})/(x_j-x_{j-1}),
 *                (f_{j+1}-f_{j-1})/(x_{j+1}-x_{j-1})).
 * Boundaries (readings):
 *   wall (left): the ghost f_{-1} is the linear extrapolation of f_0, f_1,
 *     so s_0 is the one-sided slope; for v1 > 0 the face flux is the diffuse
 *     reflection v1 sigma_w M_w(v), M_w = (2 pi T_w)^{-3/2}
 *     exp(-|v - V_w|^2 / (2 T_w)), with sigma_w chosen so the discrete
 *     incoming flux equals the discrete outgoing flux
 *     sum_{v1<0} |v1| (f_0 - dx_0/2 s_0) (Sec. 2.1, "BC");
 *   far end (right): two ghost cells of width dx_{n-1} hold f_far for
 *     v1 < 0 (the far-field gas) and f_{n-1} for v1 >= 0 (zero gradient).
 * One call advances dt with Heun's second-order Runge-Kutta (Sec. 3.1).      */

static double minmod3(double a, double b, double c)
{
    if (a > 0 && b > 0 && c > 0) return fmin(a, fmin(b, c));
    if (a < 0 && b < 0 && c < 0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* rhs = -(F_{j+1/2} - F_{j-1/2}) / dx_j for the cells first .. first+ncl-1
 * of a grid of nc cells (widths dx[0..nc-1]), read from a window fw that
 * holds the cells first-2 .. first+ncl+1 (window cell i = grid cell
 * first - 2 + i).  Window cells outside 0..nc-1 are never read: the column
 * below starts out NaN everywhere and only the window is copied into it, so
 * a read of anything else would show up as NaN in rhs.  The whole grid is
 * the case first = 0, ncl = nc.                                             */
static void transport_rhs_window(int N, double L, int nc, int first, int ncl, const double *fw,
                                 const double *dx, double Tw, const double *Vw, const double *ffar,
                                 double *rhs)
{
    int M = N * N * N;
    double dv = or_dv(N, L);
    double w3 = dv * dv * dv;
    /* cell centres, with two ghosts on the right and one on the left */
    double *x = (double *)malloc(sizeof(double) * (nc + 3)); /* x[j+1] = x_j, j=-1..nc+1 */
    double edge = 0.0;
    for (int j = 0; j < nc; ++j) {
        x[j + 1] = edge + 0.5 * dx[j];
        edge += dx[j];
    }
    x[0] = x[1] - dx[0];
    x[nc + 1] = x[nc] + dx[nc - 1];
    x[nc + 2] = x[nc + 1] + dx[nc - 1];
    double *fx = (double *)malloc(sizeof(double) * (nc + 3));
    double *slope = (double *)malloc(sizeof(double) * (nc + 2)); /* slope[j+1], j=-1..nc */
    double *face = (double *)malloc(sizeof(double) * (nc + 1));  /* F_{j-1/2}, j=0..nc */
    int lo = first - 2 < 0 ? 0 : first - 2;                      /* grid cells in the window */
    int hi = first + ncl + 1 > nc - 1 ? nc - 1 : first + ncl + 1;
#define FW(c, j) fw[(size_t)M * ((c) - first + 2) + (j)]

    /* wall: outgoing flux of the reconstructed face values, and the
     * discrete flux of M_w over v1 > 0 (needed only where the wall face
     * F_{-1/2} is one of this window's faces)                                 */
    double sigma_w = 0.0;
    if (first == 0) {
        double out_flux = 0.0, mw_flux = 0.0;
        for (int j = 0; j < M; ++j) {
            double v1 = dv * (j / (N * N) - N / 2);
            double v2 = dv * ((j / N) % N - N / 2);
            double v3 = dv * (j % N - N / 2);
            if (v1 < 0) {
                double f0 = FW(0, j), f1 = FW(1, j);
                double s0 = (f1 - f0) / (x[2] - x[1]);
                out_flux += -v1 * (f0 - 0.5 * dx[0] * s0) * w3;
            } else if (v1 > 0) {
                double e = (v1 - Vw[0]) * (v1 - Vw[0]) + (v2 - Vw[1]) * (v2 - Vw[1]) +
                           (v3 - Vw[2]) * (v3 - Vw[2]);
                double mw = pow(2.0 * OR_PI * Tw, -1.5) * exp(-e / (2.0 * Tw));
                mw_flux += v1 * mw * w3;
            }
        }
        sigma_w = out_flux / mw_flux;
    }

    for (int j = 0; j < M; ++j) {
        double v1 = dv * (j / (N * N) - N / 2);
        double v2 = dv * ((j / N) % N - N / 2);
        double v3 = dv * (j % N - N / 2);
        /* gather the column f_c(v) of the window's cells, with ghosts */
        for (int c = -1; c <= nc + 1; ++c) fx[c + 1] = NAN;
        for (int c = lo; c <= hi; ++c) fx[c + 1] = FW(c, j);
        fx[0] = 0.0; /* the left ghost only enters through s_0 below */
        if (first + ncl + 1 >= nc) { /* the far end is in the window */
            double gr = (v1 < 0) ? ffar[j] : fx[nc];
            fx[nc + 1] = gr;
            fx[nc + 2] = gr;
        }
        /* slopes for cells first-1 .. first+ncl (index c+1); cell -1 is never
         * used.  With f_{-1} the linear extrapolation of f_0, f_1 all three
         * minmod arguments of cell 0 equal the one-sided slope, taken directly. */
        for (int c = first - 1; c <= first + ncl; ++c) {
            int i = c + 1;
            if (c < 0) {
                slope[i] = 0.0;
            } else if (c == 0) {
                slope[i] = (fx[2] - fx[1]) / (x[2] - x[1]);
            } else {
                double a = (fx[i + 1] - fx[i]) / (x[i + 1] - x[i]);
                double b = (fx[i] - fx[i - 1]) / (x[i] - x[i - 1]);
                double cc = (fx[i + 1] - fx[i - 1]) / (x[i + 1] - x[i - 1]);
                slope[i] = minmod3(a, b, cc);
            }
        }
        /* faces c - 1/2 for c = first .. first+ncl */
        for (int c = first; c <= first + ncl; ++c) {
            double F;
            if (c == 0) {
                if (v1 > 0) {
                    double e = (v1 - Vw[0]) * (v1 - Vw[0]) + (v2 - Vw[1]) * (v2 - Vw[1]) +
                               (v3 - Vw[2]) * (v3 - Vw[2]);
                    double mw = pow(2.0 * OR_PI * Tw, -1.5) * exp(-e / (2.0 * Tw));
                    F = v1 * sigma_w * mw;
                } else {
                    F = v1 * (fx[1] - 0.5 * dx[0] * slope[1]);
                }
            } else {
                /* face between cell c-1 (left) and cell c (right) */
                double dxl = dx[c - 1];
                double dxr = (c < nc) ? dx[c] : dx[nc - 1];
                if (v1 >= 0)
                    F = v1 * (fx[c] + 0.5 * dxl * slope[c]);
                else
                    F = v1 * (fx[c + 1] - 0.5 * dxr * slope[c + 1]);
            }
            face[c] = F;
        }
        for (int c = first; c < first + ncl; ++c)
            rhs[(size_t)M * (c - first) + j] = -(face[c + 1] - face[c]) / dx[c];
    }
#undef FW
    free(x);
    free(fx);
    free(slope);
    free(face);
}

/* the whole grid: f [nc][M] placed in a window with two empty cells per side */
static void transport_rhs(int N, double L, int nc, const double *f, const double *dx,
                          double Tw, const double *Vw, const double *ffar, double *rhs)
{
    size_t M = (size_t)N * N * N;
    double *fw = (double *)malloc(sizeof(double) * M * (nc + 4));
    for (size_t i = 0; i < M * 2; ++i) fw[i] = NAN;
    memcpy(fw + 2 * M, f, sizeof(double) * M * nc);
    for (size_t i = 0; i < M * 2; ++i) fw[M * (nc + 2) + i] = NAN;
    transport_rhs_window(N, L, nc, 0, nc, fw, dx, Tw, Vw, ffar, rhs);
    free(fw);
}

/* The right-hand side of one shard, exposed for the sharded-transport tests:
 * rhs [ncl][M] for cells first .. first+ncl-1 from the window fw [ncl+4][M]. */
int or_transport_rhs_window(int N, double L, int nc, int first, int ncl, const double *fw,
                            const double *dx, double Tw, const double *Vw, const double *ffar,
                            double *rhs)
{
    if (first < 0 || ncl < 1 || first + ncl > nc || nc < 2) return -1;
    transport_rhs_window(N, L, nc, first, ncl, fw, dx, Tw, Vw, ffar, rhs);
    return 0;
}

int or_transport_rk2(int N, double L, int nc, double *f, const double *dx, double Tw,
                     const double *Vw, const double *ffar, double dt)
{
    size_t n = (size_t)N * N * N * nc;
    double *r = (double *)malloc(sizeof(double) * n);
    double *f1 = (double *)malloc(sizeof(double) * n);
    transport_rhs(N, L, nc, f, dx, Tw, Vw, ffar, r);
    for (size_t i = 0; i < n; ++i) f1[i] = f[i] + dt * r[i];
    transport_rhs(N, L, nc, f1, dx, Tw, Vw, ffar, r);
    for (size_t i = 0; i < n; ++i) f[i] = 0.5 * (f[i] + f1[i] + dt * r[i]);
    free(r);
    free(f1);
    return 0;
}

/* The sign-resolved wall flux used above, exposed for tests:
 * out[0] = outgoing flux, out[1] = sigma_w.                                 */
int or_wall_flux(int N, double L, int nc, const double *f, const double *dx, double Tw,
                 const double *Vw, double *out)
{
    int M = N * N * N;
    double dv = or_dv(N, L), w3 = dv * dv * dv;
    double x0 = 0.5 * dx[0], x1 = dx[0] + 0.5 * dx[1];
    double out_flux = 0.0, mw_flux = 0.0;
    (void)nc;
    for (int j = 0; j < M; ++j) {
        double v1 = dv * (j / (N * N) - N / 2);
        double v2 = dv * ((j / N) % N - N / 2);
        double v3 = dv * (j % N - N / 2);
        if (v1 < 0) {
            double f0 = f[j], f1 = f[(size_t)M + j];
            double s0 = (f1 - f0) / (x1 - x0);
            out_flux += -v1 * (f0 - 0.5 * dx[0] * s0) * w3;
        } else if (v1 > 0) {
            double e = (v1 - Vw[0]) * (v1 - Vw[0]) + (v2 - Vw[1]) * (v2 - Vw[1]) +
                       (v3 - Vw[2]) * (v3 - Vw[2]);
            mw_flux += v1 * pow(2.0 * OR_PI * Tw, -1.5) * exp(-e / (2.0 * Tw)) * w3;
        }
    }
    out[0] = out_flux;
    out[1] = out_flux / mw_flux;
    return 0;
}

/* Strang splitting, Sec. 3.1: transport dt/2, collision dt (Heun on
 * P_N Qt / eps), transport dt/2.                                            */
int or_strang_step(int N, double L, double lambda, int nc, double *f, const double *dx,
                   double Tw, const double *Vw, const double *ffar, double dt,
                   double eps, int nthreads)
{
    or_transport_rk2(N, L, nc, f, dx, Tw, Vw, ffar, 0.5 * dt);
    or_rk2_homogeneous(N, L, lambda, nc, f, dt, 1, eps, 1, nthreads);
    or_transport_rk2(N, L, nc, f, dx, Tw, Vw, ffar, 0.5 * dt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Transport in two space dimensions (the extension Sec. 3.4 says the ideas
 * carry to): cells (i, j), i = 0..nx-1 across the wall-normal direction x
 * with widths dx_i and the boundaries of the 1-D problem above, j = 0..ny-1
 * across a periodic direction y with uniform width dy.  State f[i][j][v]
 * (cell index i ny + j).  The semi-discrete scheme adds the two directions'
 * flux differences (no splitting between x and y):
 *   d f_ij / dt = -(F_{i+1/2,j} - F_{i-1/2,j}) / dx_i - (H_{i,j+1/2} - H_{i,j-1/2}) / dy,
 * F the x-flux of row j exactly as in 1-D (wall, far end, non-uniform grid),
 *   H_{j+1/2} = v2 (f_j + dy/2 s_j)           (v2 >= 0)
 *             = v2 (f_{j+1} - dy/2 s_{j+1})   (v2 <  0),
 * s_j = minmod of the forward, backward and central quotients in y, indices
 * taken modulo ny.                                                           */
static void transport_rhs_2d(int N, double L, int nx, int ny, const double *f, const double *dx,
                             double dy, double Tw, const double *Vw, const double *ffar, double *rhs)
{
    size_t M = (size_t)N * N * N;
    double dv = or_dv(N, L);
    double *row = (double *)malloc(sizeof(double) * M * nx);
    double *rr = (double *)malloc(sizeof(double) * M * nx);
    /* x: the 1-D right-hand side of every row */
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i)
            memcpy(row + M * i, f + M * ((size_t)i * ny + j), sizeof(double) * M);
        transport_rhs(N, L, nx, row, dx, Tw, Vw, ffar, rr);
        for (int i = 0; i < nx; ++i)
            memcpy(rhs + M * ((size_t)i * ny + j), rr + M * i, sizeof(double) * M);
    }
    /* y: periodic second-order upwind */
    for (int i = 0; i < nx; ++i) {
        for (size_t v = 0; v < M; ++v) {
            double v2 = dv * ((int)((v / N) % N) - N / 2);
            for (int j = 0; j < ny; ++j) {
#define FY(jj) f[M * ((size_t)i * ny + (size_t)((((jj) % ny) + ny) % ny)) + v]
#define SLOPE(jj) minmod3((FY((jj) + 1) - FY(jj)) / dy, (FY(jj) - FY((jj) - 1)) / dy, \
                          (FY((jj) + 1) - FY((jj) - 1)) / (2.0 * dy))
                double hp, hm; /* H_{j+1/2}, H_{j-1/2} */
                if (v2 >= 0) {
                    hp = v2 * (FY(j) + 0.5 * dy * SLOPE(j));
                    hm = v2 * (FY(j - 1) + 0.5 * dy * SLOPE(j - 1));
                } else {
                    hp = v2 * (FY(j + 1) - 0.5 * dy * SLOPE(j + 1));
                    hm = v2 * (FY(j) - 0.5 * dy * SLOPE(j));
                }
#undef SLOPE
#undef FY
                rhs[M * ((size_t)i * ny + j) + v] -= (hp - hm) / dy;
            }
        }
    }
    free(row);
    free(rr);
}

int or_transport2d_rhs(int N, double L, int nx, int ny, const double *f, const double *dx, double dy,
                       double Tw, const double *Vw, const double *ffar, double *rhs)
{
    if (nx < 2 || ny < 1 || !(dy > 0)) return -1;
    transport_rhs_2d(N, L, nx, ny, f, dx, dy, Tw, Vw, ffar, rhs);
    return 0;
}

/* one Heun step of length dt of the 2-D transport */
int or_transport2d_rk2(int N, double L, int nx, int ny, double *f, const double *dx, double dy,
                       double Tw, const double *Vw, const double *ffar, double dt)
{
    size_t n = (size_t)N * N * N * nx * ny;
    double *r = (double *)malloc(sizeof(double) * n);
    double *f1 = (double *)malloc(sizeof(double) * n);
    transport_rhs_2d(N, L, nx, ny, f, dx, dy, Tw, Vw, ffar, r);
    for (size_t i = 0; i < n; ++i) f1[i] = f[i] + dt * r[i];
    transport_rhs_2d(N, L, nx, ny, f1, dx, dy, Tw, Vw, ffar, r);
    for (size_t i = 0; i < n; ++i) f[i] = 0.5 * (f[i] + f1[i] + dt * r[i]);
    free(r);
    free(f1);
    return 0;
}

/* Strang step T(dt/2) C(dt) T(dt/2) with the 2-D transport */
int or_strang_step2d(int N, double L, double lambda, int nx, int ny, double *f, const double *dx,
                     double dy, double Tw, const double *Vw, const double *ffar, double dt, double eps,
                     int nthreads)
{
    or_transport2d_rk2(N, L, nx, ny, f, dx, dy, Tw, Vw, ffar, 0.5 * dt);
    or_rk2_homogeneous(N, L, lambda, nx * ny, f, dt, 1, eps, 1, nthreads);
    or_transport2d_rk2(N, L, nx, ny, f, dx, dy, Tw, Vw, ffar, 0.5 * dt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Transport in three space dimensions (Sec. 3.4: the scheme carries over to
 * higher dimensions): x is the wall direction of the 1-D problem, y and z are
 * periodic with uniform cells dy, dz.  Cell (i, j, l) is stored at
 * ((i ny + j) nz + l) N^3.  The semi-discrete scheme adds the three
 * directions' flux differences (no splitting):
 *   d f/dt = -(F_{i+1/2} - F_{i-1/2})/dx_i - (H_{j+1/2} - H_{j-1/2})/dy
 *            - (K_{l+1/2} - K_{l-1/2})/dz,
 * F the 1-D flux on each x-row, H and K the second-order upwind fluxes with
 * velocity components v2 and v3 and the three-argument minmod slope.         */
static void periodic_rhs(size_t M, int n, double h, double vel, const double *col, double *r)
{
    /* col[j] for j = 0 .. n-1 of one periodic line at one velocity; r[j] -= (P_{j+1/2} - P_{j-1/2}) / h */
    for (int j = 0; j < n; ++j) {
#define FP(jj) col[(((jj) % n) + n) % n]
#define SLP(jj) minmod3((FP((jj) + 1) - FP(jj)) / h, (FP(jj) - FP((jj) - 1)) / h, \
                        (FP((jj) + 1) - FP((jj) - 1)) / (2.0 * h))
        double pp, pm; /* P_{j+1/2}, P_{j-1/2} */
        if (vel >= 0) {
            pp = vel * (FP(j) + 0.5 * h * SLP(j));
            pm = vel * (FP(j - 1) + 0.5 * h * SLP(j - 1));
        } else {
            pp = vel * (FP(j + 1) - 0.5 * h * SLP(j + 1));
            pm = vel * (FP(j) - 0.5 * h * SLP(j));
        }
#undef SLP
#undef FP
        r[j] -= (pp - pm) / h;
    }
    (void)M;
}

static void transport_rhs_3d(int N, double L, int nx, int ny, int nz, const double *f, const double *dx,
                             double dy, double dzs, double Tw, const double *Vw, const double *ffar, double *rhs)
{
    size_t M = (size_t)N * N * N;
    double dv = or_dv(N, L);
    int nl = ny > nz ? ny : nz;
    double *row = (double *)malloc(sizeof(double) * M * nx);
    double *rr = (double *)malloc(sizeof(double) * M * nx);
    double *col = (double *)malloc(sizeof(double) * nl);
    double *rc = (double *)malloc(sizeof(double) * nl);
#define IDX(i, j, l) (M * (((size_t)(i) * ny + (j)) * nz + (l)))
    /* x: the 1-D right-hand side of every (j, l) row */
    for (int j = 0; j < ny; ++j)
        for (int l = 0; l < nz; ++l) {
            for (int i = 0; i < nx; ++i) memcpy(row + M * i, f + IDX(i, j, l), sizeof(double) * M);
            transport_rhs(N, L, nx, row, dx, Tw, Vw, ffar, rr);
            for (int i = 0; i < nx; ++i) memcpy(rhs + IDX(i, j, l), rr + M * i, sizeof(double) * M);
        }
    for (size_t v = 0; v < M; ++v) {
        double v2 = dv * ((int)((v / N) % N) - N / 2);
        double v3 = dv * ((int)(v % N) - N / 2);
        for (int i = 0; i < nx; ++i) {
            /* y: periodic lines over j at fixed (i, l) */
            for (int l = 0; l < nz; ++l) {
                for (int j = 0; j < ny; ++j) {
                    col[j] = f[IDX(i, j, l) + v];
                    rc[j] = rhs[IDX(i, j, l) + v];
                }
                periodic_rhs(M, ny, dy, v2, col, rc);
                for (int j = 0; j < ny; ++j) rhs[IDX(i, j, l) + v] = rc[j];
            }
            /* z: periodic lines over l at fixed (i, j) */
            for (int j = 0; j < ny; ++j) {
                for (int l = 0; l < nz; ++l) {
                    col[l] = f[IDX(i, j, l) + v];
                    rc[l] = rhs[IDX(i, j, l) + v];
                }
                periodic_rhs(M, nz, dzs, v3, col, rc);
                for (int l = 0; l < nz; ++l) rhs[IDX(i, j, l) + v] = rc[l];
            }
        }
    }
#undef IDX
    free(row);
    free(rr);
    free(col);
    free(rc);
}

int or_transport3d_rhs(int N, double L, int nx, int ny, int nz, const double *f, const double *dx, double dy,
                       double dzs, double Tw, const double *Vw, const double *ffar, double *rhs)
{
    if (nx < 2 || ny < 1 || nz < 1 || !(dy > 0) || !(dzs > 0)) return -1;
    transport_rhs_3d(N, L, nx, ny, nz, f, dx, dy, dzs, Tw, Vw, ffar, rhs);
    return 0;
}

/* one Heun step of length dt of the 3-D transport */
int or_transport3d_rk2(int N, double L, int nx, int ny, int nz, double *f, const double *dx, double dy,
                       double dzs, double Tw, const double *Vw, const double *ffar, double dt)
{
    if (nx < 2 || ny < 1 || nz < 1 || !(dy > 0) || !(dzs > 0)) return -1;
    size_t n = (size_t)N * N * N * nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * n);
    double *f1 = (double *)malloc(sizeof(double) * n);
    transport_rhs_3d(N, L, nx, ny, nz, f, dx, dy, dzs, Tw, Vw, ffar, r);
    for (size_t i = 0; i < n; ++i) f1[i] = f[i] + dt * r[i];
    transport_rhs_3d(N, L, nx, ny, nz, f1, dx, dy, dzs, Tw, Vw, ffar, r);
    for (size_t i = 0; i < n; ++i) f[i] = 0.5 * (f[i] + f1[i] + dt * r[i]);
    free(r);
    free(f1);
    return 0;
}

/* Strang step T(dt/2) C(dt) T(dt/2) with the 3-D transport */
int or_strang_step3d(int N, double L, double lambda, int nx, int ny, int nz, double *f, const double *dx,
                     double dy, double dzs, double Tw, const double *Vw, const double *ffar, double dt, double eps,
                     int nthreads)
{
    if (or_transport3d_rk2(N, L, nx, ny, nz, f, dx, dy, dzs, Tw, Vw, ffar, 0.5 * dt)) return -1;
    or_rk2_homogeneous(N, L, lambda, nx * ny * nz, f, dt, 1, eps, 1, nthreads);
    return or_transport3d_rk2(N, L, nx, ny, nz, f, dx, dy, dzs, Tw, Vw, ffar, 0.5 * dt);
}

/* ------------------------------------------------------------------------ */
/* Direct quadrature of the collision integral, Sec. 2 ("Q_general") with
 * the collision law "velocity_interact", B = |u|^lambda / (4 pi) and the
 * same cut |u| <= r0 as the weights, for f a sum of Maxwellians
 * mix[i] = (rho, V1, V2, V3, T).  Written in u = v - v_* = r omega:
 *   Q(v) = int_0^{r0} r^{2+lambda} dr int_{S^2} d omega int_{S^2} d sigma / (4 pi)
 *          [f(v') f(v'_*) - f(v) f(v - u)],
 *   v' = v + (r sigma - u)/2,  v'_* = v - (u + r sigma)/2.
 * Gauss-Legendre in r (npan panels of nr nodes) and in cos(theta) (nth),
 * trapezoid in phi (nph), on both spheres.                                  */
static double maxw_mix(int nmix, const double *mix, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < nmix; ++i) {
        const double *p = mix + 5 * i;
        double e = (v[0] - p[1]) * (v[0] - p[1]) + (v[1] - p[2]) * (v[1] - p[2]) +
                   (v[2] - p[3]) * (v[2] - p[3]);
        s += p[0] * pow(2.0 * OR_PI * p[4], -1.5) * exp(-e / (2.0 * p[4]));
    }
    return s;
}

/* b(t) from its Legendre moments, b(t) = sum_l (2l+1) beta_l P_l(t) / 4pi;
 * nl = 0 is the isotropic 1/4pi */
static double b_of(int nl, const double *beta, double t)
{
    if (nl == 0) return 1.0 / (4.0 * OR_PI);
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s += (2.0 * l + 1.0) * beta[l] * legendre_p(l, t);
    return s / (4.0 * OR_PI);
}

int or_q_bruteforce_b(double lambda, double r0, int nl, const double *beta, int nmix, const double *mix, int nv,
                      const double *vpts, int npan, int nr, int nth, int nph, double *out, int nthreads)
{
    double b0 = nl == 0 ? 1.0 : beta[0]; /* int b dsigma */
    double *xr = (double *)malloc(sizeof(double) * nr), *wr = (double *)malloc(sizeof(double) * nr);
    double *xt = (double *)malloc(sizeof(double) * nth), *wt = (double *)malloc(sizeof(double) * nth);
    or_gauss_legendre(nr, xr, wr);
    or_gauss_legendre(nth, xt, wt);
    int nsph = nth * nph;
    double *dir = (double *)malloc(sizeof(double) * 3 * nsph);
    double *dw = (double *)malloc(sizeof(double) * nsph);
    for (int a = 0; a < nth; ++a)
        for (int b = 0; b < nph; ++b) {
            double mu = xt[a], st = sqrt(1.0 - mu * mu), ph = 2.0 * OR_PI * b / nph;
            int i = a * nph + b;
            dir[3 * i] = st * cos(ph);
            dir[3 * i + 1] = st * sin(ph);
            dir[3 * i + 2] = mu;
            dw[i] = wt[a] * 2.0 * OR_PI / nph;
        }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int iv = 0; iv < nv; ++iv) {
        const double *v = vpts + 3 * iv;
        double fv = maxw_mix(nmix, mix, v);
        double total = 0.0;
        double h = r0 / npan;
        for (int p = 0; p < npan; ++p)
            for (int ir = 0; ir < nr; ++ir) {
                double r = p * h + 0.5 * h * (xr[ir] + 1.0);
                double wrr = 0.5 * h * wr[ir] * pow(r, 2.0 + lambda);
                for (int io = 0; io < nsph; ++io) {
                    double u[3] = {r * dir[3 * io], r * dir[3 * io + 1], r * dir[3 * io + 2]};
                    double vs[3] = {v[0] - u[0], v[1] - u[1], v[2] - u[2]};
                    double loss = b0 * fv * maxw_mix(nmix, mix, vs);
                    double gain = 0.0;
                    for (int is = 0; is < nsph; ++is) {
                        double rs[3] = {r * dir[3 * is], r * dir[3 * is + 1], r * dir[3 * is + 2]};
                        double vp[3], vps[3];
                        for (int d = 0; d < 3; ++d) {
                            vp[d] = v[d] + 0.5 * (rs[d] - u[d]);
                            vps[d] = v[d] - 0.5 * (u[d] + rs[d]);
                        }
                        double ct = dir[3 * is] * dir[3 * io] + dir[3 * is + 1] * dir[3 * io + 1] +
                                    dir[3 * is + 2] * dir[3 * io + 2]; /* cos theta = sigma . u^ */
                        gain += dw[is] * b_of(nl, beta, ct) * maxw_mix(nmix, mix, vp) * maxw_mix(nmix, mix, vps);
                    }
                    total += wrr * dw[io] * (gain - loss);
                }
            }
        out[iv] = total;
    }
    free(xr); free(wr); free(xt); free(wt); free(dir); free(dw);
    return 0;
}

/* the isotropic case, B = |u|^lambda / 4pi */
int or_q_bruteforce(double lambda, double r0, int nmix, const double *mix, int nv,
                    const double *vpts, int npan, int nr, int nth, int nph, double *out,
                    int nthreads)
{
    return or_q_bruteforce_b(lambda, r0, 0, NULL, nmix, mix, nv, vpts, npan, nr, nth, nph, out, nthreads);
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
