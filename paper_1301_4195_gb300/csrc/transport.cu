// K5: the finite-volume transport of Sec. 3.4 on a non-uniform 1-D grid,
//   d f_j / dt = -(F_{j+1/2} - F_{j-1/2}) / dx_j,
//   F_{j+1/2} = v1 (f_j + dx_j/2 s_j)            (v1 >= 0)
//             = v1 (f_{j+1} - dx_{j+1}/2 s_{j+1}) (v1 <  0),
//   s_j = minmod of the forward, backward and central difference quotients.
// On any grid the central quotient is a convex combination of the other two,
// (f_{j+1} - f_{j-1}) / (x_{j+1} - x_{j-1}) = (a (x_{j+1} - x_j) + b (x_j - x_{j-1})) / (x_{j+1} - x_{j-1}),
// so it lies between them and the three-argument minmod equals the
// two-argument one of the forward and backward quotients a, b; the kernels
// take the latter (two double operations less per face; in floating point
// the two can differ only where a and b agree to rounding).
// Boundaries: the wall face at x = 0 carries v1 sigma_w M_w(v) for v1 > 0
// (diffuse reflection, Sec. 2.1 eq. BC) with sigma_w making the discrete net
// mass flux zero; cell 0 takes the one-sided slope (linear extrapolation into
// its ghost); the far end has two ghost cells equal to f_far for v1 < 0 and
// to the last cell for v1 >= 0.
//
// Double precision is slow on this part (1/64 of float), so the kernels keep
// the double work per point small:
//   prep_kernel   once per call, one entry per thread: v1 M_w(v) per
//                 velocity (factors, normalisation and its discrete flux
//                 D = sum_{v1>0} v1 M_w dv^3 from the host), cell geometry
//                 (inverse distances, so no division later), v1 per index;
//   stage_kernel  per Runge-Kutta stage: a block takes 4 cells x 128
//                 velocities, computes their 5 faces (one slope each, from 8
//                 loaded cells) and out = a x + b y + c (F_{j-1/2} - F_{j+1/2}) / dx_j;
//                 the block at the wall first sums sigma_w = (outgoing flux of
//                 cell 0) / D itself, so no kernel boundary separates the two.
//
// The stage kernels work on a shard: cells first .. first+ncl-1 of a grid of
// nct cells (the whole grid is first = 0, ncl = nct).  Cell j of the grid is
// read at fin + (j - first + G) M, G = 0 for the caller's plain array and 2
// for a window with two ghost cells per side (grid cells first-2 ..
// first+ncl+1), which is all a shard's faces read: the flux through face c
// needs cells c-2 .. c+1.  The geometry tables always cover the whole grid,
// so a shard computes every face exactly as the unsharded grid does.
#include <algorithm>
#include <cmath>

#include "cs_internal.cuh"

namespace cs {

namespace {

// Layout of the transport tables in the workspace `scal` (doubles):
//   [0] unused   [1] D
//   inv_fwd[j] = 1 / (x_{j+1} - x_j),      j = 0 .. nc   (ghost centres past the end)
//   inv_dx[j]  = 1 / dx_j,                 j = 0 .. nc - 1
//   hdx[j]     = dx_j / 2,                 j = 0 .. nc - 1
//   v1[k]      = dv (k - N/2),              k = 0 .. N - 1
//   mw[v]      = M_w(v) for v1 > 0, else 0,  v = 0 .. N^3 - 1
// (nc above is the whole grid's cell count).  The centre distances come from
// the widths, x_{j+1} - x_j = (dx_j + dx_{j+1}) / 2 and x_{j+1} - x_{j-1} =
// dx_{j-1}/2 + dx_j + dx_{j+1}/2, with the ghosts past the end as wide as the
// last cell: every entry is local, so no running sum over the grid is needed.
constexpr int kPrepThreads = 64;

struct Tab {
    double *scal, *inv_fwd, *inv_dx, *hdx, *v1, *mw;
};

__host__ __device__ inline Tab tab_of(double *scal, int nc, int N)
{
    Tab t;
    t.scal = scal;
    t.inv_fwd = scal + 8;
    t.inv_dx = t.inv_fwd + (nc + 2);
    t.hdx = t.inv_dx + (nc + 2);
    t.v1 = t.hdx + (nc + 2);
    t.mw = t.v1 + ((N + 7) & ~7);
    return t;
}

// The wall Maxwellian factorised per axis,
//   M_w = (2 pi T_w)^{-3/2} e_1(v1) e_2(v2) e_3(v3),  e_a(v) = exp(-(v - V_a)^2 / (2 T_w)),
// with the 3N factors, the normalisation and D = sum_{v1>0} v1 M_w dv^3
// (factorised the same way) evaluated on the host: the device then needs no
// double-precision transcendental at all (each costs ~100 slow double ops).
struct WallTab {
    double e[3][kMaxN];
    double norm, D;
};

// The transport tables in one launch, one entry per thread: v1 M_w(v) for
// every velocity, the geometry of every face from the widths, v1, D.
__global__ void __launch_bounds__(kPrepThreads) prep_kernel(Geom g, WallTab w, int nc, const double *__restrict__ dx,
                                                            double *__restrict__ scal)
{
    const Tab t = tab_of(scal, nc, g.N);
    const int N = g.N;
    const int i = blockIdx.x * kPrepThreads + threadIdx.x;
    if (i < g.M) {
        const int k1 = i / (N * N), k2 = (i / N) % N, k3 = i % N;
        const double v1 = g.dv * (k1 - g.h);
        t.mw[i] = v1 > 0 ? w.norm * (w.e[0][k1] * w.e[1][k2] * w.e[2][k3]) : 0.0;
    }
    if (i <= nc) {
        const double dj = i < nc ? dx[i] : dx[nc - 1];        // dx_j (ghost: the last width)
        const double dr = i + 1 < nc ? dx[i + 1] : dx[nc - 1];  // dx_{j+1}
        t.inv_fwd[i] = 2.0 / (dj + dr);
        if (i < nc) {
            t.inv_dx[i] = 1.0 / dj;
            t.hdx[i] = 0.5 * dj;
        }
    }
    if (i < N) t.v1[i] = g.dv * (i - g.h);
    if (i == 0) t.scal[1] = w.D;
}

// minmod(a, b) on the bit patterns: 0 unless a and b share a sign, else the
// argument of least magnitude (exact; no double compares)
__device__ __forceinline__ double minmod2(double a, double b)
{
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    if ((ia ^ ib) < 0) return 0.0;
    const unsigned long long mask = 0x7fffffffffffffffull;
    const unsigned long long ma = (unsigned long long)ia & mask, mb = (unsigned long long)ib & mask;
    return ma < mb ? a : b;
}

constexpr int kStageThreads = 128;  // velocities per block
constexpr int kStageCells = 4;      // cells per block: their 5 faces from 8 loaded cells per velocity

// One transport stage for the velocities of block x and the shard cells
// cl0 .. cl1-1 (cl0 = 4 blockIdx.y): the faces first+cl0 .. first+cl1 once
// each, then out = a x + b y + c (F_{j-1/2} - F_{j+1/2}) / dx_j.  A block
// whose first face is the wall also computes sigma_w from grid cells 0 and 1
// of the stage input; every such block sums in the same order, so all of them
// hold the same value.  Reads fin only, writes out only: out must not overlap
// fin (it may alias x or y, read and written by the same thread).
//
// More space dimensions (PD periodic directions): cell (i, j, l) of an x-grid
// of nc cells, ny periodic y-cells and nz periodic z-cells (nz = 1 when
// PD = 1) is stored at index (i ny + j) nz + l; blockIdx.z = j nz + l.  The
// x-part is the 1-D stage applied to that x-row (the same arithmetic); each
// periodic direction adds -(H_{j+1/2} - H_{j-1/2}) / dy, H the second-order
// upwind flux on the uniform periodic grid with the two-argument minmod
// (equal to the three-argument one: on a uniform grid the central quotient is
// the mean of the other two), with velocity component v2 along y and v3 along
// z.  Both cells of a periodic face evaluate its flux with the same
// operations on the same values, so the periodic fluxes telescope exactly; a
// single z-layer adds exactly zero, so PD = 2 with nz = 1 is PD = 1 bit for bit.
__device__ __forceinline__ double yface(double fu, double hs, double s) { return fma(hs, s, fu); }

// (H_{j-1/2} - H_{j+1/2}) vco of one periodic direction from the values of
// the cell's line at offsets -2, -1, +1, +2 (in elements from `cell`) and its
// own value f0; vco = c v_dir / h, idh = 1/h, hh = h/2
__device__ __forceinline__ double periodic_part(const double *cell, const size_t (&o)[4], double f0, double vel,
                                                double vco, double idh, double hh)
{
    const double fm2 = cell[o[0]], fm1 = cell[o[1]], fp1 = cell[o[2]], fp2 = cell[o[3]];
    double hp, hm;
    if (vel >= 0) {  // faces j+1/2 and j-1/2 from cells j and j-1
        const double e_2 = (fm1 - fm2) * idh, e_1 = (f0 - fm1) * idh, e0 = (fp1 - f0) * idh;
        hp = yface(f0, hh, minmod2(e0, e_1));
        hm = yface(fm1, hh, minmod2(e_1, e_2));
    } else {  // from cells j+1 and j
        const double e_1 = (f0 - fm1) * idh, e0 = (fp1 - f0) * idh, e1 = (fp2 - fp1) * idh;
        hp = yface(fp1, -hh, minmod2(e1, e0));
        hm = yface(f0, -hh, minmod2(e0, e_1));
    }
    return (hm - hp) * vco;
}

template <int PD>
__global__ void __launch_bounds__(kStageThreads) stage_kernel(Geom g, const double *__restrict__ fin, int first,
                                                              int ncl, int nc, int G, const double *__restrict__ dx,
                                                              const double *__restrict__ ffar,
                                                              const double *__restrict__ scal, double a, const double *x,
                                                              double b, const double *y, double c, double *out, int ny,
                                                              double idy, double hdy, int nz, double idz, double hdz)
{
    __shared__ double sh[kStageThreads / 32];
    __shared__ double s_coef[kStageCells];  // c / dx_j of the block's cells
    const Tab t = tab_of(const_cast<double *>(scal), nc, g.N);
    const int M = g.M, NN = g.N * g.N;
    const int cl0 = blockIdx.y * kStageCells;
    const int ncb = min(kStageCells, ncl - cl0);  // cells of this block
    const int v = blockIdx.x * kStageThreads + threadIdx.x;
    const int c0 = first + cl0;                   // grid index of the block's first cell and face
    const int row = PD ? (int)blockIdx.z : 0;          // the x-row (j, l): j nz + l
    const size_t XS = (size_t)(PD ? ny * nz : 1) * M;  // stride between x-neighbours
    const size_t R0 = (size_t)row * M;                 // offset of the row

    // sigma_w enters the wall face of velocities with v1 > 0 only, i.e. index
    // k1 > N/2, v >= (N/2 + 1) N^2 (block-uniform test)
    double sigma = 0.0;
    if (c0 == 0 && (blockIdx.x + 1) * kStageThreads > (g.h + 1) * NN) {
        const int half = g.h * NN;  // velocities with v1 < 0 come first
        const double i01 = t.inv_fwd[0], hx = 0.5 * dx[0];
        const double *f0p = fin + (size_t)G * XS + R0;
        double o = 0.0;
        for (int u = threadIdx.x; u < half; u += kStageThreads) {
            const double f0 = f0p[u], f1 = f0p[XS + u];
            o -= t.v1[u / NN] * (f0 - hx * ((f1 - f0) * i01));
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = o;
        __syncthreads();
        double tot = 0.0;
#pragma unroll
        for (int k = 0; k < kStageThreads / 32; ++k) tot += sh[k];
        sigma = tot * (g.dv * g.dv * g.dv) / t.scal[1];
    }
    if (threadIdx.x < ncb) s_coef[threadIdx.x] = c * t.inv_dx[c0 + threadIdx.x];
    __syncthreads();
    if (v >= M) return;
    const double v1 = t.v1[v / NN];
    // grid cells c0-2 .. c0+ncb+1 at this velocity; j >= nc are the far-end
    // ghosts (f_far for v1 < 0, else the last cell); j < 0 is never read
    double fv[kStageCells + 4];
#pragma unroll
    for (int i = 0; i < kStageCells + 4; ++i) {
        const int j = c0 - 2 + i;
        fv[i] = 0.0;
        if (i <= ncb + 3 && j >= 0) {
            if (j < nc)
                fv[i] = fin[(ptrdiff_t)(j - first + G) * XS + R0 + v];
            else  // j >= nc only where the block reaches the grid's last cell
                fv[i] = v1 < 0 ? ffar[v] : fin[(ptrdiff_t)(nc - 1 - first + G) * XS + R0 + v];
        }
    }
    // forward difference quotients of the loaded cells, d[i] = (f_{j+1} - f_j)
    // / (x_{j+1} - x_j) for j = c0-2+i: each is the forward quotient of one
    // face's upwind cell and the backward quotient of the next face's
    double d[kStageCells + 3];
#pragma unroll
    for (int i = 0; i < kStageCells + 3; ++i) {
        const int j = c0 - 2 + i;
        d[i] = (i <= ncb + 2 && j >= 0) ? (fv[i + 1] - fv[i]) * t.inv_fwd[j] : 0.0;
    }
    // the flux is F = v1 G with G the upwind face value (sigma_w M_w at the wall
    // for v1 > 0): v1 joins the per-cell coefficient, c v1 / dx_j
    double vco[kStageCells];
#pragma unroll
    for (int i = 0; i < kStageCells; ++i) vco[i] = v1 * s_coef[i];
    const bool plain = a == 1.0 && y == nullptr;  // out = x + c R(f): one fused multiply-add per point
    // periodic parts of the block's cells: (H_{j-1/2} - H_{j+1/2}) c v2 / dy
    // (+ the same along z with v3)
    double ry[kStageCells];
    if constexpr (PD >= 1) {
        const int j = row / nz, l = row % nz;
        const double v2 = t.v1[(v / g.N) % g.N];
        const double vy = c * v2 * idy;
        size_t oy[4], oz[4];
        const int dk[4] = {-2, -1, 1, 2};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            oy[k] = ((size_t)((j + dk[k] + 2 * ny) % ny) * nz + l) * M;
            oz[k] = ((size_t)j * nz + (l + dk[k] + 2 * nz) % nz) * M;
        }
        double v3 = 0.0, vz = 0.0;
        if constexpr (PD == 2) {
            v3 = t.v1[v % g.N];
            vz = c * v3 * idz;
        }
#pragma unroll
        for (int i = 0; i < kStageCells; ++i) {
            ry[i] = 0.0;
            if (i < ncb) {
                // the cell's x-slice (every row of it) at this velocity
                const double *cell = fin + (ptrdiff_t)(c0 + i - first + G) * XS + v;
                ry[i] = periodic_part(cell, oy, fv[i + 2], v2, vy, idy, hdy);
                if constexpr (PD == 2) ry[i] += periodic_part(cell, oz, fv[i + 2], v3, vz, idz, hdz);
            }
        }
    }
    double Gprev = 0.0;
#pragma unroll
    for (int i = 0; i <= kStageCells; ++i) {
        if (i > ncb) break;
        const int cf = c0 + i;  // face between grid cells cf-1 and cf
        double G;
        if (cf == 0) {
            G = v1 > 0 ? sigma * t.mw[v] : fv[i + 2] - t.hdx[0] * d[i + 2];
        } else {
            // upwind cell u: cf-1 for v1 >= 0, cf for v1 < 0 (u = nc is a ghost, slope 0);
            // register slots are fixed: i is a compile-time index
            const bool right = v1 >= 0;
            const int u = right ? cf - 1 : cf;
            const double fu = right ? fv[i + 1] : fv[i + 2];  // cell u
            const double dF = right ? d[i + 1] : d[i + 2];     // (f_{u+1} - f_u) / (x_{u+1} - x_u)
            const double dB = right ? d[i] : d[i + 1];         // (f_u - f_{u-1}) / (x_u - x_{u-1})
            double sl = 0.0;
            if (u < nc) sl = u == 0 ? dF : minmod2(dF, dB);
            const double hw = u < nc ? t.hdx[u] : t.hdx[nc - 1];
            G = right ? fma(hw, sl, fu) : fma(-hw, sl, fu);
        }
        if (i > 0) {  // cell cf-1 = local cl0 + i - 1
            const size_t idx = (size_t)(cl0 + i - 1) * XS + R0 + v;
            double o;
            if constexpr (PD >= 1) {
                o = fma(Gprev - G, vco[i - 1], ry[i - 1]);
                if (x) o = fma(a, x[idx], o);
                if (y) o = fma(b, y[idx], o);
            } else if (plain && x) {
                o = fma(Gprev - G, vco[i - 1], x[idx]);
            } else {
                o = (Gprev - G) * vco[i - 1];
                if (x) o = fma(a, x[idx], o);
                if (y) o = fma(b, y[idx], o);
            }
            out[idx] = o;
        }
        Gprev = G;
    }
}

}  // namespace

size_t transport_table_doubles(int N, int total_cells)
{
    return 8 + 3 * ((size_t)total_cells + 2) + ((N + 7) & ~7) + (size_t)N * N * N;
}

int launch_transport_prep(const Handle &hd, int total_cells, const cs_domain &dom, cudaStream_t s)
{
    const Geom &g = hd.g;
    WallTab w{};
    const double V[3] = {dom.wall_V[0], dom.wall_V[1], dom.wall_V[2]};
    double S[3] = {0.0, 0.0, 0.0};  // S_1 = sum_{v1>0} v1 e_1, S_2 = sum e_2, S_3 = sum e_3
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < g.N; ++k) {
            const double v = g.dv * (k - g.h), d = v - V[a];
            w.e[a][k] = std::exp(-(d * d) / (2.0 * dom.wall_T));
            if (a > 0)
                S[a] += w.e[a][k];
            else if (v > 0)
                S[0] += v * w.e[0][k];
        }
    w.norm = std::pow(2.0 * M_PI * dom.wall_T, -1.5);
    w.D = w.norm * S[0] * S[1] * S[2] * (g.dv * g.dv * g.dv);
    const int n = std::max(g.M, total_cells + 1);
    prep_kernel<<<(n + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, s>>>(g, w, total_cells, dom.dx, hd.scal);
    CS_LAUNCHED(1, s, "transport tables");
    return CS_OK;
}

int launch_transport_stage(const Handle &hd, const double *fin, int ghost, int first, int ncells, int total_cells,
                           const cs_domain &dom, double a, const double *x, double b, const double *y, double c,
                           double *out, cudaStream_t s)
{
    const dim3 grid((unsigned)((hd.g.M + kStageThreads - 1) / kStageThreads),
                    (unsigned)((ncells + kStageCells - 1) / kStageCells));
    stage_kernel<0><<<grid, kStageThreads, 0, s>>>(hd.g, fin, first, ncells, total_cells, ghost, dom.dx, dom.f_far,
                                                   hd.scal, a, x, b, y, c, out, 1, 0.0, 0.0, 1, 0.0, 0.0);
    CS_LAUNCHED(1, s, "transport stage");
    return CS_OK;
}

int launch_transport_stage2d(const Handle &hd, const double *fin, int nx, int ny, double dy, const cs_domain &dom,
                             double a, const double *x, double b, const double *y, double c, double *out,
                             cudaStream_t s)
{
    const dim3 grid((unsigned)((hd.g.M + kStageThreads - 1) / kStageThreads),
                    (unsigned)((nx + kStageCells - 1) / kStageCells), (unsigned)ny);
    stage_kernel<1><<<grid, kStageThreads, 0, s>>>(hd.g, fin, 0, nx, nx, 0, dom.dx, dom.f_far, hd.scal, a, x, b, y,
                                                   c, out, ny, 1.0 / dy, 0.5 * dy, 1, 0.0, 0.0);
    CS_LAUNCHED(1, s, "transport stage (2-D)");
    return CS_OK;
}

int launch_transport_stage3d(const Handle &hd, const double *fin, int nx, int ny, int nz, double dy, double dz,
                             const cs_domain &dom, double a, const double *x, double b, const double *y, double c,
                             double *out, cudaStream_t s)
{
    const dim3 grid((unsigned)((hd.g.M + kStageThreads - 1) / kStageThreads),
                    (unsigned)((nx + kStageCells - 1) / kStageCells), (unsigned)(ny * nz));
    stage_kernel<2><<<grid, kStageThreads, 0, s>>>(hd.g, fin, 0, nx, nx, 0, dom.dx, dom.f_far, hd.scal, a, x, b, y,
                                                   c, out, ny, 1.0 / dy, 0.5 * dy, nz, 1.0 / dz, 0.5 * dz);
    CS_LAUNCHED(1, s, "transport stage (3-D)");
    return CS_OK;
}

}  // namespace cs
