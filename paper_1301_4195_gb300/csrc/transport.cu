// K5: the finite-volume transport of Sec. 3.4 on a non-uniform 1-D grid,
//   d f_j / dt = -(F_{j+1/2} - F_{j-1/2}) / dx_j,
//   F_{j+1/2} = v1 (f_j + dx_j/2 s_j)            (v1 >= 0)
//             = v1 (f_{j+1} - dx_{j+1}/2 s_{j+1}) (v1 <  0),
//   s_j = minmod of the forward, backward and central difference quotients.
// Boundaries: the wall face at x = 0 carries v1 sigma_w M_w(v) for v1 > 0
// (diffuse reflection, Sec. 2.1 eq. BC) with sigma_w making the discrete net
// mass flux zero; cell 0 takes the one-sided slope (linear extrapolation into
// its ghost); the far end has two ghost cells equal to f_far for v1 < 0 and
// to the last cell for v1 >= 0.
//
// Double precision is slow on this part (1/64 of float), so the kernels keep
// the double work per point small:
//   prep_mw_kernel, prep_geo_kernel   once per call: v1 M_w(v) per velocity
//                 and its discrete flux D = sum_{v1>0} v1 M_w dv^3 (partials
//                 summed in a fixed order), cell geometry (inverse distances,
//                 so no division later), v1 per velocity index;
//   sigma_kernel  per Heun stage: sigma_w = (outgoing flux of cell 0) / D;
//   face_kernel   per stage: every face flux once (one slope each);
//   update_kernel per stage: out = a x + b y + c (F_{j-1/2} - F_{j+1/2}) / dx_j.
//
// The stage kernels work on a shard: cells first .. first+ncl-1 of a grid of
// nct cells (the whole grid is first = 0, ncl = nct).  Cell j of the grid is
// read at fin + (j - first + G) M, G = 0 for the caller's plain array and 2
// for a window with two ghost cells per side (grid cells first-2 ..
// first+ncl+1), which is all a shard's faces read: the flux through face c
// needs cells c-2 .. c+1.  The geometry tables always cover the whole grid,
// so a shard computes every face exactly as the unsharded grid does.
#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kSigmaThreads = 512;

// Layout of the transport tables in the workspace `scal` (doubles):
//   [0] sigma_w   [1] D
//   inv_fwd[j] = 1 / (x_{j+1} - x_j),      j = 0 .. nc   (ghost centres past the end)
//   inv_ctr[j] = 1 / (x_{j+1} - x_{j-1}),  j = 1 .. nc
//   inv_dx[j]  = 1 / dx_j,                 j = 0 .. nc - 1
//   xs[j]      = cell centre,               j = 0 .. nc + 1
//   v1[k]      = dv (k - N/2),              k = 0 .. N - 1
//   mw[v]      = v1 M_w(v) for v1 > 0, else 0,  v = 0 .. N^3 - 1
//   part[b]    = partial sums of D, one per block of prep_mw_kernel
// and the face fluxes F[c][v] of the shard's faces, c = 0 .. ncl, after them
// (nc above is the whole grid's cell count).
constexpr int kPrepThreads = 256;
constexpr int kMaxPrepBlocks = (kMaxN * kMaxN * kMaxN + kPrepThreads - 1) / kPrepThreads;

struct Tab {
    double *scal, *inv_fwd, *inv_ctr, *inv_dx, *xs, *v1, *mw, *part, *face;
};

__host__ __device__ inline Tab tab_of(double *scal, int nc, int N)
{
    Tab t;
    t.scal = scal;
    t.inv_fwd = scal + 8;
    t.inv_ctr = t.inv_fwd + (nc + 2);
    t.inv_dx = t.inv_ctr + (nc + 2);
    t.xs = t.inv_dx + (nc + 2);
    t.v1 = t.xs + (nc + 2);
    t.mw = t.v1 + ((N + 7) & ~7);
    t.part = t.mw + (size_t)N * N * N;
    t.face = t.part + kMaxPrepBlocks;
    return t;
}

struct Wall {
    double T, V1, V2, V3;
};

// v1 M_w(v) for every velocity and one partial sum of D per block
__global__ void __launch_bounds__(kPrepThreads) prep_mw_kernel(Geom g, Wall w, int nc, double *__restrict__ scal)
{
    __shared__ double sh[kPrepThreads / 32];
    const Tab t = tab_of(scal, nc, g.N);
    const int N = g.N;
    const double norm = pow(2.0 * M_PI * w.T, -1.5), w3 = g.dv * g.dv * g.dv;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    double D = 0.0;
    if (v < g.M) {
        const double v1 = g.dv * (v / (N * N) - g.h);
        const double v2 = g.dv * ((v / N) % N - g.h);
        const double v3 = g.dv * (v % N - g.h);
        double m = 0.0;
        if (v1 > 0) {
            const double e = (v1 - w.V1) * (v1 - w.V1) + (v2 - w.V2) * (v2 - w.V2) + (v3 - w.V3) * (v3 - w.V3);
            m = v1 * norm * exp(-e / (2.0 * w.T));
            D = m * w3;
        }
        t.mw[v] = m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) D += __shfl_xor_sync(0xffffffffu, D, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = D;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kPrepThreads / 32; ++k) s += sh[k];
        t.part[blockIdx.x] = s;
    }
}

// cell geometry, v1 table and D (partials summed in a fixed order)
__global__ void __launch_bounds__(256) prep_geo_kernel(Geom g, int nc, int nparts, const double *__restrict__ dx,
                                                       double *__restrict__ scal)
{
    const Tab t = tab_of(scal, nc, g.N);
    if (threadIdx.x == 0) {
        double edge = 0.0;
        for (int j = 0; j < nc; ++j) {
            t.xs[j] = edge + 0.5 * dx[j];
            edge += dx[j];
        }
        t.xs[nc] = t.xs[nc - 1] + dx[nc - 1];
        t.xs[nc + 1] = t.xs[nc] + dx[nc - 1];
        double D = 0.0;
        for (int b = 0; b < nparts; ++b) D += t.part[b];
        t.scal[1] = D;
    }
    if (threadIdx.x < g.N) t.v1[threadIdx.x] = g.dv * ((int)threadIdx.x - g.h);
    __syncthreads();
    for (int j = threadIdx.x; j <= nc; j += blockDim.x) {
        t.inv_fwd[j] = 1.0 / (t.xs[j + 1] - t.xs[j]);
        if (j >= 1) t.inv_ctr[j] = 1.0 / (t.xs[j + 1] - t.xs[j - 1]);
        if (j < nc) t.inv_dx[j] = 1.0 / dx[j];
    }
}

// sigma_w of the stage input: outgoing flux of the reconstructed wall-face values
__global__ void __launch_bounds__(kSigmaThreads) sigma_kernel(Geom g, const double *__restrict__ f, int nc,
                                                              const double *__restrict__ dx, double *__restrict__ scal)
{
    __shared__ double sh[32];
    const Tab t = tab_of(scal, nc, g.N);
    const int NN = g.N * g.N;
    const int half = g.h * NN;  // velocities with v1 < 0 come first (index k1 < N/2)
    const double i01 = t.inv_fwd[0], hx = 0.5 * dx[0];
    double out = 0.0;
    for (int v = threadIdx.x; v < half; v += blockDim.x) {
        const double f0 = f[v], f1 = f[(size_t)g.M + v];
        out -= t.v1[v / NN] * (f0 - hx * ((f1 - f0) * i01));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = out;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        t.scal[0] = s * (g.dv * g.dv * g.dv) / t.scal[1];
    }
}

// 3-argument minmod on the bit patterns: 0 unless all three share a sign,
// else the argument of least magnitude (exact; no double compares)
__device__ __forceinline__ double minmod3(double a, double b, double c)
{
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b), ic = __double_as_longlong(c);
    if (((ia ^ ib) | (ia ^ ic)) < 0) return 0.0;
    const unsigned long long mask = 0x7fffffffffffffffull;
    unsigned long long m = (unsigned long long)ia & mask;
    const unsigned long long mb = (unsigned long long)ib & mask, mc = (unsigned long long)ic & mask;
    m = mb < m ? mb : m;
    m = mc < m ? mc : m;
    return __longlong_as_double((long long)(m | ((unsigned long long)ia & ~mask)));
}

// flux through face c (between cells c-1 and c), c = first .. first+ncl, one
// thread per (face, v); face c is stored at c - first
__global__ void face_kernel(Geom g, const double *__restrict__ fin, int first, int ncl, int nc, int G,
                            const double *__restrict__ dx, const double *__restrict__ ffar, double *__restrict__ scal)
{
    const Tab t = tab_of(scal, nc, g.N);
    const int M = g.M, NN = g.N * g.N;
    const int c = first + blockIdx.y;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < M; v += gridDim.x * blockDim.x) {
        const double v1 = t.v1[v / NN];
        // grid cell j (j = nc, nc + 1: far-end ghosts) as stored in fin
        auto val = [&](int j) {
            if (j >= nc) {
                if (v1 < 0) return ffar[v];
                j = nc - 1;
            }
            return fin[(ptrdiff_t)(j - first + G) * M + v];
        };
        double F;
        if (c == 0) {
            if (v1 > 0) {
                F = t.scal[0] * t.mw[v];
            } else {
                const double f0 = val(0), f1 = val(1);
                F = v1 * (f0 - 0.5 * dx[0] * ((f1 - f0) * t.inv_fwd[0]));
            }
        } else {
            // upwind cell u: c-1 for v1 >= 0, c for v1 < 0 (u = nc is a ghost, slope 0)
            const bool right = v1 >= 0;
            const int u = right ? c - 1 : c;
            const double fu = val(u);
            double s = 0.0;
            if (u < nc) {
                const double fp = val(u + 1);
                if (u == 0) {
                    s = (fp - fu) * t.inv_fwd[0];
                } else {
                    const double fm = val(u - 1);
                    s = minmod3((fp - fu) * t.inv_fwd[u], (fu - fm) * t.inv_fwd[u - 1], (fp - fm) * t.inv_ctr[u]);
                }
            }
            const double half = 0.5 * (u < nc ? dx[u] : dx[nc - 1]);
            F = v1 * (right ? fma(half, s, fu) : fma(-half, s, fu));
        }
        t.face[(size_t)blockIdx.y * M + v] = F;
    }
}

__global__ void update_kernel(Geom g, int first, int ncl, int nc, const double *__restrict__ scal, double a,
                              const double *x, double b, const double *y, double c, double *out)
{
    const Tab t = tab_of(const_cast<double *>(scal), nc, g.N);
    const size_t n = (size_t)ncl * g.M;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int cell = first + (int)(i / g.M);
        const double rhs = (t.face[i] - t.face[i + g.M]) * t.inv_dx[cell];
        double o = c * rhs;
        if (x) o = fma(a, x[i], o);
        if (y) o = fma(b, y[i], o);
        out[i] = o;
    }
}

}  // namespace

size_t transport_table_doubles(int N, int ncells, int total_cells)
{
    return 8 + 4 * ((size_t)total_cells + 2) + ((N + 7) & ~7) + kMaxPrepBlocks + (size_t)N * N * N * (ncells + 2);
}

int launch_transport_prep(const Handle &hd, int total_cells, const cs_domain &dom, cudaStream_t s)
{
    const Wall w{dom.wall_T, dom.wall_V[0], dom.wall_V[1], dom.wall_V[2]};
    const int nparts = (hd.g.M + kPrepThreads - 1) / kPrepThreads;
    prep_mw_kernel<<<nparts, kPrepThreads, 0, s>>>(hd.g, w, total_cells, hd.scal);
    prep_geo_kernel<<<1, 256, 0, s>>>(hd.g, total_cells, nparts, dom.dx, hd.scal);
    CS_LAUNCHED(2, s, "transport tables");
    return CS_OK;
}

int launch_transport_stage(const Handle &hd, const double *fin, int ghost, int first, int ncells, int total_cells,
                           const cs_domain &dom, double a, const double *x, double b, const double *y, double c,
                           double *out, cudaStream_t s)
{
    const int M = hd.g.M;
    int launched = 2;
    if (first == 0) {  // the wall face belongs to this shard: sigma_w from grid cells 0 and 1
        sigma_kernel<<<1, kSigmaThreads, 0, s>>>(hd.g, fin + (size_t)ghost * M, total_cells, dom.dx, hd.scal);
        ++launched;
    }
    const int tpb = 256;
    dim3 fgrid((unsigned)((M + tpb - 1) / tpb), (unsigned)(ncells + 1));
    face_kernel<<<fgrid, tpb, 0, s>>>(hd.g, fin, first, ncells, total_cells, ghost, dom.dx, dom.f_far, hd.scal);
    const size_t n = (size_t)ncells * M;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb < 65535 ? (n + tpb - 1) / tpb : 65535);
    update_kernel<<<blocks, tpb, 0, s>>>(hd.g, first, ncells, total_cells, hd.scal, a, x, b, y, c, out);
    CS_LAUNCHED(launched, s, "transport stage");
    return CS_OK;
}

}  // namespace cs
