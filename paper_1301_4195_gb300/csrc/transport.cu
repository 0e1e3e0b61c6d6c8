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
// Per Heun stage: wall_kernel (one block) computes the cell centres and
// sigma_w of the stage input; stage_kernel (one thread per cell and velocity)
// evaluates the two face fluxes of its cell and writes a x + b y + c rhs.
#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kWallThreads = 1024;

struct Wall {
    double T, V1, V2, V3;
};

__device__ __forceinline__ void vel(const Geom &g, int j, double &v1, double &v2, double &v3)
{
    const int N = g.N, h = g.h;
    v1 = g.dv * (j / (N * N) - h);
    v2 = g.dv * ((j / N) % N - h);
    v3 = g.dv * (j % N - h);
}

__device__ __forceinline__ double wall_maxwellian(const Wall &w, double v1, double v2, double v3)
{
    const double e = (v1 - w.V1) * (v1 - w.V1) + (v2 - w.V2) * (v2 - w.V2) + (v3 - w.V3) * (v3 - w.V3);
    return pow(2.0 * M_PI * w.T, -1.5) * exp(-e / (2.0 * w.T));
}

// scal[0] = sigma_w; scal[8 + j] = x_j for j = 0..nc-1 (cell centres)
__global__ void __launch_bounds__(kWallThreads) wall_kernel(Geom g, Wall w, const double *__restrict__ f, int nc,
                                                            const double *__restrict__ dx, double *__restrict__ scal)
{
    __shared__ double sh[2 * 32];
    double *xc = scal + 8;
    if (threadIdx.x == 0) {
        double edge = 0.0;
        for (int j = 0; j < nc; ++j) {
            xc[j] = edge + 0.5 * dx[j];
            edge += dx[j];
        }
    }
    const double w3 = g.dv * g.dv * g.dv;
    const double x0 = 0.5 * dx[0], x1 = dx[0] + 0.5 * dx[1];
    double out = 0.0, mw = 0.0;
    for (int j = threadIdx.x; j < g.M; j += blockDim.x) {
        double v1, v2, v3;
        vel(g, j, v1, v2, v3);
        if (v1 < 0) {
            const double f0 = f[j], f1 = f[(size_t)g.M + j];
            const double s0 = (f1 - f0) / (x1 - x0);
            out += -v1 * (f0 - 0.5 * dx[0] * s0) * w3;
        } else if (v1 > 0) {
            mw += v1 * wall_maxwellian(w, v1, v2, v3) * w3;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        out += __shfl_xor_sync(0xffffffffu, out, o);
        mw += __shfl_xor_sync(0xffffffffu, mw, o);
    }
    if (lane == 0) {
        sh[wid] = out;
        sh[32 + wid] = mw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double so = 0, sm = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            so += sh[k];
            sm += sh[32 + k];
        }
        scal[0] = so / sm;
    }
}

__device__ __forceinline__ double minmod3(double a, double b, double c)
{
    if (a > 0 && b > 0 && c > 0) return fmin(a, fmin(b, c));
    if (a < 0 && b < 0 && c < 0) return fmax(a, fmax(b, c));
    return 0.0;
}

struct Column {
    const double *f, *ffar, *dx, *xc;
    int nc, M, v;
    double v1;
    __device__ double val(int j) const
    {
        if (j < nc) return f[(size_t)j * M + v];
        return v1 < 0 ? ffar[v] : f[(size_t)(nc - 1) * M + v];
    }
    __device__ double pos(int j) const
    {
        if (j < nc) return xc[j];
        return xc[nc - 1] + (j - nc + 1) * dx[nc - 1];
    }
    __device__ double slope(int j) const
    {
        if (j == 0) return (val(1) - val(0)) / (pos(1) - pos(0));
        const double fm = val(j - 1), f0 = val(j), fp = val(j + 1);
        const double xm = pos(j - 1), x0 = pos(j), xp = pos(j + 1);
        return minmod3((fp - f0) / (xp - x0), (f0 - fm) / (x0 - xm), (fp - fm) / (xp - xm));
    }
    __device__ double width(int j) const { return j < nc ? dx[j] : dx[nc - 1]; }
};

__global__ void stage_kernel(Geom g, Wall w, const double *__restrict__ fin, int nc, const double *__restrict__ dx,
                             const double *__restrict__ ffar, const double *__restrict__ scal, double a,
                             const double *x, double b, const double *y, double c, double *out)
{
    const size_t n = (size_t)nc * g.M;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int cell = (int)(i / g.M), v = (int)(i % g.M);
        double v1, v2, v3;
        vel(g, v, v1, v2, v3);
        Column col{fin, ffar, dx, scal + 8, nc, g.M, v, v1};
        // face cell - 1/2
        double Fl;
        if (cell == 0) {
            if (v1 > 0)
                Fl = v1 * scal[0] * wall_maxwellian(w, v1, v2, v3);
            else
                Fl = v1 * (col.val(0) - 0.5 * dx[0] * col.slope(0));
        } else if (v1 >= 0) {
            Fl = v1 * (col.val(cell - 1) + 0.5 * col.width(cell - 1) * col.slope(cell - 1));
        } else {
            Fl = v1 * (col.val(cell) - 0.5 * col.width(cell) * col.slope(cell));
        }
        // face cell + 1/2
        double Fr;
        if (v1 >= 0)
            Fr = v1 * (col.val(cell) + 0.5 * col.width(cell) * col.slope(cell));
        else
            Fr = v1 * (col.val(cell + 1) - 0.5 * col.width(cell + 1) * col.slope(cell + 1));
        const double rhs = -(Fr - Fl) / dx[cell];
        double o = c * rhs;
        if (x) o += a * x[i];
        if (y) o += b * y[i];
        out[i] = o;
    }
}

}  // namespace

int launch_transport_stage(const Handle &hd, const double *fin, int ncells, const cs_domain &dom, double a,
                           const double *x, double b, const double *y, double c, double *out, cudaStream_t s)
{
    const Wall w{dom.wall_T, dom.wall_V[0], dom.wall_V[1], dom.wall_V[2]};
    wall_kernel<<<1, kWallThreads, 0, s>>>(hd.g, w, fin, ncells, dom.dx, hd.scal);
    const size_t n = (size_t)ncells * hd.g.M;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
    stage_kernel<<<blocks, 256, 0, s>>>(hd.g, w, fin, ncells, dom.dx, dom.f_far, hd.scal, a, x, b, y, c, out);
    CS_CHECK_LAUNCH("transport stage");
    return CS_OK;
}

}  // namespace cs
