/*
 * cs.h -- C ABI of the GB300 (sm_103a) conservative spectral collision library.
 *
 * The library evaluates the Boltzmann collision operator by the conservative
 * spectral method of Gamba and Tharkabhushanam as described in J. R. Haack,
 * "A hybrid OpenMP and MPI implementation of a conservative spectral method
 * for the Boltzmann equation" (arXiv:1301.4195): per spatial cell a forward
 * transform of f on an N^3 velocity grid, the weighted Fourier convolution
 * with the precomputed weights Ghat, an inverse transform and the
 * conservation projection; plus Heun time stepping and a finite-volume
 * transport step (one space dimension, or two or three with periodic further ones)
 * combined by Strang splitting, sharded transport stages for domain
 * decomposition, and batched calls over handles of different N.
 *
 * Conventions shared by every call
 *   - Velocity grid (Sec. 3.1, "meshpoints"): N even, 4 <= N <= 64, the cube
 *     [-L, L]^3, v_k = dv (k - N/2), dv = 2L/N, zeta_k = dzeta (k - N/2),
 *     dzeta = pi/L.  A cell's distribution is N^3 doubles in C order, flat
 *     index (k1*N + k2)*N + k3.  A batch of cells is [ncells][N^3].
 *   - Collision kernel B = |u|^lambda / (4 pi) (isotropic, Sec. 2.2), or
 *     |u|^lambda b(cos theta) with b given by its Legendre moments
 *     (cs_weights_build_aniso), -3 < lambda <= 1 (soft potentials, Maxwell
 *     molecules, variable hard potentials, hard spheres; Sec. 2), weight
 *     integral cut at r0 = L, beta = 1.
 *   - Pointers marked "device" are CUDA device pointers owned by the caller
 *     (e.g. allocated by PyTorch); "host" pointers are ordinary memory.
 *     Device arrays must be 8-byte aligned and must not overlap unless a
 *     call says so.
 *   - Every call that takes a cudaStream_t is asynchronous on that stream
 *     (0 = legacy default stream) and returns after enqueueing its work.
 *   - Every call returns CS_OK (0) or a negative CS_E* code and then leaves
 *     a message for cs_last_error().  Arguments are checked on the host
 *     before anything is enqueued; no call traps, asserts or aborts.
 *   - No call allocates device memory except cs_weights_build (the weight
 *     table), cs_reserve / the first call that needs more workspace than
 *     the handle holds, and cs_fma_probe (one word, freed before it
 *     returns).  Call cs_reserve before capturing a CUDA graph.
 *   - A handle is not thread-safe: calls on one handle must be serialised by
 *     the caller (one stream, or external synchronisation).
 */
#ifndef CS_H
#define CS_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CS_OK 0
#define CS_EINVAL (-1)     /* bad argument: N, L, lambda, pointer, size, alignment */
#define CS_ENOMEM (-2)     /* device allocation failed */
#define CS_ENOTSUP (-3)    /* valid request this build does not serve */
#define CS_ECUDA (-4)      /* a CUDA runtime call failed (message has the CUDA error) */
#define CS_ETIMEOUT (-5)   /* a bounded device-side wait expired */
#define CS_ENONFINITE (-6) /* a non-finite value was found where finiteness is checked */

#define CS_FP64 0 /* every step in double precision */
#define CS_FP32 1 /* transforms and convolution in float (compensated sum over xi),
                     weights built in double, moments and projection in double */
/* OR'd into the precision of cs_weights_build / cs_weights_bytes (CS_FP32,
 * N in {8, 16, 24, 32, 48, 64} only): build the radius tables alone, not the
 * table of every pair.  Ghat(xi_m, zeta_k) depends on the pair only through
 * |k'|^2, |2m' - k'|^2 and |m'|^2 (k' = k - N/2, m' = m - N/2; Sec. 2.2, eq.
 * GHat_calc: a = |zeta|/2, b = |xi - zeta/2|, c = |xi|), and splits into
 * A(|k'|^2, |2m'-k'|^2) - B(|m'|^2); the convolution then rebuilds every
 * weight tile from A and B (146 MB at N = 64 instead of 58 GB). */
#define CS_WEIGHTS_RADIUS 16

typedef struct cs_handle_s *cs_handle_t;

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int cs_version(void);

/* Message of the last failing call made by this host thread ("" if none).
 * The pointer stays valid until the thread's next failing call. */
const char *cs_last_error(void);

/* Bytes of device memory cs_weights_build will hold for the weights of grid
 * size N in the given precision (admission planning).  The table stores the
 * symmetrised weights Ghat(xi, zeta) + Ghat(zeta - xi, zeta) for the
 * lexicographically lower half of the valid (xi, zeta) pairs, Sec. 3.2; a
 * float handle served by the strip kernel also holds the radius tables (see
 * CS_WEIGHTS_RADIUS, which leaves the table out).
 *   bytes (host, out).  Errors: CS_EINVAL. */
int cs_weights_bytes(int N, int precision, size_t *bytes);

/* Order of the (m3, k3) pairs inside one weight tile for grid size N and a
 * precision (host only, no GPU work): map[p] = m3 * 256 + k3 for entry p, or
 * -1 for padding; *entries = the tile stride.  Pass map = NULL to query the
 * size.  Every valid pair (Sec. 3.2: k3 - m3 + N/2 in [0, N-1]) appears once.
 * Errors: CS_EINVAL (bad N or precision, or cap < stride with map != NULL). */
int cs_tile_layout(int N, int precision, int *map, int cap, int *entries);

/* Build the convolution weights of Sec. 2.2 (eq. GHat_calc; closed forms for
 * lambda = 0 and 1, radial Gauss-Legendre quadrature otherwise), in double on
 * the device (kept in float for CS_FP32), together with the constants of the
 * transforms and of the projection (C C^T)^{-1} of Sec. 3.3.  Float handles
 * with N in {8, 16, 24, 32, 48, 64} also get the radius tables, so the
 * convolution can read stored tiles or rebuild them (CS_TUNE_WEIGHTS);
 * precision CS_FP32 | CS_WEIGHTS_RADIUS builds the radius tables only.
 *   N        even, 4..64 (the float table holds about half the 27 N^6 / 64
 *            valid pairs, 4 bytes each, plus padding: 0.9 GB at N = 32,
 *            58 GB at N = 64; cs_weights_bytes gives the exact size)
 *   L        > 0, half-width of the velocity cube; r0 = L
 *   lambda   -3 < lambda <= 1 (the radial integrand behaves as r^{lambda+4}
 *            near 0, so the quadrature converges for every such lambda)
 *   stream   the build is enqueued here; the handle is usable on any stream
 *            once the build has completed on this one
 *   out      (host, out) new handle; *out is untouched on error.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_weights_build(int N, double L, double lambda, int precision, cudaStream_t stream,
                     cs_handle_t *out);

/* cs_weights_build for an anisotropic scattering kernel B = |u|^lambda
 * b(cos theta) (Sec. 2; the paper computes the weights of Sec. 2.2 only for
 * the isotropic b = 1/4pi, and notes in Sec. 4.2 that the same weighted
 * convolution serves anisotropic scattering).  b is given by its Legendre
 * moments
 *   moments[l] = int_{S^2} b(sigma . u^) P_l(sigma . u^) dsigma,  l < nmom,
 * i.e. b(t) = sum_l (2l + 1) moments[l] P_l(t) / 4pi; moments[0] is the total
 * integral of b (1 under the normalisation of Sec. 2), and {1} alone is the
 * isotropic case.  The weights are
 *   Ghat(xi, zeta) = sqrt(2/pi) [ sum_l (2l+1) (-1)^l moments[l] P_l(cos g) R_l
 *                                 - moments[0] int_0^r0 r^{lambda+2} sinc(|xi| r) dr ]
 * with R_l = int_0^r0 r^{lambda+2} j_l(|zeta| r/2) j_l(|xi - zeta/2| r) dr and
 * cos g the cosine between zeta and xi - zeta/2 (the Funk-Hecke reduction of
 * the sphere integral in G, Sec. 2.2).  Odd moments do not change Q (for
 * identical particles only b(t) + b(-t) enters the convolution); the table
 * keeps the symmetrised weights as for isotropic handles, so every other call
 * works unchanged.  Radius tables are not built (CS_TUNE_WEIGHTS = 2 is
 * refused); cs_weights_sample returns the unsymmetrised Ghat with every moment.
 *   moments (host) [nmom], 1 <= nmom <= 16, finite, moments[0] > 0
 *   precision CS_FP64 or CS_FP32 (not CS_WEIGHTS_RADIUS)
 *   other arguments and errors as cs_weights_build. */
int cs_weights_build_aniso(int N, double L, double lambda, const double *moments, int nmom, int precision,
                           cudaStream_t stream, cs_handle_t *out);

/* Free the handle, its weight table and its workspace.  NULL is a no-op.
 * The caller must make sure no work using the handle is still in flight. */
int cs_handle_destroy(cs_handle_t h);

/* Read back the parameters of a handle (any out pointer may be NULL). */
int cs_handle_info(cs_handle_t h, int *N, double *L, double *lambda, int *precision,
                   size_t *weight_bytes);

/* Grow the handle's workspace to serve up to ncells cells per call (no-op if
 * it is already large enough).  Synchronises the device when it reallocates.
 * Errors: CS_EINVAL, CS_ENOMEM. */
int cs_reserve(cs_handle_t h, int ncells);

/* Device-side status of h: synchronises the device, then returns CS_ETIMEOUT
 * if a bounded wait inside one of h's kernels expired since the last call
 * (the results of that call are invalid; no kernel traps or hangs instead),
 * else CS_ENONFINITE if the input scan (CS_TUNE_CHECK_INPUT) found a
 * non-finite value (or, in mode 2, a negative one; the message says which),
 * else CS_OK, and clears the status.  Errors: CS_EINVAL, CS_ECUDA. */
int cs_status(cs_handle_t h);

/* Ghat(xi_m, zeta_k) (unsymmetrised, Sec. 2.2) evaluated on the device by the
 * same function that fills the table, for n index pairs.
 *   km   (host) [n][6] ints: k1 k2 k3 m1 m2 m3, each in 0..N-1
 *   out  (host) [n] doubles.  Synchronous.  Errors: CS_EINVAL, CS_ECUDA. */
int cs_weights_sample(cs_handle_t h, const int *km, int n, double *out);

/* Step a1, the forward transform (Sec. 3.2 with the normalisation of
 * Sec. 2.2): fhat(zeta_k) = (2 pi)^{-3/2} dv^3 sum_j f(v_j) exp(-i zeta_k.v_j),
 * in the handle's precision.
 *   f     (device) [ncells][N^3] doubles
 *   fhat  (device, out) [ncells][N^3][2] doubles (re, im), widened from float
 *         in CS_FP32.  Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_transform(cs_handle_t h, const double *f, int ncells, double *fhat, cudaStream_t stream);

/* Step a2, the weighted convolution (Sec. 3.2, trapezoid rule, terms with
 * zeta_k - xi_m outside the grid dropped):
 *   Qhat(zeta_k) = dzeta^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m).
 *   fhat  (device) [ncells][N^3][2] doubles (rounded to float in CS_FP32)
 *   qhat  (device, out) [ncells][N^3][2] doubles.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_convolve(cs_handle_t h, const double *fhat, int ncells, double *qhat, cudaStream_t stream);

/* Step a3, the inverse transform (Sec. 3.2):
 *   Qt(v_j) = Re[(2 pi)^{-3/2} dzeta^3 sum_k Qhat(zeta_k) exp(i zeta_k.v_j)] / eps.
 *   qhat  (device) [ncells][N^3][2] doubles;  Q (device, out) [ncells][N^3].
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_inverse(cs_handle_t h, const double *qhat, int ncells, double eps, double *Q,
               cudaStream_t stream);

/* The collision operator (steps a1-a4): Q = P_N Qt(f) / eps if conserve != 0,
 * else Qt(f) / eps, for every cell.
 *   f  (device) [ncells][N^3];  Q (device, out) [ncells][N^3]; f and Q must
 *   not overlap.  eps > 0 is the Knudsen number of eq. (BTE).
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_collide(cs_handle_t h, const double *f, int ncells, double eps, double *Q, int conserve,
               cudaStream_t stream);

/* One entry of a batched collision evaluation. */
typedef struct {
    cs_handle_t handle; /* weights and workspace of this entry (N, L, lambda, precision) */
    const double *f;    /* device, [ncells][N^3] */
    double *Q;          /* device, [ncells][N^3], must not overlap f */
    int ncells;
} cs_batch_entry;

/* The collision operator for n <= 16 entries of possibly different N and
 * lambda, as one replayable unit: the first call with a given list of
 * entries captures every entry's kernels into one CUDA graph, later calls
 * with the same entries, eps and conserve replay it with a single graph
 * launch on `stream`.  When two or more entries have float handles with N in
 * {8, 16, 24, 32}, their convolutions (the O(N^6) step) run as ONE persistent
 * kernel launch that takes the items of all of them from one queue, heaviest
 * first; their transforms and projections, and the whole evaluation of every
 * other entry, run on one parallel graph branch per entry.  Each entry's
 * result is bit-identical to cs_collide on that entry.  Every entry needs its
 * own handle; handles must not be used elsewhere while the call runs.  The
 * workspace of a float handle in a shared launch is padded to whole 64-cell
 * blocks (N < 32).  Cached graphs are dropped when one of their handles is
 * destroyed or its workspace grows.
 * Errors: CS_EINVAL (NULL, duplicate handle, bad sizes), CS_ENOMEM, CS_ECUDA. */
int cs_collide_batched(const cs_batch_entry *entries, int n, double eps, int conserve, cudaStream_t stream);

/* One entry of a batched relaxation: a handle and its cells' states. */
typedef struct {
    cs_handle_t handle; /* weights and workspace of this entry (N, L, lambda, precision) */
    double *f;          /* device, [ncells][N^3], advanced in place */
    int ncells;
} cs_relax_entry;

/* nsteps Heun steps (Sec. 3.1) of df/dt = P_N Qt(f) / eps (Sec. 3.3) for
 * n <= 16 entries of possibly different N and lambda: cs_relax on each, as
 * one captured graph per step (cached like cs_collide_batched, replayed
 * nsteps times on `stream`).  Each of the step's two collision evaluations
 * runs the convolutions of the float entries with N in {8, 16, 24, 32} as
 * ONE persistent launch.  Each entry's result is bit-identical to cs_relax
 * on that entry.  The entries' states must not overlap; every entry needs
 * its own handle (its workspace holds the intermediate stage).
 * Errors: CS_EINVAL (NULL, duplicate handle, overlap, bad sizes, dt, eps),
 * CS_ENOMEM, CS_ECUDA. */
int cs_relax_batched(const cs_relax_entry *entries, int n, double dt, double eps, int nsteps, cudaStream_t stream);

/* Step a4, the conservation projection of Sec. 3.3, in place, in double:
 *   Q <- Q - C^T (C C^T)^{-1} C Q,  C = dv^3 (1, v1, v2, v3, |v|^2) (5 x N^3).
 *   Q        (device, in/out) [ncells][N^3]
 *   moments  (device, out, may be NULL) [ncells][5]: C Q before the projection.
 * Errors: CS_EINVAL, CS_ECUDA. */
int cs_conserve(cs_handle_t h, double *Q, int ncells, double *moments, cudaStream_t stream);

/* The moments of eq. (moments) as the rows of C: per cell
 * dv^3 sum_j (1, v1, v2, v3, |v|^2)_j f_j  -> out (device) [ncells][5].
 * Errors: CS_EINVAL, CS_ECUDA. */
int cs_moments(cs_handle_t h, const double *f, int ncells, double *out, cudaStream_t stream);

/* Step a5: nsteps Heun (second-order Runge-Kutta, Sec. 3.1) steps of the
 * space-homogeneous problem df/dt = P_N Qt(f) / eps, in place.
 *   f (device, in/out) [ncells][N^3].  Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_relax(cs_handle_t h, double *f, int ncells, double dt, double eps, int nsteps,
             cudaStream_t stream);

/* 1-D physical domain of the transport step (Sec. 3.4): cells of width dx_j,
 * cell 0 touching a diffusely reflecting wall at x = 0 (Sec. 2.1, eq. BC),
 * the far end open to a given gas. */
typedef struct {
    const double *dx;    /* device, [ncells] cell widths > 0 (non-uniform allowed) */
    const double *f_far; /* device, [N^3] far-field distribution, used for v1 < 0 */
    double wall_T;       /* wall temperature T_w > 0 */
    double wall_V[3];    /* wall velocity V_w */
} cs_domain;

/* One Heun step of length dt of the finite-volume transport of Sec. 3.4
 * (second-order upwind fluxes, 3-argument minmod slopes), in place.
 * Boundaries: at the wall the incoming half (v1 > 0) is sigma_w M_w(v) with
 * sigma_w set from the discrete outgoing flux so the net wall mass flux is
 * zero; the slope of cell 0 is one-sided (linear extrapolation into the
 * ghost).  At the far end two ghost cells hold f_far for v1 < 0 and copy the
 * last cell for v1 >= 0.  ncells >= 2.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_transport(cs_handle_t h, double *f, int ncells, const cs_domain *dom, double dt,
                 cudaStream_t stream);

/* Transport in two space dimensions (Sec. 3.4 notes the scheme carries over
 * to higher dimensions): x is the wall-normal direction of the 1-D problem
 * (cells of width dx, diffusely reflecting wall at x = 0, far-field gas at
 * the end), y a periodic direction of ny cells of uniform width dy.  The
 * state is [nx][ny][N^3] (cell (i, j) at index i ny + j).  A stage adds the
 * flux differences of both directions (no splitting between x and y):
 *   d f_ij/dt = -(F_{i+1/2,j} - F_{i-1/2,j})/dx_i - (H_{i,j+1/2} - H_{i,j-1/2})/dy,
 * F the x-flux of cs_transport on row j, H the second-order upwind y-flux
 * (v2 times the minmod-limited upwind face value).  ny = 1 is the 1-D
 * problem. */
typedef struct {
    const double *dx;    /* device, [nx] cell widths across x */
    const double *f_far; /* device, [N^3] far-field distribution (x end), used for v1 < 0 */
    double wall_T;       /* wall temperature T_w > 0 */
    double wall_V[3];    /* wall velocity V_w */
    int ny;              /* cells across the periodic y direction, >= 1 */
    double dy;           /* their width, > 0 */
} cs_domain2d;

/* One Heun step of length dt of the 2-D transport, in place.
 *   f (device, in/out) [nx][ny][N^3].  nx >= 2.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_transport2d(cs_handle_t h, double *f, int nx, const cs_domain2d *dom, double dt,
                   cudaStream_t stream);

/* nsteps Strang-split steps with the 2-D transport: transport dt/2,
 * collision dt (Heun on P_N Qt / eps, every cell), transport dt/2, in place;
 * captured once as a CUDA graph and replayed like cs_step.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_step2d(cs_handle_t h, double *f, int nx, const cs_domain2d *dom, double dt, double eps,
              int nsteps, cudaStream_t stream);

/* Transport in three space dimensions (Sec. 3.4): x is the wall-normal
 * direction of the 1-D problem (cells of width dx, diffusely reflecting wall
 * at x = 0, far-field gas at the end), y and z periodic directions of ny and
 * nz cells of uniform widths dy and dz.  The state is [nx][ny][nz][N^3]
 * (cell (i, j, l) at index (i ny + j) nz + l).  A stage adds the flux
 * differences of all three directions (no splitting):
 *   d f/dt = -(F_{i+1/2} - F_{i-1/2})/dx_i - (H_{j+1/2} - H_{j-1/2})/dy
 *            - (K_{l+1/2} - K_{l-1/2})/dz,
 * F the x-flux of cs_transport on each x-row, H and K the second-order upwind
 * fluxes with velocity components v2 and v3.  nz = 1 is the 2-D problem of
 * cs_transport2d (bit for bit). */
typedef struct {
    const double *dx;    /* device, [nx] cell widths across x */
    const double *f_far; /* device, [N^3] far-field distribution (x end), used for v1 < 0 */
    double wall_T;       /* wall temperature T_w > 0 */
    double wall_V[3];    /* wall velocity V_w */
    int ny;              /* cells across the periodic y direction, >= 1 */
    double dy;           /* their width, > 0 */
    int nz;              /* cells across the periodic z direction, >= 1 (ny * nz <= 65535) */
    double dz;           /* their width, > 0 */
} cs_domain3d;

/* One Heun step of length dt of the 3-D transport, in place.
 *   f (device, in/out) [nx][ny][nz][N^3].  nx >= 2.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_transport3d(cs_handle_t h, double *f, int nx, const cs_domain3d *dom, double dt, cudaStream_t stream);

/* nsteps Strang-split steps with the 3-D transport: transport dt/2,
 * collision dt (Heun on P_N Qt / eps, every cell), transport dt/2, in place;
 * captured once as a CUDA graph and replayed like cs_step.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_step3d(cs_handle_t h, double *f, int nx, const cs_domain3d *dom, double dt, double eps, int nsteps,
              cudaStream_t stream);

/* Sharded transport (Sec. 4.2, distributed memory): the x-grid of
 * total_cells cells is split into contiguous shards, one per process (or
 * several per process); the collision step is local to each cell, and the
 * transport of a shard needs two ghost cells per side, filled by the caller
 * from the neighbouring shards before every stage.  A shard's state lives in
 * a window of ncells + 4 cells: window cell i is grid cell first_cell - 2 + i
 * (cells 0, 1 and ncells+2, ncells+3 are the ghosts).  Ghosts that fall
 * outside the grid are never read: the wall and far-end boundaries of
 * cs_transport apply there.  A stage computes every face exactly as the
 * unsharded grid does, so shards reproduce cs_transport bit for bit.
 *
 * cs_transport_shard_prepare computes the handle's transport tables (cell
 * geometry of the whole grid, wall Maxwellian) and makes room for a shard of
 * ncells cells; it must precede the stages, and again after any
 * cs_transport / cs_step call on the same handle (which overwrite the
 * tables).  dom->dx has total_cells entries.  ncells >= 2,
 * 0 <= first_cell <= total_cells - ncells.
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_transport_shard_prepare(cs_handle_t h, int ncells, int first_cell, int total_cells,
                               const cs_domain *dom, cudaStream_t stream);

/* One Runge-Kutta stage of the transport on a shard:
 *   out = a x + b y + c R(f),  R_j = -(F_{j+1/2} - F_{j-1/2}) / dx_j,
 * for the shard's cells, F the fluxes of cs_transport (Sec. 3.4).
 *   f_win (device) [ncells + 4][N^3] the window, ghosts filled.
 *   x, y  (device, may be NULL: term dropped) [ncells][N^3].
 *   out   (device) [ncells][N^3]; may alias x or y, must not overlap f_win.
 * A Heun step of length dt is two stages: f1 = f + dt R(f), then, after the
 * ghosts of f1 are exchanged, f = f/2 + f1/2 + (dt/2) R(f1).
 * Errors: CS_EINVAL (also when the tables were not prepared for this
 * total_cells, dx and wall), CS_ECUDA. */
int cs_transport_shard_stage(cs_handle_t h, const double *f_win, int ncells, int first_cell,
                             int total_cells, const cs_domain *dom, double a, const double *x,
                             double b, const double *y, double c, double *out,
                             cudaStream_t stream);

/* nsteps Strang-split steps (Sec. 3.1): transport dt/2, collision dt (Heun on
 * P_N Qt / eps), transport dt/2, in place.  f (device, in/out) [ncells][N^3].
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_step(cs_handle_t h, double *f, int ncells, const cs_domain *dom, double dt, double eps,
            int nsteps, cudaStream_t stream);

/* cs_collide without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc -- code running inside
 * another runtime's host callback or plugin that owns every allocation, a
 * real-time loop that must not block on the allocator, a process whose
 * device memory is budgeted up front.  cs_collide may grow the handle's
 * workspace with cudaMalloc; this call keeps its intermediate arrays in one
 * 64 MiB array compiled into the library instead, and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   Arguments, layouts and results are those of cs_collide (same kernels).
 *   Size limit: the three spectral intermediates must fit in 64 MiB, i.e.
 *   at most 64 cells at N = 32 in CS_FP32 (32 split four ways), 32 cells at
 *   N = 32 in CS_FP64, 672 cells at N = 16 in CS_FP32 (384 split four ways);
 *   larger ncells returns CS_EINVAL and a message with the limit for the
 *   handle's N, precision and split.
 *   Every GPU that loads the library holds the 64 MiB array until the
 *   process exits.  All calls on a device share it and it keeps the last
 *   call's contents (each call writes every element it later reads, so
 *   nothing needs clearing); calls whose GPU work overlaps in time -- on two
 *   streams, or from two host threads without ordering -- race on it and
 *   return wrong results.  Order them on one stream or with events.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before capturing the stream into a CUDA graph.
 * Errors: CS_EINVAL, CS_ENOTSUP, CS_ECUDA. */
int cs_collide_noalloc(cs_handle_t h, const double *f, int ncells, double eps, double *Q, int conserve,
                       cudaStream_t stream);

/* Launch choices of the convolution (autotuner parameters).
 *   CS_TUNE_SPLIT           float handles at N = 16: 2 (default, 0 = 2) or 4
 *                           tile ranges per output pencil (4 shortens the
 *                           tail of a launch over few cells); at N = 32: 1
 *                           (default, 0 = 1), 2 or 4 (shorter launches over
 *                           one or two cells).  The ranges' partial sums are
 *                           added in a fixed order, so a choice changes the
 *                           rounding of the sum, not its terms, and holds for
 *                           every call on the handle; handles split other
 *                           than 2 ways at N = 16 or whole at N = 32 stay out
 *                           of cs_collide_batched's shared convolution launch
 *   CS_TUNE_GROUPS_PER_CTA  1, 2 or 4 groups of 32 cells share each weight
 *                           tile in shared memory (2 needs an even group
 *                           count; 4 float handles at N = 32 with stored
 *                           tiles and a group count divisible by 4, else 2;
 *                           0: 2 where the count is even at N <= 32, else 1)
 *   CS_TUNE_CTAS_PER_SM     resident CTAs per SM of the persistent kernel
 *                           (capped by what fits)
 *   CS_TUNE_WEIGHTS         1: read the stored weight tiles; 2: rebuild each
 *                           tile from the radius tables (float strip handles;
 *                           results agree to float rounding of the weights)
 *   CS_TUNE_L2_HINT         1: plain copies; 2 (default, 0 = 2): the
 *                           convolution's tile copies carry L2 eviction
 *                           priorities (the weight tiles, streamed once per
 *                           launch, evict first; the f-hat rows, read again by
 *                           every pencil that needs them, evict last): at
 *                           N = 32, 256 cells and one group per CTA 2.2 GB of
 *                           DRAM reads per launch instead of 3.1 GB in the
 *                           same time; 3: the weight
 *                           tiles' priority only; 4: the rows' only; changes
 *                           traffic, not results
 *   CS_TUNE_TILE            float handles at N = 16 and 32 with stored tiles:
 *                           the xi-tile and the ring depth, 1 (default, 0 =
 *                           1): blocks of 8 uniform rows, 3 stages (2 for two
 *                           groups per CTA at N = 32); 2: blocks of 4 rows;
 *                           3: 4 stages; 4: 2 stages.  Every output
 *                           adds its terms in the same order in all of them
 *                           (results bit for bit equal); cs_autotune times
 *                           them at the best launch shape
 *   CS_TUNE_FEW_CELLS       float handles at N = 24 and 32 with stored tiles:
 *                           the most cells a convolution launch gives to the
 *                           few-cell kernel (one warp per cell, a pencil's
 *                           outputs over its lanes) instead of the strip
 *                           kernels; 0 (default): 6 at N = 32, 9 at N = 24,
 *                           where it stops being faster; 1 .. 16 that many;
 *                           -1 never.  Both kernels add every output's terms
 *                           in the same order (results bit for bit equal)
 * Settings of the handle's checks and of its Heun steps (no counterpart in
 * the paper; failure detection and test plumbing):
 *   CS_TUNE_WAIT_US         limit of every bounded device-side wait of the
 *                           convolution, in microseconds (1 .. 10^7; 0 = the
 *                           default of 2 s).  A wait that runs out makes the
 *                           kernel record the expiry, wait (at most 0.1 s, a
 *                           limit this setting does not change) for the copies
 *                           it issued, and return; cs_status then reports
 *                           CS_ETIMEOUT
 *   CS_TUNE_TEST_STALL      1: in every convolution launch of the handle the
 *                           first CTA issues no copy for its first work item,
 *                           so its waits run out after CS_TUNE_WAIT_US (the
 *                           way a test makes the timeout path run without
 *                           faulting or hanging the GPU); 0 (default): off.
 *                           The results of such a launch are invalid
 *   CS_TUNE_CHECK_INPUT     1: every cs_collide, cs_relax, cs_step and
 *                           cs_step2d call (each step of the latter three)
 *                           first scans the distribution it is given on the
 *                           device and records non-finite values; 2: non-finite
 *                           or negative values; 0 (default): no scan.
 *                           cs_status then reports CS_ENONFINITE
 *   CS_TUNE_FORWARD_NEXT    float handles at N <= 24: 1 (default, 0 = 1): the
 *                           inverse launch of a Heun step's first evaluation
 *                           also transforms its result forward for the second
 *                           evaluation; 2: a separate forward launch does it
 *                           (the same values: a test checks both agree bit for
 *                           bit)
 * value 0 restores the automatic choice (stored tiles where the handle has
 * them).  Errors: CS_EINVAL, CS_ENOTSUP (a weight mode the handle lacks). */
#define CS_TUNE_GROUPS_PER_CTA 1
#define CS_TUNE_CTAS_PER_SM 2
#define CS_TUNE_WEIGHTS 3
#define CS_TUNE_SPLIT 4
#define CS_TUNE_WAIT_US 5
#define CS_TUNE_TEST_STALL 6
#define CS_TUNE_CHECK_INPUT 7
#define CS_TUNE_FORWARD_NEXT 8
#define CS_TUNE_L2_HINT 9
#define CS_TUNE_TILE 10
#define CS_TUNE_FEW_CELLS 11
int cs_tune(cs_handle_t h, int param, int value);

/* The current value of a launch choice (0 = automatic).
 *   value (host, out).  Errors: CS_EINVAL. */
int cs_tune_get(cs_handle_t h, int param, int *value);

/* Measured peak of one arithmetic pipe (diagnostics, no counterpart in the
 * paper): kind 0 scalar FP32 fused multiply-adds, 1 packed f32x2 ones (the
 * convolution's instructions), 2 FP64 ones; every SM full of independent
 * chains, best of three timed launches on `stream` (synchronising).
 *   lane_ops_per_s (host, out): lane operations per second (a packed f32x2
 *   instruction counts two).  Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_fma_probe(int kind, cudaStream_t stream, double *lane_ops_per_s);

/* Time the convolution's launch choices on ncells synthetic cells on
 * `stream` (synchronising), keep the fastest in the handle and return its
 * time per launch in *ms (may be NULL).  The choices are the launch shapes
 * (cell groups per CTA, CTAs per SM) times the weight modes the handle has
 * (stored tiles, radius tables): the store-versus-recompute choice of the
 * weights is timed, not assumed; at N = 16 in float it times the two splits
 * as well; then, at the best of those, the tile shapes of CS_TUNE_TILE
 * (N = 16 and 32 with stored tiles).  Uses the workspace (cs_reserve).
 * Errors: CS_EINVAL, CS_ENOMEM, CS_ECUDA. */
int cs_autotune(cs_handle_t h, int ncells, cudaStream_t stream, double *ms);

/* Per-stage timing.  While enabled on a handle, each stage that handle
 * launches is bracketed by two CUDA events recorded on the stream it is
 * launched on; cs_profile_read synchronises on those events and returns the
 * summed device time and the number of bracketed launches per stage.
 * Stage ids (index into the arrays): */
#define CS_K_FORWARD 0   /* step a1: the three transform passes */
#define CS_K_CONVOLVE 1  /* step a2: the convolution kernel */
#define CS_K_INVERSE 2   /* step a3: the three inverse passes */
#define CS_K_CONSERVE 3  /* step a4 (+ the Runge-Kutta combination) */
#define CS_K_TRANSPORT 4 /* one transport stage (wall flux + update) */
#define CS_K_COUNT 5

/* Enable (1) or disable (0) stage timing on h.  Do not enable it while a
 * stream that h launches on is being captured into a CUDA graph.
 * Errors: CS_EINVAL. */
int cs_profile(cs_handle_t h, int enable);

/* total_ms, launches (host, out) [CS_K_COUNT] each (either may be NULL);
 * reset != 0 clears the records.  Blocks until the recorded events complete.
 * Errors: CS_EINVAL, CS_ECUDA. */
int cs_profile_read(cs_handle_t h, double *total_ms, long long *launches, int reset);

/* Kernels this library has put on streams since it was loaded (or since the
 * last reset), over all handles and threads: direct launches count when they
 * are enqueued, a replayed CUDA graph counts its kernel nodes at each replay
 * (launches made while a stream is being captured count only through the
 * replays).  Memset and copy operations are not counted.  The paper has no
 * counterpart; this is measurement plumbing.
 *   kernels (host, out); reset != 0 zeroes the count after reading it.
 * Errors: CS_EINVAL (kernels NULL). */
int cs_launch_count(long long *kernels, int reset);

#ifdef __cplusplus
}
#endif
#endif /* CS_H */
