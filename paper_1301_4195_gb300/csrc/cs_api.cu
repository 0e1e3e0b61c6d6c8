// Host side of the C ABI declared in include/cs.h: argument checks, the
// handle (weights, constants, workspace) and the order of kernel launches for
// each entry point.  No exception crosses the ABI; every failure returns a
// CS_E* code and leaves a message for cs_last_error().
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_kernels{0};

bool is_finite(double x) { return std::isfinite(x); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int check_device_ptr(const void *p, const char *name, bool allow_null = false)
{
    if (p == nullptr) {
        if (allow_null) return CS_OK;
        return set_error(CS_EINVAL, std::string(name) + " is NULL");
    }
    if (((uintptr_t)p & 7u) != 0) return set_error(CS_EINVAL, std::string(name) + " is not 8-byte aligned");
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_EINVAL, std::string(name) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return set_error(CS_EINVAL, std::string(name) + " is not device memory");
    return CS_OK;
}

int check_handle(cs_handle_t h)
{
    if (h == nullptr) return set_error(CS_EINVAL, "handle is NULL");
    return CS_OK;
}

int check_cells(int ncells)
{
    if (ncells < 0) return set_error(CS_EINVAL, "ncells < 0");
    return CS_OK;
}

// Inverse of the symmetric positive definite 5x5 matrix A by Cholesky.
bool spd_inverse5(const double *A, double *inv)
{
    double Lc[25] = {0};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[5 * i + j];
            for (int k = 0; k < j; ++k) s -= Lc[5 * i + k] * Lc[5 * j + k];
            if (i == j) {
                if (!(s > 0)) return false;
                Lc[5 * i + i] = std::sqrt(s);
            } else {
                Lc[5 * i + j] = s / Lc[5 * j + j];
            }
        }
    for (int col = 0; col < 5; ++col) {
        double e[5] = {0, 0, 0, 0, 0}, z[5], x[5];
        e[col] = 1.0;
        for (int i = 0; i < 5; ++i) {
            double s = e[i];
            for (int k = 0; k < i; ++k) s -= Lc[5 * i + k] * z[k];
            z[i] = s / Lc[5 * i + i];
        }
        for (int i = 4; i >= 0; --i) {
            double s = z[i];
            for (int k = i + 1; k < 5; ++k) s -= Lc[5 * k + i] * x[k];
            x[i] = s / Lc[5 * i + i];
        }
        for (int i = 0; i < 5; ++i) inv[5 * i + col] = x[i];
    }
    return true;
}

}  // namespace

void fill_geom(Geom &g, int N, double L, double lambda, int precision)
{
    g.N = N;
    g.h = N / 2;
    g.M = N * N * N;
    g.L = L;
    g.dv = 2.0 * L / N;
    g.dz = M_PI / L;
    g.lambda = lambda;
    g.nleg = 0;  // isotropic unless cs_weights_build_aniso sets moments
    // ROWS layout: rows of a tile (one per m3) padded to a multiple of 4 entries
    g.off[0] = 0;
    g.TS = 0;
    for (int m3 = 0; m3 < N; ++m3) {
        const int w = kmax_of(m3, g.h, N) - kmin_of(m3, g.h) + 1;
        g.TS += w;
        g.off[m3 + 1] = g.off[m3] + ((w + 3) & ~3);
    }
    for (int m3 = N + 1; m3 <= kMaxN; ++m3) g.off[m3] = g.off[N];
    g.K = precision == CS_FP32 ? strip_width(N) : 0;
    if (g.K) {
        g.layout = LAYOUT_STRIP;
        g.TSp = strip_stride(N, g.K);
    } else {
        g.layout = LAYOUT_ROWS;
        g.TSp = g.off[N];
    }
}

void tile_entry_map(const Geom &g, std::vector<int> &map)
{
    const int N = g.N, H = g.h, K = g.K;
    map.assign(g.TSp, -1);
    auto put = [&](int p, int m3, int k3) { map[p] = (m3 << 8) | k3; };
    if (g.layout == LAYOUT_ROWS) {
        for (int m3 = 0; m3 < N; ++m3)
            for (int k3 = kmin_of(m3, H); k3 <= kmax_of(m3, H, N); ++k3) put(g.off[m3] + k3 - kmin_of(m3, H), m3, k3);
        return;
    }
    for (int w = 0; w < N / K; ++w) {
        const int k0 = w * K, base = strip_seg_off(N, K, w), lu = strip_lu(N, K, w);
        if (strip_is_a(N, K, w)) {
            for (int r = 0; r < lu; ++r)
                for (int j = 0; j < K; ++j) put(base + r * K + j, r, k0 + j);
            for (int t = 1; t < K; ++t)
                for (int j = t; j < K; ++j) put(base + lu * K + strip_tri_a_off(K, t) + (j - t), k0 + H + t, k0 + j);
        } else {
            for (int t = 0; t < K - 1; ++t)
                for (int j = 0; j <= t; ++j) put(base + strip_tri_b_off(t) + j, k0 - H + 1 + t, k0 + j);
            const int ub = base + strip_round4(strip_tri(K));
            for (int r = 0; r < lu; ++r)
                for (int j = 0; j < K; ++j) put(ub + r * K + j, k0 + K - H + r, k0 + j);
        }
    }
}

namespace {

size_t spectral_bytes(const Handle &hd, int ncells)
{
    return (size_t)ngroups_of(ncells) * hd.g.M * kGroup * 2 * elem_bytes(hd.precision);
}

// Carve the workspace: F, Qh, X, Y (spectral), Qt, f1 (state), scal
// (transport tables), part5 (projection partials), for a split convolution
// one more spectral buffer (its fourth partial sum) and the counters of
// finished tile ranges per (pencil, block), and for the few-cell kernel the
// f-hat of up to 16 cells in its own layout.
size_t workspace_bytes(const Handle &hd, int ncells, int geo_cells, size_t *offs)
{
    const size_t sb = align_up(spectral_bytes(hd, ncells), 256);
    const size_t st = align_up((size_t)ncells * hd.g.M * sizeof(double), 256);
    const size_t sc = align_up(sizeof(double) * (transport_table_doubles(hd.g.N, geo_cells) + 8), 256);
    const size_t sp = align_up(sizeof(double) * 5 * (size_t)ncells * conserve_parts(hd.g.M), 256);
    size_t o = 0;
    for (int i = 0; i < 4; ++i) {
        if (offs) offs[i] = o;
        o += sb;
    }
    for (int i = 4; i < 6; ++i) {
        if (offs) offs[i] = o;
        o += st;
    }
    if (offs) offs[6] = o;
    o += sc;
    if (offs) offs[7] = o;
    o += sp;
    if (offs) offs[8] = o;
    if (conv_split_max(hd) > 3) o += sb;  // Qh4
    if (offs) offs[9] = o;
    if (conv_split_max(hd) > 1) o += align_up(sizeof(int) * (size_t)hd.g.N * hd.g.N * ngroups_of(ncells), 256);
    if (offs) offs[10] = o;
    if (lane_conv_capable(hd)) o += align_up((size_t)std::min(ncells, 16) * hd.g.M * sizeof(float2), 256);
    return o;
}

void drop_graphs(Handle &hd)
{
    for (auto &g : hd.graphs) cudaGraphExecDestroy(g.exec);
    hd.graphs.clear();
}

// Workspace for ncells cells whose transport tables cover a grid of
// geo_cells cells (a shard of a larger grid; at least ncells).  Grows only.
int ensure_workspace(Handle &hd, int ncells, int geo_cells = 0)
{
    if (geo_cells < ncells) geo_cells = ncells;
    if (ncells <= hd.ws_cells && geo_cells <= hd.ws_geo_cells) return CS_OK;
    if (ncells < hd.ws_cells) ncells = hd.ws_cells;
    if (geo_cells < hd.ws_geo_cells) geo_cells = hd.ws_geo_cells;
    drop_graphs(hd);  // captured steps point into the old workspace
    size_t offs[11];
    const size_t bytes = workspace_bytes(hd, ncells, geo_cells, offs);
    if (hd.ws) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(e, "synchronise before growing the workspace");
        cudaFree(hd.ws);
        hd.ws = nullptr;
        hd.ws_cells = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_ENOMEM, "cudaMalloc of the workspace failed (" + std::to_string(bytes) + " bytes)");
    }
    char *b = (char *)p;
    hd.ws = p;
    hd.ws_bytes = bytes;
    hd.ws_cells = ncells;
    hd.ws_geo_cells = geo_cells;
    hd.shard_tables.total_cells = -1;
    ++hd.ws_generation;
    hd.F = b + offs[0];
    hd.Qh = b + offs[1];
    hd.Qh2 = b + offs[2];  // X and Y: unused by the whole-cell transforms, the only consumers of a split
    hd.Qh3 = b + offs[3];
    hd.Qh4 = conv_split_max(hd) > 3 ? b + offs[8] : nullptr;
    hd.done = conv_split_max(hd) > 1 ? (int *)(b + offs[9]) : nullptr;
    hd.Fc = lane_conv_capable(hd) ? b + offs[10] : nullptr;
    hd.X = b + offs[2];
    hd.Y = b + offs[3];
    hd.Qt = (double *)(b + offs[4]);
    hd.f1 = (double *)(b + offs[5]);
    hd.scal = (double *)(b + offs[6]);
    hd.part5 = (double *)(b + offs[7]);
    return CS_OK;
}

int timed_forward(Handle &hd, const double *f, int ncells, cudaStream_t s)
{
    StageTimer t(hd, CS_K_FORWARD, s);
    return launch_forward(hd, f, ncells, s);
}

int timed_convolve(Handle &hd, int ncells, cudaStream_t s)
{
    StageTimer t(hd, CS_K_CONVOLVE, s);
    return launch_convolve(hd, ncells, s);
}

int timed_inverse(Handle &hd, int ncells, double eps, double *Qt, cudaStream_t s)
{
    StageTimer t(hd, CS_K_INVERSE, s);
    return launch_inverse(hd, ncells, eps, Qt, s);
}

int timed_conserve(Handle &hd, const double *Qt, int ncells, int project, double a, const double *x, double b,
                   const double *y, double c, double *out, double *moments, cudaStream_t s)
{
    StageTimer t(hd, CS_K_CONSERVE, s);
    return launch_conserve(hd, Qt, ncells, project, a, x, b, y, c, out, moments, s);
}

int timed_transport(Handle &hd, const double *fin, int ncells, const cs_domain &dom, double a, const double *x,
                    double b, const double *y, double c, double *out, cudaStream_t s)
{
    StageTimer t(hd, CS_K_TRANSPORT, s);
    return launch_transport_stage(hd, fin, 0, 0, ncells, ncells, dom, a, x, b, y, c, out, s);
}

// One collision evaluation written as out = a x + b y + c P(Qt(f)/eps)
// (P = projection if project): forward transform, convolution, inverse
// transform, projection and combination.  With whole-cell kernels (float,
// N <= 24) the last three steps are one launch, timed as the inverse stage.
// collide_back: the steps after the convolution (hd.Qh -> out)
int collide_back(Handle &hd, int ncells, double eps, int project, double a, const double *x, double b,
                 const double *y, double c, double *out, cudaStream_t s, bool fwd_next = false)
{
    if (fused_available(hd)) {
        StageTimer t(hd, CS_K_INVERSE, s);
        return launch_inverse_project(hd, ncells, eps, project, a, x, b, y, c, out, s, fwd_next ? hd.F : nullptr);
    }
    const bool direct = (x == nullptr && y == nullptr && c == 1.0);
    double *qt = direct ? out : hd.Qt;
    int rc = timed_inverse(hd, ncells, eps, qt, s);
    if (rc) return rc;
    if (!project && direct) return CS_OK;
    return timed_conserve(hd, qt, ncells, project, a, x, b, y, c, out, nullptr, s);
}

// fwd_next: the inverse launch also transforms out forward into hd.F (the
// next evaluation's input); have_F: hd.F already holds f's transform
int collide_combine(Handle &hd, const double *f, int ncells, double eps, int project, double a, const double *x,
                    double b, const double *y, double c, double *out, cudaStream_t s, bool fwd_next = false,
                    bool have_F = false)
{
    int rc = have_F ? CS_OK : timed_forward(hd, f, ncells, s);
    if (rc) return rc;
    rc = timed_convolve(hd, ncells, s);
    if (rc) return rc;
    return collide_back(hd, ncells, eps, project, a, x, b, y, c, out, s, fwd_next);
}

// one Heun step of df/dt = P Qt(f) / eps, in place
// (with whole-cell kernels the first evaluation's inverse launch also
// transforms f1 forward, so the second starts at the convolution)
int heun_collision(Handle &hd, double *f, int ncells, double dt, double eps, cudaStream_t s)
{
    const bool fuse = fused_forward_next(hd);
    int rc = collide_combine(hd, f, ncells, eps, 1, 1.0, f, 0.0, nullptr, dt, hd.f1, s, fuse);
    if (rc) return rc;
    return collide_combine(hd, hd.f1, ncells, eps, 1, 0.5, f, 0.5, hd.f1, 0.5 * dt, f, s, false, fuse);
}

// one Heun step of the transport in two space dimensions, f [nx][ny][N^3]
int heun_transport2d(Handle &hd, double *f, int nx, int ny, double dy, const cs_domain &dom, double dt,
                     cudaStream_t s)
{
    int rc;
    {
        StageTimer t(hd, CS_K_TRANSPORT, s);
        rc = launch_transport_stage2d(hd, f, nx, ny, dy, dom, 1.0, f, 0.0, nullptr, dt, hd.f1, s);
    }
    if (rc) return rc;
    StageTimer t(hd, CS_K_TRANSPORT, s);
    return launch_transport_stage2d(hd, hd.f1, nx, ny, dy, dom, 0.5, f, 0.5, hd.f1, 0.5 * dt, f, s);
}

// one Heun step of the transport in three space dimensions, f [nx][ny][nz][N^3]
int heun_transport3d(Handle &hd, double *f, int nx, int ny, int nz, double dy, double dz, const cs_domain &dom,
                     double dt, cudaStream_t s)
{
    int rc;
    {
        StageTimer t(hd, CS_K_TRANSPORT, s);
        rc = launch_transport_stage3d(hd, f, nx, ny, nz, dy, dz, dom, 1.0, f, 0.0, nullptr, dt, hd.f1, s);
    }
    if (rc) return rc;
    StageTimer t(hd, CS_K_TRANSPORT, s);
    return launch_transport_stage3d(hd, hd.f1, nx, ny, nz, dy, dz, dom, 0.5, f, 0.5, hd.f1, 0.5 * dt, f, s);
}

int heun_transport(Handle &hd, double *f, int ncells, const cs_domain &dom, double dt, cudaStream_t s)
{
    int rc = timed_transport(hd, f, ncells, dom, 1.0, f, 0.0, nullptr, dt, hd.f1, s);
    if (rc) return rc;
    return timed_transport(hd, hd.f1, ncells, dom, 0.5, f, 0.5, hd.f1, 0.5 * dt, f, s);
}

// Run `body` (which enqueues one step on the stream it is given) nsteps times
// on stream s.  Without profiling, the step is captured once into a CUDA graph
// on the handle's private stream, cached under `key` (every pointer and scalar
// the captured kernels read), and replayed; capture problems fall back to
// launching the kernels directly.
template <typename Body>
int run_steps(Handle &hd, Handle::GraphEntry key, int nsteps, cudaStream_t s, Body body)
{
    if (nsteps <= 0) return CS_OK;
    if (hd.prof || !hd.use_graphs) {
        for (int i = 0; i < nsteps; ++i)
            if (int rc = body(s)) return rc;
        return CS_OK;
    }
    cudaGraphExec_t exec = nullptr;
    for (auto &g : hd.graphs)
        if (g.kind == key.kind && g.f == key.f && g.dx == key.dx && g.ffar == key.ffar && g.ncells == key.ncells &&
            g.wall_T == key.wall_T && g.wall_V[0] == key.wall_V[0] && g.wall_V[1] == key.wall_V[1] &&
            g.wall_V[2] == key.wall_V[2] && g.dt == key.dt && g.eps == key.eps && g.ny == key.ny &&
            g.dy == key.dy && g.nz == key.nz && g.dz == key.dz) {
            exec = g.exec;
            key.kernels = g.kernels;
        }
    if (!exec) {
        if (!hd.cap_stream && cudaStreamCreateWithFlags(&hd.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            hd.use_graphs = false;
            return run_steps(hd, key, nsteps, s, body);
        }
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(hd.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        const int rc = ok ? body(hd.cap_stream) : CS_OK;
        if (ok) ok = cudaStreamEndCapture(hd.cap_stream, &graph) == cudaSuccess && rc == CS_OK;
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (ok) key.kernels = graph_kernel_nodes(graph);
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            if (rc != CS_OK) return rc;
            hd.use_graphs = false;  // this build or device cannot capture: launch directly from now on
            return run_steps(hd, key, nsteps, s, body);
        }
        if (hd.graphs.size() >= 16) {
            cudaGraphExecDestroy(hd.graphs.front().exec);
            hd.graphs.erase(hd.graphs.begin());
        }
        key.exec = exec;
        hd.graphs.push_back(key);
    }
    for (int i = 0; i < nsteps; ++i) {
        cudaError_t e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) return cuda_error(e, "replay of a captured step");
        note_replay(key.kernels);
    }
    return CS_OK;
}

int check_domain(const Handle &hd, const cs_domain *dom, int ncells)
{
    if (dom == nullptr) return set_error(CS_EINVAL, "domain is NULL");
    if (ncells < 2) return set_error(CS_EINVAL, "transport needs ncells >= 2");
    if (!(dom->wall_T > 0) || !is_finite(dom->wall_T)) return set_error(CS_EINVAL, "wall_T must be finite and > 0");
    for (int i = 0; i < 3; ++i)
        if (!is_finite(dom->wall_V[i])) return set_error(CS_EINVAL, "wall_V must be finite");
    int rc = check_device_ptr(dom->dx, "domain.dx");
    if (rc) return rc;
    (void)hd;
    return check_device_ptr(dom->f_far, "domain.f_far");
}

}  // namespace

StageTimer::StageTimer(Handle &hd, int k, cudaStream_t s) : hd_(&hd), s_(s), k_(k)
{
    if (!hd.prof) return;
    cudaEvent_t a;
    if (!hd.pool.empty()) {
        a = hd.pool.back();
        hd.pool.pop_back();
    } else if (cudaEventCreate(&a) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (!hd.pool.empty()) {
        b_ = hd.pool.back();
        hd.pool.pop_back();
    } else if (cudaEventCreate(&b_) != cudaSuccess) {
        cudaGetLastError();
        hd.pool.push_back(a);
        b_ = nullptr;
        return;
    }
    cudaEventRecord(a, s);
    hd.recs.push_back({a, b_, k});
}

StageTimer::~StageTimer()
{
    if (b_) cudaEventRecord(b_, s_);
}

int set_error(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    return set_error(CS_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

void note_kernels(cudaStream_t s, int n)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        st = cudaStreamCaptureStatusNone;
    }
    if (st == cudaStreamCaptureStatusNone) g_kernels += n;
}

void note_replay(int kernels) { g_kernels += kernels; }

int graph_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// ---- batched calls (library-wide cache of captured graphs)
namespace {

struct BatchGraph {
    int kind;  // 1 = collision evaluation (cs_collide_batched), 2 = Heun step (cs_relax_batched)
    std::vector<cs_handle_t> handles;
    std::vector<unsigned> generations;
    std::vector<const void *> f, q;
    std::vector<int> ncells;
    double eps, dt;
    int conserve;
    cudaGraphExec_t exec;
    int kernels = 0;  // kernel nodes of the graph
};

std::mutex g_batch_mutex;
std::vector<BatchGraph> g_batch_graphs;
cudaStream_t g_batch_streams[17] = {};  // [0] capture root, [1..] branches

void drop_batch_graphs_of(cs_handle_t h)
{
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (size_t i = 0; i < g_batch_graphs.size();) {
        bool uses = false;
        for (auto x : g_batch_graphs[i].handles) uses |= (x == h);
        if (uses) {
            cudaGraphExecDestroy(g_batch_graphs[i].exec);
            g_batch_graphs.erase(g_batch_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

// One collision evaluation of every entry, written as
//   out_i = a x_i + b y_i + c P(Qt(src_i) / eps)
// (P the projection if project), enqueued on the capture root and one
// branch stream per entry.  With `mixed` the float strip entries' forward
// transforms run on their branches, their convolutions as one persistent
// launch on the root, and their inverse + projection on their branches
// again; every other entry runs its whole evaluation on its branch.
struct EvalSpec {
    const double *src;
    double a;
    const double *x;
    double b;
    const double *y;
    double c;
    double *out;
};

// fwd_next / have_F: as in collide_combine, for the entries whose inverse
// launch can transform forward (fused_forward_next), so each entry runs the
// same kernels as its own cs_relax.
int capture_evaluation(const std::vector<Handle *> &hs, const std::vector<int> &cells,
                       const std::vector<EvalSpec> &sp, bool mixed, double eps, int project, cudaStream_t root,
                       cudaStream_t *br, const std::vector<cudaEvent_t> &ev, bool fwd_next = false,
                       bool have_F = false)
{
    const int n = (int)hs.size();
    auto in_mix = [&](int i) { return mixed && cells[i] > 0 && strip_mixable(*hs[i]); };
    int rc = CS_OK;
    cudaEventRecord(ev[0], root);
    for (int i = 0; i < n && rc == CS_OK; ++i) {
        cudaStreamWaitEvent(br[i], ev[0], 0);
        Handle &hd = *hs[i];
        const bool ffn = fused_forward_next(hd);
        if (in_mix(i)) {
            if (!(have_F && ffn))
                rc = fused_available(hd)
                         ? launch_forward_fused(hd, sp[i].src, cells[i], br[i], strip_mixed_cells(hd, cells[i]))
                         : launch_forward(hd, sp[i].src, cells[i], br[i]);
        } else if (cells[i] > 0) {
            rc = collide_combine(hd, sp[i].src, cells[i], eps, project, sp[i].a, sp[i].x, sp[i].b, sp[i].y, sp[i].c,
                                 sp[i].out, br[i], fwd_next && ffn, have_F && ffn);
        }
        cudaEventRecord(ev[i + 1], br[i]);
        cudaStreamWaitEvent(root, ev[i + 1], 0);
    }
    if (!mixed || rc != CS_OK) return rc;
    std::vector<const Handle *> mh;
    std::vector<int> mc;
    for (int i = 0; i < n; ++i)
        if (in_mix(i)) {
            mh.push_back(hs[i]);
            mc.push_back(cells[i]);
        }
    rc = launch_strip_mixed(mh.data(), mc.data(), (int)mh.size(), root);
    cudaEventRecord(ev[n + 1], root);
    for (int i = 0; i < n && rc == CS_OK; ++i) {
        if (!in_mix(i)) continue;
        cudaStreamWaitEvent(br[i], ev[n + 1], 0);
        rc = collide_back(*hs[i], cells[i], eps, project, sp[i].a, sp[i].x, sp[i].b, sp[i].y, sp[i].c, sp[i].out,
                          br[i], fwd_next && fused_forward_next(*hs[i]));
        cudaEventRecord(ev[n + 2 + i], br[i]);
        cudaStreamWaitEvent(root, ev[n + 2 + i], 0);
    }
    return rc;
}

// Validation, workspace, the graph cache and the replay shared by the
// batched calls.  kind 1: one collision evaluation, f[i] -> q[i]; kind 2:
// Heun steps of df/dt = P Qt(f) / eps on the states f[i] (q unused),
// nsteps replays of one captured step.
int batched_call(int kind, const std::vector<cs_handle_t> &handles, const std::vector<const double *> &f,
                 const std::vector<double *> &q, const std::vector<int> &ncells, double eps, double dt,
                 int conserve, int nsteps, cudaStream_t stream)
{
    const int n = (int)handles.size();
    if (n > 16) return set_error(CS_EINVAL, "at most 16 entries per batched call");
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (kind == 2 && !is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    if (nsteps < 0) return set_error(CS_EINVAL, "nsteps < 0");
    for (int i = 0; i < n; ++i) {
        if (int rc = check_handle(handles[i])) return rc;
        if (int rc = check_cells(ncells[i])) return rc;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return set_error(CS_EINVAL, "each batch entry needs its own handle");
        if (ncells[i] == 0) continue;
        if (int rc = check_device_ptr(f[i], "entry f")) return rc;
        const size_t bytes = (size_t)ncells[i] * handles[i]->h.g.M * sizeof(double);
        if (kind == 1) {
            if (int rc = check_device_ptr(q[i], "entry Q")) return rc;
            if ((const char *)f[i] < (const char *)q[i] + bytes && (const char *)q[i] < (const char *)f[i] + bytes)
                return set_error(CS_EINVAL, "entry f and Q overlap");
        } else {
            for (int j = 0; j < i; ++j) {
                if (ncells[j] == 0) continue;
                const size_t bj = (size_t)ncells[j] * handles[j]->h.g.M * sizeof(double);
                if ((const char *)f[i] < (const char *)f[j] + bj && (const char *)f[j] < (const char *)f[i] + bytes)
                    return set_error(CS_EINVAL, "the states of two entries overlap");
            }
        }
        if (handles[i]->h.prof) return set_error(CS_EINVAL, "stage timing must be off for batched calls");
    }
    if (n == 0 || nsteps == 0) return CS_OK;
    // float strip handles share one persistent convolution launch when the
    // call has two or more of them; their cells are padded to whole CTA groups
    int nmix = 0;
    for (int i = 0; i < n; ++i) nmix += ncells[i] > 0 && strip_mixable(handles[i]->h);
    const bool mixed = nmix >= 2;
    for (int i = 0; i < n; ++i) {
        if (ncells[i] == 0) continue;
        Handle &hd = handles[i]->h;
        const int cells = mixed && strip_mixable(hd) ? strip_mixed_cells(hd, ncells[i]) : ncells[i];
        if (int rc = ensure_workspace(hd, cells)) return rc;
    }
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    cudaGraphExec_t exec = nullptr;
    int kernels_of_exec = 0;
    for (auto &g : g_batch_graphs) {
        if (g.kind != kind || (int)g.handles.size() != n || g.eps != eps || g.conserve != conserve ||
            (kind == 2 && g.dt != dt))
            continue;
        bool same = true;
        for (int i = 0; i < n && same; ++i)
            same = g.handles[i] == handles[i] && g.generations[i] == handles[i]->h.ws_generation && g.f[i] == f[i] &&
                   g.q[i] == (kind == 1 ? (const void *)q[i] : nullptr) && g.ncells[i] == ncells[i];
        if (same) {
            exec = g.exec;
            kernels_of_exec = g.kernels;
        }
    }
    if (!exec) {
        for (int i = 0; i <= n; ++i)
            if (!g_batch_streams[i] &&
                cudaStreamCreateWithFlags(&g_batch_streams[i], cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return set_error(CS_ECUDA, "batched call: stream creation failed");
            }
        cudaStream_t root = g_batch_streams[0];
        const int nev = (kind == 2 ? 2 : 1) * (2 * n + 2);
        std::vector<cudaEvent_t> ev(nev, nullptr);
        for (auto &e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                for (auto x : ev)
                    if (x) cudaEventDestroy(x);
                return set_error(CS_ECUDA, "batched call: event creation failed");
            }
        std::vector<Handle *> hs(n);
        for (int i = 0; i < n; ++i) hs[i] = &handles[i]->h;
        cudaGraph_t graph = nullptr;
        int rc = CS_OK;
        cudaError_t e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int project = conserve ? 1 : 0;
            std::vector<EvalSpec> sp(n);
            if (kind == 1) {
                for (int i = 0; i < n; ++i) sp[i] = EvalSpec{f[i], 0.0, nullptr, 0.0, nullptr, 1.0, q[i]};
                rc = capture_evaluation(hs, ncells, sp, mixed, eps, project, root, g_batch_streams + 1, ev);
            } else {
                // Heun: f1 = f + dt P Q(f); f = f/2 + (f1 + dt P Q(f1))/2, each entry's f1 in its workspace
                std::vector<cudaEvent_t> ev1(ev.begin(), ev.begin() + (2 * n + 2));
                std::vector<cudaEvent_t> ev2(ev.begin() + (2 * n + 2), ev.end());
                for (int i = 0; i < n; ++i) sp[i] = EvalSpec{f[i], 1.0, f[i], 0.0, nullptr, dt, hs[i]->f1};
                rc = capture_evaluation(hs, ncells, sp, mixed, eps, project, root, g_batch_streams + 1, ev1, true);
                for (int i = 0; i < n; ++i)
                    sp[i] = EvalSpec{hs[i]->f1, 0.5, f[i], 0.5, hs[i]->f1, 0.5 * dt, const_cast<double *>(f[i])};
                if (rc == CS_OK)
                    rc = capture_evaluation(hs, ncells, sp, mixed, eps, project, root, g_batch_streams + 1, ev2,
                                            false, true);
            }
            e = cudaStreamEndCapture(root, &graph);
        }
        if (e == cudaSuccess && rc == CS_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        int kernels = 0;
        if (e == cudaSuccess && rc == CS_OK) kernels = graph_kernel_nodes(graph);
        if (graph) cudaGraphDestroy(graph);
        for (auto x : ev) cudaEventDestroy(x);
        if (rc != CS_OK) return rc;
        if (e != cudaSuccess) return cuda_error(e, "batched call: graph capture");
        if (g_batch_graphs.size() >= 16) {
            cudaGraphExecDestroy(g_batch_graphs.front().exec);
            g_batch_graphs.erase(g_batch_graphs.begin());
        }
        BatchGraph bg;
        bg.kind = kind;
        for (int i = 0; i < n; ++i) {
            bg.handles.push_back(handles[i]);
            bg.generations.push_back(handles[i]->h.ws_generation);
            bg.f.push_back(f[i]);
            bg.q.push_back(kind == 1 ? (const void *)q[i] : nullptr);
            bg.ncells.push_back(ncells[i]);
        }
        bg.eps = eps;
        bg.dt = kind == 2 ? dt : 0.0;
        bg.conserve = conserve;
        bg.exec = exec;
        bg.kernels = kernels;
        kernels_of_exec = kernels;
        g_batch_graphs.push_back(bg);
    }
    for (int r = 0; r < (kind == 2 ? nsteps : 1); ++r) {
        cudaError_t e = cudaGraphLaunch(exec, stream);
        if (e != cudaSuccess) return cuda_error(e, "batched call: replay");
        note_replay(kernels_of_exec);
    }
    return CS_OK;
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" {

int cs_collide_batched(const cs_batch_entry *entries, int n, double eps, int conserve, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && !entries)) return set_error(CS_EINVAL, "bad entry list");
    std::vector<cs_handle_t> hs;
    std::vector<const double *> f;
    std::vector<double *> q;
    std::vector<int> nc;
    for (int i = 0; i < n; ++i) {
        hs.push_back(entries[i].handle);
        f.push_back(entries[i].f);
        q.push_back(entries[i].Q);
        nc.push_back(entries[i].ncells);
    }
    return batched_call(1, hs, f, q, nc, eps, 0.0, conserve, 1, stream);
}

int cs_relax_batched(const cs_relax_entry *entries, int n, double dt, double eps, int nsteps, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && !entries)) return set_error(CS_EINVAL, "bad entry list");
    std::vector<cs_handle_t> hs;
    std::vector<const double *> f;
    std::vector<double *> q;
    std::vector<int> nc;
    for (int i = 0; i < n; ++i) {
        hs.push_back(entries[i].handle);
        f.push_back(entries[i].f);
        q.push_back(nullptr);
        nc.push_back(entries[i].ncells);
    }
    return batched_call(2, hs, f, q, nc, eps, dt, 1, nsteps, stream);
}

int cs_launch_count(long long *kernels, int reset)
{
    if (!kernels) return set_error(CS_EINVAL, "kernels is NULL");
    *kernels = reset ? g_kernels.exchange(0) : g_kernels.load();
    return CS_OK;
}


int cs_version(void) { return 100; }

const char *cs_last_error(void) { return g_last_error.c_str(); }

int cs_weights_bytes(int N, int precision, size_t *bytes)
{
    const bool radius_only = (precision & CS_WEIGHTS_RADIUS) != 0;
    precision &= ~CS_WEIGHTS_RADIUS;
    if (N < 4 || N > kMaxN || (N & 1)) return set_error(CS_EINVAL, "N must be even, 4 <= N <= 64");
    if (precision != CS_FP64 && precision != CS_FP32) return set_error(CS_EINVAL, "precision must be CS_FP64 or CS_FP32");
    if (radius_only && !(precision == CS_FP32 && strip_width(N)))
        return set_error(CS_EINVAL, "CS_WEIGHTS_RADIUS needs CS_FP32 and N in {8, 16, 24, 32, 48, 64}");
    if (!bytes) return set_error(CS_EINVAL, "bytes is NULL");
    Geom g{};
    fill_geom(g, N, 1.0, 0.0, precision);
    const long long tiles = count_tiles(N, nullptr);
    size_t b = sizeof(int) * (2 * N * N + 1) + (size_t)N * N * (sizeof(double2) + sizeof(float2));
    if (!radius_only) b += (size_t)tiles * g.TSp * elem_bytes(precision);
    if (g.layout == LAYOUT_STRIP) b += radius_bytes(N);
    *bytes = b;
    return CS_OK;
}

int cs_tile_layout(int N, int precision, int *map, int cap, int *entries)
{
    if (N < 4 || N > kMaxN || (N & 1)) return set_error(CS_EINVAL, "N must be even, 4 <= N <= 64");
    if (precision != CS_FP64 && precision != CS_FP32) return set_error(CS_EINVAL, "precision must be CS_FP64 or CS_FP32");
    Geom g{};
    fill_geom(g, N, 1.0, 0.0, precision);
    if (entries) *entries = g.TSp;
    if (!map) return CS_OK;
    if (cap < g.TSp) return set_error(CS_EINVAL, "map capacity below the tile stride");
    std::vector<int> m;
    tile_entry_map(g, m);
    for (int i = 0; i < g.TSp; ++i) map[i] = m[i];
    return CS_OK;
}

namespace {
int build_handle(int N, double L, double lambda, int precision, const double *moments, int nmom,
                 cudaStream_t stream, cs_handle_t *out);
}

int cs_weights_build(int N, double L, double lambda, int precision, cudaStream_t stream, cs_handle_t *out)
{
    return build_handle(N, L, lambda, precision, nullptr, 0, stream, out);
}

int cs_weights_build_aniso(int N, double L, double lambda, const double *moments, int nmom, int precision,
                           cudaStream_t stream, cs_handle_t *out)
{
    if (!moments || nmom < 1 || nmom > kMaxLeg)
        return set_error(CS_EINVAL, "anisotropic b: 1 to 16 Legendre moments");
    for (int l = 0; l < nmom; ++l)
        if (!is_finite(moments[l])) return set_error(CS_EINVAL, "anisotropic b: moments must be finite");
    if (!(moments[0] > 0)) return set_error(CS_EINVAL, "anisotropic b: moment 0 (int b dsigma) must be > 0");
    if (precision & CS_WEIGHTS_RADIUS)
        return set_error(CS_EINVAL, "anisotropic b: the radius tables describe isotropic weights only");
    return build_handle(N, L, lambda, precision, moments, nmom, stream, out);
}

}  // extern "C"

namespace {

int build_handle(int N, double L, double lambda, int precision, const double *moments, int nmom,
                 cudaStream_t stream, cs_handle_t *out)
{
    const bool radius_only = (precision & CS_WEIGHTS_RADIUS) != 0;
    precision &= ~CS_WEIGHTS_RADIUS;
    if (N < 4 || N > kMaxN || (N & 1)) return set_error(CS_EINVAL, "N must be even, 4 <= N <= 64");
    if (!(L > 0) || !is_finite(L)) return set_error(CS_EINVAL, "L must be finite and > 0");
    if (!(lambda > -3.0 && lambda <= 1.0)) return set_error(CS_EINVAL, "lambda must lie in (-3, 1]");
    if (precision != CS_FP64 && precision != CS_FP32) return set_error(CS_EINVAL, "precision must be CS_FP64 or CS_FP32");
    if (radius_only && !(precision == CS_FP32 && strip_width(N)))
        return set_error(CS_EINVAL, "CS_WEIGHTS_RADIUS needs CS_FP32 and N in {8, 16, 24, 32, 48, 64}");
    if (!out) return set_error(CS_EINVAL, "out is NULL");
    cs_handle_s *hs = new (std::nothrow) cs_handle_s();
    if (!hs) return set_error(CS_ENOMEM, "host allocation of the handle failed");
    Handle &hd = hs->h;
    cudaGetDevice(&hd.device);
    hd.precision = precision;
    hd.has_table = !radius_only;
    fill_geom(hd.g, N, L, lambda, precision);
    hd.g.nleg = nmom;
    for (int l = 0; l < nmom; ++l) hd.g.bl[l] = moments[l];
    // twiddles exp(-i 2 pi ((k-h)(j-h) mod N) / N)
    std::vector<double2> t64(N * N);
    std::vector<float2> t32(N * N);
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j) {
            long r = (long)(k - N / 2) * (long)(j - N / 2) % N;
            if (r < 0) r += N;
            const double ang = 2.0 * M_PI * (double)r / (double)N;
            t64[k * N + j] = make_double2(std::cos(ang), -std::sin(ang));
            t32[k * N + j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
        }
    // (C C^T)^{-1}
    {
        double A[25] = {0};
        const double w = hd.g.dv * hd.g.dv * hd.g.dv;
        for (int j = 0; j < hd.g.M; ++j) {
            const double v1 = hd.g.dv * (j / (N * N) - N / 2);
            const double v2 = hd.g.dv * ((j / N) % N - N / 2);
            const double v3 = hd.g.dv * (j % N - N / 2);
            const double r[5] = {w, w * v1, w * v2, w * v3, w * (v1 * v1 + v2 * v2 + v3 * v3)};
            for (int a = 0; a < 5; ++a)
                for (int b = 0; b < 5; ++b) A[5 * a + b] += r[a] * r[b];
        }
        if (!spd_inverse5(A, hd.cct_inv)) {
            delete hs;
            return set_error(CS_EINVAL, "C C^T is not positive definite");
        }
    }
    cudaError_t e = cudaMalloc(&hd.tw64, sizeof(double2) * N * N);
    if (e == cudaSuccess) e = cudaMalloc(&hd.tw32, sizeof(float2) * N * N);
    if (e == cudaSuccess) e = cudaMalloc(&hd.err, 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(hd.err, 0, 256, stream);
    hd.counter = hd.err ? hd.err + 32 : nullptr;
    if (e != cudaSuccess) {
        cudaGetLastError();
        cs_handle_destroy(hs);
        return set_error(CS_ENOMEM, "cudaMalloc of the twiddle tables failed");
    }
    e = cudaMemcpyAsync(hd.tw64, t64.data(), sizeof(double2) * N * N, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.tw32, t32.data(), sizeof(float2) * N * N, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) {
        const int rc = cuda_error(e, "copy of the twiddle tables");
        cs_handle_destroy(hs);
        return rc;
    }
    int rc = build_weights(hd, stream);
    if (rc == CS_OK && hd.g.layout == LAYOUT_STRIP && hd.g.nleg == 0) rc = build_radius_tables(hd, stream);
    if (rc == CS_OK) {
        // host vectors above must outlive the async copies
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) rc = cuda_error(e, "weight build");
    }
    if (rc != CS_OK) {
        const std::string msg = g_last_error;
        cudaStreamSynchronize(stream);
        cs_handle_destroy(hs);
        return set_error(rc, msg);
    }
    *out = hs;
    return CS_OK;
}

}  // namespace

extern "C" {

int cs_tune(cs_handle_t h, int param, int value)
{
    if (int rc = check_handle(h)) return rc;
    Handle &hd = h->h;
    switch (param) {
    case CS_TUNE_GROUPS_PER_CTA:
        if (value < 0 || value > 4 || value == 3) return set_error(CS_EINVAL, "groups per CTA must be 0, 1, 2 or 4");
        hd.tune_gpc = value;
        break;
    case CS_TUNE_CTAS_PER_SM:
        if (value < 0 || value > 64) return set_error(CS_EINVAL, "CTAs per SM must be in 0..64");
        hd.tune_ctas = value;
        break;
    case CS_TUNE_SPLIT:
        if (value != 0 && value != 2 && value != 4) return set_error(CS_EINVAL, "split must be 0, 2 or 4");
        hd.tune_split = value;
        break;
    case CS_TUNE_WEIGHTS:
        if (value < 0 || value > 2) return set_error(CS_EINVAL, "weights must be 0, 1 (stored) or 2 (radius tables)");
        if (value == 1 && !hd.has_table) return set_error(CS_ENOTSUP, "the handle was built without the stored table");
        if (value == 2 && !hd.radA) return set_error(CS_ENOTSUP, "the handle has no radius tables");
        hd.tune_weights = value;
        break;
    case CS_TUNE_WAIT_US:
        if (value < 0 || value > 10000000) return set_error(CS_EINVAL, "wait limit must be 0 .. 10^7 microseconds");
        hd.wait_us = (unsigned)value;
        break;
    case CS_TUNE_TEST_STALL:
        if (value < 0 || value > 1) return set_error(CS_EINVAL, "test stall must be 0 or 1");
        hd.test_stall = value;
        break;
    case CS_TUNE_CHECK_INPUT:
        if (value < 0 || value > 2) return set_error(CS_EINVAL, "input check must be 0, 1 or 2");
        hd.check_input = value;
        break;
    case CS_TUNE_FORWARD_NEXT:
        if (value < 0 || value > 2) return set_error(CS_EINVAL, "forward-next must be 0, 1 or 2");
        hd.tune_fwd_next = value;
        break;
    case CS_TUNE_L2_HINT:
        if (value < 0 || value > 4) return set_error(CS_EINVAL, "L2 hint must be 0 .. 4");
        hd.tune_l2 = value;
        break;
    case CS_TUNE_TILE:
        if (value < 0 || value > 4) return set_error(CS_EINVAL, "tile shape must be 0 .. 4");
        if (value >= 2 && !tile_shapes_available(hd))
            return set_error(CS_ENOTSUP, "other tile shapes: float handles at N = 16 and 32 with stored tiles");
        hd.tune_tile = value;
        break;
    case CS_TUNE_FEW_CELLS:
        if (value < -1 || value > 16) return set_error(CS_EINVAL, "few-cell limit must be -1 .. 16");
        hd.tune_few = value;
        break;
    default: return set_error(CS_EINVAL, "unknown tuning parameter");
    }
    drop_graphs(hd);  // captured steps and batches hold the old launch configuration
    drop_batch_graphs_of(h);
    return CS_OK;
}

int cs_tune_get(cs_handle_t h, int param, int *value)
{
    if (int rc = check_handle(h)) return rc;
    if (!value) return set_error(CS_EINVAL, "value is NULL");
    switch (param) {
    case CS_TUNE_GROUPS_PER_CTA: *value = h->h.tune_gpc; return CS_OK;
    case CS_TUNE_CTAS_PER_SM: *value = h->h.tune_ctas; return CS_OK;
    case CS_TUNE_WEIGHTS: *value = h->h.tune_weights; return CS_OK;
    case CS_TUNE_SPLIT: *value = h->h.tune_split; return CS_OK;
    case CS_TUNE_WAIT_US: *value = (int)h->h.wait_us; return CS_OK;
    case CS_TUNE_TEST_STALL: *value = h->h.test_stall; return CS_OK;
    case CS_TUNE_CHECK_INPUT: *value = h->h.check_input; return CS_OK;
    case CS_TUNE_FORWARD_NEXT: *value = h->h.tune_fwd_next; return CS_OK;
    case CS_TUNE_L2_HINT: *value = h->h.tune_l2; return CS_OK;
    case CS_TUNE_TILE: *value = h->h.tune_tile; return CS_OK;
    case CS_TUNE_FEW_CELLS: *value = h->h.tune_few; return CS_OK;
    default: return set_error(CS_EINVAL, "unknown tuning parameter");
    }
}

int cs_autotune(cs_handle_t h, int ncells, cudaStream_t s, double *ms)
{
    if (int rc = check_handle(h)) return rc;
    if (ncells < 1) return set_error(CS_EINVAL, "ncells must be >= 1");
    Handle &hd = h->h;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    // spectral input: any finite values exercise the same work
    cudaError_t e = cudaMemsetAsync(hd.F, 0, (size_t)ngroups_of(ncells) * hd.g.M * kGroup * 2 * elem_bytes(hd.precision), s);
    if (e != cudaSuccess) return cuda_error(e, "cs_autotune: input");
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return set_error(CS_ECUDA, "cs_autotune: events");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hd.device);
    const int cand[][2] = {{0, 0}, {1, 0}, {2, 1}, {2, 2}, {2, 3}, {2, 4}, {2, 6}, {1, 2},
                           {1, 3}, {1, 4}, {1, 6}, {1, 8}, {1, 12}, {4, 0}};  // four groups fill an SM alone
    // weight modes to time: the stored tiles and the radius tables, where the handle has both
    std::vector<int> modes;
    if (hd.has_table) modes.push_back(1);
    if (hd.radA) modes.push_back(2);
    if (modes.empty()) modes.push_back(0);
    // and the tile split where the handle has one (float, N = 16: 2 or 4; N = 32: 1, 2 or 4)
    std::vector<int> splits = conv_split_max(hd) == 1 ? std::vector<int>{0}
                              : hd.g.N == 32         ? std::vector<int>{0, 2, 4}
                                                     : std::vector<int>{4, 2};
    const size_t nc = sizeof(cand) / sizeof(cand[0]);
    double best = 1e300;
    int bg = 0, bc = 0, bw = 0, bs = 0, bt = 0;
    const int keep_g = hd.tune_gpc, keep_c = hd.tune_ctas, keep_w = hd.tune_weights, keep_s = hd.tune_split,
              keep_t = hd.tune_tile;
    int rc = CS_OK;
    // the average time of three launches in the current choices (one more first, untimed)
    auto time_it = [&](double *out) -> int {
        int r = launch_convolve(hd, ncells, s);
        if (r != CS_OK) return r;
        cudaEventRecord(a, s);
        for (int k = 0; k < 3 && r == CS_OK; ++k) r = launch_convolve(hd, ncells, s);
        cudaEventRecord(b, s);
        if (r != CS_OK) return r;
        cudaError_t err = cudaEventSynchronize(b);
        float t = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, a, b);
        if (err != cudaSuccess) return cuda_error(err, "cs_autotune: timing");
        *out = t / 3.0;
        return CS_OK;
    };
    // launch shapes x weight modes x splits, with the default tile shape
    struct Timed {
        double t;
        int g, c, w, s;
    };
    std::vector<Timed> timed;
    hd.tune_tile = 0;
    for (size_t ci = 0; ci < splits.size() * modes.size() * nc && rc == CS_OK; ++ci) {
        const auto &c = cand[ci % nc];
        hd.tune_weights = modes[(ci / nc) % modes.size()];
        hd.tune_split = splits[ci / (nc * modes.size())];
        hd.tune_gpc = c[0];
        hd.tune_ctas = c[1];
        double t = 0.0;
        if ((rc = time_it(&t)) != CS_OK) break;
        timed.push_back({t, c[0], c[1], hd.tune_weights, hd.tune_split});
    }
    // The choice: among the shapes within 1 % of the fastest (a gap inside the
    // noise of a few launches), at N = 32 four groups per CTA with whole
    // pencils first, then any whole-pencil shape, then the rest, each class
    // by time.  Four groups read the weight table about 1.7 times fewer
    // (256 cells: 1.49 against 2.50 GB per launch) and a tile split about
    // 0.5 GB more while changing the rounding; the same arithmetic with
    // fewer table reads leaves HBM to whatever runs beside the convolution.
    if (rc == CS_OK && !timed.empty()) {
        double tmin = 1e300;
        for (const auto &x : timed) tmin = std::min(tmin, x.t);
        const bool four_ok = ngroups_of(ncells) % 4 == 0;
        auto rank = [&](const Timed &x) {
            if (hd.g.N != 32) return 0;
            return (x.g == 4 && four_ok && x.s <= 1) ? 0 : x.s <= 1 ? 1 : 2;
        };
        const Timed *pick = nullptr;
        for (const auto &x : timed) {
            if (x.t > 1.01 * tmin) continue;
            if (!pick || rank(x) < rank(*pick) || (rank(x) == rank(*pick) && x.t < pick->t)) pick = &x;
        }
        best = pick->t;
        bg = pick->g;
        bc = pick->c;
        bw = pick->w;
        bs = pick->s;
    }
    // then the tile shapes (xi-tile U, ring depth) at the best of those
    if (rc == CS_OK) {
        hd.tune_gpc = bg;
        hd.tune_ctas = bc;
        hd.tune_weights = bw;
        hd.tune_split = bs;
        if (tile_shapes_available(hd))
            for (int tile = 2; tile <= 4 && rc == CS_OK; ++tile) {
                hd.tune_tile = tile;
                double t = 0.0;
                if ((rc = time_it(&t)) != CS_OK) break;
                if (t < 0.99 * best) {  // another tile shape must win by 1 % too
                    best = t;
                    bt = tile;
                }
            }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != CS_OK) {
        hd.tune_gpc = keep_g;
        hd.tune_ctas = keep_c;
        hd.tune_weights = keep_w;
        hd.tune_split = keep_s;
        hd.tune_tile = keep_t;
        return rc;
    }
    hd.tune_gpc = bg;
    hd.tune_ctas = bc;
    hd.tune_weights = bw;
    hd.tune_split = bs;
    hd.tune_tile = bt;
    drop_graphs(hd);
    drop_batch_graphs_of(h);
    if (ms) *ms = best;
    (void)sms;
    (void)e;
    return CS_OK;
}

int cs_status(cs_handle_t h)
{
    if (int rc = check_handle(h)) return rc;
    Handle &hd = h->h;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "cs_status: synchronise");
    int word = 0;
    e = cudaMemcpy(&word, hd.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(hd.err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "cs_status: read");
    if (word & 1) return set_error(CS_ETIMEOUT, "a bounded wait inside a kernel expired; its results are invalid");
    if (word & 2) return set_error(CS_ENONFINITE, "the input scan found a non-finite value in a distribution");
    if (word & 4) return set_error(CS_ENONFINITE, "the input scan found a negative value in a distribution");
    return CS_OK;
}

int cs_profile(cs_handle_t h, int enable)
{
    if (int rc = check_handle(h)) return rc;
    h->h.prof = enable != 0;
    return CS_OK;
}

int cs_profile_read(cs_handle_t h, double *total_ms, long long *launches, int reset)
{
    if (int rc = check_handle(h)) return rc;
    Handle &hd = h->h;
    double ms[CS_K_COUNT] = {0};
    long long n[CS_K_COUNT] = {0};
    for (const auto &r : hd.recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_error(e, "cs_profile_read");
        ms[r.k] += t;
        n[r.k] += 1;
    }
    if (total_ms)
        for (int i = 0; i < CS_K_COUNT; ++i) total_ms[i] = ms[i];
    if (launches)
        for (int i = 0; i < CS_K_COUNT; ++i) launches[i] = n[i];
    if (reset) {
        for (const auto &r : hd.recs) {
            hd.pool.push_back(r.a);
            hd.pool.push_back(r.b);
        }
        hd.recs.clear();
    }
    return CS_OK;
}

int cs_handle_destroy(cs_handle_t h)
{
    if (!h) return CS_OK;
    drop_batch_graphs_of(h);
    Handle &hd = h->h;
    for (const auto &r : hd.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : hd.pool) cudaEventDestroy(e);
    drop_graphs(hd);
    if (hd.cap_stream) cudaStreamDestroy(hd.cap_stream);
    cudaFree(hd.ghat);
    cudaFree(hd.radA);
    cudaFree(hd.radB);
    cudaFree(hd.emap);
    cudaFree(hd.pencil_tile0);
    cudaFree(hd.pencil_order);
    cudaFree(hd.err);
    cudaFree(hd.tw64);
    cudaFree(hd.tw32);
    cudaFree(hd.ws);
    delete h;
    return CS_OK;
}

int cs_handle_info(cs_handle_t h, int *N, double *L, double *lambda, int *precision, size_t *weight_bytes)
{
    if (int rc = check_handle(h)) return rc;
    const Handle &hd = h->h;
    if (N) *N = hd.g.N;
    if (L) *L = hd.g.L;
    if (lambda) *lambda = hd.g.lambda;
    if (precision) *precision = hd.precision;
    if (weight_bytes)
        *weight_bytes = hd.ghat_bytes + hd.rad_bytes + sizeof(int) * (2 * hd.g.N * hd.g.N + 1) +
                        (size_t)hd.g.N * hd.g.N * (sizeof(double2) + sizeof(float2));
    return CS_OK;
}

int cs_reserve(cs_handle_t h, int ncells)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    return ensure_workspace(h->h, ncells);
}

int cs_weights_sample(cs_handle_t h, const int *km, int n, double *out)
{
    if (int rc = check_handle(h)) return rc;
    if (n < 0 || (n > 0 && (!km || !out))) return set_error(CS_EINVAL, "bad sample arrays");
    const int N = h->h.g.N;
    for (int i = 0; i < 6 * n; ++i)
        if (km[i] < 0 || km[i] >= N) return set_error(CS_EINVAL, "sample index out of range");
    if (n == 0) return CS_OK;
    return sample_weights(h->h, km, n, out);
}

int cs_transform(cs_handle_t h, const double *f, int ncells, double *fhat, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (ncells == 0) return CS_OK;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = check_device_ptr(fhat, "fhat")) return rc;
    Handle &hd = h->h;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    if (int rc = timed_forward(hd, f, ncells, s)) return rc;
    return launch_spectral_to_natural(hd, hd.F, ncells, fhat, s);
}

int cs_convolve(cs_handle_t h, const double *fhat, int ncells, double *qhat, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (ncells == 0) return CS_OK;
    if (int rc = check_device_ptr(fhat, "fhat")) return rc;
    if (int rc = check_device_ptr(qhat, "qhat")) return rc;
    Handle &hd = h->h;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    if (int rc = launch_natural_to_spectral(hd, fhat, ncells, hd.F, s)) return rc;
    if (int rc = timed_convolve(hd, ncells, s)) return rc;
    return launch_spectral_to_natural(hd, hd.Qh, ncells, qhat, s);
}

int cs_inverse(cs_handle_t h, const double *qhat, int ncells, double eps, double *Q, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (ncells == 0) return CS_OK;
    if (int rc = check_device_ptr(qhat, "qhat")) return rc;
    if (int rc = check_device_ptr(Q, "Q")) return rc;
    Handle &hd = h->h;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    if (int rc = launch_natural_to_spectral(hd, qhat, ncells, hd.Qh, s)) return rc;
    StageTimer t(hd, CS_K_INVERSE, s);
    return launch_inverse(hd, ncells, eps, Q, s);  // one given sum, no second part
}

int cs_collide(cs_handle_t h, const double *f, int ncells, double eps, double *Q, int conserve, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (ncells == 0) return CS_OK;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = check_device_ptr(Q, "Q")) return rc;
    Handle &hd = h->h;
    const size_t bytes = (size_t)ncells * hd.g.M * sizeof(double);
    if ((const char *)f < (const char *)Q + bytes && (const char *)Q < (const char *)f + bytes)
        return set_error(CS_EINVAL, "f and Q overlap");
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    if (int rc = launch_input_check(hd, f, (long long)ncells * hd.g.M, s)) return rc;
    return collide_combine(hd, f, ncells, eps, conserve ? 1 : 0, 0.0, nullptr, 0.0, nullptr, 1.0, Q, s);
}

int cs_conserve(cs_handle_t h, double *Q, int ncells, double *moments, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (ncells == 0) return CS_OK;
    if (int rc = check_device_ptr(Q, "Q")) return rc;
    if (int rc = check_device_ptr(moments, "moments", true)) return rc;
    return timed_conserve(h->h, Q, ncells, 1, 0.0, nullptr, 0.0, nullptr, 1.0, Q, moments, s);
}

int cs_moments(cs_handle_t h, const double *f, int ncells, double *out, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (ncells == 0) return CS_OK;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = check_device_ptr(out, "out")) return rc;
    return launch_moments(h->h, f, ncells, out, s);
}

int cs_relax(cs_handle_t h, double *f, int ncells, double dt, double eps, int nsteps, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (nsteps < 0) return set_error(CS_EINVAL, "nsteps < 0");
    if (ncells == 0 || nsteps == 0) return CS_OK;
    if (int rc = check_device_ptr(f, "f")) return rc;
    Handle &hd = h->h;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    Handle::GraphEntry key{2, f, nullptr, nullptr, ncells, 0.0, {0.0, 0.0, 0.0}, dt, eps, nullptr, 0, 1, 0.0};
    return run_steps(hd, key, nsteps, s, [&](cudaStream_t st) {
        if (int rc = launch_input_check(hd, f, (long long)ncells * hd.g.M, st)) return rc;
        return heun_collision(hd, f, ncells, dt, eps, st);
    });
}

int cs_transport(cs_handle_t h, double *f, int ncells, const cs_domain *dom, double dt, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    Handle &hd = h->h;
    if (int rc = check_domain(hd, dom, ncells)) return rc;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    hd.shard_tables.total_cells = -1;
    if (int rc = launch_transport_prep(hd, ncells, *dom, s)) return rc;
    return heun_transport(hd, f, ncells, *dom, dt, s);
}

int cs_step(cs_handle_t h, double *f, int ncells, const cs_domain *dom, double dt, double eps, int nsteps,
            cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (nsteps < 0) return set_error(CS_EINVAL, "nsteps < 0");
    Handle &hd = h->h;
    if (int rc = check_domain(hd, dom, ncells)) return rc;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = ensure_workspace(hd, ncells)) return rc;
    const cs_domain d = *dom;
    hd.shard_tables.total_cells = -1;
    Handle::GraphEntry key{1, f, d.dx, d.f_far, ncells, d.wall_T, {d.wall_V[0], d.wall_V[1], d.wall_V[2]},
                           dt, eps, nullptr, 0, 1, 0.0};
    return run_steps(hd, key, nsteps, s, [&](cudaStream_t st) {
        if (int rc = launch_input_check(hd, f, (long long)ncells * hd.g.M, st)) return rc;
        if (int rc = launch_transport_prep(hd, ncells, d, st)) return rc;
        if (int rc = heun_transport(hd, f, ncells, d, 0.5 * dt, st)) return rc;
        if (int rc = heun_collision(hd, f, ncells, dt, eps, st)) return rc;
        return heun_transport(hd, f, ncells, d, 0.5 * dt, st);
    });
}


int cs_transport_shard_prepare(cs_handle_t h, int ncells, int first_cell, int total_cells, const cs_domain *dom,
                               cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    if (int rc = check_cells(total_cells)) return rc;
    if (ncells < 2 || first_cell < 0 || first_cell > total_cells - ncells)
        return set_error(CS_EINVAL, "shard must hold >= 2 cells inside 0 .. total_cells-1");
    Handle &hd = h->h;
    if (int rc = check_domain(hd, dom, total_cells)) return rc;
    if (int rc = ensure_workspace(hd, ncells, total_cells)) return rc;
    if (int rc = launch_transport_prep(hd, total_cells, *dom, s)) return rc;
    hd.shard_tables.total_cells = total_cells;
    hd.shard_tables.dx = dom->dx;
    hd.shard_tables.wall_T = dom->wall_T;
    for (int i = 0; i < 3; ++i) hd.shard_tables.wall_V[i] = dom->wall_V[i];
    return CS_OK;
}

int cs_transport_shard_stage(cs_handle_t h, const double *f_win, int ncells, int first_cell, int total_cells,
                             const cs_domain *dom, double a, const double *x, double b, const double *y, double c,
                             double *out, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(ncells)) return rc;
    Handle &hd = h->h;
    if (dom == nullptr) return set_error(CS_EINVAL, "domain is NULL");
    const auto &t = hd.shard_tables;
    if (t.total_cells != total_cells || t.dx != dom->dx || t.wall_T != dom->wall_T || t.wall_V[0] != dom->wall_V[0] ||
        t.wall_V[1] != dom->wall_V[1] || t.wall_V[2] != dom->wall_V[2])
        return set_error(CS_EINVAL, "transport tables not prepared for this grid and wall "
                                    "(call cs_transport_shard_prepare first)");
    if (ncells < 2 || first_cell < 0 || first_cell > total_cells - ncells || ncells > hd.ws_cells)
        return set_error(CS_EINVAL, "shard must hold 2 .. reserved cells inside 0 .. total_cells-1");
    if (!is_finite(a) || !is_finite(b) || !is_finite(c)) return set_error(CS_EINVAL, "a, b, c must be finite");
    if (int rc = check_device_ptr(f_win, "f_win")) return rc;
    if (int rc = check_device_ptr(dom->f_far, "domain.f_far")) return rc;
    if (int rc = check_device_ptr(out, "out")) return rc;
    if (int rc = check_device_ptr(x, "x", true)) return rc;
    if (int rc = check_device_ptr(y, "y", true)) return rc;
    const size_t M = hd.g.M;
    const double *o0 = out, *o1 = out + (size_t)ncells * M, *w0 = f_win, *w1 = f_win + (size_t)(ncells + 4) * M;
    if (o0 < w1 && w0 < o1) return set_error(CS_EINVAL, "out overlaps f_win");
    StageTimer tm(hd, CS_K_TRANSPORT, s);
    return launch_transport_stage(hd, f_win, 2, first_cell, ncells, total_cells, *dom, a, x, b, y, c, out, s);
}


// ---- two space dimensions
static int check_domain2d(const Handle &hd, const cs_domain2d *dom, int nx, cs_domain *d1)
{
    if (dom == nullptr) return set_error(CS_EINVAL, "domain is NULL");
    if (dom->ny < 1) return set_error(CS_EINVAL, "ny must be >= 1");
    if (!(dom->dy > 0) || !is_finite(dom->dy)) return set_error(CS_EINVAL, "dy must be finite and > 0");
    if ((long long)nx * dom->ny > (1ll << 30)) return set_error(CS_EINVAL, "too many cells");
    d1->dx = dom->dx;
    d1->f_far = dom->f_far;
    d1->wall_T = dom->wall_T;
    for (int i = 0; i < 3; ++i) d1->wall_V[i] = dom->wall_V[i];
    return check_domain(hd, d1, nx);
}

int cs_transport2d(cs_handle_t h, double *f, int nx, const cs_domain2d *dom, double dt, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(nx)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    Handle &hd = h->h;
    cs_domain d;
    if (int rc = check_domain2d(hd, dom, nx, &d)) return rc;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = ensure_workspace(hd, nx * dom->ny, nx)) return rc;
    hd.shard_tables.total_cells = -1;
    if (int rc = launch_transport_prep(hd, nx, d, s)) return rc;
    return heun_transport2d(hd, f, nx, dom->ny, dom->dy, d, dt, s);
}

int cs_step2d(cs_handle_t h, double *f, int nx, const cs_domain2d *dom, double dt, double eps, int nsteps,
              cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(nx)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (nsteps < 0) return set_error(CS_EINVAL, "nsteps < 0");
    Handle &hd = h->h;
    cs_domain d;
    if (int rc = check_domain2d(hd, dom, nx, &d)) return rc;
    if (int rc = check_device_ptr(f, "f")) return rc;
    const int ny = dom->ny, ncells = nx * ny;
    const double dy = dom->dy;
    if (int rc = ensure_workspace(hd, ncells, nx)) return rc;
    hd.shard_tables.total_cells = -1;
    Handle::GraphEntry key{3, f, d.dx, d.f_far, ncells, d.wall_T, {d.wall_V[0], d.wall_V[1], d.wall_V[2]},
                           dt, eps, nullptr, 0, ny, dy};
    return run_steps(hd, key, nsteps, s, [&](cudaStream_t st) {
        if (int rc = launch_input_check(hd, f, (long long)ncells * hd.g.M, st)) return rc;
        if (int rc = launch_transport_prep(hd, nx, d, st)) return rc;
        if (int rc = heun_transport2d(hd, f, nx, ny, dy, d, 0.5 * dt, st)) return rc;
        if (int rc = heun_collision(hd, f, ncells, dt, eps, st)) return rc;
        return heun_transport2d(hd, f, nx, ny, dy, d, 0.5 * dt, st);
    });
}

// ---- three space dimensions
static int check_domain3d(const Handle &hd, const cs_domain3d *dom, int nx, cs_domain *d1)
{
    if (dom == nullptr) return set_error(CS_EINVAL, "domain is NULL");
    if (dom->ny < 1 || dom->nz < 1) return set_error(CS_EINVAL, "ny and nz must be >= 1");
    if (!(dom->dy > 0) || !is_finite(dom->dy) || !(dom->dz > 0) || !is_finite(dom->dz))
        return set_error(CS_EINVAL, "dy and dz must be finite and > 0");
    if ((long long)dom->ny * dom->nz > 65535) return set_error(CS_EINVAL, "ny * nz must be at most 65535");
    if ((long long)nx * dom->ny * dom->nz > (1ll << 30)) return set_error(CS_EINVAL, "too many cells");
    d1->dx = dom->dx;
    d1->f_far = dom->f_far;
    d1->wall_T = dom->wall_T;
    for (int i = 0; i < 3; ++i) d1->wall_V[i] = dom->wall_V[i];
    return check_domain(hd, d1, nx);
}

int cs_transport3d(cs_handle_t h, double *f, int nx, const cs_domain3d *dom, double dt, cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(nx)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    Handle &hd = h->h;
    cs_domain d;
    if (int rc = check_domain3d(hd, dom, nx, &d)) return rc;
    if (int rc = check_device_ptr(f, "f")) return rc;
    if (int rc = ensure_workspace(hd, nx * dom->ny * dom->nz, nx)) return rc;
    hd.shard_tables.total_cells = -1;
    if (int rc = launch_transport_prep(hd, nx, d, s)) return rc;
    return heun_transport3d(hd, f, nx, dom->ny, dom->nz, dom->dy, dom->dz, d, dt, s);
}

int cs_step3d(cs_handle_t h, double *f, int nx, const cs_domain3d *dom, double dt, double eps, int nsteps,
              cudaStream_t s)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_cells(nx)) return rc;
    if (!is_finite(dt)) return set_error(CS_EINVAL, "dt must be finite");
    if (!(eps > 0) || !is_finite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (nsteps < 0) return set_error(CS_EINVAL, "nsteps < 0");
    Handle &hd = h->h;
    cs_domain d;
    if (int rc = check_domain3d(hd, dom, nx, &d)) return rc;
    if (int rc = check_device_ptr(f, "f")) return rc;
    const int ny = dom->ny, nz = dom->nz, ncells = nx * ny * nz;
    const double dy = dom->dy, dz = dom->dz;
    if (int rc = ensure_workspace(hd, ncells, nx)) return rc;
    hd.shard_tables.total_cells = -1;
    Handle::GraphEntry key{4, f, d.dx, d.f_far, ncells, d.wall_T, {d.wall_V[0], d.wall_V[1], d.wall_V[2]},
                           dt, eps, nullptr, 0, ny, dy, nz, dz};
    return run_steps(hd, key, nsteps, s, [&](cudaStream_t st) {
        if (int rc = launch_input_check(hd, f, (long long)ncells * hd.g.M, st)) return rc;
        if (int rc = launch_transport_prep(hd, nx, d, st)) return rc;
        if (int rc = heun_transport3d(hd, f, nx, ny, nz, dy, dz, d, 0.5 * dt, st)) return rc;
        if (int rc = heun_collision(hd, f, ncells, dt, eps, st)) return rc;
        return heun_transport3d(hd, f, nx, ny, nz, dy, dz, d, 0.5 * dt, st);
    });
}

}  // extern "C"
