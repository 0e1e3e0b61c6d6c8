// cs_collide_noalloc: the collision operator of cs_collide for callers that
// must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is unavailable or
// forbidden -- for example inside a host callback or a plugin of another
// runtime that owns all allocations and hands out only the buffers it
// created, a real-time loop that may not block on the allocator, or a
// process whose memory budget is fixed up front.  cs_collide grows the
// handle's workspace with cudaMalloc on first use; this entry point instead
// keeps the intermediate spectral arrays in one array compiled into the
// library (g_scratch below), so it calls neither cudaMalloc nor cudaFree nor
// any allocating library routine.
//
// Cost of that choice: every GPU that loads this library holds g_scratch
// (kScratchBytes) until the process exits, and every call on a device uses
// the same array, so two calls whose GPU work overlaps (two streams, or two
// host threads without ordering) overwrite each other's intermediates and
// return wrong results.  Order such calls on one stream or with events.
#include <cmath>
#include <mutex>
#include <string>

#include "cs_internal.cuh"

namespace cs {

namespace {

// 64 MiB: at N = 32 this holds the three spectral buffers of two 32-cell
// groups in float (64 cells) or one group in double (32 cells).
constexpr size_t kScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Host code may not use g_scratch's name as an address: on the host it is a
// stand-in object, not device memory.  Ask the runtime for the device address
// once per device, with that device current.
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cs_collide_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(CS_ENOTSUP, "cs_collide_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cs_collide_noalloc: cudaGetSymbolAddress of the scratch array");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CS_OK;
}

// A handle that shares hd's weights and constants but owns no host containers
// (so building it allocates nothing) and points at caller-chosen scratch.
Handle view_of(const Handle &hd)
{
    Handle v;
    v.device = hd.device;
    v.precision = hd.precision;
    v.g = hd.g;
    v.ghat = hd.ghat;
    v.ghat_bytes = hd.ghat_bytes;
    v.total_tiles = hd.total_tiles;
    v.pencil_tile0 = hd.pencil_tile0;
    v.pencil_order = hd.pencil_order;
    v.radA = hd.radA;
    v.radB = hd.radB;
    v.emap = hd.emap;
    v.rad_bb = hd.rad_bb;
    v.has_table = hd.has_table;
    v.tune_weights = hd.tune_weights;
    v.tune_split = hd.tune_split;
    v.tune_gpc = hd.tune_gpc;
    v.tune_ctas = hd.tune_ctas;
    v.wait_us = hd.wait_us;
    v.test_stall = hd.test_stall;
    v.tune_l2 = hd.tune_l2;
    v.tune_tile = hd.tune_tile;
    v.tune_few = hd.tune_few;
    v.err = hd.err;
    v.counter = hd.counter;
    v.tw64 = hd.tw64;
    v.tw32 = hd.tw32;
    for (int i = 0; i < 25; ++i) v.cct_inv[i] = hd.cct_inv[i];
    return v;
}

size_t buffer_bytes(const Handle &hd, int ncells)
{
    const size_t b = (size_t)ngroups_of(ncells) * hd.g.M * kGroup * 2 * elem_bytes(hd.precision);
    return (b + 255) / 256 * 256;
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" int cs_collide_noalloc(cs_handle_t h, const double *f, int ncells, double eps, double *Q, int conserve,
                                  cudaStream_t stream)
{
    if (h == nullptr) return set_error(CS_EINVAL, "handle is NULL");
    if (ncells < 0) return set_error(CS_EINVAL, "ncells < 0");
    if (!(eps > 0) || !std::isfinite(eps)) return set_error(CS_EINVAL, "eps must be finite and > 0");
    if (ncells == 0) return CS_OK;
    if (!f || !Q) return set_error(CS_EINVAL, "f and Q must not be NULL");
    if ((((uintptr_t)f) | ((uintptr_t)Q)) & 7u) return set_error(CS_EINVAL, "f and Q must be 8-byte aligned");
    const Handle &hd = h->h;
    const size_t state = (size_t)ncells * hd.g.M * sizeof(double);
    if ((const char *)f < (const char *)Q + state && (const char *)Q < (const char *)f + state)
        return set_error(CS_EINVAL, "f and Q overlap");
    // three spectral buffers: forward X, Y -> F; convolution F -> Qh (reusing X's
    // space, and Y's for a split's second partial sum, two more buffers for a
    // third and fourth, and the split's counters); inverse Qh -> X', Y'
    // (reusing Y's and F's space); then the per-block partial moments of the
    // projection
    const int split = conv_split(hd);
    const int nbuf = 3 + (split > 2 ? split - 2 : 0);
    const size_t part_bytes = (sizeof(double) * 5 * (size_t)ncells * conserve_parts(hd.g.M) + 255) / 256 * 256;
    const size_t done_bytes =
        split > 1 ? (sizeof(int) * (size_t)hd.g.N * hd.g.N * ngroups_of(ncells) + 255) / 256 * 256 : 0;
    const size_t need = nbuf * buffer_bytes(hd, ncells) + part_bytes + done_bytes;
    if (need > kScratchBytes) {
        const size_t per_group = nbuf * buffer_bytes(hd, 1) + 5 * sizeof(double) * kGroup * conserve_parts(hd.g.M) +
                                 (split > 1 ? sizeof(int) * hd.g.N * hd.g.N : 0);
        return set_error(CS_EINVAL, "cs_collide_noalloc: " + std::to_string(ncells) + " cells need " +
                                        std::to_string(need) + " bytes of scratch; the fixed array holds " +
                                        std::to_string(kScratchBytes) + " (at most " +
                                        std::to_string(kScratchBytes / per_group * kGroup) +
                                        " cells for this N and precision)");
    }
    // Nothing in the array needs clearing: the forward passes write every
    // element of X, Y and F (zeros for the padding cells of the last group),
    // the convolution every element of Qh, the inverse passes (where the
    // handle has no whole-cell inverse) all of X', Y'.
    void *base = nullptr;
    if (int rc = scratch_address(&base)) return rc;
    char *A = (char *)base;
    char *B = A + buffer_bytes(hd, ncells);
    char *C = B + buffer_bytes(hd, ncells);
    char *D = C + buffer_bytes(hd, ncells);  // third and fourth partial sums (nbuf == 5)
    char *E = D + buffer_bytes(hd, ncells);
    // same kernels as cs_collide, pointed at the fixed array
    Handle fwd = view_of(hd);
    fwd.X = A;
    fwd.Y = B;
    fwd.F = C;
    fwd.Qh = A;
    fwd.Qh2 = B;  // a split convolution's further partial sums (Y is free again after the forward passes)
    fwd.Qh3 = nbuf > 3 ? D : nullptr;
    fwd.Qh4 = nbuf > 4 ? E : nullptr;
    fwd.done = split > 1 ? (int *)(C + (nbuf - 2) * buffer_bytes(hd, ncells) + part_bytes) : nullptr;
    Handle inv = view_of(hd);
    inv.Qh = A;

    inv.X = B;
    inv.Y = C;
    inv.part5 = (double *)(C + (nbuf - 2) * buffer_bytes(hd, ncells));
    if (int rc = launch_forward(fwd, f, ncells, stream)) return rc;
    if (int rc = launch_convolve(fwd, ncells, stream)) return rc;
    // the steps after the convolution exactly as cs_collide takes them: the
    // whole-cell inverse with the projection in the same launch where the
    // handle has it (float, N <= 32), else the inverse passes and the
    // projection kernels, so both entry points give the same bits
    if (fused_available(inv))
        return launch_inverse_project(inv, ncells, eps, conserve ? 1 : 0, 0.0, nullptr, 0.0, nullptr, 1.0, Q, stream);
    if (int rc = launch_inverse(inv, ncells, eps, Q, stream)) return rc;
    if (conserve) return launch_conserve(inv, Q, ncells, 1, 0.0, nullptr, 0.0, nullptr, 1.0, Q, nullptr, stream);
    return CS_OK;
}
