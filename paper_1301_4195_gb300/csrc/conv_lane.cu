// K2 for a few cells (float, N = 24 and 32, stored weight tiles): the
// weighted convolution of Sec. 3.2,
//   Qhat(zeta_k) = dzeta^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m),
// with the outputs of a pencil spread over a warp's lanes instead of its
// cells.
//
// The strip kernel puts one cell on each lane of a warp, so a launch over a
// few cells costs as much as one over 32 (N = 32: 1.4 ms for 1 to 16 cells,
// with two strips per warp).  Here a warp holds ONE cell and lane k3 sums
// output (k1, k2, k3) of the CTA's pencil: per tile it walks the rows m3 in
// increasing order and adds, for each row its output takes, the same packed
// multiply-add on the same weight, f-hat values and accumulator as the strip
// kernel; it folds each m1 slab into the same compensated (hi, lo) pair and
// scales and stores the same way.  Every output is therefore the strip
// kernel's bit for bit (a GPU test checks it), and the two kernels may
// serve the same handle in any mix.  A CTA holds one warp per cell, so the
// weight tiles cross HBM once per launch whatever the cell count.
//
// Cost.  Each lane issues about ten instructions per row it visits (three
// shared loads, the packed multiply-add, the predicate) where the strip
// kernel spreads one row over 32 cells, and each output's sum is one chain
// through all of its pencil's tiles, so a launch lasts at least as long as
// its heaviest pencil takes one warp (at two cells and whole pencils the SMs
// are busy 70 % of the launch).  It wins at few cells only: N = 32 up to 6 cells (one cell
// 0.41 ms against 1.36 ms), N = 24 up to 9 (0.19 against 0.47 ms).
//
// Layout.  f-hat of the few cells is first transposed from the grouped
// layout (32 cells per m, one per lane) into "row-major by cell": for each
// (m1, m2) row the C cells' N values one after another, so one bulk copy
// stages a row of all cells and lane k3 reads partner m3' = k3 + N/2 - m3 of
// its cell from consecutive words (no bank conflicts).  The transpose writes
// into a workspace region of its own (16 cells' f-hat at most); where a
// handle has none (cs_collide_noalloc's view) the strip kernels serve.
//
// Tile split.  With S > 1 (CS_TUNE_SPLIT at N = 32) a work item is one of S
// consecutive ranges of a pencil's tiles, summed into its own partial buffer
// and added in range order by the last range to finish, the strip kernel's
// cut and order, so the two kernels stay bit-identical; the shorter items
// shorten the launch at one or two cells, which the heaviest pencils set
// (N = 32, one cell: 0.43 ms whole, 0.30 ms in two ranges, SMs busy 95 %).
//
// Per lane the tile offsets of its weights (the STRIP layout of its strip,
// see cs_internal.cuh) are fixed for the whole launch and sit in registers,
// with a mask of the rows the lane takes.  Waits, the error word, the abort
// path and the test stall are the strip kernel's.
#include <algorithm>

#include "strip.cuh"

namespace cs {

namespace {

constexpr int kLaneMaxCells = 16;  // cells of one launch (one warp each)

// most cells it serves unless the handle says otherwise: where it stops
// beating the strip kernels (measured, one cell per warp against two strips
// per warp: N = 32 1 cell 0.41 / 1.36 ms, 4 cells 0.83 / 1.36, 8 cells 1.56 /
// 1.36; N = 24 1 cell 0.19 / 0.47, 8 cells 0.35 / 0.47, 12 cells 0.60 / 0.47)
constexpr int lane_default(int N) { return N == 32 ? 6 : 9; }

struct LaneJob {
    const float *ghat;
    const int *tile0, *order;
    const float2 *Fc;              // f-hat, row-major by cell: [(m1 N + m2) C + c] N + m3
    float2 *Qh, *Qh2, *Qh3, *Qh4;  // grouped layout, as the strip kernel writes them (partial sums of S ranges)
    int *done;                     // S > 1: finished ranges per pencil, zero at the launch
    int S;
    int *err;
    float omega;
    int ncells;
    unsigned wait_us;
    int stall;
    int l2hint;
};

template <int N>
struct LaneCfg {
    static constexpr int H = N / 2;
    static constexpr int K = strip_width(N);
    static constexpr int TSV = strip_stride(N, K);
    static constexpr uint32_t GB = TSV * sizeof(float);
    static constexpr uint32_t rowb(int C) { return (uint32_t)(C * N * sizeof(float2)); }
    static constexpr uint32_t stage(int C) { return (2 * rowb(C) + GB + 127) / 128 * 128; }
    // ring depth: four stages (measured at N = 32: one cell 0.41 ms with 4,
    // 0.46 ms with 11 and 0.48 ms with 7; deeper rings only left fewer CTAs
    // per SM)
    __host__ __device__ static constexpr int nst(int) { return 4; }
    static constexpr size_t smem(int C) { return kRingHead + (size_t)nst(C) * stage(C); }
};

// grouped f-hat (cells 0 .. C-1 of group 0) -> row-major by cell; one block
// per (m1, m2) row, N C threads, through shared memory so both sides coalesce
template <int N>
__global__ void lane_transpose_kernel(const float2 *__restrict__ F, int C, float2 *__restrict__ Fc)
{
    __shared__ float2 s[N * kLaneMaxCells];
    const int r = blockIdx.x, t = threadIdx.x;
    if (t < N * C) {
        const int m3 = t / C, c = t % C;
        s[m3 * C + c] = F[((size_t)r * N + m3) * kGroup + c];
    }
    __syncthreads();
    if (t < N * C) {
        const int c = t / N, m3 = t % N;
        Fc[((size_t)r * C + c) * N + m3] = s[m3 * C + c];
    }
}

// weight offset of (output k3, row m3) inside a tile, or -1 where the pair is
// not in the tile (the row takes no partner for this output)
template <int N>
__device__ int lane_weight_offset(int k3, int m3)
{
    using L = LaneCfg<N>;
    constexpr int K = L::K, H = L::H;
    const int w = k3 / K, j = k3 % K, k0 = w * K;
    const int seg = strip_seg_off(N, K, w), lu = strip_lu(N, K, w);
    if (k0 < H) {  // kind A: uniform rows 0 .. k0+H, triangle t = 1 .. K-1 for j >= t
        if (m3 < lu) return seg + m3 * K + j;
        const int t = m3 - (k0 + H);
        if (t < 1 || t > j) return -1;
        return seg + lu * K + strip_tri_a_off(K, t) + j - t;
    }
    // kind B: triangle t = 0 .. K-2 (m3 = k0-H+1+t) for j <= t, then uniform rows
    const int t = m3 - (k0 - H + 1);
    if (t < 0) return -1;
    if (t < K - 1) return j <= t ? seg + strip_tri_b_off(t) + j : -1;
    const int i = m3 - (k0 + K - H);
    return seg + strip_round4(strip_tri(K)) + i * K + j;
}

template <int N>
__global__ void __launch_bounds__(32 * kLaneMaxCells, 1) conv_lane_kernel(LaneJob jb, int *counter)
{
    using L = LaneCfg<N>;
    constexpr int H = L::H;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    const int C = jb.ncells, nwarps = blockDim.x >> 5;
    const int warp_id = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ROWB = L::rowb(C), STAGE = L::stage(C);
    const int NST = L::nst(C);

    // ring head: NST full and NST empty barriers, the abort word
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + NST;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NST);
    unsigned char *stages = smem + kRingHead;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nwarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // this lane's weight offsets, row by row, and the rows it takes (bit m3),
    // fixed for every tile
    const int k3 = lane < N ? lane : N - 1;
    int off[N];
    unsigned takes = 0;
#pragma unroll
    for (int m3 = 0; m3 < N; ++m3) {
        const int o = lane < N ? lane_weight_offset<N>(k3, m3) : -1;
        off[m3] = o < 0 ? 0 : o;
        takes |= (o >= 0 ? 1u : 0u) << m3;
    }

    const int S = jb.S;
    const int nitems = N * N * S;
    uint32_t tt = 0, issued = 0;  // ring uses consumed before the current item; uses issued (thread 0)
    bool ok = true;
    for (;;) {
        if (threadIdx.x == 0) s_item = *abort_flag ? nitems : atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;

        // a pencil, or with S > 1 the part-th of S consecutive ranges of its
        // tiles, exactly as the strip kernel cuts them
        const int part = item % S, rest = item / S;
        const int pencil = jb.order[rest];
        const int k1 = pencil / N, k2 = pencil % N;
        const int K1 = k1 + H, K2 = k2 + H;
        const int lo1 = max(0, K1 - N + 1);
        const int lo2 = max(0, K2 - N + 1), hi2 = min(N - 1, K2);
        const int Tall = jb.tile0[pencil + 1] - jb.tile0[pencil];
        const int tb = (part * Tall + S - 1) / S, te = ((part + 1) * Tall + S - 1) / S;
        const int T = te - tb;
        const float *Gp = jb.ghat + (size_t)(jb.tile0[pencil] + tb) * L::TSV;
        float2 *Qout = part == 0 ? jb.Qh : part == 1 ? jb.Qh2 : part == 2 ? jb.Qh3 : jb.Qh4;

        TileWalk pw;  // producer's walk (thread 0), NST tiles ahead
        int pt = 0;
        auto issue_next = [&]() -> bool {
            const uint32_t u = tt + pt;
            const int s = u % NST;
            if (u >= (uint32_t)NST && !wait_phase(&empty[s], ((u / NST) + 1) & 1u, abort_flag, jb.err, jb.wait_us))
                return false;
            unsigned char *st = stages + s * STAGE;
            mbar_arrive_expect_tx(&full[s], 2 * ROWB + L::GB);
            const float2 *ra = jb.Fc + (size_t)(pw.m1 * N + pw.m2) * C * N;
            const float2 *rb = jb.Fc + (size_t)((K1 - pw.m1) * N + (K2 - pw.m2)) * C * N;
            if (jb.l2hint & 2) {
                const uint64_t pol = l2_policy_evict_last();
                bulk_copy_hint(st, ra, ROWB, &full[s], pol);
                bulk_copy_hint(st + ROWB, rb, ROWB, &full[s], pol);
            } else {
                bulk_copy(st, ra, ROWB, &full[s]);
                bulk_copy(st + ROWB, rb, ROWB, &full[s]);
            }
            if (jb.l2hint & 1)
                bulk_copy_hint(st + 2 * ROWB, Gp + (size_t)pt * L::TSV, L::GB, &full[s], l2_policy_evict_first());
            else
                bulk_copy(st + 2 * ROWB, Gp + (size_t)pt * L::TSV, L::GB, &full[s]);
            ++pt;
            ++issued;
            pw.next();
            return true;
        };
        const bool stalled = jb.stall && blockIdx.x == 0 && tt == 0;  // the test stall
        if (threadIdx.x == 0 && !stalled) {
            pw.start(lo1, lo2, hi2, K1, K2);
            for (int i = 0; i < tb; ++i) pw.next();
            while (pt < NST && pt < T)
                if (!issue_next()) {
                    ok = false;
                    break;
                }
        }

        float2 acc = make_float2(0.f, 0.f), hi = acc, lo = acc;
        TileWalk cw;
        cw.start(lo1, lo2, hi2, K1, K2);
        for (int i = 0; i < tb; ++i) cw.next();
        int cur_m1 = cw.m1;
        for (int t = 0; t < T && ok; ++t) {
            const uint32_t u = tt + t;
            const int s = u % NST;
            if (!wait_phase(&full[s], (u / NST) & 1u, abort_flag, jb.err, jb.wait_us)) {
                ok = false;
                break;
            }
            if (cw.m1 != cur_m1) {  // new m1 slab: fold the finished one
                two_sum(hi.x, lo.x, acc.x);
                two_sum(hi.y, lo.y, acc.y);
                acc = make_float2(0.f, 0.f);
                cur_m1 = cw.m1;
            }
            const unsigned char *st = stages + s * STAGE;
            const float2 *arow = reinterpret_cast<const float2 *>(st) + warp_id * N;
            const float2 *brow = reinterpret_cast<const float2 *>(st + ROWB) + warp_id * N + k3 + H;
            const float *gt = reinterpret_cast<const float *>(st + 2 * ROWB);
            // the loads of a row the lane does not take stay inside this
            // stage (the partner index runs at most N/2 - 1 values past the
            // cell's row, into the a rows below or the weights above)
#pragma unroll
            for (int m3 = 0; m3 < N; ++m3) {
                const float2 a = arow[m3];
                const float2 b = brow[-m3];
                const float2 gg = wpair(gt, off[m3]);
                if ((takes >> m3) & 1u) cmad2(acc, gg, dup_x(a), dup_y(a), b, rot_i(b));
            }
            cw.next();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (threadIdx.x == 0 && pt < T && !stalled)
                if (!issue_next()) ok = false;
            __syncwarp();
        }
        if (__syncthreads_or(!ok || *abort_flag)) {
            ok = false;
            break;
        }
        two_sum(hi.x, lo.x, acc.x);
        two_sum(hi.y, lo.y, acc.y);
        const size_t qi = ((size_t)pencil * N + k3) * kGroup + warp_id;
        if (lane < N && warp_id < C) {
            const float2 v = make_float2(hi.x + lo.x, hi.y + lo.y);
            Qout[qi] = make_float2(jb.omega * v.x, jb.omega * v.y);
        }
        tt += T;
        if (S > 1) {
            // the last of a pencil's S ranges adds the partial sums into Qh in
            // range order, as the strip kernel does (same release / acquire
            // count, same order of additions, loads that bypass L1)
            __shared__ int s_last;
            __syncthreads();
            if (threadIdx.x == 0) {
                int old;
                asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], 1;" : "=r"(old) : "l"(jb.done + rest) : "memory");
                s_last = old == S - 1;
            }
            __syncthreads();
            if (s_last && lane < N && warp_id < C) {
                const float2 *more[3] = {jb.Qh2, jb.Qh3, jb.Qh4};
                float2 v = __ldcg(jb.Qh + qi);
                for (int m = 0; m < S - 1; ++m) {
                    const float2 w = __ldcg(more[m] + qi);
                    v = make_float2(v.x + w.x, v.y + w.y);
                }
                jb.Qh[qi] = v;
            }
        }
    }
    // after an abort: the copies thread 0 issued get a bounded time to land
    if (threadIdx.x == 0 && (!ok || *abort_flag)) {
        const uint32_t from = issued > tt + NST ? issued - NST : tt;
        for (uint32_t u = from; u < issued; ++u) {
            volatile int dummy = 0;
            wait_phase(&full[u % NST], (u / NST) & 1u, &dummy, jb.err, kWaitUs / 20);
        }
    }
}

template <int N>
int launch_lane_n(const Handle &hd, int ncells, cudaStream_t s)
{
    using L = LaneCfg<N>;
    static_assert(2 * L::nst(1) * sizeof(uint64_t) + sizeof(int) <= kRingHead, "ring head");
    auto kern = conv_lane_kernel<N>;
    const size_t smem = L::smem(ncells);  // 45 KB at most (16 cells at N = 32)
    static_assert(L::smem(kLaneMaxCells) <= 48 * 1024, "the few-cell kernel needs no shared-memory opt-in");
    const int threads = 32 * ncells;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hd.device);
    const int grid = std::min(N * N, std::max(1, sms) * occ);
    float2 *Fc = (float2 *)hd.Fc;
    const int S = conv_split(hd);
    lane_transpose_kernel<N><<<N * N, N * ncells, 0, s>>>((const float2 *)hd.F, ncells, Fc);
    CS_LAUNCHED(1, s, "few-cell convolution: f-hat by cell");
    cudaError_t e = cudaMemsetAsync(hd.counter, 0, sizeof(int), s);
    if (e == cudaSuccess && S > 1) e = cudaMemsetAsync(hd.done, 0, sizeof(int) * N * N, s);
    if (e != cudaSuccess) return cuda_error(e, "few-cell kernel work counters");
    LaneJob jb{(const float *)hd.ghat,
               hd.pencil_tile0,
               hd.pencil_order,
               Fc,
               (float2 *)hd.Qh,
               (float2 *)hd.Qh2,
               (float2 *)hd.Qh3,
               (float2 *)hd.Qh4,
               hd.done,
               S,
               hd.err,
               (float)(hd.g.dz * hd.g.dz * hd.g.dz),
               ncells,
               hd.wait_us ? hd.wait_us : kWaitUs,
               hd.test_stall,
               l2_hint_bits(hd.tune_l2)};
    kern<<<grid, threads, smem, s>>>(jb, hd.counter);
    CS_LAUNCHED(1, s, "few-cell convolution (one cell per warp, outputs over lanes)");
    return CS_OK;
}

}  // namespace

bool lane_conv_capable(const Handle &hd)
{
    return hd.precision == CS_FP32 && hd.g.layout == LAYOUT_STRIP && (hd.g.N == 24 || hd.g.N == 32);
}

bool lane_conv_applies(const Handle &hd, int ncells)
{
    const int most = hd.tune_few < 0   ? 0
                     : hd.tune_few > 0 ? std::min(hd.tune_few, kLaneMaxCells)
                                       : lane_default(hd.g.N);
    return lane_conv_capable(hd) && !strip_uses_radius(hd) && hd.Fc != nullptr && ncells >= 1 && ncells <= most;
}

int launch_strip_lane(const Handle &hd, int ncells, cudaStream_t s)
{
    switch (hd.g.N) {
    case 24: return launch_lane_n<24>(hd, ncells, s);
    case 32: return launch_lane_n<32>(hd, ncells, s);
    default: return set_error(CS_ENOTSUP, "few-cell convolution: N = 24 and 32 only");
    }
}

}  // namespace cs
