// Peak probes of the arithmetic pipes the path is bound by (diagnostics, no
// counterpart in the paper): the measured rate of scalar FP32 fused
// multiply-adds, packed f32x2 ones (the convolution's instructions) and FP64
// ones, in lane operations per second, to set beside the rooflines derived
// from unit counts and clocks.  Every thread runs 8 independent chains
// x <- x a + b (a < 1, so nothing overflows) for `iters` rounds; the sum is
// stored only on an impossible value, which keeps the work live.
#include <algorithm>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float *out, int iters, float a, float b)
{
    float s = 0.f;
    if constexpr (KIND == 0) {
        float x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3f + j;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += x[j];
    } else if constexpr (KIND == 1) {
        float2 x[kChains];
        const float2 aa = make_float2(a, a), bb = make_float2(b, b);
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = make_float2(threadIdx.x * 1e-3f + j, j);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], aa, bb);
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
    } else {
        double x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3 + j;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], (double)a, (double)b);
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += (float)x[j];
    }
    if (s == -1.2345e30f) out[0] = s;
}

template <int KIND>
int probe(const int sms, float *out, int iters, cudaStream_t s, double *rate)
{
    const dim3 grid(sms * (2048 / kProbeThreads));
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(CS_ECUDA, "cs_fma_probe: events");
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // the first run warms up
        cudaEventRecord(e0, s);
        fma_probe_kernel<KIND><<<grid, kProbeThreads, 0, s>>>(out, iters, 0.999f, 1e-3f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_error(e, "cs_fma_probe");
    note_kernels(s, 4);
    const double lanes = (KIND == 1 ? 2.0 : 1.0) * kChains * (double)iters * grid.x * kProbeThreads;
    *rate = lanes / (best * 1e-3);
    return CS_OK;
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" int cs_fma_probe(int kind, cudaStream_t stream, double *lane_ops_per_s)
{
    if (kind < 0 || kind > 2) return set_error(CS_EINVAL, "kind must be 0 (FFMA), 1 (FFMA2) or 2 (DFMA)");
    if (!lane_ops_per_s) return set_error(CS_EINVAL, "lane_ops_per_s is NULL");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "cs_fma_probe: device");
    float *out = nullptr;
    e = cudaMalloc(&out, sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CS_ENOMEM, "cs_fma_probe: cudaMalloc");
    }
    int rc;
    if (kind == 0)
        rc = probe<0>(sms, out, 4096, stream, lane_ops_per_s);
    else if (kind == 1)
        rc = probe<1>(sms, out, 2048, stream, lane_ops_per_s);
    else
        rc = probe<2>(sms, out, 64, stream, lane_ops_per_s);
    cudaFree(out);
    return rc;
}
