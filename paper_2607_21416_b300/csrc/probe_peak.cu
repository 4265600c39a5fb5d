// probe_peak.cu -- issue-rate microbenchmarks that give the compositing
// kernels' roofline denominators on the running device: FP32 fused
// multiply-adds and SFU base-2 exponentials per second.  Measurement
// helper only; no step of the rendering method runs here.
#include "gs_common.cuh"

namespace gs {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;   // independent dependency chains per thread

__global__ void __launch_bounds__(kProbeThreads) probe_fma_kernel(int iters, float *sink)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    const float a = 0.999f, b = 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) probe_ex2_kernel(int iters, float *sink)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = -(threadIdx.x * 1e-4f + c * 0.01f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
            x[c] = -y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

}  // namespace gs

extern "C" int gs_probe_peak(int32_t kind, int32_t blocks, int32_t iters, float *sink, int64_t *ops, void *stream)
{
    if ((kind != 0 && kind != 1) || blocks < 1 || iters < 1 || sink == nullptr || ops == nullptr)
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0) gs::probe_fma_kernel<<<blocks, gs::kProbeThreads, 0, s>>>(iters, sink);
    else gs::probe_ex2_kernel<<<blocks, gs::kProbeThreads, 0, s>>>(iters, sink);
    gs::count_launches(1);
    *ops = (int64_t)blocks * gs::kProbeThreads * iters * gs::kProbeChains;
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
