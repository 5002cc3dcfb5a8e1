// Throughput of the units the sweep runs on: cvo_measure_throughput
// (include/cvo.h).
//
// An addition of this library for roofline reporting; the paper has no
// counterpart.  The sweep is bound by FP32 arithmetic and by one ex2 per
// pair, so its roofline denominators are the device's FP32 fused
// multiply-add rate and its ex2.approx rate.  Counting units (SMs x FP32
// lanes x clock) gives a ceiling the hardware may not reach; these kernels
// measure what it does reach on the GPU at hand, under the clocks it runs at
// when measured.
//
// Each thread runs kChains independent dependency chains (enough to cover
// the pipes' latency at the launched occupancy), kUnroll steps per loop
// trip so that loop control takes a few percent of the issue slots.  The
// FMA chains compute v = v * a + b with |a| < 1 (bounded, finite values);
// the ex2 chains compute v = 2^(-v), which settles near 0.64.  The results
// are kept live by a store that the compiler cannot prove unreachable: both
// chains stay positive (v starts in [0, 0.27]; v * 0.999 + 0.001 stays in
// [0, 1] and 2^(-v) in (0, 1]), so their sum is never -1, and the store
// would go to a one-word array of the library's own in any case.
#include <cuda_runtime.h>

#include "cvo.h"
#include "cvo_internal.cuh"

namespace cvo {
void set_error_message(const char* msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ float g_sink[1];

__global__ void __launch_bounds__(kThreads) k_ffma_rate(int trips, float a, float b)
{
    float v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = 1.0e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(v[k]) : "f"(a), "f"(b));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += v[k];
    if (s == -1.0f) g_sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_ex2_rate(int trips)
{
    float v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = 1.0e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm volatile("{\n\t.reg .f32 t;\n\tneg.f32 t, %0;\n\tex2.approx.ftz.f32 %0, t;\n\t}" : "+f"(v[k]));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += v[k];
    if (s == -1.0f) g_sink[0] = s;
}

// Best of `reps` timed launches (after one untimed launch), in ms.
template <class Launch>
cudaError_t time_best(cudaStream_t s, int reps, Launch&& launch, float* best_ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    cvo::g_launch_count.fetch_add(reps + 1, std::memory_order_relaxed);
    float best = 0.0f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (r == 0 || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *best_ms = best;
    return e;
}

}  // namespace

extern "C" cvo_status cvo_measure_throughput(void* cuda_stream, cvo_throughput* out)
{
    if (out == nullptr) {
        cvo::set_error_message("cvo_measure_throughput: out is NULL");
        return CVO_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = kBlocksPerSm * sms;
    const int ffma_trips = 2048, ex2_trips = 256;
    float ms_f = 0.0f, ms_x = 0.0f;
    if (e == cudaSuccess)
        e = time_best(s, 5, [&]() { k_ffma_rate<<<blocks, kThreads, 0, s>>>(ffma_trips, 0.999f, 1.0e-3f); },
                      &ms_f);
    if (e == cudaSuccess)
        e = time_best(s, 5, [&]() { k_ex2_rate<<<blocks, kThreads, 0, s>>>(ex2_trips); }, &ms_x);
    if (e != cudaSuccess) {
        cvo::set_error_message(cudaGetErrorString(e));
        return CVO_ERR_CUDA;
    }
    const double lanes = (double)blocks * kThreads * kChains * kUnroll;
    out->ffma_flops = ms_f > 0.0f ? 2.0 * lanes * ffma_trips / (ms_f * 1e-3) : 0.0;
    out->ex2_per_s = ms_x > 0.0f ? lanes * ex2_trips / (ms_x * 1e-3) : 0.0;
    out->ms_ffma = ms_f;
    out->ms_ex2 = ms_x;
    out->sms = sms;
    return CVO_OK;
}
