// hf_probe.cu -- measured FP32 peak of the GPU, the denominator of the
// FP32 roofline of the reconstruction kernels.
//
// Two throughput kernels: scalar fused multiply-add (fmaf) and the packed
// two-lane form (PTX fma.rn.f32x2, sm_100 and later), each thread running
// 16 independent dependency chains so that neither latency nor occupancy
// limits the issue rate.  A full grid (every SM at its thread limit) runs for
// a fixed number of iterations after a warm-up launch, timed with CUDA events
// on a private stream.  Flops = 2 per lane per fma.
#include <cstdint>
#include <cuda_runtime.h>
#include "hf.h"

namespace {

constexpr int CHAINS = 16;
constexpr int PROBE_BLOCK = 256;

__global__ void __launch_bounds__(PROBE_BLOCK) k_ffma(float* sink, int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1.0e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(PROBE_BLOCK) k_ffma2(float* sink, int iters, float a, float b)
{
    uint64_t x[CHAINS / 2];
#pragma unroll
    for (int c = 0; c < CHAINS / 2; ++c) {
        float2 v = make_float2((float)(threadIdx.x + 2 * c) * 1.0e-3f, (float)(threadIdx.x + 2 * c + 1) * 1.0e-3f);
        x[c] = *reinterpret_cast<uint64_t*>(&v);
    }
    float2 av = make_float2(a, a), bv = make_float2(b, b);
    const uint64_t ra = *reinterpret_cast<uint64_t*>(&av), rb = *reinterpret_cast<uint64_t*>(&bv);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS / 2; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(ra), "l"(rb));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS / 2; ++c) {
        float2 v = *reinterpret_cast<float2*>(&x[c]);
        s += v.x + v.y;
    }
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" hf_status hf_fp32_peak(int32_t device, hf_fp32_peak_result* out)
{
    if (!out) return HF_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return HF_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return HF_EINVAL;
    hf_status st = HF_OK;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* sink = nullptr;
    int sms = 0, per_sm = 0;
    do {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess) {
            st = HF_ECUDA;
            break;
        }
        const int blocks = sms * (per_sm / PROBE_BLOCK);
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
            cudaMalloc(&sink, sizeof(float) * (size_t)blocks) != cudaSuccess) {
            st = HF_ECUDA;
            break;
        }
        const int iters = 1 << 11;  // about 0.25 s per launch at 80 TFLOP/s
        const double flops = 2.0 * CHAINS * (double)iters * (double)blocks * PROBE_BLOCK;
        double best[2] = {0.0, 0.0};
        for (int kind = 0; kind < 2 && st == HF_OK; ++kind) {
            for (int rep = 0; rep < 4; ++rep) {  // rep 0 warms up the clocks
                cudaEventRecord(e0, s);
                if (kind == 0) k_ffma<<<blocks, PROBE_BLOCK, 0, s>>>(sink, iters, 0.999999f, 1.0e-7f);
                else k_ffma2<<<blocks, PROBE_BLOCK, 0, s>>>(sink, iters, 0.999999f, 1.0e-7f);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                    st = HF_ECUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms > 0.f) {
                    const double tf = flops / (ms * 1.0e-3) / 1.0e12;
                    if (tf > best[kind]) best[kind] = tf;
                }
            }
        }
        out->sm_count = sms;
        out->tflops_ffma = best[0];
        out->tflops_ffma2 = best[1];
    } while (0);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(prev);
    return st;
}
