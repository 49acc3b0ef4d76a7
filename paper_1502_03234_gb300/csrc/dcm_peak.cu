// dcm_peak.cu -- the measured FP32 FMA throughput of the device, the
// denominator against which the force kernels' FP32-pipe roofline can be
// read (no counterpart in the thesis: a measurement aid).  Every thread runs
// 8 independent chains of dependent FMAs on operands the compiler cannot
// fold; blocks fill every SM.
#include "dcm_device.cuh"

namespace dcm {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(PEAK_THREADS) k_ffma_chain(float *out, int iters, float a,
                                                             float b)
{
    float x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    if (s == -1.f) out[blockIdx.x] = s;      // (never true: keeps the chains live)
}

}  // namespace dcm

using namespace dcm;

extern "C" int dcm_fp32_peak(int iters, double *tflops, double *ms)
{
    if (iters < 1 || !tflops) return fail(DCM_ERR_ARG, "need iters >= 1 and an output");
    int dev = 0, sms = 0;
    DCM_CHECK_CUDA(cudaGetDevice(&dev));
    DCM_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = nullptr;
    DCM_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *out = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out, sizeof(float) * 8 * sms, s);
    const int grid = 8 * sms;                // 64 warps per SM
    float t = 0.f;
    if (e == cudaSuccess) {
        k_ffma_chain<<<grid, PEAK_THREADS, 0, s>>>(out, iters / 8 + 1, 0.999999f, 1e-6f);   // warm-up
        cudaEventRecord(e0, s);
        k_ffma_chain<<<grid, PEAK_THREADS, 0, s>>>(out, iters, 0.999999f, 1e-6f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    }
    if (out) cudaFreeAsync(out, s);
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return fail_cuda(e, "fp32 peak", __FILE__, __LINE__);
    const double flops = 2.0 * PEAK_CHAINS * (double)iters * grid * PEAK_THREADS;
    *tflops = flops / ((double)t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return DCM_OK;
}
