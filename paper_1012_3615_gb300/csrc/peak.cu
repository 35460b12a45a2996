// Measured arithmetic peaks of this GPU (the ALU rooflines of the stencil):
// independent chains of fused multiply-adds, long enough that issue and the
// FMA pipe are the only limits, timed with CUDA events.  FP32 uses the packed
// fma.rn.f32x2 form the FP32 stencil is built from (two FMAs per lane and
// instruction); FP64 plain fma.rn.f64.  Nothing here changes a GPU setting:
// the rates are those of the clocks the GPU runs at.
#include "ctx.h"

namespace {

constexpr int CHAINS = 16;  // independent chains per thread (hides the FMA latency)

__global__ void k_fma_f32x2(float2 *out, float seed, int iters) {
    float2 a[CHAINS];
    const float2 m = make_float2(0.999999f, 1.000001f), c = make_float2(seed * 1e-7f, -seed * 1e-7f);
#pragma unroll
    for (int i = 0; i < CHAINS; i++) a[i] = make_float2(seed + threadIdx.x + i, seed - threadIdx.x - i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < CHAINS; i++) a[i] = __ffma2_rn(a[i], m, c);
    }
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < CHAINS; i++) s = make_float2(s.x + a[i].x, s.y + a[i].y);
    // every chain stays positive, so this store never happens; the compiler
    // cannot know that and keeps the chains
    if (out && s.x < 0.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fma_f64(double *out, double seed, int iters) {
    double a[CHAINS];
    const double m = 0.9999999999, c = seed * 1e-12;
#pragma unroll
    for (int i = 0; i < CHAINS; i++) a[i] = seed + threadIdx.x + i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < CHAINS; i++) a[i] = fma(a[i], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CHAINS; i++) s += a[i];
    if (out && s < 0.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" bri_status bri_alu_peak(int prec, double *tflops) {
    if (!tflops || (prec != BRI_F32 && prec != BRI_F64))
        return bri_fail(nullptr, BRI_EINVAL, "bri_alu_peak: prec must be BRI_F32 or BRI_F64, tflops non-null");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bri_fail(nullptr, BRI_ECUDA, "bri_alu_peak: no CUDA device");
    const int threads = 256, blocks = sms * 8;
    const int iters = prec == BRI_F32 ? 4096 : 512;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bri_fail(nullptr, BRI_ECUDA, "bri_alu_peak: cudaEventCreate failed");
    float best = 1e30f;
    for (int rep = 0; rep < 6; rep++) {  // the first launch warms up; the fastest counts
        cudaEventRecord(e0, 0);
        if (prec == BRI_F32) k_fma_f32x2<<<blocks, threads>>>(nullptr, 1.0f + rep, iters);
        else k_fma_f64<<<blocks, threads>>>(nullptr, 1.0 + rep, iters);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bri_fail(nullptr, BRI_ECUDA, std::string("bri_alu_peak: ") + cudaGetErrorString(e));
    const double fmas = (double)blocks * threads * CHAINS * iters * (prec == BRI_F32 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return BRI_OK;
}
