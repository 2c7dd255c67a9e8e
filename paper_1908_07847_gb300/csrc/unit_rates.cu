// Measured execution rates of the units the training kernels lean on: the
// FP32 FMA pipe, and the special-function unit for tanh (the bf16 sigmoid) and
// exp2 (the FP32 sigmoid).  Used to state roofline peaks from measurement
// rather than from data sheets.  Each block runs 8 independent dependency
// chains per thread on registers; the rate is instructions per second over the
// whole device, timed with CUDA events.
#include <cuda_runtime.h>

#include "mlp_internal.cuh"

namespace {

template <int MODE>
__global__ void k_rate(unsigned *out, int iters) {
    unsigned v[8];
    for (int i = 0; i < 8; ++i) v[i] = 0x3E003E00u + threadIdx.x * 7u + (unsigned)i;   // small positive values
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (MODE == 0) asm volatile("fma.rn.f32 %0, %0, %0, %0;" : "+r"(v[i]));
            if (MODE == 1) asm volatile("tanh.approx.f32 %0, %0;" : "+r"(v[i]));
            if (MODE == 2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+r"(v[i]));
        }
    }
    unsigned x = 0;
    for (int i = 0; i < 8; ++i) x ^= v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

template <int MODE>
cudaError_t rate(unsigned *buf, int blocks, int threads, double *per_s) {
    const int iters = 1 << 14;
    k_rate<MODE><<<blocks, threads>>>(buf, 64);   // warm-up
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    cudaEventRecord(a);
    k_rate<MODE><<<blocks, threads>>>(buf, iters);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e == cudaSuccess) *per_s = (double)blocks * threads * iters * 8 / (ms * 1e-3);
    return e;
}

}  // namespace

extern "C" mlp_status mlp_unit_rates(double *ffma_per_s, double *tanh_per_s, double *ex2_per_s) {
    if (!ffma_per_s || !tanh_per_s || !ex2_per_s) return mlp::set_error(MLP_EINVAL, "mlp_unit_rates: null pointer");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return mlp::set_error(MLP_ECUDA, "mlp_unit_rates: no device");
    const int blocks = 4 * sms, threads = 512;
    unsigned *buf = nullptr;
    if (cudaMalloc((void **)&buf, sizeof(unsigned) * blocks * threads) != cudaSuccess) {
        cudaGetLastError();
        return mlp::set_error(MLP_ENOMEM, "mlp_unit_rates: cannot allocate");
    }
    cudaError_t e = rate<0>(buf, blocks, threads, ffma_per_s);
    if (e == cudaSuccess) e = rate<1>(buf, blocks, threads, tanh_per_s);
    if (e == cudaSuccess) e = rate<2>(buf, blocks, threads, ex2_per_s);
    cudaFree(buf);
    return e == cudaSuccess ? MLP_OK : mlp::set_error(MLP_ECUDA, cudaGetErrorString(e));
}
