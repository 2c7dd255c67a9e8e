// mlp_train_fused_noalloc: the fused training kernel run on caller-owned
// weights with its scratch in a fixed device array, so that the call allocates
// no device memory.  For callers that cannot allocate: code inside a framework
// that hands out every byte of device memory from its own pool (a cudaMalloc
// beside the pool would fail or fragment it), or a real-time loop that must not
// block on the allocator's device-wide synchronisation.
#include "mlp_internal.cuh"

namespace {

// Largest network accepted: D <= 64 and H <= 128, that is at most
// (64 + 2) * 128 + 1 = 8449 parameters.
constexpr int NA_MAX_D = 64;
constexpr int NA_MAX_H = 128;
// Three fixed-point accumulators of (P + 1) int64 and the barrier counter
// (the fused kernel's scratch at the largest size), then the status word:
// 203,520 bytes in all.
constexpr size_t NA_SCRATCH = 203264;
constexpr size_t NA_BYTES = NA_SCRATCH + 256;

// One copy per device that loads this library, kept until the process exits.
// Every call uses all of it from the start, so calls that overlap on the GPU
// (any two streams, any two threads) race and must not be issued that way.
__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// The array's device address on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in for the symbol; kernels must
// be given this address instead.  It is looked up on every call (the lookup
// allocates nothing): after cudaDeviceReset, or any other teardown of the
// device's primary context, the module is loaded again and the array may sit
// at a new address, so a cached one could be stale.
cudaError_t scratch_address(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (unsigned char *)p;
    return cudaSuccess;
}

}  // namespace

mlp_status noalloc_fail(mlp_status s, const char *msg);

extern "C" mlp_status mlp_train_fused_noalloc(int32_t act, int32_t D, int32_t H, int64_t n, const float *X,
                                              const float *y, float *params, float lr, int32_t loss_mean,
                                              int32_t epochs, int64_t minibatch, double *loss_hist,
                                              int32_t *status_out, void *stream) {
    if (act != MLP_ACT_SIGMOID && act != MLP_ACT_TANH)
        return noalloc_fail(MLP_EINVAL, "mlp_train_fused_noalloc: bad activation");
    if (D < 1 || D > NA_MAX_D || H < 1 || H > NA_MAX_H)
        return noalloc_fail(MLP_EINVAL,
                            "mlp_train_fused_noalloc: the network must have 1 <= D <= 64 and 1 <= H <= 128 "
                            "(the size of its fixed scratch array)");
    if (n < 0 || epochs < 0 || !params || (n > 0 && (!X || !y)))
        return noalloc_fail(MLP_EINVAL, "mlp_train_fused_noalloc: bad arguments");
    if (((uintptr_t)params & 15) != 0)
        return noalloc_fail(MLP_EINVAL, "mlp_train_fused_noalloc: params must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess)
        return noalloc_fail(MLP_ECUDA, "mlp_train_fused_noalloc: cannot resolve the scratch array");
    int *status = (int *)(base + NA_SCRATCH);
    const size_t need = mlp::fused_scratch_bytes(D, H, 0);
    if (need > NA_SCRATCH) return noalloc_fail(MLP_EINVAL, "mlp_train_fused_noalloc: network too large");
    // The array keeps the previous call's contents: clear the accumulators,
    // the barrier counter and the status word.
    if (cudaMemsetAsync(base, 0, need, st) != cudaSuccess || cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        return noalloc_fail(MLP_ECUDA, "mlp_train_fused_noalloc: clearing the scratch failed");
    if (epochs > 0 && n == 0 && loss_hist &&
        cudaMemsetAsync(loss_hist, 0, sizeof(double) * (size_t)epochs, st) != cudaSuccess)
        return noalloc_fail(MLP_ECUDA, "mlp_train_fused_noalloc: clearing the loss history failed");
    if (epochs > 0 && n > 0) {
        mlp::FusedScratch fsc;
        mlp::fused_scratch_carve(base, D, H, 0, &fsc);
        mlp::FusedCounters ctr;
        cudaError_t e = mlp::fused_train(act, D, H, n, X, y, params, lr, loss_mean ? 1 : 0, epochs, minibatch,
                                         loss_hist, nullptr, status, fsc, &ctr, 32, -1, st, nullptr);
        if (e != cudaSuccess) return noalloc_fail(MLP_ECUDA, cudaGetErrorString(e));
    }
    if (status_out &&
        cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return noalloc_fail(MLP_ECUDA, "mlp_train_fused_noalloc: copying the status failed");
    return MLP_OK;
}
