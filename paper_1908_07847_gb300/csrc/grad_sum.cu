// The exchange step of data-parallel training of one network.  Mini-batch
// gradient descent (Sec. 2.2 of arXiv 1908.07847) updates with the gradient
// of the batch's squared error, which is a sum over the batch's rows; when
// each rank computes the summed gradient of its own shard of the rows, the
// batch's gradient is the sum of the ranks' vectors.  Every rank receives all
// of them (an all-gather) and adds them here in rank order, so every replica
// gets the same bits and applies the same update:
//   out[i]    = scale * (((p_0[i] + p_1[i]) + p_2[i]) + ...)
//   *loss_acc += loss_scale * (((l_0 + l_1) + l_2) + ...)      (FP64)
#include "mlp_internal.cuh"

namespace {

__global__ void k_grad_sum(const float *__restrict__ parts, int nparts, int64_t len, float scale,
                           float *__restrict__ out) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += step) {
        float s = parts[i];
        for (int p = 1; p < nparts; ++p) s += parts[(int64_t)p * len + i];
        out[i] = s * scale;
    }
}

__global__ void k_loss_sum(const double *__restrict__ parts, int nparts, double scale, double *acc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = parts[0];
        for (int p = 1; p < nparts; ++p) s += parts[p];
        *acc += scale * s;
    }
}

}  // namespace

extern "C" mlp_status mlp_grad_sum(const float *parts, const double *loss_parts, int32_t nparts, int64_t len,
                                   float scale, double loss_scale, float *out, double *loss_acc, void *stream) {
    if (nparts < 1 || len < 0 || (len > 0 && (!parts || !out)) || (!loss_parts != !loss_acc))
        return mlp::set_error(MLP_EINVAL, "mlp_grad_sum: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (len > 0) {
        int64_t blocks = (len + 255) / 256;
        const int64_t cap = 4 * (int64_t)mlp::device_sm_count();
        if (blocks > cap) blocks = cap;
        k_grad_sum<<<(unsigned)blocks, 256, 0, st>>>(parts, nparts, len, scale, out);
    }
    if (loss_parts) k_loss_sum<<<1, 32, 0, st>>>(loss_parts, nparts, loss_scale, loss_acc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp::set_error(MLP_ECUDA, cudaGetErrorString(e));
    return MLP_OK;
}
