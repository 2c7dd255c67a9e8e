// Z-score normalisation of the feature table (Sec. 2.2 normalises the data
// before training; the reading: per-column mean and population standard
// deviation of the training rows, applied to every row; a column with no
// spread maps to 0), fused with the conversion to the padded layout the
// training kernels read (FP32, or bf16 with zero columns up to D_out).
//
// Statistics: two passes over the fit rows (sum, then squared deviations from
// the mean), FP64 accumulation.  Each block sums a contiguous slice of rows;
// inside a block, with D <= 256, 256 / D "row lanes" take every (256/D)-th row
// and are combined in lane order; the block partials are combined in block
// order.  Every sum has a fixed order, so the statistics are bitwise
// reproducible.  The normalisation pass is FP32: (x - m_hi) - m_lo with the
// mean split into two floats, times 1/s rounded to float; it is bound by HBM.
#include <cuda_bf16.h>

#include "mlp_internal.cuh"

namespace mlp {
namespace {

constexpr int ZT = 256;

// partial[b][j] = sum over the block's rows of (X[i][j] - centre[j])^p, p = 1 or 2
template <int P>
__global__ void __launch_bounds__(ZT) k_colsum(const float *__restrict__ X, int64_t n_fit, int D,
                                               const double *__restrict__ centre, double *__restrict__ partial) {
    __shared__ double red[ZT];
    const int b = blockIdx.x, G = gridDim.x, t = threadIdx.x;
    const int64_t r0 = n_fit * b / G, r1 = n_fit * (b + 1) / G;
    if (D <= ZT) {
        const int RL = ZT / D;                 // row lanes
        const int rl = t / D, j = t % D;
        double acc = 0.0;
        if (rl < RL) {
            const double c = P == 2 ? centre[j] : 0.0;
            for (int64_t i = r0 + rl; i < r1; i += RL) {
                const double v = (double)X[i * D + j] - c;
                acc += P == 2 ? v * v : v;
            }
        }
        red[t] = acc;
        __syncthreads();
        if (t < D) {
            double s = 0.0;
            for (int l = 0; l < RL; ++l) s += red[l * D + t];
            partial[(size_t)b * D + t] = s;
        }
    } else {
        for (int j = t; j < D; j += ZT) {
            const double c = P == 2 ? centre[j] : 0.0;
            double acc = 0.0;
            for (int64_t i = r0; i < r1; ++i) {
                const double v = (double)X[i * D + j] - c;
                acc += P == 2 ? v * v : v;
            }
            partial[(size_t)b * D + j] = acc;
        }
    }
}

// out[j] = sum_b partial[b][j] / n_fit (P = 1: the mean), or its square root
// (P = 2: the population deviation)
template <int P>
__global__ void k_colcombine(const double *__restrict__ partial, int G, int D, int64_t n_fit, double *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += partial[(size_t)b * D + j];
    const double v = s / (double)n_fit;
    out[j] = P == 2 ? sqrt(v) : v;
}

template <typename TO>
__device__ __forceinline__ TO to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename TO>
__global__ void __launch_bounds__(ZT) k_zapply(const float *__restrict__ X, int64_t n, int D, int D_out,
                                               const double *__restrict__ mean, const double *__restrict__ sdev,
                                               TO *__restrict__ Y) {
    extern __shared__ float zs[];   // [D] m_hi, [D] m_lo, [D] 1/s (0 where s = 0)
    for (int j = threadIdx.x; j < D; j += ZT) {
        const double m = mean[j], s = sdev[j];
        const float hi = (float)m;
        zs[j] = hi;
        zs[D + j] = (float)(m - (double)hi);
        zs[2 * D + j] = s > 0.0 ? (float)(1.0 / s) : 0.f;
    }
    __syncthreads();
    const int64_t total = n * D_out;
    const bool narrow = total < ((int64_t)1 << 32);   // 32-bit index division suffices
    for (int64_t e = (int64_t)blockIdx.x * ZT + threadIdx.x; e < total; e += (int64_t)gridDim.x * ZT) {
        const int64_t i = narrow ? (int64_t)((uint32_t)e / (uint32_t)D_out) : e / D_out;
        const int j = (int)(e - i * D_out);
        float v = 0.f;
        if (j < D) v = ((X[i * D + j] - zs[j]) - zs[D + j]) * zs[2 * D + j];
        Y[e] = to_out<TO>(v);
    }
}

int zscore_blocks(int64_t n_fit) {
    int64_t g = (n_fit + 63) / 64;
    const int64_t cap = 4 * (int64_t)device_sm_count();
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace mlp

extern "C" mlp_status mlp_zscore_workspace_bytes(int32_t D, uint64_t *bytes) {
    if (!bytes || D < 1) return mlp::set_error(MLP_EINVAL, "mlp_zscore_workspace_bytes: bad arguments");
    *bytes = sizeof(double) * (uint64_t)D * 4 * (uint64_t)mlp::device_sm_count();
    return MLP_OK;
}

extern "C" mlp_status mlp_zscore(const float *X, int64_t n, int32_t D, int64_t n_fit, int32_t out_prec, int32_t D_out,
                                 void *Y, double *mean, double *sdev, void *workspace, uint64_t workspace_bytes,
                                 void *stream) {
    using namespace mlp;
    if (D < 1 || D_out < D || n < 0 || (out_prec != MLP_FP32 && out_prec != MLP_BF16) || !mean || !sdev)
        return set_error(MLP_EINVAL, "mlp_zscore: bad D, D_out, n, precision or statistics pointer");
    if (n == 0) return MLP_OK;
    if (!X || !Y || !workspace || n_fit < 1 || n_fit > n)
        return set_error(MLP_EINVAL, "mlp_zscore: null buffer or n_fit outside 1..n");
    const int G = zscore_blocks(n_fit);
    if (workspace_bytes < sizeof(double) * (uint64_t)G * (uint64_t)D)
        return set_error(MLP_EINVAL, "mlp_zscore: workspace smaller than mlp_zscore_workspace_bytes");
    cudaStream_t st = (cudaStream_t)stream;
    double *partial = (double *)workspace;
    const int cb = (D + 127) / 128;
    k_colsum<1><<<G, ZT, 0, st>>>(X, n_fit, D, nullptr, partial);
    k_colcombine<1><<<cb, 128, 0, st>>>(partial, G, D, n_fit, mean);
    k_colsum<2><<<G, ZT, 0, st>>>(X, n_fit, D, mean, partial);
    k_colcombine<2><<<cb, 128, 0, st>>>(partial, G, D, n_fit, sdev);
    const int64_t total = n * (int64_t)D_out;
    int64_t blocks = (total + ZT - 1) / ZT;
    const int64_t cap = 16 * (int64_t)device_sm_count();
    if (blocks > cap) blocks = cap;
    const size_t smem = sizeof(float) * 3 * (size_t)D;
    if (smem > 48 * 1024) return set_error(MLP_EUNSUPPORTED, "mlp_zscore: D above 4096");
    if (out_prec == MLP_FP32)
        k_zapply<float><<<(unsigned)blocks, ZT, smem, st>>>(X, n, D, D_out, mean, sdev, (float *)Y);
    else
        k_zapply<__nv_bfloat16><<<(unsigned)blocks, ZT, smem, st>>>(X, n, D, D_out, mean, sdev, (__nv_bfloat16 *)Y);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : set_error(MLP_ECUDA, cudaGetErrorString(e));
}
