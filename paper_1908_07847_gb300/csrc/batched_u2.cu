// Many independent networks in one launch with two hidden units a lane
// (row_engine2.cuh), for inputs up to 36 wide (the paper's 33 markers among
// them).  The method per net is the one of batched_kernels.cu (Sec. 2.2 of
// arXiv 1908.07847: feed-forward, output error, backpropagation, full-batch
// gradient descent without momentum, one update per epoch in shared memory in
// a fixed order); only the mapping of hidden units to lanes differs: each lane
// holds two units' weights and gradient rows, so every row word read from
// shared memory feeds two multiply-adds and the per-row z2 butterfly and
// output delta are shared by two units.  Blocks of four warps, two per SM (the
// two units' registers leave room for eight warps an SM).
#include "row_engine2.cuh"

namespace mlp {

namespace {

constexpr int NW2 = 4;
constexpr int BNT2 = NW2 * 32;
constexpr int BCAP2 = 128;       // rows staged in shared memory at a time

// The same per-net training with the two-units-a-lane engine (D = 4 DQ + DT,
// D <= 36).  Shared memory: rows (BCAP2 x DPR), labels, master weights, the
// row groups' gradient partials and the z2 exchange.
template <int DQ, int DT, int WU, int ACT, int RB>
__device__ __forceinline__ void net_body2(const BatchNet &nd, int D, int epochs, float lr, int loss_mean,
                                          int *status, float *Xs, float *ys, float *Wm, float *part, float *zx,
                                          double *s_sse, double *s_gn) {
    using Eng = RowEngine2<DQ, DT, 2, WU, ACT, RB, NW2>;
    constexpr int DPR = Eng::DPR, NG = Eng::NG;
    Eng eng;
    eng.setup(nd.H, D);
    const int64_t n = nd.n;
    const int P = (D + 2) * nd.H + 1;
    const int tid = threadIdx.x;

    for (int i = tid; i < P; i += BNT2) Wm[i] = nd.params[i];
    const bool resident = n <= BCAP2;
    auto load_rows = [&](int64_t r0, int cn) {
        const float *Xg = nd.X + r0 * D;
        for (int i = tid; i < cn * D; i += BNT2) {
            const int s = i / D, k = i - s * D;
            Xs[s * DPR + k] = Xg[i];
        }
        for (int i = tid; i < cn; i += BNT2) ys[i] = nd.y[r0 + i];
    };
    if (resident) load_rows(0, (int)n);
    __syncthreads();
    const float c = loss_mean ? 1.0f / (float)n : 1.0f;
    const double C = loss_mean ? 1.0 / (double)n : 1.0;
    const bool want_gn = nd.gnorm_hist != nullptr;

    for (int e = 0; e < epochs; ++e) {
        eng.load_weights(Wm);
        for (int64_t cs = 0; cs < n; cs += BCAP2) {
            const int cn = (int)min((int64_t)BCAP2, n - cs);
            if (!resident) {
                __syncthreads();
                load_rows(cs, cn);
                __syncthreads();
            }
            eng.rows(Xs, ys, cn, c, zx);
        }
        eng.write_group(part, s_sse);
        __syncthreads();
        // Update, and (only when asked for: FP64 is slow on this part) the FP64
        // squared norm of the gradient it applies, in a fixed order.
        double gn = 0.0;
        for (int p = tid; p < P; p += BNT2) {
            float g = part[p];
#pragma unroll
            for (int q = 1; q < NG; ++q) g += part[q * P + p];
            Wm[p] -= lr * g;
            if (want_gn) gn = fma((double)g, (double)g, gn);
        }
        if (want_gn) {
            gn = warp_sum(gn);
            if ((tid & 31) == 0) s_gn[tid >> 5] = gn;
            __syncthreads();
        }
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NG; ++q) t += s_sse[q];
            const double L = 0.5 * C * t;
            if (nd.loss_hist) nd.loss_hist[e] = L;
            if (!isfinite(L)) atomicOr(status, ST_NONFINITE);
            if (want_gn) {
                double u = 0.0;
                for (int q = 0; q < NW2; ++q) u += s_gn[q];
                nd.gnorm_hist[e] = sqrt(u);
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < P; i += BNT2) nd.params[i] = Wm[i];
    __syncthreads();
}

template <int DQ, int DT, int ACT, int RB, int MINB = 2>
__global__ void __launch_bounds__(BNT2, MINB) k_batched_train2(const BatchNet *__restrict__ nets,
                                                           const int *__restrict__ order, int n_nets, int D,
                                                           int epochs, float lr, int loss_mean, int *status,
                                                           int part_floats, int wm_floats) {
    constexpr int DPR = RowEngine2<DQ, DT, 2, 1, ACT, RB, NW2>::DPR;
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_sse[NW2];
    __shared__ double s_gn[NW2];
    float *Xs = smem;                      // BCAP2 x DPR
    float *ys = Xs + BCAP2 * DPR;          // BCAP2
    float *Wm = ys + BCAP2;                // wm_floats
    float *part = Wm + wm_floats;          // part_floats
    float *zx = part + part_floats;        // z2 exchange
    for (int i = threadIdx.x; i < BCAP2 * DPR; i += BNT2) Xs[i] = 0.f;
    __syncthreads();
    for (int idx = blockIdx.x; idx < n_nets; idx += gridDim.x) {
        const BatchNet nd = nets[order ? order[idx] : idx];
        if (nd.n <= 0 || nd.H <= 0) {
            if (threadIdx.x == 0)
                for (int e = 0; e < epochs; ++e) {
                    if (nd.loss_hist) nd.loss_hist[e] = 0.0;
                    if (nd.gnorm_hist) nd.gnorm_hist[e] = 0.0;
                }
            continue;
        }
        if (nd.H <= 64)
            net_body2<DQ, DT, 1, ACT, RB>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse, s_gn);
        else
            net_body2<DQ, DT, 2, ACT, RB>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse, s_gn);
    }
}


template <int DQ, int DT, int RB, int MINB = 2>
void *pick2(int act) {
    if (act == MLP_ACT_TANH) return (void *)k_batched_train2<DQ, DT, MLP_ACT_TANH, RB, MINB>;
    return (void *)k_batched_train2<DQ, DT, MLP_ACT_SIGMOID, RB, MINB>;
}

// (DQ, DT) of the input-width class, the row buffer's stride in floats.
bool width_class(int D, int *DQ, int *DT, int *DPR) {
    if (D < 1 || D > 36) return false;
    if (D == 33) { *DQ = 8; *DT = 1; *DPR = 36; return true; }
    const int DP = D <= 8 ? 8 : (D <= 16 ? 16 : (D <= 32 ? 32 : 36));
    *DQ = DP / 4;
    *DT = 0;
    *DPR = DP;
    return true;
}

}  // namespace

// rb: rows in flight (1, 2) or 3 = one row in flight at three blocks an SM
// (168 registers a thread); 2 and 3 only for the paper's D = 33.
bool batched_u2_supported(int D, int rb) {
    int a, b, c;
    return width_class(D, &a, &b, &c) && (rb == 1 || D == 33) && rb >= 1 && rb <= 3;
}

cudaError_t batched_train_u2(int act, int D, int Hmax, const BatchNet *nets_dev, const int *order_dev, int n_nets,
                             int epochs, float lr, int loss_mean, int *status, int rb, cudaStream_t st) {
    int DQ, DT, DPR;
    if (!batched_u2_supported(D, rb) || Hmax > 128 || !width_class(D, &DQ, &DT, &DPR)) return cudaErrorInvalidValue;
    if (n_nets == 0 || epochs == 0) return cudaSuccess;
    void *fn = nullptr;
    if (rb == 3) fn = pick2<8, 1, 1, 3>(act);
    else if (rb == 2) fn = pick2<8, 1, 2>(act);
    else if (DT == 1) fn = pick2<8, 1, 1>(act);
    else if (DQ == 2) fn = pick2<2, 0, 1>(act);
    else if (DQ == 4) fn = pick2<4, 0, 1>(act);
    else if (DQ == 8) fn = pick2<8, 0, 1>(act);
    else fn = pick2<9, 0, 1>(act);
    const int pf = re2_part_floats(D, Hmax, 2, NW2);
    const int wm = ((D + 2) * Hmax + 1 + 3) & ~3;
    const size_t smem = sizeof(float) * ((size_t)BCAP2 * DPR + BCAP2 + wm + pf + 2 * NW2 * 2);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&nets_dev, (void *)&order_dev, (void *)&n_nets, (void *)&D, (void *)&epochs,
                    (void *)&lr, (void *)&loss_mean, (void *)&status, (void *)&pf, (void *)&wm};
    return cudaLaunchKernel(fn, dim3((unsigned)n_nets), dim3(BNT2), args, smem, st);
}

}  // namespace mlp
