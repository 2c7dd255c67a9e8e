// Many independent networks in one launch (Sec. 2.1 of arXiv 1908.07847 trains
// the male and female subsets as separate networks; here thousands of nets with
// their own hidden width H <= 128 and row count n).  One block trains one net
// for all epochs without leaving the chip: its rows of X (when they fit) and
// its master weights live in shared memory, the row engine (row_engine.cuh)
// runs forward and backward with one hidden neuron per lane, and the per-epoch
// gradient reduction and update (Sec. 2.2: full-batch gradient descent, no
// momentum) run in shared memory in a fixed order.  Blocks take nets in the
// order given (the host sorts them by cost, largest first).
#include "row_engine.cuh"

namespace mlp {

namespace {

constexpr int BNT = RE_NT;       // threads per block
constexpr int BCAP = 256;        // rows staged in shared memory at a time

template <int DP, int WU, int ACT>
__device__ __forceinline__ void net_body(const BatchNet &nd, int D, int epochs, float lr, int loss_mean,
                                         int *status, float *Xs, float *ys, float *Wm, float *part,
                                         float *zx, double *s_sse, double *s_gn) {
    // One row in flight per lane for H <= 32: at two blocks per SM the second
    // row's registers spill (measured 4.7 % slower on the 4096-net workload).
    using Eng = RowEngine<DP, WU, ACT, 1>;
    Eng eng;
    eng.setup(nd.H, D);
    constexpr int NG = Eng::NG;
    const int64_t n = nd.n;
    const int P = (D + 2) * nd.H + 1;
    const int tid = threadIdx.x;

    for (int i = tid; i < P; i += BNT) Wm[i] = nd.params[i];
    const bool resident = n <= BCAP;
    auto load_rows = [&](int64_t r0, int cn) {
        const float *Xg = nd.X + r0 * D;
        for (int i = tid; i < cn * D; i += BNT) {
            int s = i / D, k = i - s * D;
            Xs[s * DP + k] = Xg[i];
        }
        for (int i = tid; i < cn; i += BNT) ys[i] = nd.y[r0 + i];
    };
    if (resident) load_rows(0, (int)n);
    __syncthreads();
    const float c = loss_mean ? 1.0f / (float)n : 1.0f;
    const double C = loss_mean ? 1.0 / (double)n : 1.0;

    for (int e = 0; e < epochs; ++e) {
        eng.load_weights(Wm);
        for (int64_t cs = 0; cs < n; cs += BCAP) {
            const int cn = (int)min((int64_t)BCAP, n - cs);
            if (!resident) {
                __syncthreads();
                load_rows(cs, cn);
                __syncthreads();
            }
            eng.rows(Xs, ys, cn, c, zx);
        }
        eng.write_group(part, s_sse);
        __syncthreads();
        // Update, and the FP64 squared norm of the gradient it applies: each
        // thread's values in index order, then a fixed butterfly per warp and
        // the warps in order.
        // (FP64 arithmetic is slow on this part: only when asked for.)
        double gn = 0.0;
        const bool want_gn = nd.gnorm_hist != nullptr;
        for (int p = tid; p < P; p += BNT) {
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
            if (nd.gnorm_hist) {
                double u = 0.0;
                for (int q = 0; q < RE_NW; ++q) u += s_gn[q];
                nd.gnorm_hist[e] = sqrt(u);
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < P; i += BNT) nd.params[i] = Wm[i];
    __syncthreads();
}

template <int DP, int ACT>
__global__ void __launch_bounds__(BNT, (DP <= 36 ? 2 : 1)) k_batched_train(const BatchNet *__restrict__ nets,
                                                         const int *__restrict__ order, int n_nets, int D,
                                                         int epochs, float lr, int loss_mean, int *status,
                                                         int part_floats, int wm_floats) {
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_sse[RE_NW];
    __shared__ double s_gn[RE_NW];
    float *Xs = smem;                      // BCAP x DP
    float *ys = Xs + BCAP * DP;            // BCAP
    float *Wm = ys + BCAP;                 // wm_floats
    float *part = Wm + wm_floats;          // part_floats
    float *zx = part + part_floats;        // z2 exchange
    for (int i = threadIdx.x; i < BCAP * DP; i += BNT) Xs[i] = 0.f;
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
        if (nd.H <= 32)
            net_body<DP, 1, ACT>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse, s_gn);
        else if (nd.H <= 64)
            net_body<DP, 2, ACT>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse, s_gn);
        else
            net_body<DP, 4, ACT>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse, s_gn);
    }
}

template <int DP>
void *pick(int act) {
    if (act == MLP_ACT_TANH) return (void *)k_batched_train<DP, MLP_ACT_TANH>;
    return (void *)k_batched_train<DP, MLP_ACT_SIGMOID>;
}

int dp_for(int D) {
    if (D <= 8) return 8;
    if (D <= 16) return 16;
    if (D <= 36) return 36;
    if (D <= 48) return 48;
    if (D <= 64) return 64;
    return 0;
}

}  // namespace

bool batched_shape_supported(int D, int shape) {
    if (shape == BATCH_SHAPE_U1) return dp_for(D) != 0;
    if (shape == BATCH_SHAPE_U2_RB1) return batched_u2_supported(D, 1);
    if (shape == BATCH_SHAPE_U2_RB2) return batched_u2_supported(D, 2);
    if (shape == BATCH_SHAPE_U2_3B) return batched_u2_supported(D, 3);
    if (shape == BATCH_SHAPE_TILED128 || shape == BATCH_SHAPE_TILED64 || shape == BATCH_SHAPE_TILED32)
        return batched_tiled_supported(D, 128);
    return false;
}

int batched_max_H() { return 128; }
int batched_max_D() { return 64; }

void batched_smem_layout(int D, int Hmax, int *part_floats, int *wm_floats, size_t *bytes) {
    const int DP = dp_for(D);
    const int pf = re_part_floats(D, Hmax);
    const int wm = ((D + 2) * Hmax + 1 + 3) & ~3;
    *part_floats = pf;
    *wm_floats = wm;
    *bytes = sizeof(float) * ((size_t)BCAP * DP + BCAP + wm + pf + RE_ZX);
}

cudaError_t batched_train(int act, int D, int Hmax, int64_t nmax, const BatchNet *nets_dev, const int *order_dev,
                          int n_nets, int epochs, float lr, int loss_mean, int *status, int shape, cudaStream_t st) {
    if (shape == BATCH_SHAPE_TILED128 || shape == BATCH_SHAPE_TILED64 || shape == BATCH_SHAPE_TILED32)
        return batched_train_tiled(act, D, Hmax, nmax, nets_dev, order_dev, n_nets, epochs, lr, loss_mean, status,
                                   shape == BATCH_SHAPE_TILED32 ? 32 : (shape == BATCH_SHAPE_TILED64 ? 64 : 128), st);
    if (shape != BATCH_SHAPE_U1)
        return batched_train_u2(act, D, Hmax, nets_dev, order_dev, n_nets, epochs, lr, loss_mean, status,
                                shape == BATCH_SHAPE_U2_RB2 ? 2 : (shape == BATCH_SHAPE_U2_3B ? 3 : 1), st);
    const int DP = dp_for(D);
    if (DP == 0 || Hmax > 128) return cudaErrorInvalidValue;
    if (n_nets == 0 || epochs == 0) return cudaSuccess;
    void *fn = nullptr;
    switch (DP) {
        case 8: fn = pick<8>(act); break;
        case 16: fn = pick<16>(act); break;
        case 36: fn = pick<36>(act); break;
        case 48: fn = pick<48>(act); break;
        default: fn = pick<64>(act); break;
    }
    int pf, wm;
    size_t smem;
    batched_smem_layout(D, Hmax, &pf, &wm, &smem);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&nets_dev, (void *)&order_dev, (void *)&n_nets, (void *)&D, (void *)&epochs,
                    (void *)&lr, (void *)&loss_mean, (void *)&status, (void *)&pf, (void *)&wm};
    return cudaLaunchKernel(fn, dim3((unsigned)n_nets), dim3(BNT), args, smem, st);
}

}  // namespace mlp
