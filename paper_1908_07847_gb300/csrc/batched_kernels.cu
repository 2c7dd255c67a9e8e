// Many independent networks in one launch (Sec. 2.1 of arXiv 1908.07847 trains
// the male and female subsets as separate networks; here thousands of nets with
// their own hidden width H <= 128 and row count n).  One block trains one net
// for all epochs without leaving the chip: its rows of X (when they fit) and
// its master weights live in shared memory, each lane owns one or two hidden
// neurons with their incoming weights and gradient rows in registers, and the
// per-epoch gradient reduction and update (Sec. 2.2: full-batch gradient
// descent, no momentum) run in shared memory in a fixed order.
//
// Small widths pack several rows into one warp: a warp is cut into segments of
// S = next power of two >= H lanes (S >= 4), lane j of a segment owns hidden
// unit j, and the output sum z2 is a butterfly over the segment.  Widths 65..128
// use two warps per row group that exchange their halves of z2 through shared
// memory.  Blocks take nets in the order given (the host sorts by cost,
// longest first).
#include "mlp_internal.cuh"

namespace mlp {

namespace {

constexpr int BNW = 4;           // warps per block
constexpr int BNT = BNW * 32;    // threads per block
constexpr int RB = 4;            // rows per lane slot per iteration
constexpr int BCAP = 256;        // rows staged in shared memory at a time

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <int DP, int UPL, int WU, int ACT>
__device__ __forceinline__ void net_body(const BatchNet &nd, int D, int epochs, float lr, int loss_mean,
                                         int *status, float *Xs, float *ys, float *Wm, float *part,
                                         float *zx, double *s_sse) {
    const int H = nd.H;
    const int64_t n = nd.n;
    const int HD = H * D, P = HD + 2 * H + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NG = BNW / WU;  // row groups per block
    const int grp = warp / WU, wu = warp % WU;
    int S = 32;
    if (UPL == 1 && WU == 1) {
        S = 4;
        while (S < H) S <<= 1;
    }
    const int slot = lane / S, sl = lane % S, nslots = 32 / S;
    const int RPI = nslots * RB;  // rows per group iteration

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
    int par = 0;

    for (int e = 0; e < epochs; ++e) {
        float w[UPL][DP], b1r[UPL], w2r[UPL];
        int jj[UPL];
#pragma unroll
        for (int u = 0; u < UPL; ++u) {
            const int j = wu * (32 * UPL) + u * 32 + sl;
            jj[u] = j;
            const bool ok = j < H;
#pragma unroll
            for (int k = 0; k < DP; ++k) w[u][k] = (ok && k < D) ? Wm[j * D + k] : 0.f;
            b1r[u] = ok ? Wm[HD + j] : 0.f;
            w2r[u] = ok ? Wm[HD + H + j] : 0.f;
        }
        const float b2 = Wm[P - 1];
        float acc[UPL][DP], gb1a[UPL], gw2a[UPL], gb2a = 0.f;
        double sse = 0.0;
#pragma unroll
        for (int u = 0; u < UPL; ++u) {
            gb1a[u] = 0.f;
            gw2a[u] = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) acc[u][k] = 0.f;
        }

        for (int64_t cs = 0; cs < n; cs += BCAP) {
            const int cn = (int)min((int64_t)BCAP, n - cs);
            if (!resident) {
                __syncthreads();
                load_rows(cs, cn);
                __syncthreads();
            }
            for (int base = grp * RPI; base < cn; base += NG * RPI) {
                int r[RB];
                bool valid[RB];
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const int rr = base + slot * RB + t;
                    valid[t] = rr < cn;
                    r[t] = valid[t] ? rr : 0;
                }
                float z[RB][UPL];
#pragma unroll
                for (int t = 0; t < RB; ++t)
#pragma unroll
                    for (int u = 0; u < UPL; ++u) z[t][u] = b1r[u];
#pragma unroll
                for (int q = 0; q < DP / 4; ++q) {
#pragma unroll
                    for (int t = 0; t < RB; ++t) {
                        const float4 xv = *reinterpret_cast<const float4 *>(Xs + r[t] * DP + 4 * q);
#pragma unroll
                        for (int u = 0; u < UPL; ++u) {
                            z[t][u] = fmaf(xv.x, w[u][4 * q + 0], z[t][u]);
                            z[t][u] = fmaf(xv.y, w[u][4 * q + 1], z[t][u]);
                            z[t][u] = fmaf(xv.z, w[u][4 * q + 2], z[t][u]);
                            z[t][u] = fmaf(xv.w, w[u][4 * q + 3], z[t][u]);
                        }
                    }
                }
                float hv[RB][UPL], zp[RB];
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    zp[t] = 0.f;
#pragma unroll
                    for (int u = 0; u < UPL; ++u) {
                        hv[t][u] = Act<ACT>::f(z[t][u]);
                        zp[t] = fmaf(hv[t][u], w2r[u], zp[t]);
                    }
                }
#pragma unroll
                for (int t = 0; t < RB; ++t)
                    for (int off = S >> 1; off > 0; off >>= 1) zp[t] += __shfl_xor_sync(0xffffffffu, zp[t], off);
                if (WU == 2) {
                    float *zg = zx + (par * NG + grp) * (2 * RB);
                    if (lane == 0) {
#pragma unroll
                        for (int t = 0; t < RB; ++t) zg[wu * RB + t] = zp[t];
                    }
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(64) : "memory");
#pragma unroll
                    for (int t = 0; t < RB; ++t) zp[t] = zg[t] + zg[RB + t];
                    par ^= 1;
                }
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float o = sigmoid_out(zp[t] + b2);
                    const float err = o - ys[r[t]];
                    const float d2 = valid[t] ? c * err * o * (1.0f - o) : 0.f;
                    if (valid[t]) sse += (double)err * (double)err;
                    gb2a += d2;
#pragma unroll
                    for (int u = 0; u < UPL; ++u) {
                        gw2a[u] = fmaf(d2, hv[t][u], gw2a[u]);
                        const float d1 = d2 * w2r[u] * Act<ACT>::df(hv[t][u]);
                        gb1a[u] += d1;
                        hv[t][u] = d1;
                    }
                }
#pragma unroll
                for (int q = 0; q < DP / 4; ++q) {
#pragma unroll
                    for (int t = 0; t < RB; ++t) {
                        const float4 xv = *reinterpret_cast<const float4 *>(Xs + r[t] * DP + 4 * q);
#pragma unroll
                        for (int u = 0; u < UPL; ++u) {
                            acc[u][4 * q + 0] = fmaf(hv[t][u], xv.x, acc[u][4 * q + 0]);
                            acc[u][4 * q + 1] = fmaf(hv[t][u], xv.y, acc[u][4 * q + 1]);
                            acc[u][4 * q + 2] = fmaf(hv[t][u], xv.z, acc[u][4 * q + 2]);
                            acc[u][4 * q + 3] = fmaf(hv[t][u], xv.w, acc[u][4 * q + 3]);
                        }
                    }
                }
            }
        }
        // Sum the row slots of each warp (segments), fixed butterfly order.
        for (int off = S; off < 32; off <<= 1) {
#pragma unroll
            for (int u = 0; u < UPL; ++u) {
#pragma unroll
                for (int k = 0; k < DP; ++k) acc[u][k] += __shfl_xor_sync(0xffffffffu, acc[u][k], off);
                gb1a[u] += __shfl_xor_sync(0xffffffffu, gb1a[u], off);
                gw2a[u] += __shfl_xor_sync(0xffffffffu, gw2a[u], off);
            }
            gb2a += __shfl_xor_sync(0xffffffffu, gb2a, off);
            sse += __shfl_xor_sync(0xffffffffu, sse, off);
        }
        float *pg = part + grp * P;
        if (slot == 0) {
#pragma unroll
            for (int u = 0; u < UPL; ++u) {
                const int j = jj[u];
                if (j < H) {
#pragma unroll
                    for (int k = 0; k < DP; ++k)
                        if (k < D) pg[j * D + k] = acc[u][k];
                    pg[HD + j] = gb1a[u];
                    pg[HD + H + j] = gw2a[u];
                }
            }
        }
        if (wu == 0 && lane == 0) {
            pg[P - 1] = gb2a;
            s_sse[grp] = sse;
        }
        __syncthreads();
        for (int p = tid; p < P; p += BNT) {
            float g = part[p];
#pragma unroll
            for (int q = 1; q < NG; ++q) g += part[q * P + p];
            Wm[p] -= lr * g;
        }
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NG; ++q) t += s_sse[q];
            const double L = 0.5 * C * t;
            if (nd.loss_hist) nd.loss_hist[e] = L;
            if (!isfinite(L)) atomicOr(status, ST_NONFINITE);
        }
        __syncthreads();
    }
    for (int i = tid; i < P; i += BNT) nd.params[i] = Wm[i];
    __syncthreads();
}

template <int DP, int ACT>
__global__ void __launch_bounds__(BNT, 2) k_batched_train(const BatchNet *__restrict__ nets,
                                                         const int *__restrict__ order, int n_nets, int D,
                                                         int epochs, float lr, int loss_mean, int *status,
                                                         int part_floats, int wm_floats) {
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_sse[BNW];
    float *Xs = smem;                      // BCAP x DP
    float *ys = Xs + BCAP * DP;            // BCAP
    float *Wm = ys + BCAP;                 // wm_floats
    float *part = Wm + wm_floats;          // part_floats
    float *zx = part + part_floats;        // 2 x 2 x 2 x RB
    for (int i = threadIdx.x; i < BCAP * DP; i += BNT) Xs[i] = 0.f;
    __syncthreads();
    for (int idx = blockIdx.x; idx < n_nets; idx += gridDim.x) {
        const BatchNet nd = nets[order ? order[idx] : idx];
        if (nd.n <= 0 || nd.H <= 0) {
            if (nd.loss_hist && threadIdx.x == 0)
                for (int e = 0; e < epochs; ++e) nd.loss_hist[e] = 0.0;
            continue;
        }
        if (nd.H <= 32)
            net_body<DP, 1, 1, ACT>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse);
        else if (nd.H <= 64)
            net_body<DP, 2, 1, ACT>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse);
        else
            net_body<DP, 2, 2, ACT>(nd, D, epochs, lr, loss_mean, status, Xs, ys, Wm, part, zx, s_sse);
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

int batched_max_H() { return 128; }
int batched_max_D() { return 64; }

void batched_smem_layout(int D, int Hmax, int *part_floats, int *wm_floats, size_t *bytes) {
    const int DP = dp_for(D);
    // Row groups: 4 for H <= 64, 2 for 65..128 (two warps per group).
    int pf = 0;
    for (int H : {32, 64, Hmax}) {
        if (H > Hmax) continue;
        const int P = (D + 2) * H + 1;
        const int NG = (H <= 64) ? BNW : BNW / 2;
        pf = pf > NG * P ? pf : NG * P;
    }
    const int wm = ((D + 2) * Hmax + 1 + 3) & ~3;
    pf = (pf + 3) & ~3;
    *part_floats = pf;
    *wm_floats = wm;
    *bytes = sizeof(float) * ((size_t)BCAP * DP + BCAP + wm + pf + 2 * 2 * 2 * RB);
}

cudaError_t batched_train(int act, int D, int Hmax, const BatchNet *nets_dev, const int *order_dev, int n_nets,
                          int epochs, float lr, int loss_mean, int *status, cudaStream_t st) {
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
