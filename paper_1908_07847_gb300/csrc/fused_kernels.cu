// Fused training kernel for small networks (D <= 64, H <= 64): one cooperative
// launch runs every step of every epoch.  Per step (Sec. 2.2 of arXiv
// 1908.07847: feed-forward, output error, backpropagation, gradient descent
// with no momentum):
//   1. every block stages the weights and its rows of X in shared memory with
//      asynchronous copies (all in flight at once); each warp takes a row at a
//      time, each lane owns up to two hidden neurons (the paper's "each neuron
//      on its own thread") with their incoming weights in registers, computes
//      z1, h, the warp-shuffle sum z2, o (Eq. 1), the output delta and the
//      hidden deltas, and accumulates the neuron's gradient row in registers;
//      activations never leave the chip;
//   2. warp partials are summed in shared memory in warp order and written as
//      one partial per block;
//   3. grid barrier; every warp then owns a few parameters: its lanes load the
//      block partials of a parameter in parallel (lane q takes blocks q, q+32,
//      ...), add them in that order and finish with a butterfly -- a fixed
//      order, so results are bitwise reproducible -- and lane 0 applies
//      w -= lr g and adds g^2 to an FP64 norm partial;
//   4. grid barrier; block 0 folds the FP64 loss and norm partials the same way.
#include <mutex>

#include "mlp_internal.cuh"

namespace mlp {

namespace {

constexpr int FNT = 256;         // threads per block
constexpr int FNW = FNT / 32;    // warps per block
constexpr int CAP = 64;          // rows staged in shared memory at a time
constexpr int QMAX = 5;          // blocks per lane in the cross-block sums
constexpr int GMAX = 32 * QMAX;  // largest grid
constexpr int PPW = 4;           // parameters per warp per round

struct FArgs {
    int D, H;
    int64_t n;
    const float *X;
    const float *y;
    float *params;
    float lr;
    int loss_mean;
    int epochs;
    int64_t mb;
    double *loss_hist;
    double *gnorm_hist;
    int *status;
    float *part;
    double *lossp;
    double *gnp;
    unsigned *bar;
    int skip_block;
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Shared-memory layout (floats): [weights staging | per-warp partials] (aliased),
// then b1, w2, b2 staging, then CAP rows of X (DP wide, zero padded), CAP labels.
__host__ __device__ inline int weights_floats(int D, int H) { return H * (D | 1); }
__host__ __device__ inline int partial_floats(int D, int H) { return FNW * ((D + 2) * H + 1); }
__host__ __device__ inline int bias_offset(int D, int H) {
    int a = weights_floats(D, H), b = partial_floats(D, H);
    return ((a > b ? a : b) + 3) & ~3;
}
__host__ __device__ inline int xs_offset(int D, int H) { return (bias_offset(D, H) + 2 * H + 1 + 3) & ~3; }

template <int DP>
size_t smem_bytes(int D, int H) {
    return sizeof(float) * ((size_t)xs_offset(D, H) + (size_t)CAP * DP + CAP);
}

// Sum of v[q] for q < G in a fixed order: lane l adds q = l, l+32, ... in turn,
// then a butterfly over the lanes.  Every lane returns the same value.
template <typename T>
__device__ __forceinline__ T fixed_sum(const T *__restrict__ v, int G, int lane) {
    T s = T(0);
#pragma unroll
    for (int t = 0; t < QMAX; ++t) {
        const int q = lane + 32 * t;
        if (q < G) s += __ldcg(v + q);
    }
    return warp_sum(s);
}

template <int DP, int UPL, int ACT>
__global__ void __launch_bounds__(FNT, 1) k_fused_train(FArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_red[FNW];
    const int D = a.D, H = a.H;
    const int HD = H * D;
    const int P = HD + 2 * H + 1;
    const int WSTR = D | 1;
    float *Ws = smem;                        // H x WSTR weights staging (aliased with
    float *parts = smem;                     // the FNW x P per-warp partials)
    float *Bs = smem + bias_offset(D, H);    // b1 [H], w2 [H], b2
    float *Xs = smem + xs_offset(D, H);      // CAP x DP rows, zero padded
    float *ys = Xs + CAP * DP;               // CAP labels
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, g = blockIdx.x;
    if (g == a.skip_block) return;           // fault-injection hook (tests only)
    unsigned nbar = 0;
    const float *__restrict__ X = a.X;
    const float *__restrict__ Y = a.y;
    float *__restrict__ params = a.params;
    float *__restrict__ part = a.part;

    for (int i = tid; i < CAP * DP; i += FNT) Xs[i] = 0.f;

    const int64_t mbs = (a.mb <= 0 || a.mb >= a.n) ? a.n : a.mb;
    double sse_epoch = 0.0, gn_last = 0.0;

    for (int e = 0; e < a.epochs; ++e) {
        sse_epoch = 0.0;
        for (int64_t b0 = 0; b0 < a.n; b0 += mbs) {
            const int64_t m = min(mbs, a.n - b0);
            const float c = a.loss_mean ? 1.0f / (float)m : 1.0f;
            const int64_t r0 = b0 + (m * g) / G, r1 = b0 + (m * (g + 1)) / G;

            // ---- stage the first rows asynchronously (X and y are read-only for
            // the whole launch, so L1-allocating copies are safe) and the weights
            // through L2 (other blocks rewrote them), eight loads in flight per
            // thread
            __syncthreads();
            int64_t cs = r0;
            int cn = (int)min((int64_t)CAP, r1 - cs);
            if (cn > 0) {
                const float *Xg = X + cs * D;
                for (int i = tid; i < cn * D; i += FNT) {
                    const int s = i / D, k = i - s * D;
                    cp_async4(Xs + s * DP + k, Xg + i);
                }
                for (int i = tid; i < cn; i += FNT) cp_async4(ys + i, Y + cs + i);
            }
            for (int base = 0; base < P; base += 8 * FNT) {
                float v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = base + r * FNT + tid;
                    v[r] = (i < P) ? __ldcg(params + i) : 0.f;
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = base + r * FNT + tid;
                    if (i < HD) {
                        const int j = i / D, k = i - j * D;
                        Ws[j * WSTR + k] = v[r];
                    } else if (i < P) {
                        Bs[i - HD] = v[r];
                    }
                }
            }
            cp_async_wait_all();
            __syncthreads();
            float w[UPL][DP], b1r[UPL], w2r[UPL];
#pragma unroll
            for (int u = 0; u < UPL; ++u) {
                const int j = u * 32 + lane;
#pragma unroll
                for (int k = 0; k < DP; ++k) w[u][k] = (j < H && k < D) ? Ws[j * WSTR + k] : 0.f;
                b1r[u] = (j < H) ? Bs[j] : 0.f;
                w2r[u] = (j < H) ? Bs[H + j] : 0.f;
            }
            const float b2 = Bs[2 * H];

            float acc[UPL][DP], gb1a[UPL], gw2a[UPL], gb2a = 0.f;
            double sse = 0.0;
#pragma unroll
            for (int u = 0; u < UPL; ++u) {
                gb1a[u] = 0.f;
                gw2a[u] = 0.f;
#pragma unroll
                for (int k = 0; k < DP; ++k) acc[u][k] = 0.f;
            }

            // ---- forward + backward over this block's rows of the step
            while (cn > 0) {
                for (int s = warp; s < cn; s += FNW) {
                    const float4 *xr = reinterpret_cast<const float4 *>(Xs + s * DP);
                    float z[UPL];
#pragma unroll
                    for (int u = 0; u < UPL; ++u) z[u] = b1r[u];
#pragma unroll
                    for (int q = 0; q < DP / 4; ++q) {
                        const float4 xv = xr[q];
#pragma unroll
                        for (int u = 0; u < UPL; ++u) {
                            z[u] = fmaf(xv.x, w[u][4 * q + 0], z[u]);
                            z[u] = fmaf(xv.y, w[u][4 * q + 1], z[u]);
                            z[u] = fmaf(xv.z, w[u][4 * q + 2], z[u]);
                            z[u] = fmaf(xv.w, w[u][4 * q + 3], z[u]);
                        }
                    }
                    float hv[UPL], zp = 0.f;
#pragma unroll
                    for (int u = 0; u < UPL; ++u) {
                        hv[u] = Act<ACT>::f(z[u]);
                        zp = fmaf(hv[u], w2r[u], zp);
                    }
                    zp = warp_sum(zp);
                    const float o = sigmoid_out(zp + b2);
                    const float err = o - ys[s];
                    const float d2 = c * err * o * (1.0f - o);
                    sse += (double)err * (double)err;
                    gb2a += d2;
#pragma unroll
                    for (int u = 0; u < UPL; ++u) {
                        gw2a[u] = fmaf(d2, hv[u], gw2a[u]);
                        const float d1 = d2 * w2r[u] * Act<ACT>::df(hv[u]);
                        gb1a[u] += d1;
#pragma unroll
                        for (int q = 0; q < DP / 4; ++q) {
                            const float4 xv = xr[q];
                            acc[u][4 * q + 0] = fmaf(d1, xv.x, acc[u][4 * q + 0]);
                            acc[u][4 * q + 1] = fmaf(d1, xv.y, acc[u][4 * q + 1]);
                            acc[u][4 * q + 2] = fmaf(d1, xv.z, acc[u][4 * q + 2]);
                            acc[u][4 * q + 3] = fmaf(d1, xv.w, acc[u][4 * q + 3]);
                        }
                    }
                }
                cs += cn;
                cn = (int)min((int64_t)CAP, r1 - cs);
                if (cn > 0) {
                    __syncthreads();
                    const float *Xg = X + cs * D;
                    for (int i = tid; i < cn * D; i += FNT) {
                        const int s = i / D, k = i - s * D;
                        cp_async4(Xs + s * DP + k, Xg + i);
                    }
                    for (int i = tid; i < cn; i += FNT) cp_async4(ys + i, Y + cs + i);
                    cp_async_wait_all();
                    __syncthreads();
                }
            }

            // ---- block partial: warp partials summed in warp order
            __syncthreads();
            float *pw = parts + warp * P;
#pragma unroll
            for (int u = 0; u < UPL; ++u) {
                const int j = u * 32 + lane;
                if (j < H) {
#pragma unroll
                    for (int k = 0; k < DP; ++k)
                        if (k < D) pw[j * D + k] = acc[u][k];
                    pw[HD + j] = gb1a[u];
                    pw[HD + H + j] = gw2a[u];
                }
            }
            if (lane == 0) {
                pw[P - 1] = gb2a;
                s_red[warp] = sse;
            }
            __syncthreads();
            float *pg = part + (int64_t)g * P;
            for (int p = tid; p < P; p += FNT) {
                float s = parts[p];
#pragma unroll
                for (int q = 1; q < FNW; ++q) s += parts[q * P + p];
                pg[p] = s;
            }
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < FNW; ++q) t += s_red[q];
                a.lossp[g] = t;
            }
            if (!grid_barrier(a.bar, (++nbar) * (unsigned)G, a.status)) return;

            // ---- cross-block reduction in a fixed order, update, norm partial
            double gn = 0.0;
            const int64_t gw = (int64_t)g * FNW + warp;
            for (int64_t p0 = gw * PPW; p0 < P; p0 += (int64_t)G * FNW * PPW) {
                float v[PPW][QMAX];
#pragma unroll
                for (int i = 0; i < PPW; ++i)
#pragma unroll
                    for (int t = 0; t < QMAX; ++t) {
                        const int q = lane + 32 * t;
                        v[i][t] = (q < G && p0 + i < P) ? __ldcg(part + (int64_t)q * P + p0 + i) : 0.f;
                    }
                float old[PPW];
#pragma unroll
                for (int i = 0; i < PPW; ++i) old[i] = (lane == 0 && p0 + i < P) ? __ldcg(params + p0 + i) : 0.f;
#pragma unroll
                for (int i = 0; i < PPW; ++i) {
                    float s = v[i][0];
#pragma unroll
                    for (int t = 1; t < QMAX; ++t) s += v[i][t];
                    s = warp_sum(s);
                    if (lane == 0 && p0 + i < P) {
                        params[p0 + i] = old[i] - a.lr * s;
                        gn += (double)s * (double)s;
                    }
                }
            }
            if (lane == 0) s_red[warp] = gn;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < FNW; ++q) t += s_red[q];
                a.gnp[g] = t;
            }
            if (g == 0 && warp == 0) sse_epoch += fixed_sum(a.lossp, G, lane);
            if (!grid_barrier(a.bar, (++nbar) * (unsigned)G, a.status)) return;
            if (g == 0 && warp == 0) gn_last = fixed_sum(a.gnp, G, lane);
        }
        if (g == 0 && tid == 0) {
            const double C = a.loss_mean ? (a.n > 0 ? 1.0 / (double)a.n : 0.0) : 1.0;
            const double L = 0.5 * sse_epoch * C;
            if (a.loss_hist) a.loss_hist[e] = L;
            if (a.gnorm_hist) a.gnorm_hist[e] = sqrt(gn_last);
            if (!isfinite(L)) atomicOr(a.status, ST_NONFINITE);
        }
    }
}

template <int DP, int UPL>
void *pick_kernel(int act) {
    if (act == MLP_ACT_TANH) return (void *)k_fused_train<DP, UPL, MLP_ACT_TANH>;
    return (void *)k_fused_train<DP, UPL, MLP_ACT_SIGMOID>;
}

struct Choice {
    void *fn;
    size_t smem;
};

bool choose(int act, int D, int H, Choice *c) {
    if (D < 1 || H < 1) return false;
    if (D <= 8) {
        if (H <= 32) *c = {pick_kernel<8, 1>(act), smem_bytes<8>(D, H)};
        else if (H <= 64) *c = {pick_kernel<8, 2>(act), smem_bytes<8>(D, H)};
        else return false;
    } else if (D <= 16) {
        if (H <= 32) *c = {pick_kernel<16, 1>(act), smem_bytes<16>(D, H)};
        else if (H <= 64) *c = {pick_kernel<16, 2>(act), smem_bytes<16>(D, H)};
        else return false;
    } else if (D <= 36) {
        if (H <= 32) *c = {pick_kernel<36, 1>(act), smem_bytes<36>(D, H)};
        else if (H <= 64) *c = {pick_kernel<36, 2>(act), smem_bytes<36>(D, H)};
        else return false;
    } else if (D <= 48) {
        if (H <= 32) *c = {pick_kernel<48, 1>(act), smem_bytes<48>(D, H)};
        else if (H <= 64) *c = {pick_kernel<48, 2>(act), smem_bytes<48>(D, H)};
        else return false;
    } else if (D <= 64) {
        if (H <= 32) *c = {pick_kernel<64, 1>(act), smem_bytes<64>(D, H)};
        else return false;
    } else {
        return false;
    }
    return true;
}

// Resident blocks per SM for (kernel, dynamic smem) on the current device,
// computed once (the attribute call and the occupancy query are not free).
int blocks_per_sm(void *fn, size_t smem, cudaError_t *err) {
    struct Entry {
        void *fn;
        size_t smem;
        int dev;
        int per_sm;
    };
    static std::mutex mu;
    static Entry cache[64];
    static int ncache = 0;
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (int i = 0; i < ncache; ++i)
            if (cache[i].fn == fn && cache[i].smem == smem && cache[i].dev == dev) return cache[i].per_sm;
    }
    if (smem > 48 * 1024) {
        *err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (*err != cudaSuccess) return 0;
    }
    int per_sm = 0;
    *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FNT, smem);
    if (*err != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (ncache < 64) cache[ncache++] = {fn, smem, dev, per_sm};
    return per_sm;
}

}  // namespace

bool fused_supported(int D, int H) {
    Choice c;
    return choose(MLP_ACT_SIGMOID, D, H, &c);
}

size_t fused_scratch_bytes(int D, int H, int sms) {
    FusedScratch s;
    fused_scratch_carve(nullptr, D, H, sms, &s);
    return (size_t)(uintptr_t)s.bar + 256;
}

void fused_scratch_carve(void *base, int D, int H, int sms, FusedScratch *s) {
    (void)sms;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t P = (size_t)(D + 2) * H + 1;
    char *b = (char *)base;
    size_t off = 0;
    s->part = (float *)(b + off);
    off = al(off + sizeof(float) * GMAX * P);
    s->lossp = (double *)(b + off);
    off = al(off + sizeof(double) * GMAX);
    s->gnp = (double *)(b + off);
    off = al(off + sizeof(double) * GMAX);
    s->bar = (unsigned *)(b + off);
}

cudaError_t fused_train(int act, int D, int H, int64_t n, const float *X, const float *y, float *params,
                        float lr, int loss_mean, int epochs, int64_t mb, double *loss_hist, double *gnorm_hist,
                        int *status, const FusedScratch &s, int rows_per_block, int skip_block,
                        cudaStream_t st, int *grid_used) {
    Choice ch;
    if (!choose(act, D, H, &ch)) return cudaErrorInvalidValue;
    cudaError_t e;
    int per_sm = blocks_per_sm(ch.fn, ch.smem, &e);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int sms = device_sm_count();
    const int64_t mbs = (mb <= 0 || mb >= n) ? n : mb;
    if (rows_per_block < 1) rows_per_block = 64;
    int64_t G = cdiv(mbs > 0 ? mbs : 1, rows_per_block);
    if (G > (int64_t)per_sm * sms) G = (int64_t)per_sm * sms;
    if (G > GMAX) G = GMAX;
    if (G < 1) G = 1;
    if (grid_used) *grid_used = (int)G;
    const int64_t steps_per_epoch = n > 0 ? cdiv(n, mbs) : 0;
    // Barrier targets are 32-bit: split the epochs over launches if needed.
    int64_t max_epochs = steps_per_epoch > 0 ? (int64_t)(0x7fffffff / (2 * G * steps_per_epoch)) : epochs;
    if (max_epochs < 1) return cudaErrorInvalidValue;
    for (int e0 = 0; e0 < epochs; e0 += (int)max_epochs) {
        int ne = (int)((epochs - e0) < max_epochs ? (epochs - e0) : max_epochs);
        e = cudaMemsetAsync(s.bar, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        FArgs a;
        a.D = D;
        a.H = H;
        a.n = n;
        a.X = X;
        a.y = y;
        a.params = params;
        a.lr = lr;
        a.loss_mean = loss_mean;
        a.epochs = ne;
        a.mb = mb;
        a.loss_hist = loss_hist ? loss_hist + e0 : nullptr;
        a.gnorm_hist = gnorm_hist ? gnorm_hist + e0 : nullptr;
        a.status = status;
        a.part = s.part;
        a.lossp = s.lossp;
        a.gnp = s.gnp;
        a.bar = s.bar;
        a.skip_block = skip_block;
        void *args[] = {&a};
        e = cudaLaunchCooperativeKernel(ch.fn, dim3((unsigned)G), dim3(FNT), args, ch.smem, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mlp
