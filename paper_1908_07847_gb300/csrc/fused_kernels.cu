// Fused training kernel for small networks (D <= 64, H <= 128): one cooperative
// launch runs every step of every epoch.  Per step (Sec. 2.2 of arXiv
// 1908.07847: feed-forward, output error, backpropagation, gradient descent
// with no momentum):
//   1. every block stages the packed weights (through L2: other blocks rewrote
//      them) and its rows of X (asynchronous copies) in shared memory; the row
//      engine (row_engine.cuh) runs forward and backward with one hidden neuron
//      per lane and accumulates the gradient rows in registers; activations
//      never leave the chip;
//   2. row-group partials are summed in shared memory in group order and
//      written as one partial per block, with the block's FP64 squared error;
//   3. grid barrier; every warp then owns a few parameters: its lanes load the
//      block partials of a parameter in parallel (lane q takes blocks q, q+32,
//      ...), add them in that order and finish with a butterfly -- a fixed
//      order, so results are bitwise reproducible -- and lane 0 applies
//      w -= lr g.  Warp 0 of block 0 folds the loss partials in the same round.
//   4. a second grid barrier only before another step.  The gradient norm, if
//      asked for, is folded by the last block to finish (an arrival ticket).
#include <mutex>

#include "row_engine.cuh"

namespace mlp {

namespace {

constexpr int FNT = RE_NT;       // threads per block
constexpr int CAP = 64;          // rows staged in shared memory at a time
constexpr int QMAX = 5;          // blocks per lane in the cross-block sums
constexpr int GMAX = 32 * QMAX;  // largest grid
constexpr int PPW = 8;           // parameters per warp per round

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
    unsigned long long *bar;        // [0] barrier arrivals, [1] finish tickets
    unsigned long long bar_base;    // their values at launch
    unsigned long long ticket_base;
    int skip_block;
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Shared-memory layout (floats): packed weights [P], row-group partials
// [NG x P], CAP rows of X (DP wide, zero padded), CAP labels, z2 exchange.
__host__ __device__ inline int wm_floats(int D, int H) { return ((D + 2) * H + 1 + 3) & ~3; }

template <int DP>
size_t smem_bytes(int D, int H) {
    return sizeof(float) * ((size_t)wm_floats(D, H) + re_part_floats(D, H) + (size_t)CAP * DP + CAP + RE_ZX);
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

template <int DP, int WU, int ACT>
__global__ void __launch_bounds__(FNT, 2) k_fused_train(FArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_red[RE_NW];
    __shared__ int s_last;
    using Eng = RowEngine<DP, WU, ACT>;
    constexpr int NG = Eng::NG;
    const int D = a.D, H = a.H;
    const int P = (D + 2) * H + 1;
    float *Wm = smem;                               // packed weights
    float *gpart = Wm + wm_floats(D, H);            // NG x P row-group partials
    float *Xs = gpart + re_part_floats(D, H);       // CAP x DP rows
    float *ys = Xs + CAP * DP;                      // CAP labels
    float *zx = ys + CAP;                           // z2 exchange
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, g = blockIdx.x;
    // A launch after a failed one must not touch the counters; the status load
    // is consumed only before the first barrier, so it overlaps the staging.
    const int status0 = ld_volatile(a.status);
    if (g == a.skip_block) return;                  // fault-injection hook (tests only)
    unsigned long long target = a.bar_base;
    const float *__restrict__ X = a.X;
    const float *__restrict__ Y = a.y;
    float *__restrict__ params = a.params;
    float *__restrict__ part = a.part;
    Eng eng;
    eng.setup(H, D);

    for (int i = tid; i < CAP * DP; i += FNT) Xs[i] = 0.f;

    const int64_t mbs = (a.mb <= 0 || a.mb >= a.n) ? a.n : a.mb;
    const double Cl = a.loss_mean ? (a.n > 0 ? 1.0 / (double)a.n : 0.0) : 1.0;
    double sse_epoch = 0.0;

    for (int e = 0; e < a.epochs; ++e) {
        sse_epoch = 0.0;
        for (int64_t b0 = 0; b0 < a.n; b0 += mbs) {
            const int64_t m = min(mbs, a.n - b0);
            const bool epoch_end = b0 + mbs >= a.n;
            const bool last_step = (e == a.epochs - 1) && epoch_end;
            const float c = a.loss_mean ? 1.0f / (float)m : 1.0f;
            const int64_t r0 = b0 + (m * g) / G, r1 = b0 + (m * (g + 1)) / G;

            // ---- stage the first rows asynchronously (X and y are read-only for
            // the whole launch, so L1-allocating copies are safe) and the
            // weights with 16-byte copies through L2 (other blocks rewrote them)
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
            {
                const int P4 = P & ~3;
                for (int i = 4 * tid; i < P4; i += 4 * FNT) cp_async16_cg(Wm + i, params + i);
                if (tid < P - P4) Wm[P4 + tid] = __ldcg(params + P4 + tid);
            }
            cp_async_wait_all();
            __syncthreads();
            eng.load_weights(Wm);

            // ---- forward + backward over this block's rows of the step
            while (cn > 0) {
                eng.rows(Xs, ys, cn, c, zx);
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

            // ---- block partial: row-group partials summed in group order
            eng.write_group(gpart, s_red);
            __syncthreads();
            float *pg = part + (int64_t)g * P;
            for (int p = tid; p < P; p += FNT) {
                float s = gpart[p];
#pragma unroll
                for (int q = 1; q < NG; ++q) s += gpart[q * P + p];
                pg[p] = s;
            }
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < NG; ++q) t += s_red[q];
                a.lossp[g] = t;
            }
            if (status0 & ST_TIMEOUT) return;
            target += (unsigned long long)G;
            if (!grid_barrier(a.bar, target, a.status)) return;

            // ---- cross-block reduction in a fixed order and update; block 0's
            // warp 0 folds the loss partials in the same round of loads
            double gn = 0.0;
            if (g == 0 && warp == 0) sse_epoch += fixed_sum(a.lossp, G, lane);
            const int64_t gw = (int64_t)g * RE_NW + warp;
            for (int64_t p0 = gw * PPW; p0 < P; p0 += (int64_t)G * RE_NW * PPW) {
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
            if (epoch_end && g == 0 && tid == 0) {
                const double L = 0.5 * sse_epoch * Cl;
                if (a.loss_hist) a.loss_hist[e] = L;
                if (!isfinite(L)) atomicOr(a.status, ST_NONFINITE);
            }
            const bool want_gn = a.gnorm_hist && epoch_end;
            if (want_gn) {
                __syncthreads();
                if (lane == 0) s_red[warp] = gn;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int q = 0; q < RE_NW; ++q) t += s_red[q];
                    a.gnp[g] = t;
                }
            }
            if (!last_step) {
                target += (unsigned long long)G;
                if (!grid_barrier(a.bar, target, a.status)) return;
                if (want_gn && g == 0 && warp == 0) {
                    const double t = fixed_sum(a.gnp, G, lane);
                    if (lane == 0) a.gnorm_hist[e] = sqrt(t);
                }
            } else if (want_gn) {
                // The last block to finish folds the norm partials.
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    s_last = (atomicAdd(a.bar + 1, 1ull) == a.ticket_base + (unsigned long long)G - 1);
                    __threadfence();
                }
                __syncthreads();
                if (s_last && warp == 0) {
                    const double t = fixed_sum(a.gnp, G, lane);
                    if (lane == 0) a.gnorm_hist[e] = sqrt(t);
                }
            }
        }
    }
}

template <int DP>
void *pick_kernel(int act, int H) {
    const int wu = re_wu(H);
    if (act == MLP_ACT_TANH) {
        if (wu == 1) return (void *)k_fused_train<DP, 1, MLP_ACT_TANH>;
        if (wu == 2) return (void *)k_fused_train<DP, 2, MLP_ACT_TANH>;
        return (void *)k_fused_train<DP, 4, MLP_ACT_TANH>;
    }
    if (wu == 1) return (void *)k_fused_train<DP, 1, MLP_ACT_SIGMOID>;
    if (wu == 2) return (void *)k_fused_train<DP, 2, MLP_ACT_SIGMOID>;
    return (void *)k_fused_train<DP, 4, MLP_ACT_SIGMOID>;
}

struct Choice {
    void *fn;
    size_t smem;
};

bool choose(int act, int D, int H, Choice *c) {
    if (D < 1 || H < 1 || H > 128) return false;
    if (D <= 8) *c = {pick_kernel<8>(act, H), smem_bytes<8>(D, H)};
    else if (D <= 16) *c = {pick_kernel<16>(act, H), smem_bytes<16>(D, H)};
    else if (D <= 36) *c = {pick_kernel<36>(act, H), smem_bytes<36>(D, H)};
    else if (D <= 48) *c = {pick_kernel<48>(act, H), smem_bytes<48>(D, H)};
    else if (D <= 64) *c = {pick_kernel<64>(act, H), smem_bytes<64>(D, H)};
    else return false;
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
    s->bar = (unsigned long long *)(b + off);
}

cudaError_t fused_train(int act, int D, int H, int64_t n, const float *X, const float *y, float *params,
                        float lr, int loss_mean, int epochs, int64_t mb, double *loss_hist, double *gnorm_hist,
                        int *status, const FusedScratch &s, FusedCounters *ctr, int rows_per_block,
                        int skip_block, cudaStream_t st, int *grid_used) {
    Choice ch;
    if (!choose(act, D, H, &ch)) return cudaErrorInvalidValue;
    cudaError_t e;
    int per_sm = blocks_per_sm(ch.fn, ch.smem, &e);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int sms = device_sm_count();
    const int64_t mbs = (mb <= 0 || mb >= n) ? n : mb;
    if (rows_per_block < 1) rows_per_block = 32;
    int64_t G = cdiv(mbs > 0 ? mbs : 1, rows_per_block);
    if (G > (int64_t)per_sm * sms) G = (int64_t)per_sm * sms;
    if (G > GMAX) G = GMAX;
    if (G < 1) G = 1;
    if (grid_used) *grid_used = (int)G;
    const int64_t steps = n > 0 ? cdiv(n, mbs) * (int64_t)epochs : 0;
    if (steps == 0) return cudaSuccess;
    FArgs a;
    a.D = D;
    a.H = H;
    a.n = n;
    a.X = X;
    a.y = y;
    a.params = params;
    a.lr = lr;
    a.loss_mean = loss_mean;
    a.epochs = epochs;
    a.mb = mb;
    a.loss_hist = loss_hist;
    a.gnorm_hist = gnorm_hist;
    a.status = status;
    a.part = s.part;
    a.lossp = s.lossp;
    a.gnp = s.gnp;
    a.bar = s.bar;
    a.bar_base = ctr->bar;
    a.ticket_base = ctr->ticket;
    a.skip_block = skip_block;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(ch.fn, dim3((unsigned)G), dim3(FNT), args, ch.smem, st);
    if (e != cudaSuccess) return e;
    // Every block arrives at 2 * steps - 1 barriers and, when the norm is
    // folded at the end, takes one ticket.
    ctr->bar += (unsigned long long)G * (unsigned long long)(2 * steps - 1);
    if (gnorm_hist) ctr->ticket += (unsigned long long)G;
    return cudaSuccess;
}

}  // namespace mlp
