// Fused training kernel for small networks (D <= 64, H <= 128): one cooperative
// launch runs every step of every epoch, with one grid barrier per step.
//
// Per step (Sec. 2.2 of arXiv 1908.07847: feed-forward, output error,
// backpropagation, gradient descent with no momentum):
//   1. every block holds a copy of the packed weights in shared memory and its
//      rows of X (staged with asynchronous copies, kept there across epochs when
//      they fit); the row engine (row_engine.cuh) runs forward and backward
//      with one hidden neuron per lane and accumulates the gradient rows in
//      registers; activations never leave the chip;
//   2. the row groups' partial gradients are summed in shared memory in group
//      order, converted to 64-bit fixed point (scale 2^E) and added into a
//      global accumulator with integer atomics.  Integer addition does not
//      depend on the order, so the cross-block sum is exact and bitwise
//      reproducible; the block's squared error joins it the same way;
//   3. one grid barrier; every block then reads the whole summed gradient,
//      converts it back and applies w -= lr g to its own copy of the weights,
//      so all copies stay identical and no second barrier is needed; block 0
//      also records the epoch loss (and, if asked, the FP64 gradient norm);
//   4. the accumulator is triple-buffered: while reading buffer s, each block
//      clears its share of buffer s + 2, which the barrier of step s + 1 then
//      publishes before anyone adds into it.
// A grid of one block skips 2-4: it rounds its own partial the same way and
// updates in shared memory.  At the end block 0 writes its copy of the weights
// back.
#include <mutex>

#include "row_engine.cuh"

namespace mlp {

namespace {

constexpr int FNT = RE_NT;       // threads per block
constexpr int CAP = 64;          // rows staged in shared memory at a time
constexpr int RESIDENT = 192;    // rows a block keeps resident across steps
constexpr int GMAX = 320;        // largest grid

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
    int gshift;                     // fixed-point scale 2^gshift of the gradient
    double *loss_hist;
    double *gnorm_hist;
    int *status;
    long long *acc;                 // 3 x (P + 1) fixed-point accumulators
    int rot;                        // buffer of the first step
    unsigned long long *bar;        // barrier arrivals
    unsigned long long bar_base;    // its value at launch
    int skip_block;
};

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Shared-memory layout (floats): packed weights [P], row-group partials
// [NG x P], rows of X (DP wide, zero padded), labels, z2 exchange.
__host__ __device__ inline int wm_floats(int D, int H) { return ((D + 2) * H + 1 + 3) & ~3; }

template <int DP>
size_t smem_bytes(int D, int H, int rows) {
    return sizeof(float) * ((size_t)wm_floats(D, H) + re_part_floats(D, H) + (size_t)rows * DP + rows + RE_ZX);
}

__device__ __forceinline__ void red_add(long long *p, long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One block per SM (the fused grid rarely needs more than one wave): with the
// register file to itself a lane keeps eight rows in flight for H > 32, and
// three for H <= 32 with D <= 36, without spilling.
template <int DP, int WU>
__host__ __device__ constexpr int fused_rb1() { return (WU == 1 && DP <= 36) ? 3 : 2; }

template <int DP, int WU, int ACT>
__global__ void __launch_bounds__(FNT, 1) k_fused_train(FArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_red[RE_NW];
    __shared__ long long s_sse;   // the step's fixed-point squared-error sum
    __shared__ double s_gn[RE_NW];
    using Eng = RowEngine<DP, WU, ACT, fused_rb1<DP, WU>(), 8>;
    constexpr int NG = Eng::NG;
    const int D = a.D, H = a.H;
    const int P = (D + 2) * H + 1;
    const int P1 = P + 1;                           // + the squared error
    const int tid = threadIdx.x;
    const int G = gridDim.x, g = blockIdx.x;
    // A launch after a failed one must not touch the counters; the status load
    // is consumed only before the first barrier, so it overlaps the staging.
    const int status0 = ld_volatile(a.status);
    if (g == a.skip_block) return;                  // fault-injection hook (tests only)

    const int64_t mbs = (a.mb <= 0 || a.mb >= a.n) ? a.n : a.mb;
    // Rows of a step per block, and whether they stay resident for the launch.
    const int64_t rows_max = cdiv(mbs, G);
    const bool resident = (mbs == a.n) && rows_max <= RESIDENT;
    const int xcap = resident ? RESIDENT : CAP;
    float *Wm = smem;                               // packed weights
    float *gpart = Wm + wm_floats(D, H);            // NG x P row-group partials
    float *Xs = gpart + re_part_floats(D, H);       // xcap x DP rows
    float *ys = Xs + xcap * DP;                     // xcap labels
    float *zx = ys + xcap;                          // z2 exchange
    unsigned long long target = a.bar_base;
    const float *__restrict__ X = a.X;
    const float *__restrict__ Y = a.y;
    Eng eng;
    eng.setup(H, D);
    const float gscale = __int_as_float((127 - a.gshift) << 23);   // 2^-gshift
    const float gup = __int_as_float((127 + a.gshift) << 23);      // 2^gshift
    const double Cl = a.loss_mean ? (a.n > 0 ? 1.0 / (double)a.n : 0.0) : 1.0;

    {
        // Initial weights: 16-byte copies through L2, then the tail.
        const int P4 = P & ~3;
        for (int i = 4 * tid; i < P4; i += 4 * FNT) cp_async16_cg(Wm + i, a.params + i);
        if (tid < P - P4) Wm[P4 + tid] = __ldcg(a.params + P4 + tid);
    }
    auto stage = [&](int64_t r0, int cn) {
        const float *Xg = X + r0 * D;
        for (int i = tid; i < cn * D; i += FNT) {
            const int s = i / D, k = i - s * D;
            cp_async4(Xs + s * DP + k, Xg + i);
        }
        for (int i = tid; i < cn; i += FNT) cp_async4(ys + i, Y + r0 + i);
    };
    if (resident) {
        const int64_t r0 = (mbs * g) / G, r1 = (mbs * (g + 1)) / G;
        if (r1 > r0) stage(r0, (int)(r1 - r0));
    }
    // Only the padding columns D..DP-1 of the row buffer are read without
    // being copied; zero them while the copies are in flight (disjoint words).
    if (DP > D)
        for (int i = tid; i < xcap * (DP - D); i += FNT) Xs[(i / (DP - D)) * DP + D + i % (DP - D)] = 0.f;
    cp_async_wait_all();
    __syncthreads();

    double sse_epoch = 0.0;
    int64_t step = 0;
    for (int e = 0; e < a.epochs; ++e) {
        sse_epoch = 0.0;
        for (int64_t b0 = 0; b0 < a.n; b0 += mbs, ++step) {
            const int64_t m = min(mbs, a.n - b0);
            const bool epoch_end = b0 + mbs >= a.n;
            const float c = a.loss_mean ? 1.0f / (float)m : 1.0f;
            const int64_t r0 = b0 + (m * g) / G, r1 = b0 + (m * (g + 1)) / G;
            long long *acc = a.acc + (size_t)((a.rot + step) % 3) * P1;
            long long *acc_clear = a.acc + (size_t)((a.rot + step + 2) % 3) * P1;

            // ---- forward + backward over this block's rows of the step
            eng.load_weights(Wm);
            if (resident) {
                if (r1 > r0) eng.rows(Xs, ys, (int)(r1 - r0), c, zx);
            } else {
                for (int64_t cs = r0; cs < r1; cs += CAP) {
                    const int cn = (int)min((int64_t)CAP, r1 - cs);
                    __syncthreads();
                    stage(cs, cn);
                    cp_async_wait_all();
                    __syncthreads();
                    eng.rows(Xs, ys, cn, c, zx);
                }
            }

            // ---- block partial, in fixed point, into the global accumulator
            eng.write_group(gpart, s_red);
            __syncthreads();
            if (G == 1) {
                // A single block holds the whole step: its partial is the sum.  The
                // same fixed-point rounding as the cross-block path, applied here,
                // without the global accumulator, the barrier or the counters.
                if (status0 & ST_TIMEOUT) return;
                const bool want_gn = a.gnorm_hist && epoch_end;
                double gn = 0.0;
                int bad = 0;
                for (int p = tid; p < P; p += FNT) {
                    float s = gpart[p];
#pragma unroll
                    for (int q = 1; q < NG; ++q) s += gpart[q * P + p];
                    const float v = s * gup;
                    if (!(fabsf(v) < 4.0e18f)) bad = 1;
                    // = (float)llrint(v) * 2^-gshift: below 2^23 both round v to the
                    // same integer, above it v already is one (no 64-bit conversion)
                    const float gsum = rintf(v) * gscale;
                    Wm[p] -= a.lr * gsum;
                    if (want_gn) gn = fma((double)gsum, (double)gsum, gn);
                }
                if (bad) atomicOr(a.status, ST_NONFINITE);
                if (want_gn) {
                    gn = warp_sum(gn);
                    if ((tid & 31) == 0) s_gn[tid >> 5] = gn;
                }
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int q = 0; q < NG; ++q) t += s_red[q];
                    const double v = t * 4294967296.0;
                    if (!(v < 4.0e18)) atomicOr(a.status, ST_NONFINITE);
                    sse_epoch += (double)__double2ll_rn(v) * (1.0 / 4294967296.0);
                    if (epoch_end) {
                        const double L = 0.5 * sse_epoch * Cl;
                        if (a.loss_hist) a.loss_hist[e] = L;
                        if (!isfinite(L)) atomicOr(a.status, ST_NONFINITE);
                        if (want_gn) {
                            double u = 0.0;
                            for (int q = 0; q < RE_NW; ++q) u += s_gn[q];
                            a.gnorm_hist[e] = sqrt(u);
                        }
                    }
                }
                __syncthreads();
                continue;
            }
            // Each of the G block partials stays below 2^63 / G in magnitude, so
            // their integer sum cannot wrap; a partial beyond that (or NaN) is
            // flagged as non-finite instead of silently corrupting the update.
            const float lim = 9.2e18f / (float)G;
            int bad = 0;
            for (int p = tid; p < P; p += FNT) {
                float s = gpart[p];
#pragma unroll
                for (int q = 1; q < NG; ++q) s += gpart[q * P + p];
                const float v = s * gup;
                if (!(fabsf(v) < lim)) bad = 1;   // out of range or NaN
                red_add(acc + p, __float2ll_rn(v));
            }
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < NG; ++q) t += s_red[q];
                const double v = t * 4294967296.0;
                if (!(v < (double)lim)) bad = 1;
                red_add(acc + P, __double2ll_rn(v));
            }
            if (bad) atomicOr(a.status, ST_NONFINITE);
            if (status0 & ST_TIMEOUT) return;
            target += (unsigned long long)G;
            if (!grid_barrier(a.bar, target, a.status)) return;

            // ---- every block applies the summed gradient to its own copy
            const bool want_gn = g == 0 && a.gnorm_hist && epoch_end;
            double gn = 0.0;
            // the gradient and the squared error (entry P) in one round trip
            for (int base = 0; base < P1; base += 12 * FNT) {
                long long v[12];  // twelve loads in flight per thread: one round trip up to P = 3071
#pragma unroll
                for (int r = 0; r < 12; ++r) {
                    const int p = base + r * FNT + tid;
                    v[r] = (p < P1) ? __ldcg(acc + p) : 0ll;
                }
#pragma unroll
                for (int r = 0; r < 12; ++r) {
                    const int p = base + r * FNT + tid;
                    if (p == P) s_sse = v[r];
                    if (p < P) {
                        const float gsum = (float)v[r] * gscale;
                        Wm[p] -= a.lr * gsum;
                        if (want_gn) gn = fma((double)gsum, (double)gsum, gn);
                    }
                }
            }
            for (int p = (int)(((int64_t)P1 * g) / G) + tid; p < (int)(((int64_t)P1 * (g + 1)) / G); p += FNT)
                acc_clear[p] = 0;
            if (g == 0) {
                if (want_gn) {
                    gn = warp_sum(gn);
                    if ((tid & 31) == 0) s_red[tid >> 5] = gn;
                }
                __syncthreads();
                if (tid == 0) {
                    sse_epoch += (double)s_sse * (1.0 / 4294967296.0);
                    if (epoch_end) {
                        const double L = 0.5 * sse_epoch * Cl;
                        if (a.loss_hist) a.loss_hist[e] = L;
                        if (!isfinite(L)) atomicOr(a.status, ST_NONFINITE);
                        if (want_gn) {
                            double t = 0.0;
                            for (int q = 0; q < RE_NW; ++q) t += s_red[q];
                            a.gnorm_hist[e] = sqrt(t);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (g == 0)
        for (int p = tid; p < P; p += FNT) a.params[p] = Wm[p];
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
    int DP;
};

bool choose(int act, int D, int H, Choice *c) {
    if (D < 1 || H < 1 || H > 128) return false;
    if (D <= 8) *c = {pick_kernel<8>(act, H), 8};
    else if (D <= 16) *c = {pick_kernel<16>(act, H), 16};
    else if (D <= 36) *c = {pick_kernel<36>(act, H), 36};
    else if (D <= 48) *c = {pick_kernel<48>(act, H), 48};
    else if (D <= 64) *c = {pick_kernel<64>(act, H), 64};
    else return false;
    return true;
}

size_t choice_smem(const Choice &c, int D, int H, int rows) {
    switch (c.DP) {
        case 8: return smem_bytes<8>(D, H, rows);
        case 16: return smem_bytes<16>(D, H, rows);
        case 36: return smem_bytes<36>(D, H, rows);
        case 48: return smem_bytes<48>(D, H, rows);
        default: return smem_bytes<64>(D, H, rows);
    }
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
    {
        // Raise the kernel's ceiling to the device's opt-in limit rather than to
        // this request: a cached entry for a larger request must not find the
        // ceiling lowered by a smaller one made since.  Always: the default
        // ceiling (48 KB) covers the kernel's static shared memory as well.
        int optin = 0;
        cudaFuncAttributes fa;
        *err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (*err == cudaSuccess) *err = cudaFuncGetAttributes(&fa, fn);
        if (*err != cudaSuccess) return 0;
        const size_t ceiling = (size_t)optin - fa.sharedSizeBytes;
        if (smem > ceiling) {
            *err = cudaErrorInvalidValue;
            return 0;
        }
        *err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ceiling);
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
    const size_t P1 = (size_t)(D + 2) * H + 2;
    char *b = (char *)base;
    s->acc = (long long *)b;
    s->bar = (unsigned long long *)(b + al(sizeof(long long) * 3 * P1));
}

cudaError_t fused_train(int act, int D, int H, int64_t n, const float *X, const float *y, float *params,
                        float lr, int loss_mean, int epochs, int64_t mb, double *loss_hist, double *gnorm_hist,
                        int *status, const FusedScratch &s, FusedCounters *ctr, int rows_per_block,
                        int skip_block, cudaStream_t st, int *grid_used) {
    Choice ch;
    if (!choose(act, D, H, &ch)) return cudaErrorInvalidValue;
    const int64_t mbs = (mb <= 0 || mb >= n) ? n : mb;
    if (rows_per_block < 1) rows_per_block = 32;
    int64_t G = cdiv(mbs > 0 ? mbs : 1, rows_per_block);
    if (G > GMAX) G = GMAX;
    if (G < 1) G = 1;
    // Shared memory depends on whether the rows stay resident.
    bool resident = (mbs == n) && cdiv(mbs, G) <= RESIDENT;
    size_t smem = choice_smem(ch, D, H, resident ? RESIDENT : CAP);
    cudaError_t e;
    int per_sm = blocks_per_sm(ch.fn, smem, &e);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)per_sm * device_sm_count();
    if (G > cap) {
        G = cap;
        resident = (mbs == n) && cdiv(mbs, G) <= RESIDENT;
        smem = choice_smem(ch, D, H, resident ? RESIDENT : CAP);
        per_sm = blocks_per_sm(ch.fn, smem, &e);
        if (e != cudaSuccess) return e;
        if ((int64_t)per_sm * device_sm_count() < G) return cudaErrorInvalidConfiguration;
    }
    if (grid_used) *grid_used = (int)G;
    const int64_t steps = n > 0 ? cdiv(n, mbs) * (int64_t)epochs : 0;
    if (steps == 0) return cudaSuccess;
    // Fixed-point scale of the gradient sums: 2^40 leaves 2^23 of range for a
    // mean loss; a summed loss scales the range with the rows of a step.
    int gshift = 40;
    if (!loss_mean) {
        int lg = 0;
        while (((int64_t)1 << lg) < mbs) ++lg;
        gshift = 40 - lg;
        if (gshift < 8) gshift = 8;
    }
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
    a.gshift = gshift;
    a.loss_hist = loss_hist;
    a.gnorm_hist = gnorm_hist;
    a.status = status;
    a.acc = s.acc;
    a.rot = ctr->rot;
    a.bar = s.bar;
    a.bar_base = ctr->bar;
    a.skip_block = skip_block;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(ch.fn, dim3((unsigned)G), dim3(FNT), args, smem, st);
    if (e != cudaSuccess) return e;
    // One barrier per step for every block; the accumulator rotates by a step.
    // A single block uses neither (it sums and updates on chip).
    if (G > 1) {
        ctr->bar += (unsigned long long)G * (unsigned long long)steps;
        ctr->rot = (int)((ctr->rot + steps) % 3);
    }
    return cudaSuccess;
}

}  // namespace mlp
