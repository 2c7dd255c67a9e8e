// Many independent networks in one launch, each net's epoch computed as two
// small register-tiled products (inputs up to 36 wide).  The method per net is
// the one of batched_kernels.cu (Sec. 2.2 of arXiv 1908.07847: feed-forward,
// output error, backpropagation, full-batch gradient descent without
// momentum); only the schedule differs.  Per pass of rows (as many as the
// h / d1 buffer holds at the net's own width -- W^T is stored at the net's
// own width too and the buffer takes the rest of the space the widest net of
// the launch needs; X^T holds up to 128 rows, a net's whole set when it fits):
//
//   1. Z = [X | 1] [W1 | b1]^T, every thread a 4-row x 4-unit tile of Z with
//      its 16 sums in registers (one 16-byte word of X^T and one of W^T a
//      step: 16 multiply-adds per two shared-memory loads); h = f(Z) goes to
//      shared memory;
//   2. one thread a row: z2 = b2 + h w2, o = sigmoid(z2), d2 = c (o - y) o (1 - o);
//   3. d1 = d2 w2 f'(h) written over h, and the row subsets' partial
//      gw2 = sum_rows h d2, in registers;
//   4. [gW1 | gb1] += d1^T [X | 1], every thread up to three 4-unit x 4-input
//      tiles held in registers across the chunks (per 4 rows: 8 loads, 64
//      multiply-adds).
// At the end of the epoch each thread applies its own tiles' update to the
// transposed weights in shared memory; gw2, gb2, the loss and the gradient
// norm are summed in fixed orders.  Every sum has one fixed order, so a run
// is bitwise reproducible.  X^T (ncap columns), W^T, and h / d1 (hcap rows)
// live in shared memory; padding rows of X^T and padding units of W^T and w2
// are zero, so their d1 and their share of z2 are zero and they add nothing.
// Nets with more than 128 rows stream their rows in chunks of 128.
//
// The products are bound by shared-memory bandwidth, so tiles are handed to
// lanes for the fewest wavefronts.  A 16-byte load is served a half-warp at a
// time; the two quarter-warps of a half share one wavefront only if the
// distinct words they read add up to at most 128 bytes, without two of them in
// one bank.  Both products therefore give a quarter-warp 4 unit quads x 2 row
// (or input) quads, so a load reads at most 4 distinct words a quarter, and
// X^T rows are 4 mod 8 words apart so that neighbouring input quads sit in
// different banks.
#include "mlp_internal.cuh"

namespace mlp {

namespace {

constexpr int TNT = 128;          // threads per block
constexpr int TSLOTS = 3;         // gradient tiles a thread holds (<= 32 x 10 tiles)

struct TLayout {
    int K;       // D + 1 (the ones column carries the bias)
    int KQ;      // K rounded up to 4, / 4
    int ncap;    // rows of X^T held at a time (multiple of 4; all of a net's rows when they fit)
    int xs;      // row stride of X^T: ncap, or ncap + 4, whichever is 4 mod 8 (so that the rows of
                 //   two neighbouring input quads start 16 words apart: no bank conflict between them)
    int hcap;    // rows of h / d1 a pass computes (multiple of 4, <= ncap)
    int HP;      // Hmax rounded up to 4
    int HSS;     // h / d1 buffer: hcap rows of HP + 4 floats (nets narrower than Hmax fit more rows)
    // float offsets
    int xt, wt, hs, w2, d2, gwp, red;
    int total;
};

__host__ __device__ inline TLayout t_layout(int D, int Hmax, int ncap, int hcap) {
    TLayout L;
    L.K = D + 1;
    L.KQ = (L.K + 3) / 4;
    L.ncap = ncap;
    L.xs = (ncap & 7) ? ncap : ncap + 4;
    L.hcap = hcap;
    L.HP = (Hmax + 3) & ~3;
    L.HSS = L.HP + 4;
    L.xt = 0;                                   // X^T: 4 KQ rows x xs
    L.wt = L.xt + 4 * L.KQ * L.xs;              // W^T: 4 KQ rows x HP
    L.hs = L.wt + 4 * L.KQ * L.HP;              // h / d1: hcap x HSS, and at least four rows at
    const int hsz = hcap * L.HSS;               //   the widest stride a net can use (HSS + 4), so
    const int hmin = 4 * (L.HSS + 4);           //   that a pass always takes at least four rows
    L.w2 = L.hs + (hsz > hmin ? hsz : hmin);    // w2: HP
    L.d2 = L.w2 + L.HP;                         // d2: ncap (a pass never exceeds it)
    L.gwp = L.d2 + ncap;                        // gw2 partials: TNT x 4
    L.red = L.gwp + 4 * TNT;                    // reductions: 4 warps x (sse, gb2) + 4 doubles
    L.total = L.red + 32;
    return L;
}

// Hidden-unit activation.  Sigmoid (Eq. 1) as 1 / (1 + 2^(-x log2 e)): one
// exp2 and one reciprocal (ex2.approx, rcp.approx refined by a Newton step),
// half the instructions of the output unit's sigmoid_f32.  It drops that
// function's split-constant reduction, so its error is bounded in absolute
// terms: the relative error of 2^(-x log2 e) grows like |x| 2^-24 while the
// value it feeds, sigmoid(x), shrinks like e^x for x < 0.  Measured on the
// GPU against FP64 over [-100, 100]: absolute error <= 9.2e-8; relative
// error <= 2.6e-7 for x >= -3 and <= 5.0e-7 for x >= -8.
// Inputs below -87 are raised to -87 so that 1 + e stays finite (the result
// is then below 2e-38); NaN passes through.
template <int ACT> __device__ __forceinline__ float hidden_f(float x) { return Act<ACT>::f(x); }
template <> __device__ __forceinline__ float hidden_f<MLP_ACT_SIGMOID>(float x) {
    const float L2E = 1.44269504088896341f;
    x = x < -87.0f ? -87.0f : x;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-x * L2E));
    const float d = 1.0f + e;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return fmaf(r, fmaf(-d, r, 1.0f), r);
}

// f'(z) through the value h = f(z), as one fused multiply-add: h - h^2 for
// sigmoid, 1 - h^2 for tanh.
template <int ACT> __device__ __forceinline__ float dact(float h);
template <> __device__ __forceinline__ float dact<MLP_ACT_SIGMOID>(float h) { return fmaf(-h, h, h); }
template <> __device__ __forceinline__ float dact<MLP_ACT_TANH>(float h) { return fmaf(-h, h, 1.0f); }

// Gradient tile t (of HQ x KQ) -> its input quad kq and unit quad uq.  Input
// quads go in pairs, unit-major inside a pair, so a quarter-warp covers 4 unit
// quads x 2 input quads (at most 4 distinct 16-byte words a load: one
// wavefront a half-warp); an odd last input quad follows, unit-major.
__device__ __forceinline__ void grad_tile(int t, int HQ, int KQ, int &kq, int &uq) {
    const int TA = (KQ >> 1) * 2 * HQ;
    if (t < TA) {
        const int p = t / (2 * HQ), rem = t - p * 2 * HQ;
        uq = rem >> 1;
        kq = 2 * p + (rem & 1);
    } else {
        uq = t - TA;
        kq = KQ - 1;
    }
}

template <int ACT>
__device__ __forceinline__ void net_tiled(const BatchNet &nd, int D, int epochs, float lr, int loss_mean,
                                          int *status, float *sm, const TLayout &L) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = nd.H, K = L.K, HQ = (H + 3) / 4, HP = L.HP;
    // W^T rows are as wide as this net's units (HN floats); the h / d1 buffer
    // starts right after them, so a net narrower than the widest of the
    // launch gets the rest of the widest net's W^T as extra h / d1 rows
    const int HN = 4 * HQ;
    const int64_t n = nd.n;
    float *XT = sm + L.xt, *WT = sm + L.wt, *HS = sm + L.wt + 4 * L.KQ * HN, *w2s = sm + L.w2, *d2s = sm + L.d2;
    float *gwp = sm + L.gwp, *red = sm + L.red;
    double *redd = (double *)(red + 16);
    const float *P = nd.params;
    const int HD = H * D;

    // W^T (row k < D: W1[., k]; row D: b1; rows above and units >= H: 0), w2
    for (int i = tid; i < 4 * L.KQ * HN; i += TNT) {
        const int k = i / HN, j = i - k * HN;
        float v = 0.f;
        if (j < H) v = k < D ? P[j * D + k] : (k == D ? P[HD + j] : 0.f);
        WT[i] = v;
    }
    for (int j = tid; j < HP; j += TNT) w2s[j] = j < H ? P[HD + H + j] : 0.f;
    float b2 = P[HD + 2 * H];
    // X^T of rows r0 .. r0 + nc - 1 (row D: ones; padding rows and columns 0)
    auto load_chunk = [&](int64_t r0, int nc) {
        const int cols = L.ncap;
        for (int i = tid; i < 4 * L.KQ * cols; i += TNT) {
            const int k = i / cols, r = i - k * cols;
            float v = 0.f;
            if (r < nc) v = k < D ? nd.X[(r0 + r) * D + k] : (k == D ? 1.f : 0.f);
            XT[k * L.xs + r] = v;
        }
    };
    const bool resident = n <= L.ncap;
    if (resident) load_chunk(0, (int)n);
    __syncthreads();
    const float c = loss_mean ? 1.0f / (float)n : 1.0f;
    const double C = loss_mean ? 1.0 / (double)n : 1.0;
    const bool want_gn = nd.gnorm_hist != nullptr;
    const int KQ = L.KQ;
    const int T2 = HQ * KQ;             // gradient tiles (4 units x 4 inputs)
    const int RS = TNT / HQ;            // row subsets of step 3
    const int uq3 = tid % HQ, rs3 = tid / HQ;
    // h / d1 rows are as wide as this net's units (in 16-byte words: HQ,
    // plus one or two so that the stride is odd and rows start in different
    // banks); a pass takes as many rows as the buffer holds at that stride
    const int hss = 4 * (HQ + 1 + (HQ & 1));
    const int hpass = min(128, ((L.w2 - (L.wt + 4 * L.KQ * HN)) / hss) & ~3);

    for (int e = 0; e < epochs; ++e) {
        float g[TSLOTS][4][4];
#pragma unroll
        for (int s = 0; s < TSLOTS; ++s)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < 4; ++k) g[s][u][k] = 0.f;
        float gw2a[4] = {0.f, 0.f, 0.f, 0.f};
        float sse_f = 0.f, gb2_f = 0.f;

        for (int64_t r0 = 0; r0 < n; r0 += L.ncap) {
            const int ncx = (int)min((int64_t)L.ncap, n - r0);
            if (!resident) {
                __syncthreads();
                load_chunk(r0, ncx);
                __syncthreads();
            }
            // passes of up to hcap rows over the rows of X^T held
            for (int h0 = 0; h0 < ncx; h0 += hpass) {
                const int nc = min(hpass, ncx - h0);
                const int nc4 = (nc + 3) & ~3;
                const float *XTc = XT + h0;   // column h0 of X^T: this pass's first row
                if (h0 > 0) __syncthreads();  // the previous pass is done with h / d1
                // ---- 1. Z = [X | 1] [W1 | b1]^T by 4 x 4 tiles, h = f(Z)
                // tiles in pairs of row quads, unit-major inside a pair: a
                // quarter-warp covers 2 row quads x 4 unit quads, so each of its
                // 16-byte loads touches at most 4 distinct words (one wavefront
                // a half-warp); an odd last row quad leaves its pair's second
                // half idle
                const int RQ = nc4 >> 2, T1 = ((RQ + 1) >> 1) * 2 * HQ;
                for (int t = tid; t < T1; t += TNT) {
                    const int rp = t / (2 * HQ), rem = t - rp * 2 * HQ;
                    const int uq = rem >> 1, rq = 2 * rp + (rem & 1);
                    if (rq >= RQ) continue;
                    float z[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int u = 0; u < 4; ++u) z[i][u] = 0.f;
                    const float *xa = XTc + 4 * rq, *wb = WT + 4 * uq;
#pragma unroll 8
                    for (int k = 0; k < K; ++k) {
                        const float4 a = *reinterpret_cast<const float4 *>(xa + k * L.xs);
                        const float4 b = *reinterpret_cast<const float4 *>(wb + k * HN);
                        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int u = 0; u < 4; ++u) z[i][u] = fmaf(av[i], bv[u], z[i][u]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        *reinterpret_cast<float4 *>(HS + (4 * rq + i) * hss + 4 * uq) =
                            make_float4(hidden_f<ACT>(z[i][0]), hidden_f<ACT>(z[i][1]), hidden_f<ACT>(z[i][2]),
                                        hidden_f<ACT>(z[i][3]));
                }
                __syncthreads();
                // ---- 2. one thread a row: z2, o, d2 (rows nc .. nc4 - 1 get d2 = 0)
                for (int r = tid; r < nc4; r += TNT) {
                    float d2 = 0.f;
                    if (r < nc) {
                        const float *hr = HS + r * hss;
                        float za = 0.f, zb = 0.f, zc = 0.f, zd = 0.f;
                        for (int q = 0; q < HQ; ++q) {
                            const float4 h4 = *reinterpret_cast<const float4 *>(hr + 4 * q);
                            const float4 w4 = *reinterpret_cast<const float4 *>(w2s + 4 * q);
                            za = fmaf(h4.x, w4.x, za);
                            zb = fmaf(h4.y, w4.y, zb);
                            zc = fmaf(h4.z, w4.z, zc);
                            zd = fmaf(h4.w, w4.w, zd);
                        }
                        const float o = sigmoid_out(((za + zb) + (zc + zd)) + b2);
                        const float err = o - nd.y[r0 + h0 + r];
                        d2 = c * err * o * (1.0f - o);
                        sse_f = fmaf(err, err, sse_f);
                        gb2_f += d2;
                    }
                    d2s[r] = d2;
                }
                __syncthreads();
                // ---- 3. d1 = d2 w2 f'(h) over h; partial gw2 = sum h d2 per row subset
                if (rs3 < RS) {
                    const float4 w4 = *reinterpret_cast<const float4 *>(w2s + 4 * uq3);
                    for (int r = rs3; r < nc4; r += RS) {
                        float *hp = HS + r * hss + 4 * uq3;
                        const float4 h4 = *reinterpret_cast<const float4 *>(hp);
                        const float d2 = d2s[r];
                        gw2a[0] = fmaf(h4.x, d2, gw2a[0]);
                        gw2a[1] = fmaf(h4.y, d2, gw2a[1]);
                        gw2a[2] = fmaf(h4.z, d2, gw2a[2]);
                        gw2a[3] = fmaf(h4.w, d2, gw2a[3]);
                        *reinterpret_cast<float4 *>(hp) =
                            make_float4((d2 * w4.x) * dact<ACT>(h4.x), (d2 * w4.y) * dact<ACT>(h4.y),
                                        (d2 * w4.z) * dact<ACT>(h4.z), (d2 * w4.w) * dact<ACT>(h4.w));
                    }
                }
                __syncthreads();
                // ---- 4. [gW1 | gb1] += d1^T [X | 1], 4 rows at a time
#pragma unroll
                for (int s = 0; s < TSLOTS; ++s) {
                    const int t = tid + s * TNT;
                    if (t < T2) {
                        int kq, uq;
                        grad_tile(t, HQ, KQ, kq, uq);
                        const float *da = HS + 4 * uq;
                        const float *xb = XTc + 4 * kq * L.xs;
                        for (int rr = 0; rr < nc4; rr += 4) {
                            float4 dv[4], xv[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                dv[i] = *reinterpret_cast<const float4 *>(da + (rr + i) * hss);
#pragma unroll
                            for (int k = 0; k < 4; ++k) xv[k] = *reinterpret_cast<const float4 *>(xb + k * L.xs + rr);
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float d[4] = {dv[i].x, dv[i].y, dv[i].z, dv[i].w};
                                const float xr[4] = {i == 0 ? xv[0].x : i == 1 ? xv[0].y : i == 2 ? xv[0].z : xv[0].w,
                                                     i == 0 ? xv[1].x : i == 1 ? xv[1].y : i == 2 ? xv[1].z : xv[1].w,
                                                     i == 0 ? xv[2].x : i == 1 ? xv[2].y : i == 2 ? xv[2].z : xv[2].w,
                                                     i == 0 ? xv[3].x : i == 1 ? xv[3].y : i == 2 ? xv[3].z : xv[3].w};
#pragma unroll
                                for (int u = 0; u < 4; ++u)
#pragma unroll
                                    for (int k = 0; k < 4; ++k) g[s][u][k] = fmaf(d[u], xr[k], g[s][u][k]);
                            }
                        }
                    }
                }
            }
            if (!resident) __syncthreads();   // the next chunk overwrites X^T and h
        }

        // ---- end of epoch: reductions in fixed orders, then the update
        if (rs3 < RS)
            *reinterpret_cast<float4 *>(gwp + rs3 * 4 * HQ + 4 * uq3) = make_float4(gw2a[0], gw2a[1], gw2a[2], gw2a[3]);
        sse_f = warp_sum(sse_f);
        gb2_f = warp_sum(gb2_f);
        if (lane == 0) {
            red[2 * warp] = sse_f;
            red[2 * warp + 1] = gb2_f;
        }
        __syncthreads();
        float gb2 = 0.f;
        double sse = 0.0;
        for (int w = 0; w < TNT / 32; ++w) {
            sse += (double)red[2 * w];
            gb2 += red[2 * w + 1];
        }
        double gn = 0.0;
        // gw2 (rows subsets in order) and the w2 / b2 update
        for (int j = tid; j < H; j += TNT) {
            float v = 0.f;
            for (int q = 0; q < RS; ++q) v += gwp[q * 4 * HQ + j];
            w2s[j] -= lr * v;
            if (want_gn) gn = fma((double)v, (double)v, gn);
        }
        b2 -= lr * gb2;
        // this thread's tiles of [gW1 | gb1] update W^T (row D of W^T is b1),
        // a 16-byte word a row of the tile.  Padding units (j >= H) and inputs
        // (k > D) have zero gradient (their d1, or their X^T row, is zero), so
        // the whole word is updated and their weights stay zero.
#pragma unroll
        for (int s = 0; s < TSLOTS; ++s) {
            const int t = tid + s * TNT;
            if (t < T2) {
                int kq, uq;
                grad_tile(t, HQ, KQ, kq, uq);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 *wp = reinterpret_cast<float4 *>(WT + (4 * kq + k) * HN + 4 * uq);
                    float4 w = *wp;
                    w.x -= lr * g[s][0][k];
                    w.y -= lr * g[s][1][k];
                    w.z -= lr * g[s][2][k];
                    w.w -= lr * g[s][3][k];
                    *wp = w;
                    if (want_gn) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) gn = fma((double)g[s][u][k], (double)g[s][u][k], gn);
                    }
                }
            }
        }
        if (want_gn) {
            gn = warp_sum(gn);
            if (lane == 0) redd[warp] = gn;
        }
        if (tid == 0) {
            const double Lv = 0.5 * C * sse;
            if (nd.loss_hist) nd.loss_hist[e] = Lv;
            if (!isfinite(Lv)) atomicOr(status, ST_NONFINITE);
        }
        __syncthreads();
        if (want_gn && tid == 0) {
            double u = 0.0;
            for (int w = 0; w < TNT / 32; ++w) u += redd[w];
            nd.gnorm_hist[e] = sqrt(fma((double)gb2, (double)gb2, u));
        }
    }
    // write the trained weights back in the packed layout
    float *Pw = nd.params;
    for (int i = tid; i < HD; i += TNT) {
        const int j = i / D, k = i - j * D;
        Pw[i] = WT[k * HN + j];
    }
    for (int j = tid; j < H; j += TNT) {
        Pw[HD + j] = WT[D * HN + j];
        Pw[HD + H + j] = w2s[j];
    }
    if (tid == 0) Pw[HD + 2 * H] = b2;
    __syncthreads();
}

template <int ACT>
__global__ void __launch_bounds__(TNT) k_batched_tiled(const BatchNet *__restrict__ nets, const int *__restrict__ order,
                                                       int n_nets, int D, int Hmax, int ncap, int hcap, int epochs,
                                                       float lr, int loss_mean, int *status) {
    extern __shared__ __align__(16) float smem[];
    const TLayout L = t_layout(D, Hmax, ncap, hcap);
    // every region is written before it is read (padding rows and units of
    // h hold finite values whose d1, and whose weight in z2, are 0)
    for (int i = threadIdx.x; i < L.total; i += TNT) smem[i] = 0.f;
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
        net_tiled<ACT>(nd, D, epochs, lr, loss_mean, status, smem, L);
    }
}

}  // namespace

bool batched_tiled_supported(int D, int Hmax) { return D >= 1 && D <= 36 && Hmax >= 1 && Hmax <= 128; }

size_t batched_tiled_smem(int D, int Hmax, int ncap, int hcap) {
    return sizeof(float) * (size_t)t_layout(D, Hmax, ncap, hcap).total;
}

cudaError_t batched_train_tiled(int act, int D, int Hmax, int64_t nmax, const BatchNet *nets_dev,
                                const int *order_dev, int n_nets, int epochs, float lr, int loss_mean, int *status,
                                int hcap_max, cudaStream_t st) {
    if (!batched_tiled_supported(D, Hmax)) return cudaErrorInvalidValue;
    if (n_nets == 0 || epochs == 0) return cudaSuccess;
    // X^T holds a net's rows up to 128 (resident across epochs); h / d1 holds
    // hcap_max rows, a pass
    int ncap = (int)((nmax + 3) & ~(int64_t)3);
    if (ncap > 128) ncap = 128;
    if (ncap < 4) ncap = 4;
    const int hcap = ncap < hcap_max ? ncap : hcap_max;
    const size_t smem = batched_tiled_smem(D, Hmax, ncap, hcap);
    void *fn = act == MLP_ACT_TANH ? (void *)k_batched_tiled<MLP_ACT_TANH> : (void *)k_batched_tiled<MLP_ACT_SIGMOID>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&nets_dev, (void *)&order_dev, (void *)&n_nets, (void *)&D, (void *)&Hmax,
                    (void *)&ncap, (void *)&hcap, (void *)&epochs, (void *)&lr, (void *)&loss_mean, (void *)&status};
    return cudaLaunchKernel(fn, dim3((unsigned)n_nets), dim3(TNT), args, smem, st);
}

}  // namespace mlp
