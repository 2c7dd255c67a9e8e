// BF16 tensor-core (tcgen05) training of one wide network (H = 256 x S hidden
// units, S <= 8) by mini-batch gradient descent (Sec. 2.2 of arXiv 1908.07847:
// feed-forward, output error, backpropagation, w <- w - lr g, no momentum),
// with sigmoid (Eq. 1) or tanh hidden units.
//
// The grid is made of clusters of S blocks; block c of a cluster owns hidden
// units [256 c, 256 c + 256).  Per step (one mini-batch of m rows), cluster k
// takes the 128-row tiles k, k + K, ... (K clusters).  Per tile, every block of
// the cluster loads the same X tile (TMA, 128-byte swizzle), computes its slice
// of Z1 = X W1^T on the tensor cores, its share of z2 = h w2 (h = sigmoid), and
// pushes the share into every block's receive buffer in distributed shared
// memory (st.async, completion counted by the receiver's mbarrier); each block
// adds the shares in rank order, so all blocks of a cluster have the same z2,
// o and d2 for the tile; every block then builds its slice of d1 and
// accumulates its slice of gW1 | gb1 and gw2 in tensor memory (as in the
// many-nets kernel, tc_kernels.cu).  At the end of the step the gradient is
// summed over clusters by a reduce-scatter in global memory among the K blocks
// that own the same hidden slice: every block stores its slice, a barrier of
// those K blocks, block k adds the K clusters' values of 1/K of the slice in
// cluster order (deterministic), a second barrier, and every cluster applies
// the summed gradient to its own copy of the FP32 master weights: the
// epilogue thread that owns hidden unit j keeps row j of W1 in its lane of
// tensor memory (columns the accumulators leave free), b1 and w2 live in
// shared memory, b2 in every thread.  Cluster 0 writes the result back at the
// end.
#include <mutex>

#include "tc_common.cuh"

namespace mlp {

namespace {

using namespace tcd;

constexpr int TR = 128;
constexpr int HS = 256;            // hidden units per block
constexpr int NSTAGE = 2;
constexpr int NEPI = 8;
constexpr int NT = (2 + NEPI) * 32;
constexpr uint32_t NEPI_T = NEPI * 32;
constexpr uint32_t TM_Z1 = 0, TM_GW1 = 256, TM_GW2 = 384, TM_WM = 416;   // TM_WM: 2 x 48 master columns
constexpr int DMAX = 48;

constexpr uint32_t SM_X = 0;                                // 2 stages of 128 x 64 bf16, SW128
constexpr uint32_t SM_W1 = SM_X + NSTAGE * 16384;          // W1/2 slice, 256 x 64 bf16, SW128
constexpr uint32_t SM_HT = SM_W1 + HS * 128;               // h^T, MN-major SW128
constexpr uint32_t SM_DT = SM_HT + 4 * 16384;              // d1^T, MN-major SW128
constexpr uint32_t SM_B3 = SM_DT + 4 * 16384;              // d2 as a 16-wide K-major operand
constexpr uint32_t SM_ONES = SM_B3 + 4096;                 // 128 x 16 bf16, column 0 = 1
constexpr uint32_t SM_B1T = SM_ONES + 4096;                // 256 x 16 bf16, column 0 = b1/2
constexpr uint32_t SM_B1 = SM_B1T + 8192;                  // b1 FP32 master
constexpr uint32_t SM_W2 = SM_B1 + HS * 4;                 // w2 FP32 master
constexpr uint32_t SM_W2B = SM_W2 + HS * 4;                // w2 as bf16
constexpr uint32_t SM_BAR = SM_W2B + HS * 2;
constexpr uint32_t SM_MISC = SM_BAR + 256;
constexpr uint32_t SM_ZX = SM_MISC + 256;   // [2][128] floats: one half's z2 share, the block's
constexpr uint32_t SM_ZR = SM_ZX + 1024;    // [2 parities][8 source blocks][128 rows] floats
constexpr uint32_t SM_TOTAL = SM_ZR + 2 * 8 * 128 * 4;
constexpr uint32_t SM_ALLOC = SM_TOTAL + 1024;
static_assert(SM_ALLOC <= 227 * 1024, "shared memory");

struct ClArgs {
    const float *y;
    float *params;                // initial weights in, trained weights out
    float *part;                  // [K][S][D + 2][256] per-cluster gradient slices
    float *sum;                   // [S][D + 2][256] summed gradient
    double *spart;                // [S][K][2] per-block (sse, gb2) of its cluster
    unsigned long long *bar;      // per-slice barrier arrivals, 16 apart
    unsigned long long bar_base;  // value at launch
    double *loss_hist;
    double *gn_part;              // [epochs][S + 1] or NULL: slice squared norms, then gb2
    int *status;
    int64_t n, mb;
    int D, H, epochs;
    float lr;
    int loss_mean;
    int act;                      // hidden activation (mlp_activation)
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t remote_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
// Asynchronous 16-byte store into a cluster peer's shared memory that
// completes `16 bytes` of the transaction count of the peer's mbarrier.
__device__ __forceinline__ void st_async_v4(uint32_t addr, float4 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)), "r"(__float_as_uint(v.w)),
                 "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int ACT>
__global__ void __launch_bounds__(NT, 1) k_tc_cluster(const __grid_constant__ CUtensorMap tmap, ClArgs a) {
    // Launch-shape check before any tensor-memory, cluster or peer access: the
    // kernel needs clusters of exactly H/256 blocks of NT threads.
    {
        uint32_t ncta;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
        if ((int)ncta * HS != a.H || gridDim.x % ncta != 0 || blockDim.x != NT || a.H > 8 * HS) {
            if (threadIdx.x == 0) atomicOr(a.status, ST_BADLAUNCH);
            return;
        }
    }
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sb = s32(sm);
    float *b1s = (float *)(sm + SM_B1);
    float *w2s = (float *)(sm + SM_W2);
    __nv_bfloat16 *w2b = (__nv_bfloat16 *)(sm + SM_W2B);
    const uint32_t bar0 = sb + SM_BAR;
    // TMA -> MMA: FULL; MMA -> TMA: EMPTY; MMA -> epilogue: Z1F (forward done),
    // HE (h^T and d2 read), DE (d1^T read), STEP; epilogue -> MMA: Z1E (Z1
    // read), HF (h^T, d2 written), DF (d1^T written); cluster peers -> block:
    // ZR0 / ZR1 (z2 shares of even / odd tiles landed, by transaction count).
    const uint32_t BAR_FULL = bar0, BAR_EMPTY = bar0 + 16, BAR_Z1F = bar0 + 32, BAR_Z1E = bar0 + 40,
                   BAR_HF = bar0 + 48, BAR_HE = bar0 + 56, BAR_DF = bar0 + 64, BAR_DE = bar0 + 72,
                   BAR_STEP = bar0 + 80, BAR_ZR0 = bar0 + 88, BAR_DRAIN = bar0 + 96, BAR_EPI = bar0 + 104,
                   BAR_ZR1 = bar0 + 112;
    uint32_t *tmem_slot = (uint32_t *)(sm + SM_MISC);
    volatile int *abort = (volatile int *)(sm + SM_MISC + 16);
    float *red = (float *)(sm + SM_MISC + 64);
    double *gnw = (double *)(sm + SM_MISC + 128);   // 8 epilogue warps' squared gradient norms
    float *zx = (float *)(sm + SM_ZX);
    const float *zrb = (const float *)(sm + SM_ZR);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = a.D, H = a.H;
    // Hidden activation from the forward accumulator: the sigmoid as
    // 1/2 + tanh(z/2)/2 (the operands hold W1/2 and b1/2, so the accumulator
    // is z/2), tanh (Sec. 2.2's other activation) directly from z.
    constexpr bool tanh_act = ACT == MLP_ACT_TANH;
    constexpr float wscale = tanh_act ? 1.0f : 0.5f;
    // h = act_a tanh(acc) + act_b; the tanh form keeps the sigmoid's instruction
    // pattern (one packed fma after the tanh)
    constexpr uint32_t act_a = tanh_act ? BF2_ONE : BF2_HALF, act_b = tanh_act ? 0u : BF2_HALF;
    const int S = H / HS;                            // blocks per cluster
    const int crank = (int)cluster_rank();
    const int k = blockIdx.x / S, K = gridDim.x / S;
    const int j0 = crank * HS;
    const int HD = H * D, P = HD + 2 * H + 1;
    const int E = (D + 2) * HS;                      // gradient values per slice

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(BAR_FULL + 8 * s, 1);
            mbar_init(BAR_EMPTY + 8 * s, 1);
        }
        mbar_init(BAR_Z1F, 1);
        mbar_init(BAR_Z1E, NEPI_T);
        mbar_init(BAR_HF, NEPI_T);
        mbar_init(BAR_HE, 1);
        mbar_init(BAR_DF, NEPI_T);
        mbar_init(BAR_DE, 1);
        mbar_init(BAR_STEP, 1);
        mbar_init(BAR_ZR0, 1);
        mbar_init(BAR_ZR1, 1);
        mbar_init(BAR_DRAIN, 1);
        mbar_init(BAR_EPI, NEPI_T);
        // a launch after a timeout that mlp_check has not cleared does nothing
        *abort = (ld_volatile(a.status) & ST_TIMEOUT) ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(s32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // constant operands: d2 tile and b1 tile zero, ones tile column 0 = 1
    for (int i = tid; i < (4096 + 4096 + 8192) / 4; i += NT) ((uint32_t *)(sm + SM_B3))[i] = 0u;
    __syncthreads();
    for (int row = tid; row < TR; row += NT)
        *(__nv_bfloat16 *)(sm + SM_ONES + k16_off(row, 0)) = __float2bfloat16_rn(1.0f);
    const int q = warp & 3, half = (warp - 2) >> 2, r = q * 32 + lane;
    float b2 = a.params[P - 1];
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    // FP32 master row of the hidden unit this epilogue thread owns, into its
    // tensor-memory lane; the MMA operands hold W1/2 and b1/2 in bf16 so that
    // the forward accumulator is z1/2, the argument sigmoid's tanh form needs.
    if (warp >= 2) {
        const int jl = half * 128 + r, j = j0 + jl;
#pragma unroll
        for (int c16 = 0; c16 < DMAX; c16 += 16) {
            float w[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) w[u] = (c16 + u < D) ? a.params[(size_t)j * D + c16 + u] : 0.f;
            tmem_st16(lane_base + TM_WM + DMAX * half + c16, w);
#pragma unroll
            for (int u = 0; u < 16; ++u)
                *(__nv_bfloat16 *)(sm + SM_W1 + kmajor_off(jl, c16 + u)) = __float2bfloat16_rn(wscale * w[u]);
        }
#pragma unroll
        for (int kk = DMAX; kk < 64; ++kk) *(__nv_bfloat16 *)(sm + SM_W1 + kmajor_off(jl, kk)) = __float2bfloat16_rn(0.f);
        b1s[jl] = a.params[HD + j];
        w2s[jl] = a.params[HD + H + j];
        w2b[jl] = __float2bfloat16_rn(w2s[jl]);
        *(__nv_bfloat16 *)(sm + SM_B1T + k16_off(jl, 0)) = __float2bfloat16_rn(wscale * b1s[jl]);
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync_all();  // every block's barriers exist before any peer's store
    // arm the receive barriers for the first two tiles: S shares of 512 bytes
    if (tid == 64) {
        mbar_expect_tx(BAR_ZR0, (uint32_t)S * 512u);
        mbar_expect_tx(BAR_ZR1, (uint32_t)S * 512u);
    }

    const int64_t mbs = (a.mb <= 0 || a.mb >= a.n) ? a.n : a.mb;
    const double Cl = a.loss_mean ? 1.0 / (double)a.n : 1.0;
    unsigned long long target = a.bar_base;
    // per-role phase counters (they persist across steps)
    int it_tma = 0, it_mma = 0, z1e_use = 0, hf_use = 0, df_use = 0, stepd_use = 0;
    int z1f_use = 0, he_use = 0, de_use = 0, epi_use = 0, tcount = 0;
    double sse_epoch = 0.0;
    bool ok = !*abort;
    // A launch that starts after an unread timeout does nothing, and no block
    // of its cluster sends it anything (all of them read the same status as
    // they start together).
    const bool skipped = !ok;
    int64_t step = 0;
    auto epi_sync = [&]() -> bool {
        mbar_arrive(BAR_EPI);
        return mbar_wait(BAR_EPI, epi_use++ & 1, abort);
    };

    for (int e = 0; e < a.epochs && ok; ++e) {
        sse_epoch = 0.0;
        for (int64_t b0 = 0; b0 < a.n && ok; b0 += mbs, ++step) {
            const int64_t m = min(mbs, a.n - b0);
            const int Ts = (int)((m + TR - 1) / TR);
            const int Tk = (k < Ts) ? (Ts - k + K - 1) / K : 0;    // this cluster's tiles
            const float c = a.loss_mean ? 1.0f / (float)m : 1.0f;

            if (warp == 0) {
                if (lane == 0)
                    for (int i = 0; i < Tk; ++i, ++it_tma) {
                        const int s = it_tma % NSTAGE, use = it_tma / NSTAGE;
                        if (!mbar_wait(BAR_EMPTY + 8 * s, (use & 1) ^ 1, abort)) break;
                        mbar_expect_tx(BAR_FULL + 8 * s, 16384);
                        tma_load_2d(sb + SM_X + 16384 * s, &tmap, 0, (int)(b0 + (int64_t)(k + i * K) * TR),
                                    BAR_FULL + 8 * s);
                    }
            } else if (warp == 1) {
                if (lane == 0) {
                    const uint32_t id_fwd = idesc_bf16(128, HS, 0, 0);
                    const uint32_t id_gw1 = idesc_bf16(128, 64, 1, 1);
                    const uint32_t id_gw2 = idesc_bf16(128, 16, 1, 0);
                    const int Dk = (D + 15) & ~15;
                    int itf = it_mma;   // next forward to issue
                    // Z1 = X (W1/2)^T + 1 (b1/2)^T for tile itf, once its X tile has
                    // landed and the epilogue has read the previous Z1
                    auto forward = [&]() -> bool {
                        const int s = itf % NSTAGE;
                        if (!mbar_wait(BAR_FULL + 8 * s, (itf / NSTAGE) & 1, abort)) return false;
                        if (!mbar_wait(BAR_Z1E, (z1e_use++ & 1) ^ 1, abort)) return false;
                        tc_fence_after();
                        const uint32_t xs = sb + SM_X + 16384 * s;
                        for (int ks = 0; ks < Dk / 16; ++ks)
                            mma_bf16(tmem + TM_Z1, sdesc(xs + ks * 32, 16, 1024, 2), sdesc(sb + SM_W1 + ks * 32, 16, 1024, 2),
                                     id_fwd, ks > 0 ? 1u : 0u);
                        mma_bf16(tmem + TM_Z1, sdesc(sb + SM_ONES, 128, 256, 0), sdesc(sb + SM_B1T, 128, 256, 0), id_fwd, 1u);
                        mma_commit(BAR_Z1F);
                        ++itf;
                        return true;
                    };
                    tc_fence_after();
                    bool mok = Tk == 0 || forward();
                    for (int i = 0; i < Tk && mok; ++i, ++it_mma) {
                        if (i + 1 < Tk && !forward()) { mok = false; break; }
                        const int s = it_mma % NSTAGE;
                        const uint32_t xs = sb + SM_X + 16384 * s;
                        // gw2 += h^T d2 as soon as h^T and d2 are written
                        if (!mbar_wait(BAR_HF, hf_use++ & 1, abort)) { mok = false; break; }
                        tc_fence_after();
                        for (int hb = 0; hb < 2; ++hb)
                            for (int kk = 0; kk < TR / 16; ++kk)
                                mma_bf16(tmem + TM_GW2 + 16 * hb, sdesc(sb + SM_HT + hb * 32768 + kk * 2048, 16384, 1024, 2),
                                         sdesc(sb + SM_B3 + kk * 256, 128, 2048, 0), id_gw2, (i > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(BAR_HE);
                        // [gW1 | gb1] += d1^T [X | 1]
                        if (!mbar_wait(BAR_DF, df_use++ & 1, abort)) { mok = false; break; }
                        tc_fence_after();
                        for (int hb = 0; hb < 2; ++hb)
                            for (int kk = 0; kk < TR / 16; ++kk)
                                mma_bf16(tmem + TM_GW1 + 64 * hb, sdesc(sb + SM_DT + hb * 32768 + kk * 2048, 16384, 1024, 2),
                                         sdesc(xs + kk * 2048, 16384, 1024, 2), id_gw1, (i > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(BAR_DE);
                        mma_commit(BAR_EMPTY + 8 * s);
                    }
                    mma_commit(BAR_STEP);
                }
            } else {
                // epilogue: thread = row = lane; half of the slice's columns
                const int cb = half * 128;
                float sse = 0.f, gb2s = 0.f;
                bool eok = true;
                for (int i = 0; i < Tk && eok; ++i, ++tcount) {
                    const int64_t trow = (int64_t)(k + i * K) * TR + r;   // row within the step
                    const bool valid = trow < m;
                    const float yv = valid ? a.y[b0 + trow] : 0.f;
                    if (!mbar_wait(BAR_Z1F, z1f_use++ & 1, abort)) { eok = false; break; }
                    tc_fence_after();
                    // pass 1: h = sigmoid(z1) in bf16 pairs (written as h^T), this
                    // block's share of z2 = h w2 with FP32 accumulation
                    uint32_t hp[64];
                    float zp[4] = {0.f, 0.f, 0.f, 0.f};
                    bool heok = true;
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        const int c0 = cb + 32 * ch;
                        float z[32];
                        tmem_ld32(lane_base + TM_Z1 + c0, z);
#pragma unroll
                        for (int u = 0; u < 16; ++u) hp[16 * ch + u] = hfma2(tanh_bf2(pack_bf16(z[2 * u], z[2 * u + 1])), act_a, act_b);
#pragma unroll
                        for (int u = 0; u < 16; u += 4) {
                            const uint4 w = *(const uint4 *)(w2b + c0 + 2 * u);
                            zp[0] = dot2_bf16(hp[16 * ch + u], w.x, zp[0]);
                            zp[1] = dot2_bf16(hp[16 * ch + u + 1], w.y, zp[1]);
                            zp[2] = dot2_bf16(hp[16 * ch + u + 2], w.z, zp[2]);
                            zp[3] = dot2_bf16(hp[16 * ch + u + 3], w.w, zp[3]);
                        }
                        // h^T from the second chunk on: the previous tile's gw2 MMA
                        // is done with h^T and d2 by then (waited for here, halfway)
                        if (ch == 1) {
                            if (!mbar_wait(BAR_HE, (he_use++ & 1) ^ 1, abort)) { heok = false; break; }
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                *(uint4 *)(sm + SM_HT + mnmajor_chunk(cb + 8 * v, r)) =
                                    make_uint4(hp[4 * v], hp[4 * v + 1], hp[4 * v + 2], hp[4 * v + 3]);
                        }
                        if (ch >= 1) {
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                *(uint4 *)(sm + SM_HT + mnmajor_chunk(c0 + 8 * v, r)) =
                                    make_uint4(hp[16 * ch + 4 * v], hp[16 * ch + 4 * v + 1], hp[16 * ch + 4 * v + 2],
                                               hp[16 * ch + 4 * v + 3]);
                        }
                    }
                    if (!heok) { eok = false; break; }
                    tc_fence_before();
                    mbar_arrive(BAR_Z1E);
                    // this block's share of z2 (both halves), pushed into every
                    // cluster block's receive buffer; z2 = the shares in rank order
                    const float zs = (zp[0] + zp[1]) + (zp[2] + zp[3]);
                    if (half == 1) zx[r] = zs;
                    if (!epi_sync()) { eok = false; break; }
                    const int par = tcount & 1;
                    const uint32_t zbar = par ? BAR_ZR1 : BAR_ZR0;
                    if (half == 0) {
                        zx[128 + r] = zs + zx[r];
                        __syncwarp();
                        if (lane < 8) {
                            const float4 v = *(const float4 *)(zx + 128 + q * 32 + 4 * lane);
                            const uint32_t src = sb + SM_ZR + (uint32_t)((par * 8 + crank) * 128 + q * 32 + 4 * lane) * 4;
                            for (int cr = 0; cr < S; ++cr)
                                st_async_v4(remote_addr(src, (uint32_t)cr), v, remote_addr(zbar, (uint32_t)cr));
                        }
                    }
                    // while the shares travel: u = w2 f'(h) in bf16 pairs, in place
#pragma unroll
                    for (int ch = 0; ch < 16; ++ch) {
                        const uint4 wv = *(const uint4 *)(w2b + cb + 8 * ch);
                        const uint32_t wp[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const uint32_t h = hp[4 * ch + v];
                            // f'(h): h (1 - h) for the sigmoid, 1 - h^2 for tanh
                            hp[4 * ch + v] = tanh_act ? hmul2(wp[v], hfma2(h ^ 0x80008000u, h, BF2_ONE))
                                                      : hmul2(wp[v], hmul2(h, hfma2(h, BF2_NEG1, BF2_ONE)));
                        }
                    }
                    if (!mbar_wait(zbar, (tcount >> 1) & 1, abort)) { eok = false; break; }
                    // re-arm this parity for tile tcount + 2 (its shares can only be
                    // sent after every block has read this tile's)
                    if (tid == 64) mbar_expect_tx(zbar, (uint32_t)S * 512u);
                    float z2 = 0.f;
                    for (int cr = 0; cr < S; ++cr) z2 += zrb[(par * 8 + cr) * 128 + r];
                    const float o = sigmoid_bf(z2 + b2);
                    const float err = o - yv;
                    const float d2 = valid ? c * err * o * (1.0f - o) : 0.f;
                    if (half == 0) {
                        if (valid) sse = fmaf(err, err, sse);
                        gb2s += d2;
                        *(__nv_bfloat16 *)(sm + SM_B3 + (r & 7) * 2 + (r >> 3) * 128) = __float2bfloat16_rn(d2);
                    }
                    proxy_fence();
                    mbar_arrive(BAR_HF);
                    // pass 2: d1 = d2 u in bf16 pairs, written as d1^T
                    if (!mbar_wait(BAR_DE, (de_use++ & 1) ^ 1, abort)) { eok = false; break; }
                    const uint32_t d2p = pack_bf16(d2, d2);
#pragma unroll
                    for (int ch = 0; ch < 16; ++ch)
                        *(uint4 *)(sm + SM_DT + mnmajor_chunk(cb + 8 * ch, r)) =
                            make_uint4(hmul2(hp[4 * ch], d2p), hmul2(hp[4 * ch + 1], d2p), hmul2(hp[4 * ch + 2], d2p),
                                       hmul2(hp[4 * ch + 3], d2p));
                    if (half == 0) {
                        const int s = tcount % NSTAGE;   // the ones column of [X | 1]
                        *(__nv_bfloat16 *)(sm + SM_X + 16384 * s + kmajor_off(r, D)) = __float2bfloat16_rn(1.0f);
                    }
                    proxy_fence();
                    mbar_arrive(BAR_DF);
                }
                // this cluster's gradient slice (zeros if it had no tile) to global
                if (eok && mbar_wait(BAR_STEP, stepd_use & 1, abort)) {
                    tc_fence_after();
                    const int jl = half * 128 + r;
                    float *pp = a.part + ((size_t)(k * S + crank) * (D + 2)) * HS + jl;
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        float g[32];
                        tmem_ld32(lane_base + TM_GW1 + 64 * half + 32 * part, g);
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            const int kk = 32 * part + u;   // column D holds gb1 (the ones column)
                            if (kk <= D) __stcg(pp + (size_t)kk * HS, Tk > 0 ? g[u] : 0.f);
                        }
                    }
                    const float gw2 = tmem_ld1(lane_base + TM_GW2 + 16 * half);
                    __stcg(pp + (size_t)(D + 1) * HS, Tk > 0 ? gw2 : 0.f);
                    const float ws = warp_sum(sse), wg = warp_sum(gb2s);
                    if (half == 0 && lane == 0) {
                        red[2 * q] = ws;
                        red[2 * q + 1] = wg;
                    }
                    if (epi_sync() && tid == 64) {
                        // every block of a cluster has the same rows' errors
                        double st = 0.0, gb = 0.0;
                        for (int w = 0; w < 4; ++w) {
                            st += (double)red[2 * w];
                            gb += (double)red[2 * w + 1];
                        }
                        __stcg(a.spart + 2 * (crank * K + k), st);
                        __stcg(a.spart + 2 * (crank * K + k) + 1, gb);
                    }
                }
                if (*abort) eok = false;
                ok = ok && eok;
            }
            ++stepd_use;
            // ---- reduce-scatter over clusters, then every cluster updates its copy
            tc_fence_before();
            __syncthreads();
            if (*abort) ok = false;
            if (!ok) break;
            unsigned long long *sbar = a.bar + 16 * crank;
            target += (unsigned long long)K;
            if (!grid_barrier(sbar, target, a.status)) {
                ok = false;
                break;
            }
            {
                // elements [e0, e1) of this slice, each summed over the K
                // clusters in cluster order; up to 3 x 16 loads in flight a thread
                const int e0 = (int)(((int64_t)E * k) / K), e1 = (int)(((int64_t)E * (k + 1)) / K);
                const size_t cs = (size_t)S * E;   // cluster stride in part
                const float *src = a.part + (size_t)crank * E;
                float *dst = a.sum + (size_t)crank * E;
                const int R = K <= 16 ? 3 : 1;     // elements a thread takes per round
                int bad = 0;
                for (int base = e0 + tid * R; base < e1; base += NT * R) {
                    float v[3] = {0.f, 0.f, 0.f};
                    for (int kb = 0; kb < K; kb += 16) {
                        float t[3][16];
#pragma unroll
                        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                            for (int u = 0; u < 16; ++u)
                                t[rr][u] = (rr < R && base + rr < e1 && kb + u < K)
                                               ? __ldcg(src + (size_t)(kb + u) * cs + base + rr)
                                               : 0.f;
#pragma unroll
                        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                            for (int u = 0; u < 16; ++u) v[rr] += t[rr][u];
                    }
#pragma unroll
                    for (int rr = 0; rr < 3; ++rr)
                        if (rr < R && base + rr < e1) {
                            bad |= !isfinite(v[rr]);
                            __stcg(dst + base + rr, v[rr]);
                        }
                }
                if (tid == 64) {
                    // the step's loss and gb2: every block sums its slice's copies
                    double st = 0.0, gb = 0.0;
                    for (int kc = 0; kc < K; ++kc) {
                        st += __ldcg(a.spart + 2 * (crank * K + kc));
                        gb += __ldcg(a.spart + 2 * (crank * K + kc) + 1);
                    }
                    bad |= !isfinite(st) | !isfinite(gb);
                    red[8] = (float)gb;
                    if (k == 0 && crank == 0) sse_epoch += st;
                }
                if (bad) atomicOr(a.status, ST_NONFINITE);
            }
            target += (unsigned long long)K;
            if (!grid_barrier(sbar, target, a.status)) {
                ok = false;
                break;
            }
            // the epoch's last update: cluster 0's blocks record the squared
            // norm of their slice of the gradient (FP64, fixed order)
            const bool want_gn = a.gn_part && k == 0 && b0 + mbs >= a.n;
            if (warp >= 2) {
                const int jl = half * 128 + r;
                const float *gs = a.sum + (size_t)crank * E + jl;
                // all loads first, then the updates (one memory round trip)
                float g[DMAX + 2];
#pragma unroll
                for (int kk = 0; kk < DMAX; ++kk) g[kk] = (kk < D) ? __ldcg(gs + (size_t)kk * HS) : 0.f;
                g[DMAX] = __ldcg(gs + (size_t)D * HS);
                g[DMAX + 1] = __ldcg(gs + (size_t)(D + 1) * HS);
#pragma unroll
                for (int c16 = 0; c16 < DMAX; c16 += 16) {
                    float w[16];
                    tmem_ld16(lane_base + TM_WM + DMAX * half + c16, w);
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        w[u] -= a.lr * g[c16 + u];   // columns >= D stay 0
                        *(__nv_bfloat16 *)(sm + SM_W1 + kmajor_off(jl, c16 + u)) = __float2bfloat16_rn(wscale * w[u]);
                    }
                    tmem_st16(lane_base + TM_WM + DMAX * half + c16, w);
                }
                if (want_gn) {
                    double gn = 0.0;
#pragma unroll
                    for (int kk = 0; kk < DMAX + 2; ++kk) gn = fma((double)g[kk], (double)g[kk], gn);
                    gn = warp_sum(gn);
                    if (lane == 0) gnw[warp - 2] = gn;
                }
                b1s[jl] -= a.lr * g[DMAX];
                w2s[jl] -= a.lr * g[DMAX + 1];
                w2b[jl] = __float2bfloat16_rn(w2s[jl]);
                *(__nv_bfloat16 *)(sm + SM_B1T + k16_off(jl, 0)) = __float2bfloat16_rn(wscale * b1s[jl]);
            }
            b2 -= a.lr * red[8];
            if (k == 0 && crank == 0 && tid == 64) {
                if (b0 + mbs >= a.n) {
                    const double L = 0.5 * sse_epoch * Cl;
                    if (a.loss_hist) a.loss_hist[e] = L;
                    if (!isfinite(L)) atomicOr(a.status, ST_NONFINITE);
                }
            }
            proxy_fence();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (want_gn && tid == 64) {
                double u = 0.0;
                for (int w = 0; w < NEPI; ++w) u += gnw[w];
                a.gn_part[(size_t)e * (S + 1) + crank] = u;
                if (crank == 0) a.gn_part[(size_t)e * (S + 1) + S] = (double)red[8];
            }
        }
    }
    // a failed step-end barrier stops the block without raising its flag
    const bool aborted = *abort || (!ok && !skipped);
    if (aborted && tid == 0) atomicOr(a.status, ST_TIMEOUT);
    if (k == 0 && !aborted) {
        if (warp >= 2) {
            const int jl = half * 128 + r, j = j0 + jl;
#pragma unroll
            for (int c16 = 0; c16 < DMAX; c16 += 16) {
                float w[16];
                tmem_ld16(lane_base + TM_WM + DMAX * half + c16, w);
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (c16 + u < D) a.params[(size_t)j * D + c16 + u] = w[u];
            }
            a.params[HD + j] = b1s[jl];
            a.params[HD + H + j] = w2s[jl];
        }
        if (crank == 0 && tid == 64) a.params[P - 1] = b2;
    }
    // drain: no tensor-core work, copy or remote access may outlive the block
    if (warp == 1 && lane == 0) {
        mma_commit(BAR_DRAIN);
        mbar_wait(BAR_DRAIN, 0, abort, true);
    }
    if (warp == 0 && lane == 0)
        for (int qd = (it_tma > NSTAGE ? it_tma - NSTAGE : 0); qd < it_tma; ++qd)
            mbar_wait(BAR_FULL + 8 * (qd % NSTAGE), (qd / NSTAGE) & 1, abort, true);
    tc_fence_before();
    __syncthreads();
    // Every block of the cluster stops here, so after this barrier no peer
    // issues another z2 share.  Every wait on the way is bounded, so every
    // block gets here.
    cluster_sync_all();
    if (aborted && !skipped && tid == 64) {
        // Shares a peer issued before stopping may still be landing in this
        // block's receive buffers (the st.async stores are tracked only by the
        // receive barriers).  Only the tiles tcount and tcount + 1 can have
        // any: a peer sends tile t + 1's share only after it has received
        // every share of tile t, this block's included.  Wait (bounded) for
        // both phases, so that nothing targets this block's shared memory
        // once it has left; a phase whose sender stopped first never
        // completes and the wait gives up after the time limit.
        for (int t = tcount; t < tcount + 2; ++t)
            mbar_wait((t & 1) ? BAR_ZR1 : BAR_ZR0, (t >> 1) & 1, abort, true);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// gnorm[e] = sqrt(sum over slices of their squared norms + gb2^2), in slice
// order (the slices' values come from cluster 0's blocks).
__global__ void k_cluster_gnorm(const double *part, int S, int epochs, double *gnorm) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < epochs; e += gridDim.x * blockDim.x) {
        const double *p = part + (size_t)e * (S + 1);
        double u = 0.0;
        for (int c = 0; c < S; ++c) u += p[c];
        gnorm[e] = sqrt(fma(p[S], p[S], u));
    }
}

}  // namespace

bool tc_cluster_supported(int D, int H) {
    return D >= 8 && D <= DMAX && D % 8 == 0 && H >= HS && H <= 8 * HS && H % HS == 0;
}

// part [Kmax][S][D + 2][256] floats, sum [S][D + 2][256], spart [S][Kmax][2]
// doubles, 8 barrier counters 128 bytes apart; Kmax = the device's cluster limit.
size_t tc_cluster_scratch_bytes(int D, int H) {
    const size_t E = (size_t)(D + 2) * HS, S = (size_t)(H / HS), Kmax = (size_t)tc_cluster_max_clusters(H);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(sizeof(float) * Kmax * S * E) + al(sizeof(float) * S * E) + al(sizeof(double) * 2 * S * Kmax) + 1024;
}

int tc_cluster_max_clusters(int H) {
    // cached per device and cluster size (devices may differ in SM count)
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static int cache[MAXDEV][9] = {};
    const int S = H / HS;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) {
        cudaGetLastError();
        dev = 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    int &slot = cache[dev][S];
    if (slot == 0) {
        cudaFuncSetAttribute(k_tc_cluster<MLP_ACT_SIGMOID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_ALLOC);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)S);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = SM_ALLOC;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)S;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        // (both activations' instantiations use the same resources)
        if (cudaOccupancyMaxActiveClusters(&n, (void *)k_tc_cluster<MLP_ACT_SIGMOID>, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 1;
        }
        slot = n;
    }
    return slot;
}

cudaError_t tc_cluster_train(const void *X, const float *y, float *params, int D, int H, int64_t n, int epochs,
                             int64_t mb, float lr, int loss_mean, int act, double *loss_hist, double *gnorm_hist,
                             double *gn_part, int *status, void *scratch, int max_clusters, FusedCounters *ctr,
                             cudaStream_t st) {
    if (!tc_cluster_supported(D, H)) return cudaErrorInvalidValue;
    if (n <= 0 || epochs <= 0) return cudaSuccess;
    const int S = H / HS;
    const int64_t mbs = (mb <= 0 || mb >= n) ? n : mb;
    const int tiles = (int)((mbs + TR - 1) / TR);
    int K = tc_cluster_max_clusters(H);
    if (K > max_clusters) K = max_clusters;
    if (K > tiles) K = tiles;
    if (K < 1) K = 1;
    CUtensorMap tmap;
    cudaError_t e = tc_encode_map(&tmap, X, D, n);
    if (e != cudaSuccess) return e;
    auto kern = act == MLP_ACT_TANH ? k_tc_cluster<MLP_ACT_TANH> : k_tc_cluster<MLP_ACT_SIGMOID>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_ALLOC);
    if (e != cudaSuccess) return e;
    const size_t E = (size_t)(D + 2) * HS, Kmax = (size_t)tc_cluster_max_clusters(H);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *b = (char *)scratch;
    ClArgs a;
    a.y = y;
    a.params = params;
    a.part = (float *)b;
    b += al(sizeof(float) * Kmax * S * E);
    a.sum = (float *)b;
    b += al(sizeof(float) * S * E);
    a.spart = (double *)b;
    b += al(sizeof(double) * 2 * S * Kmax);
    a.bar = (unsigned long long *)b;
    a.bar_base = ctr->bar;
    a.loss_hist = loss_hist;
    a.gn_part = gnorm_hist ? gn_part : nullptr;
    a.status = status;
    a.n = n;
    a.mb = mb;
    a.D = D;
    a.H = H;
    a.epochs = epochs;
    a.lr = lr;
    a.loss_mean = loss_mean;
    a.act = act;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(K * S));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SM_ALLOC;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)S;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    // Only a cooperative launch guarantees that every cluster is resident at
    // once, which the step-end barriers between clusters need; if the device
    // refuses it, the call fails (there is no launch without that guarantee).
    e = cudaLaunchKernelEx(&cfg, kern, tmap, a);
    if (e != cudaSuccess) return e;
    const int64_t steps = ((n + mbs - 1) / mbs) * (int64_t)epochs;
    ctr->bar += 2ull * (unsigned long long)K * (unsigned long long)steps;   // every slice's counter
    if (gnorm_hist) {
        k_cluster_gnorm<<<(epochs + 127) / 128, 128, 0, st>>>(gn_part, S, epochs, gnorm_hist);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mlp
