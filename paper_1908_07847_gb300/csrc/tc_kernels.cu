// BF16 tensor-core (tcgen05) training of many independent D-H-1 networks, one
// block per network for all epochs (Sec. 2.2 of arXiv 1908.07847: feed-forward,
// output error, backpropagation, full-batch gradient descent, no momentum).
//
// Per tile of 128 rows of X (bf16, loaded by TMA into a 128-byte-swizzled tile):
//   forward    Z1 = X (W1/2)^T + 1 (b1/2)^T    tcgen05.mma M = 128 rows, N = H,
//                                    K = D, A = X tile (K-major), B = bf16 copy
//                                    of W1/2 (K-major), plus one K = 16 MMA of a
//                                    ones column against b1/2; FP32 accumulator
//                                    in tensor memory holds z1/2;
//   epilogue   thread r of 4 warps owns row r (= tensor-memory lane r):
//              h = sigmoid(z1) = 1/2 + tanh(z1/2)/2 in bf16 pairs (or, for tanh
//              hidden units, h = tanh(z1) with W1 and b1 unscaled), z2 = h w2 + b2
//              (FP32), o = sigmoid(z2), d2 = c (o - y) o (1 - o),
//              u = w2 f'(h) and d1 = d2 u in bf16 pairs;
//              h and d1 go to shared memory as bf16, transposed on the fly
//              (MN-major operand tiles), d2 to a small K-major operand;
//   gradient   gW1 += d1^T X         M = 128 hidden units, N = 64, K = 128 rows,
//                                    A = d1 tile (MN-major), B = the same X tile
//                                    read as MN-major; column D of the X tile is
//                                    set to 1 so column D of the result is gb1;
//              gw2 += h^T d2         M = 128, N = 16, K = 128 rows.
// At the end of an epoch the epilogue threads read the accumulators (one hidden
// unit per tensor-memory lane), update the FP32 master weights in global memory
// (w -= lr g) and rebuild the bf16 copy of W1 for the next epoch.
//
// Roles: warp 0 issues the TMA loads, warp 1 issues the MMAs (one thread each),
// warps 2..9 run the epilogue: the two warps that share a tensor-memory lane
// quarter take one half of the hidden columns each and add their halves of z2
// through shared memory.  The gw2 MMA of a tile is issued as soon as h^T and
// d2 are written and the gW1 MMA when d1^T is, so the next tile's first pass
// only waits for the former.  Every wait is bounded; on a timeout the block
// records MLP_ETIMEOUT, stops issuing, drains what it issued (again bounded),
// frees its tensor memory and leaves.
#include <mutex>

#include "tc_common.cuh"

namespace mlp {

namespace {

constexpr int TR = 128;           // rows per tile
constexpr int HMAX = 256;
constexpr int NSTAGE = 2;
constexpr int NEPI = 8;           // epilogue warps: two per tensor-memory lane quarter
constexpr int NT = (2 + NEPI) * 32;  // threads: TMA warp, MMA warp, epilogue warps
constexpr uint32_t NEPI_T = NEPI * 32;
constexpr uint32_t TM_Z1 = 0;     // tensor-memory columns: Z1 [0, H)
constexpr uint32_t TM_GW1 = 256;  // gW1 | gb1 for hidden block hb at 256 + 64 hb
constexpr uint32_t TM_GW2 = 384;  // gw2 for hidden block hb at 384 + 16 hb

// shared-memory layout (bytes); operand tiles 1024-byte aligned
constexpr uint32_t SM_X = 0;                               // NSTAGE x 16 KB
constexpr uint32_t SM_W1 = SM_X + NSTAGE * 16384;          // H x 128 B
constexpr uint32_t SM_HT = SM_W1 + HMAX * 128;             // 4 x 16 KB (h^T)
constexpr uint32_t SM_DT = SM_HT + 4 * 16384;              // 4 x 16 KB (d1^T)
constexpr uint32_t SM_B3 = SM_DT + 4 * 16384;              // 4 KB (d2)
constexpr uint32_t SM_ONES = SM_B3 + 4096;                 // 128 x 16 bf16, column 0 = 1
constexpr uint32_t SM_B1T = SM_ONES + 4096;                // H x 16 bf16, column 0 = b1/2
constexpr uint32_t SM_B1 = SM_B1T + HMAX * 32;             // fp32 b1
constexpr uint32_t SM_W2 = SM_B1 + HMAX * 4;               // fp32 w2
constexpr uint32_t SM_W2B = SM_W2 + HMAX * 4;              // bf16 w2
constexpr uint32_t SM_BAR = SM_W2B + HMAX * 2;             // mbarriers
constexpr uint32_t SM_MISC = SM_BAR + 256;                 // tmem slot, flags, reductions
constexpr uint32_t SM_ZX = SM_MISC + 256;                  // z2 halves: 2 parities x 2 halves x 128 rows
constexpr uint32_t SM_TOTAL = SM_ZX + 2 * 2 * 128 * 4;
constexpr uint32_t SM_ALLOC = SM_TOTAL + 1024;             // + alignment slack
static_assert(SM_ALLOC <= 227 * 1024, "shared memory");

// 16-byte aligned: the host packs the descriptors sizeof(TcNet) apart.
struct __align__(16) TcNet {
    const CUtensorMap *tmap;  // X: bf16 [n x D], box 64 x 128, 128-byte swizzle
    const float *y;           // n labels
    float *params;            // packed FP32 [W1 (H x D), b1, w2, b2]
    double *loss_hist;        // [epochs] or NULL
    double *gnorm_hist;       // [epochs] or NULL
    int64_t n;
    int32_t H;
    int32_t pad;
};

struct TcArgs {
    const TcNet *nets;
    const int *order;
    int n_nets;
    int D;
    int epochs;
    float lr;
    int loss_mean;
    int act;                  // hidden activation (mlp_activation)
    int *status;
    int *next;                // nets taken after the first wave (zeroed before the launch), or NULL
};

using namespace tcd;

template <int ACT>
__global__ void __launch_bounds__(NT, 1) k_tc_batched(TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sb = s32(sm);
    float *b1s = (float *)(sm + SM_B1);
    float *w2s = (float *)(sm + SM_W2);
    __nv_bfloat16 *w2b = (__nv_bfloat16 *)(sm + SM_W2B);
    const uint32_t bar0 = sb + SM_BAR;
    // TMA -> MMA: FULL; MMA -> TMA: EMPTY; MMA -> epilogue: Z1F (forward done),
    // HE (h^T, d2 read), DE (d1^T read), EPOCH; epilogue -> MMA: Z1E (Z1 read),
    // HF (h^T, d2 written), DF (d1^T written), W (weights updated).
    const uint32_t BAR_FULL = bar0, BAR_EMPTY = bar0 + 16, BAR_Z1F = bar0 + 32, BAR_Z1E = bar0 + 40,
                   BAR_HF = bar0 + 48, BAR_HE = bar0 + 56, BAR_DF = bar0 + 64, BAR_DE = bar0 + 72,
                   BAR_EPOCH = bar0 + 80, BAR_W = bar0 + 88, BAR_DRAIN = bar0 + 96, BAR_EPI = bar0 + 104;
    uint32_t *tmem_slot = (uint32_t *)(sm + SM_MISC);
    volatile int *abort = (volatile int *)(sm + SM_MISC + 16);
    float *red = (float *)(sm + SM_MISC + 64);     // 4 warps x (sse, gb2)
    double *gnr = (double *)(sm + SM_MISC + 128);  // 8 epilogue warps' squared gradient norms
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = a.D;
    // Hidden activation from the forward accumulator: the sigmoid as
    // 1/2 + tanh(z/2)/2 (the operands hold W1/2 and b1/2, so the accumulator
    // is z/2), tanh (Sec. 2.2's other activation) directly from z.
    constexpr bool tanh_act = ACT == MLP_ACT_TANH;
    constexpr float wscale = tanh_act ? 1.0f : 0.5f;
    // h = act_a tanh(acc) + act_b; the tanh form keeps the sigmoid's instruction
    // pattern (one packed fma after the tanh)
    constexpr uint32_t act_a = tanh_act ? BF2_ONE : BF2_HALF, act_b = tanh_act ? 0u : BF2_HALF;
    const uint32_t bars[12] = {BAR_FULL, BAR_FULL + 8, BAR_EMPTY, BAR_EMPTY + 8, BAR_Z1F, BAR_Z1E,
                               BAR_HF,   BAR_HE,       BAR_DF,    BAR_DE,        BAR_EPOCH, BAR_W};
    const uint32_t counts[12] = {1, 1, 1, 1, 1, NEPI_T, NEPI_T, 1, NEPI_T, 1, 1, NEPI_T};

    if (tid == 0) {
        for (int i = 0; i < 12; ++i) mbar_init(bars[i], counts[i]);
        mbar_init(BAR_DRAIN, 1);
        mbar_init(BAR_EPI, NEPI_T);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(s32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // constant operands: the d2 tile and b1 tile zero (only column 0 is ever
    // written), the ones tile with column 0 = 1
    for (int i = tid; i < (4096 + 4096 + HMAX * 32) / 4; i += NT) ((uint32_t *)(sm + SM_B3))[i] = 0u;
    __syncthreads();
    for (int row = tid; row < TR; row += NT)
        *(__nv_bfloat16 *)(sm + SM_ONES + k16_off(row, 0)) = __float2bfloat16_rn(1.0f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // Nets go to blocks in decreasing cost: block b takes net b first, then
    // each block that finishes takes the next net not yet taken (one atomic
    // increment), so the longest nets start first and no block waits on a
    // fixed share; which block trains a net does not change its result.
    int *s_idx = (int *)(sm + SM_MISC + 32);
    auto next_net = [&](int cur) -> int {
        if (!a.next) return cur + (int)gridDim.x;
        __syncthreads();
        if (tid == 0) *s_idx = (int)gridDim.x + atomicAdd(a.next, 1);
        __syncthreads();
        return *s_idx;
    };
    for (int idx = blockIdx.x; idx < a.n_nets; idx = next_net(idx)) {
        const TcNet nd = a.nets[a.order ? a.order[idx] : idx];
        const int H = nd.H;
        const int64_t n = nd.n;
        const int T = (int)((n + TR - 1) / TR);
        const int Dk = (D + 15) & ~15;        // forward K covered by MMAs
        const float c = a.loss_mean ? 1.0f / (float)n : 1.0f;
        const double Cl = a.loss_mean ? 1.0 / (double)n : 1.0;
        float *P = nd.params;
        const int HD = H * D;

        // ---- weights into shared memory: bf16 W1/2 (swizzled, zero padded),
        // b1/2 as the bias operand, b1, w2 (FP32) and w2 (bf16)
        for (int i = tid; i < H * 64; i += NT) {
            const int j = i >> 6, k = i & 63;
            const float v = (k < D) ? P[j * D + k] : 0.f;
            *(__nv_bfloat16 *)(sm + SM_W1 + kmajor_off(j, k)) = __float2bfloat16_rn(wscale * v);
        }
        for (int j = tid; j < H; j += NT) {
            b1s[j] = P[HD + j];
            w2s[j] = P[HD + H + j];
            w2b[j] = __float2bfloat16_rn(w2s[j]);
            *(__nv_bfloat16 *)(sm + SM_B1T + k16_off(j, 0)) = __float2bfloat16_rn(wscale * b1s[j]);
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        float b2 = P[HD + 2 * H];

        if (T == 0 || a.epochs == 0) {
            if (tid == 0)
                for (int e = 0; e < a.epochs; ++e) {
                    if (nd.loss_hist) nd.loss_hist[e] = 0.0;
                    if (nd.gnorm_hist) nd.gnorm_hist[e] = 0.0;
                }
            continue;
        }

        // Barrier phase counters restart for every net: the previous net's
        // waits were all completed, so re-initialising is safe after a sync.
        if (tid == 0) {
            for (int i = 0; i < 12; ++i) {
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bars[i]));
                mbar_init(bars[i], counts[i]);
            }
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(BAR_DRAIN));
            mbar_init(BAR_DRAIN, 1);
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(BAR_EPI));
            mbar_init(BAR_EPI, NEPI_T);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();

        if (warp == 0) {
            // ================= TMA producer =================
            if (lane == 0) {
                int it = 0;
                for (int e = 0; e < a.epochs && !*abort; ++e)
                    for (int t = 0; t < T; ++t, ++it) {
                        const int s = it % NSTAGE, use = it / NSTAGE;
                        if (!mbar_wait(BAR_EMPTY + 8 * s, (use & 1) ^ 1, abort)) break;
                        mbar_expect_tx(BAR_FULL + 8 * s, 16384);
                        tma_load_2d(sb + SM_X + 16384 * s, nd.tmap, 0, t * TR, BAR_FULL + 8 * s);
                    }
                // drain: every issued load completes before the block moves on
                const int issued = it;
                for (int q = (issued > NSTAGE ? issued - NSTAGE : 0); q < issued; ++q)
                    mbar_wait(BAR_FULL + 8 * (q % NSTAGE), (q / NSTAGE) & 1, abort, true);
            }
        } else if (warp == 1) {
            // ================= MMA issuer =================
            if (lane == 0) {
                const uint32_t id_fwd = idesc_bf16(128, H, 0, 0);
                const uint32_t id_gw1 = idesc_bf16(128, 64, 1, 1);
                const uint32_t id_gw2 = idesc_bf16(128, 16, 1, 0);
                int it = 0, itf = 0, z1e_use = 0, hf_use = 0, df_use = 0;
                // Z1 = X (W1/2)^T + 1 (b1/2)^T for tile itf once its X tile has landed
                // and the epilogue has read the previous Z1
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
                bool ok = true;
                for (int e = 0; e < a.epochs && ok; ++e) {
                    if (e > 0 && !mbar_wait(BAR_W, (e - 1) & 1, abort)) { ok = false; break; }
                    tc_fence_after();
                    if (!forward()) { ok = false; break; }
                    for (int t = 0; t < T; ++t, ++it) {
                        if (t + 1 < T && !forward()) { ok = false; break; }
                        const int s = it % NSTAGE;
                        const uint32_t xs = sb + SM_X + 16384 * s;
                        // gw2 += h^T d2 as soon as h^T and d2 are written
                        if (!mbar_wait(BAR_HF, hf_use++ & 1, abort)) { ok = false; break; }
                        tc_fence_after();
                        for (int hb = 0; hb < H / 128; ++hb)
                            for (int kk = 0; kk < TR / 16; ++kk)
                                mma_bf16(tmem + TM_GW2 + 16 * hb, sdesc(sb + SM_HT + hb * 32768 + kk * 2048, 16384, 1024, 2),
                                         sdesc(sb + SM_B3 + kk * 256, 128, 2048, 0), id_gw2, (t > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(BAR_HE);
                        // [gW1 | gb1] += d1^T [X | 1]
                        if (!mbar_wait(BAR_DF, df_use++ & 1, abort)) { ok = false; break; }
                        tc_fence_after();
                        for (int hb = 0; hb < H / 128; ++hb)
                            for (int kk = 0; kk < TR / 16; ++kk)
                                mma_bf16(tmem + TM_GW1 + 64 * hb, sdesc(sb + SM_DT + hb * 32768 + kk * 2048, 16384, 1024, 2),
                                         sdesc(xs + kk * 2048, 16384, 1024, 2), id_gw1, (t > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(BAR_DE);
                        mma_commit(BAR_EMPTY + 8 * s);
                    }
                    if (!ok) break;
                    mma_commit(BAR_EPOCH);
                }
                // drain every MMA issued before tensor memory is released
                mma_commit(BAR_DRAIN);
                mbar_wait(BAR_DRAIN, 0, abort, true);
            }
        } else {
            // ========== epilogue: thread = row = TMEM lane, one half of the columns ==========
            const int q = warp & 3;                 // tensor-memory lane quarter
            const int half = (warp - 2) >> 2;      // which half of the hidden columns
            const int r = q * 32 + lane;            // row within the tile / lane
            const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
            const int cw = H / 2, cb = half * cw;   // this thread's columns [cb, cb + cw)
            const int nch = cw / 32;                // 32-column chunks: 2 (H = 128) or 4
            float *zx = (float *)(sm + SM_ZX);
            int z1f_use = 0, he_use = 0, de_use = 0, epi_use = 0;
            bool ok = true;
            // Barrier of the epilogue threads with a bounded wait (an mbarrier,
            // so that a block that aborts cannot leave it hanging).
            auto epi_sync = [&]() -> bool {
                mbar_arrive(BAR_EPI);
                return mbar_wait(BAR_EPI, epi_use++ & 1, abort);
            };
            int tcount = 0;
            for (int e = 0; e < a.epochs && ok; ++e) {
                float sse = 0.f, gb2s = 0.f;
                float y_next = (r < n) ? nd.y[r] : 0.f;  // label of this thread's row, one tile ahead
                for (int t = 0; t < T; ++t, ++tcount) {
                    const int64_t row = (int64_t)t * TR + r;
                    const bool valid = row < n;
                    const float yv = y_next;
                    if (row + TR < n) y_next = nd.y[row + TR];
                    if (!mbar_wait(BAR_Z1F, z1f_use++ & 1, abort)) { ok = false; break; }
                    tc_fence_after();
                    // pass 1: h = sigmoid(z1) in bf16 pairs -> h^T, this half's
                    // share of z2 = h w2 in FP32
                    uint32_t hp[64];
                    float zp[4] = {0.f, 0.f, 0.f, 0.f};
                    bool heok = true;
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        if (ch >= nch) break;
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
                    if (!heok) { ok = false; break; }
                    tc_fence_before();
                    mbar_arrive(BAR_Z1E);  // Z1 in tensor memory may be overwritten
                    // the two halves' shares of z2 meet in shared memory; while the
                    // other half arrives: u = w2 f'(h) in bf16 pairs, in place
                    float *zxp = zx + (tcount & 1) * 256;
                    zxp[half * 128 + r] = (zp[0] + zp[1]) + (zp[2] + zp[3]);
                    mbar_arrive(BAR_EPI);
#pragma unroll
                    for (int ch = 0; ch < 16; ++ch) {
                        if (ch >= 4 * nch) break;
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
                    if (!mbar_wait(BAR_EPI, epi_use++ & 1, abort)) { ok = false; break; }
                    const float o = sigmoid_bf(zxp[r] + zxp[128 + r] + b2);
                    const float err = o - yv;
                    const float d2 = valid ? c * err * o * (1.0f - o) : 0.f;
                    if (half == 0) {
                        if (valid) sse = fmaf(err, err, sse);
                        gb2s += d2;
                        *(__nv_bfloat16 *)(sm + SM_B3 + (r & 7) * 2 + (r >> 3) * 128) = __float2bfloat16_rn(d2);
                    }
                    proxy_fence();
                    mbar_arrive(BAR_HF);
                    // pass 2: d1 = d2 u in bf16 pairs -> d1^T, once the previous
                    // tile's gW1 MMA has read d1^T
                    if (!mbar_wait(BAR_DE, (de_use++ & 1) ^ 1, abort)) { ok = false; break; }
                    const uint32_t d2p = pack_bf16(d2, d2);
#pragma unroll
                    for (int ch = 0; ch < 16; ++ch) {
                        if (ch >= 4 * nch) break;
                        *(uint4 *)(sm + SM_DT + mnmajor_chunk(cb + 8 * ch, r)) =
                            make_uint4(hmul2(hp[4 * ch], d2p), hmul2(hp[4 * ch + 1], d2p), hmul2(hp[4 * ch + 2], d2p),
                                       hmul2(hp[4 * ch + 3], d2p));
                    }
                    if (half == 0) {
                        const int s = tcount % NSTAGE;   // the ones column of [X | 1]
                        *(__nv_bfloat16 *)(sm + SM_X + 16384 * s + kmajor_off(r, D)) = __float2bfloat16_rn(1.0f);
                    }
                    proxy_fence();
                    mbar_arrive(BAR_DF);
                }
                if (!ok) break;
                // ---- end of epoch: reductions and the update
                if (!mbar_wait(BAR_EPOCH, e & 1, abort)) { ok = false; break; }
                tc_fence_after();
                const float ws = warp_sum(sse), wg = warp_sum(gb2s);
                // fixed order over the four half-0 warps (by lane quarter)
                if (half == 0 && lane == 0) {
                    red[2 * q] = ws;
                    red[2 * q + 1] = wg;
                }
                if (!epi_sync()) { ok = false; break; }
                double sse_t = 0.0;
                float gb2 = 0.f;
                for (int w = 0; w < 4; ++w) {
                    sse_t += (double)red[2 * w];
                    gb2 += red[2 * w + 1];
                }
                // The gradient rows go to shared memory (the h^T buffer is free
                // once every MMA of the epoch has completed) so that the FP32
                // master weights in global memory are updated with coalesced
                // accesses: a row per thread there would touch a cache line per
                // lane and load.  Hidden unit of this thread: block hb = half
                // (H = 256) or 0 (H = 128).
                float *gs = (float *)(sm + SM_HT);   // H x D gradient, row-major
                if (half < H / 128) {
                    const int hb = half;
                    const int j = hb * 128 + r;  // hidden unit = lane
                    const float gw2 = tmem_ld1(lane_base + TM_GW2 + 16 * hb);
                    const float gb1 = tmem_ld1(lane_base + TM_GW1 + 64 * hb + D);   // the ones column
#pragma unroll
                    for (int c16 = 0; c16 < 64; c16 += 16) {
                        if (c16 >= D) break;
                        float g[16];
                        tmem_ld16(lane_base + TM_GW1 + 64 * hb + c16, g);
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (c16 + u < D) gs[j * D + c16 + u] = g[u];
                    }
                    gs[HD + j] = gb1;       // kept for the gradient norm
                    gs[HD + H + j] = gw2;
                    const float nb1 = b1s[j] - a.lr * gb1;
                    const float nw2 = w2s[j] - a.lr * gw2;
                    P[HD + j] = nb1;
                    P[HD + H + j] = nw2;
                    b1s[j] = nb1;
                    w2s[j] = nw2;
                    w2b[j] = __float2bfloat16_rn(nw2);
                    *(__nv_bfloat16 *)(sm + SM_B1T + k16_off(j, 0)) = __float2bfloat16_rn(wscale * nb1);
                }
                if (!epi_sync()) { ok = false; break; }
                // FP64 squared norm of the gradient this update applies (only
                // when asked for): each thread's elements of [gW1, gb1, gw2] in
                // index order, a fixed butterfly per warp, the warps in order,
                // then gb2
                // (the pointer is read here, not kept in registers for the epoch)
                double *const gnorm_hist = a.nets[a.order ? a.order[idx] : idx].gnorm_hist;
                const bool want_gn = gnorm_hist != nullptr;
                if (want_gn) {
                    double gn = 0.0;
                    for (int i = (warp - 2) * 32 + lane; i < HD + 2 * H; i += (int)NEPI_T)
                        gn = fma((double)gs[i], (double)gs[i], gn);
                    gn = warp_sum(gn);
                    if (lane == 0) gnr[warp - 2] = gn;
                }
                {
                    // w -= lr g over the flat H x D array, 16 loads in flight per thread
                    const int et = (warp - 2) * 32 + lane;   // epilogue thread 0..255
                    for (int i0 = et; i0 < HD; i0 += (int)NEPI_T * 16) {
                        float w[16];
#pragma unroll
                        for (int v = 0; v < 16; ++v) {
                            const int i = i0 + v * (int)NEPI_T;
                            w[v] = i < HD ? P[i] : 0.f;
                        }
#pragma unroll
                        for (int v = 0; v < 16; ++v) {
                            const int i = i0 + v * (int)NEPI_T;
                            if (i < HD) {
                                const int j = i / D, k = i - j * D;
                                w[v] -= a.lr * gs[i];
                                P[i] = w[v];
                                *(__nv_bfloat16 *)(sm + SM_W1 + kmajor_off(j, k)) = __float2bfloat16_rn(wscale * w[v]);
                            }
                        }
                    }
                }
                b2 -= a.lr * gb2;
                if (half == 0 && r == 0) {
                    P[HD + 2 * H] = b2;
                    const double L = 0.5 * Cl * sse_t;
                    if (nd.loss_hist) nd.loss_hist[e] = L;
                    if (!isfinite(L)) atomicOr(a.status, ST_NONFINITE);
                }
                proxy_fence();
                tc_fence_before();
                if (!epi_sync()) { ok = false; break; }
                mbar_arrive(BAR_W);
                if (want_gn && half == 0 && r == 0) {
                    double u = 0.0;
                    for (int w = 0; w < NEPI; ++w) u += gnr[w];
                    gnorm_hist[e] = sqrt(fma((double)gb2, (double)gb2, u));
                }
            }
        }
        if (*abort && tid == 0) atomicOr(a.status, ST_TIMEOUT);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*abort) break;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

static_assert(sizeof(TcNet) % 16 == 0, "descriptor stride");
size_t tc_desc_bytes() { return sizeof(TcNet); }
size_t tc_tmap_bytes() { return sizeof(CUtensorMap); }

bool tc_supported(int D, int H) { return D >= 8 && D <= 56 && D % 8 == 0 && (H == 128 || H == 256); }

// Encodes the tensor map of one net's X (bf16 n x D, row-major) into *map.
cudaError_t tc_encode_map(void *map, const void *X, int D, int64_t n) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)X & 15) != 0) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)(n > 0 ? n : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)D * 2};
    cuuint32_t box[2] = {64, TR};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn((CUtensorMap *)map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(X), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Fills the device-side descriptor (host image) of one net.
void tc_fill_desc(void *desc, const void *tmap_dev, const float *y, float *params, double *loss_hist,
                  double *gnorm_hist, int64_t n, int H) {
    TcNet *d = (TcNet *)desc;
    d->tmap = (const CUtensorMap *)tmap_dev;
    d->y = y;
    d->params = params;
    d->loss_hist = loss_hist;
    d->gnorm_hist = gnorm_hist;
    d->n = n;
    d->H = H;
    d->pad = 0;
}

cudaError_t tc_batched_train(const void *descs_dev, const int *order_dev, int n_nets, int D, int epochs, float lr,
                             int loss_mean, int act, int *status, int *next, cudaStream_t st) {
    if (n_nets == 0 || epochs == 0) return cudaSuccess;
    auto kern = act == MLP_ACT_TANH ? k_tc_batched<MLP_ACT_TANH> : k_tc_batched<MLP_ACT_SIGMOID>;
    static bool attr_set[2] = {false, false};
    if (!attr_set[act == MLP_ACT_TANH]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_ALLOC);
        if (e != cudaSuccess) return e;
        attr_set[act == MLP_ACT_TANH] = true;
    }
    TcArgs a;
    a.nets = (const TcNet *)descs_dev;
    a.order = order_dev;
    a.n_nets = n_nets;
    a.D = D;
    a.epochs = epochs;
    a.lr = lr;
    a.loss_mean = loss_mean;
    a.act = act;
    a.status = status;
    const int grid = n_nets < device_sm_count() ? n_nets : device_sm_count();
    a.next = nullptr;
    if (next && n_nets > grid) {
        cudaError_t e = cudaMemsetAsync(next, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        a.next = next;
    }
    kern<<<grid, NT, SM_ALLOC, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mlp
