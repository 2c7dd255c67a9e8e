// Per-block forward + backward over rows staged in shared memory, shared by the
// single-network fused kernel and the many-networks kernel.
//
// The method (Sec. 2.2 and Eq. 1 of arXiv 1908.07847) for one row x:
//   z1_j = b1_j + sum_k W1_jk x_k,  h_j = f(z1_j),  z2 = b2 + sum_j w2_j h_j,
//   o = sigmoid(z2),  d2 = c (o - y) o (1 - o),  d1_j = d2 w2_j f'(h_j),
//   and the gradient sums gW1_jk += d1_j x_k, gb1_j += d1_j, gw2_j += d2 h_j,
//   gb2 += d2.
//
// Mapping: a block of BNW warps.  Lane sl of a segment of S lanes owns hidden
// neuron j = wu * 32 + sl (the paper's one neuron per thread), holding its D
// incoming weights and its gradient row in registers.  H <= 32: one warp per row
// group, cut into 32 / S segments (S = next power of two >= H, at least 4) that
// each take their own rows, and z2 is a butterfly over the segment.  H in
// 33..64 (65..128): row groups of WU = 2 (4) warps, whose partial z2 are added
// through shared memory in warp order once per RB rows.  Each lane keeps RB
// rows in flight so that its fused multiply-add chains overlap.
#pragma once

#include "mlp_internal.cuh"

namespace mlp {

constexpr int RE_NW = 8;               // warps per block
constexpr int RE_NT = RE_NW * 32;      // threads per block
constexpr int RE_RB = 4;               // rows per lane per iteration (default)
constexpr int RE_RB_MAX = 8;           // most rows per lane any kernel asks for
constexpr int RE_ZX = 2 * RE_NW * RE_RB_MAX;  // floats of z2 exchange space

// Warps per row group for a width H (1, 2 or 4).
__host__ __device__ inline int re_wu(int H) { return H <= 32 ? 1 : (H <= 64 ? 2 : 4); }
// Row groups per block.
__host__ __device__ inline int re_groups(int H) { return RE_NW / re_wu(H); }

// Rows in flight per lane: RB1 when H <= 32 (segments of a warp already take
// separate rows there), RBN otherwise; a kernel with the register file to
// itself can afford more than the defaults.
template <int DP, int WU, int ACT, int RB1 = 2, int RBN = RE_RB>
struct RowEngine {
    static_assert(RB1 <= RE_RB_MAX && RBN <= RE_RB_MAX, "z2 exchange space");
    static constexpr int NG = RE_NW / WU;
    static constexpr int RB = (WU == 1) ? RB1 : RBN;
    // Per-lane state: the neuron's weights and gradient sums.
    float w[DP];
    float acc[DP];
    float b1r, w2r, b2;
    float gb1a, gw2a, gb2a;
    double sse;
    int H, D;
    int S;    // lanes per segment
    int par;  // z2 exchange buffer parity

    __device__ __forceinline__ void setup(int H_, int D_) {
        H = H_;
        D = D_;
        S = 32;
        if (WU == 1) {
            S = 4;
            while (S < H) S <<= 1;
        }
        par = 0;
    }
    __device__ __forceinline__ int unit() const { return ((threadIdx.x >> 5) % WU) * 32 + (threadIdx.x & 31) % S; }

    // Weights from the packed parameters [W1 (H x D), b1, w2, b2] in shared
    // memory; zero the gradient sums.
    __device__ __forceinline__ void load_weights(const float *Wm) {
        const int j = unit(), HD = H * D;
        const bool own = j < H;
        const float *wr = Wm + j * D;
#pragma unroll
        for (int k = 0; k < DP; ++k) w[k] = (own && k < D) ? wr[k] : 0.f;
        b1r = own ? Wm[HD + j] : 0.f;
        w2r = own ? Wm[HD + H + j] : 0.f;
        b2 = Wm[HD + 2 * H];
#pragma unroll
        for (int k = 0; k < DP; ++k) acc[k] = 0.f;
        gb1a = gw2a = gb2a = 0.f;
        sse = 0.0;
    }

    // Rows 0..cn-1 of the staged chunk Xs (DP floats per row, zero padded) with
    // labels ys; c scales the output delta (1/m or 1).
    __device__ __forceinline__ void rows(const float *Xs, const float *ys, int cn, float c, float *zx) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int grp = warp / WU, wu = warp % WU;
        const int slot = lane / S;
        const int RPI = (32 / S) * RB;
        // Squared errors of this call are summed in FP32 per lane and folded
        // into the FP64 sum once (FP64 arithmetic is slow on this part).
        float sse_f = 0.f;
        // Row t of a slot's batch is base + t * nslots + slot: neighbouring
        // segments read neighbouring rows, whose float4 words fall in distinct
        // shared-memory banks (row stride DP = 4 mod 32 words or a multiple of 8).
        const int nslots = 32 / S;
        for (int base = grp * RPI; base < cn; base += NG * RPI) {
            int xo[RB], rr[RB];
            bool valid[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) {
                rr[t] = base + t * nslots + slot;
                valid[t] = rr[t] < cn;
                xo[t] = (valid[t] ? rr[t] : 0) * DP;
            }
            float z[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) z[t] = b1r;
#pragma unroll
            for (int q = 0; q < DP / 4; ++q) {
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(Xs + xo[t] + 4 * q);
                    z[t] = fmaf(xv.x, w[4 * q + 0], z[t]);
                    z[t] = fmaf(xv.y, w[4 * q + 1], z[t]);
                    z[t] = fmaf(xv.z, w[4 * q + 2], z[t]);
                    z[t] = fmaf(xv.w, w[4 * q + 3], z[t]);
                }
            }
            // Re-read the rows from shared memory in the backward pass instead of
            // keeping RB x DP values live in registers.
            asm volatile("" ::: "memory");
            float hv[RB], zp[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) {
                hv[t] = Act<ACT>::f(z[t]);
                zp[t] = hv[t] * w2r;
            }
            // Butterfly over the segment, level by level so that the RB rows'
            // shuffles overlap.
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                if (WU > 1 || off < S) {
#pragma unroll
                    for (int t = 0; t < RB; ++t) zp[t] += __shfl_xor_sync(0xffffffffu, zp[t], off);
                }
            }
            if (WU > 1) {
                float *zg = zx + (par * NG + grp) * (WU * RB);
                if (lane == 0) {
#pragma unroll
                    for (int t = 0; t < RB; ++t) zg[wu * RB + t] = zp[t];
                }
                asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(WU * 32) : "memory");
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    float v = zg[t];
#pragma unroll
                    for (int q = 1; q < WU; ++q) v += zg[q * RB + t];
                    zp[t] = v;
                }
                par ^= 1;
            }
#pragma unroll
            for (int t = 0; t < RB; ++t) {
                const float o = sigmoid_out(zp[t] + b2);
                const float err = o - ys[valid[t] ? rr[t] : 0];
                const float d2 = valid[t] ? c * err * o * (1.0f - o) : 0.f;
                if (valid[t]) sse_f = fmaf(err, err, sse_f);
                gb2a += d2;
                gw2a = fmaf(d2, hv[t], gw2a);
                const float d1 = d2 * w2r * Act<ACT>::df(hv[t]);
                gb1a += d1;
                hv[t] = d1;
            }
#pragma unroll
            for (int q = 0; q < DP / 4; ++q) {
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(Xs + xo[t] + 4 * q);
                    acc[4 * q + 0] = fmaf(hv[t], xv.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(hv[t], xv.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(hv[t], xv.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(hv[t], xv.w, acc[4 * q + 3]);
                }
            }
        }
        sse += (double)sse_f;
    }

    // Sum the segments of each warp (fixed butterfly) and write this row group's
    // gradient sums to part[grp * P ...] (packed layout) and its squared-error
    // sum to s_sse[grp].  The caller synchronises the block afterwards.
    __device__ __forceinline__ void write_group(float *part, double *s_sse) {
        if (WU == 1) {
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                if (off >= S) {
#pragma unroll
                    for (int k = 0; k < DP; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
                    gb1a += __shfl_xor_sync(0xffffffffu, gb1a, off);
                    gw2a += __shfl_xor_sync(0xffffffffu, gw2a, off);
                    gb2a += __shfl_xor_sync(0xffffffffu, gb2a, off);
                    sse += __shfl_xor_sync(0xffffffffu, sse, off);
                }
            }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int grp = warp / WU, wu = warp % WU;
        const int j = unit(), HD = H * D, P = HD + 2 * H + 1;
        float *pg = part + grp * P;
        if (lane < S && j < H) {
            float *gr = pg + j * D;
#pragma unroll
            for (int k = 0; k < DP; ++k)
                if (k < D) gr[k] = acc[k];
            pg[HD + j] = gb1a;
            pg[HD + H + j] = gw2a;
        }
        if (wu == 0 && lane == 0) {
            pg[P - 1] = gb2a;
            s_sse[grp] = sse;
        }
    }
};

// Shared-memory floats for the group partials of a block (largest width class
// up to Hmax).
__host__ __device__ inline int re_part_floats(int D, int Hmax) {
    int pf = 0;
    const int caps[3] = {32, 64, Hmax};
    for (int i = 0; i < 3; ++i) {
        const int H = caps[i] < Hmax ? caps[i] : Hmax;
        const int v = re_groups(H) * ((D + 2) * H + 1);
        pf = pf > v ? pf : v;
    }
    return (pf + 3) & ~3;
}

}  // namespace mlp
