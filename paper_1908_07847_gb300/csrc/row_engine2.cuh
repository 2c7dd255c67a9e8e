// Per-block forward + backward over rows staged in shared memory with U hidden
// units per lane, used by the many-networks kernel for inputs up to 36 wide.
//
// The method (Sec. 2.2 and Eq. 1 of arXiv 1908.07847) for one row x:
//   z1_j = b1_j + sum_k W1_jk x_k,  h_j = f(z1_j),  z2 = b2 + sum_j w2_j h_j,
//   o = sigmoid(z2),  d2 = c (o - y) o (1 - o),  d1_j = d2 w2_j f'(h_j),
//   and the gradient sums gW1_jk += d1_j x_k, gb1_j += d1_j, gw2_j += d2 h_j,
//   gb2 += d2.
//
// Mapping: a block of NW warps cut into row groups of WU warps.  Lane gl of a
// group (gl = warp-in-group * 32 + lane-in-segment) owns the hidden units
// j = gl + i * WU * S, i < U, and keeps their D incoming weights and gradient
// rows in registers.  Each row x (broadcast from shared memory in 16-byte
// words) then feeds U fused multiply-adds per word element instead of one,
// and the per-row work shared by the lanes of a row (the z2 butterfly, the
// output sigmoid and delta) is spread over U units.  WU = 1: a warp is cut into
// segments of S lanes (S = the power of two >= ceil(H / U), at least 2) that
// take separate rows; WU = 2: rows span two warps, whose partial z2 meet in
// shared memory.  D = 4 DQ + DT with DT < 4: the row buffer is 4 (DQ + 1)
// floats wide when DT > 0 (zero padded) and DW = 4 DQ + DT multiply-adds are
// issued per unit; the paper's 33 markers are DQ = 8, DT = 1, with no padding.
// Narrower nets (D < DW) read zero padding columns.
#pragma once

#include "mlp_internal.cuh"

namespace mlp {

template <int DQ, int DT, int U, int WU, int ACT, int RB, int NW>
struct RowEngine2 {
    static_assert(DT >= 0 && DT < 4, "D tail");
    static constexpr int DW = 4 * DQ + DT;                 // inputs covered by the multiply-adds
    static constexpr int DPR = 4 * (DQ + (DT > 0 ? 1 : 0)); // row stride in shared memory
    static constexpr int NG = NW / WU;                      // row groups per block
    static constexpr int ZX = 2 * NW * RB;                  // floats of z2 exchange space
    float w[U][DW];
    float acc[U][DW];
    float b1r[U], w2r[U], gb1a[U], gw2a[U];
    float b2, gb2a;
    double sse;
    int H, Dr, S, par;   // Dr: the nets' D (<= DW; the row buffer's columns Dr..DW-1 are 0)

    __device__ __forceinline__ void setup(int H_, int D_) {
        H = H_;
        Dr = D_;
        S = 32;
        if (WU == 1) {
            const int lanes = (H + U - 1) / U;
            S = 2;
            while (S < lanes) S <<= 1;
        }
        par = 0;
    }
    // Group-lane index gl; unit i of this lane is gl + i * WU * S.
    __device__ __forceinline__ int glane() const { return ((threadIdx.x >> 5) % WU) * 32 + (threadIdx.x & 31) % S; }
    __device__ __forceinline__ int unit(int i) const { return glane() + i * WU * S; }

    // Weights from the packed parameters [W1 (H x D), b1, w2, b2] in shared
    // memory; zero the gradient sums.
    __device__ __forceinline__ void load_weights(const float *Wm) {
        const int HD = H * Dr;
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int j = unit(i);
            const bool own = j < H;
            const float *wr = Wm + (own ? j : 0) * Dr;
#pragma unroll
            for (int k = 0; k < DW; ++k) w[i][k] = (own && k < Dr) ? wr[k] : 0.f;
            b1r[i] = own ? Wm[HD + j] : 0.f;
            w2r[i] = own ? Wm[HD + H + j] : 0.f;
#pragma unroll
            for (int k = 0; k < DW; ++k) acc[i][k] = 0.f;
            gb1a[i] = gw2a[i] = 0.f;
        }
        b2 = Wm[HD + 2 * H];
        gb2a = 0.f;
        sse = 0.0;
    }

    // Rows 0..cn-1 of the staged chunk Xs (DPR floats per row, zero padded)
    // with labels ys; c scales the output delta (1/m or 1).
    __device__ __forceinline__ void rows(const float *Xs, const float *ys, int cn, float c, float *zx) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int grp = warp / WU, wu = warp % WU;
        const int slot = lane / S;
        const int nslots = 32 / S;
        const int RPI = nslots * RB;
        float sse_f = 0.f;
        for (int base = grp * RPI; base < cn; base += NG * RPI) {
            int xo[RB], rr[RB];
            bool valid[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) {
                rr[t] = base + t * nslots + slot;
                valid[t] = rr[t] < cn;
                xo[t] = (valid[t] ? rr[t] : 0) * DPR;
            }
            // Two partial sums a (row, unit), even and odd inputs, so that each
            // lane has 2 U RB independent multiply-add chains in flight.
            float z[RB][U], zo[RB][U];
#pragma unroll
            for (int t = 0; t < RB; ++t)
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    z[t][i] = b1r[i];
                    zo[t][i] = 0.f;
                }
#pragma unroll
            for (int q = 0; q < DQ; ++q) {
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(Xs + xo[t] + 4 * q);
#pragma unroll
                    for (int i = 0; i < U; ++i) {
                        z[t][i] = fmaf(xv.x, w[i][4 * q + 0], z[t][i]);
                        zo[t][i] = fmaf(xv.y, w[i][4 * q + 1], zo[t][i]);
                        z[t][i] = fmaf(xv.z, w[i][4 * q + 2], z[t][i]);
                        zo[t][i] = fmaf(xv.w, w[i][4 * q + 3], zo[t][i]);
                    }
                }
            }
            if (DT > 0) {
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(Xs + xo[t] + 4 * DQ);
                    const float xt[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                    for (int i = 0; i < U; ++i)
#pragma unroll
                        for (int d = 0; d < DT; ++d) z[t][i] = fmaf(xt[d], w[i][4 * DQ + d], z[t][i]);
                }
            }
#pragma unroll
            for (int t = 0; t < RB; ++t)
#pragma unroll
                for (int i = 0; i < U; ++i) z[t][i] += zo[t][i];
            // Re-read the rows from shared memory in the backward pass instead of
            // keeping RB x D values live in registers.
            asm volatile("" ::: "memory");
            float zp[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) {
                zp[t] = 0.f;
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    z[t][i] = Act<ACT>::f(z[t][i]);      // z now holds h
                    zp[t] = fmaf(z[t][i], w2r[i], zp[t]);
                }
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
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    gw2a[i] = fmaf(d2, z[t][i], gw2a[i]);
                    const float d1 = d2 * w2r[i] * Act<ACT>::df(z[t][i]);
                    gb1a[i] += d1;
                    z[t][i] = d1;                       // z now holds d1
                }
            }
#pragma unroll
            for (int q = 0; q < DQ; ++q) {
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(Xs + xo[t] + 4 * q);
#pragma unroll
                    for (int i = 0; i < U; ++i) {
                        acc[i][4 * q + 0] = fmaf(z[t][i], xv.x, acc[i][4 * q + 0]);
                        acc[i][4 * q + 1] = fmaf(z[t][i], xv.y, acc[i][4 * q + 1]);
                        acc[i][4 * q + 2] = fmaf(z[t][i], xv.z, acc[i][4 * q + 2]);
                        acc[i][4 * q + 3] = fmaf(z[t][i], xv.w, acc[i][4 * q + 3]);
                    }
                }
            }
            if (DT > 0) {
#pragma unroll
                for (int t = 0; t < RB; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(Xs + xo[t] + 4 * DQ);
                    const float xt[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                    for (int i = 0; i < U; ++i)
#pragma unroll
                        for (int d = 0; d < DT; ++d) acc[i][4 * DQ + d] = fmaf(z[t][i], xt[d], acc[i][4 * DQ + d]);
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
            for (int off = 2; off < 32; off <<= 1) {
                if (off >= S) {
#pragma unroll
                    for (int i = 0; i < U; ++i) {
#pragma unroll
                        for (int k = 0; k < DW; ++k) acc[i][k] += __shfl_xor_sync(0xffffffffu, acc[i][k], off);
                        gb1a[i] += __shfl_xor_sync(0xffffffffu, gb1a[i], off);
                        gw2a[i] += __shfl_xor_sync(0xffffffffu, gw2a[i], off);
                    }
                    gb2a += __shfl_xor_sync(0xffffffffu, gb2a, off);
                    sse += __shfl_xor_sync(0xffffffffu, sse, off);
                }
            }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int grp = warp / WU, wu = warp % WU;
        const int HD = H * Dr, P = HD + 2 * H + 1;
        float *pg = part + grp * P;
        if (lane < S) {
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const int j = unit(i);
                if (j < H) {
                    float *gr = pg + j * Dr;
#pragma unroll
                    for (int k = 0; k < DW; ++k)
                        if (k < Dr) gr[k] = acc[i][k];
                    pg[HD + j] = gb1a[i];
                    pg[HD + H + j] = gw2a[i];
                }
            }
        }
        if (wu == 0 && lane == 0) {
            pg[P - 1] = gb2a;
            s_sse[grp] = sse;
        }
    }
};

// Shared-memory floats for the group partials of a block of NW warps whose
// nets have up to Hmax hidden units (U units a lane: a group is one warp up to
// 32 U units, two warps above).
__host__ __device__ inline int re2_part_floats(int D, int Hmax, int U, int NW) {
    const int H1 = 32 * U < Hmax ? 32 * U : Hmax;
    const int v1 = NW * ((D + 2) * H1 + 1);
    const int v2 = Hmax > 32 * U ? (NW / 2) * ((D + 2) * Hmax + 1) : 0;
    const int pf = v1 > v2 ? v1 : v2;
    return (pf + 3) & ~3;
}

}  // namespace mlp
