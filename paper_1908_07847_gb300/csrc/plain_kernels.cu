// Plain path: separate forward, output, gradient, reduction and update kernels
// for any D and H, with the hidden activations materialised in device memory.
// This is the straightforward data-parallel mapping of Sec. 2.2 of
// arXiv 1908.07847 (feed-forward, output error, backpropagation, gradient
// descent) and the baseline the fused kernels are measured against.  It also
// provides the FP64 kernels used for gradient checking.
#include "mlp_internal.cuh"

namespace mlp {

namespace {

constexpr int TS = 64;   // rows per tile
constexpr int TJ = 64;   // hidden units per tile
constexpr int TK = 16;   // reduction slice
constexpr int NTH = 256; // threads per block (16 x 16, 4 x 4 outputs each)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// z1 = X W1^T + b1 on a 64-row x 64-unit tile, h = f(z1), and the tile's share
// of z2 = h w2 (summed over the tile's units) written to z2part[tile_j][row].
template <typename T, typename TX, int ACT>
__global__ void __launch_bounds__(NTH) k_fwd_hidden(int D, int H, int64_t n, const TX *__restrict__ X,
                                                    const T *__restrict__ W1, const T *__restrict__ b1,
                                                    const T *__restrict__ w2, T *__restrict__ hid,
                                                    T *__restrict__ z2part) {
    __shared__ T Xs[TK][TS + 1];
    __shared__ T Ws[TK][TJ + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t s0 = (int64_t)blockIdx.x * TS;
    const int j0 = blockIdx.y * TJ;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

    for (int k0 = 0; k0 < D; k0 += TK) {
#pragma unroll
        for (int r = 0; r < (TS * TK) / NTH; ++r) {
            int e = tid + r * NTH, s = e / TK, k = e % TK;
            int64_t row = s0 + s;
            Xs[k][s] = (row < n && k0 + k < D) ? ldx<T, TX>(X, row * D + k0 + k) : T(0);
            int j = j0 + s;  // TJ == TS
            Ws[k][s] = (j < H && k0 + k < D) ? W1[(int64_t)j * D + k0 + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[k][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Ws[k][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }

    T zp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        zp[i] = T(0);
        int64_t row = s0 + ty * 4 + i;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            int j = j0 + tx * 4 + jj;
            if (row < n && j < H) {
                T h = Act<ACT>::f(acc[i][jj] + b1[j]);
                if (hid) hid[row * H + j] = h;
                zp[i] = fma(h, w2[j], zp[i]);
            }
        }
    }
    // Sum over the 16 threads (tx) that share these rows: lanes of one half-warp.
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) zp[i] += __shfl_xor_sync(0xffffffffu, zp[i], off);
        int64_t row = s0 + ty * 4 + i;
        if (tx == 0 && row < n) z2part[(int64_t)blockIdx.y * n + row] = zp[i];
    }
}

// o = sigmoid(b2 + sum_t z2part[t]) (Eq. 1); optional output delta and
// squared-error partial per block (FP64, fixed tree order).
template <typename T>
__global__ void __launch_bounds__(256) k_fwd_output(int ntj, int64_t n, const T *__restrict__ z2part,
                                                    const T *__restrict__ b2, T *__restrict__ o,
                                                    const T *__restrict__ y, const T *__restrict__ dLdo,
                                                    T c, T *__restrict__ d2, double *__restrict__ ssep) {
    __shared__ double red[8];
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double se = 0.0;
    if (i < n) {
        T z = b2[0];
        for (int t = 0; t < ntj; ++t) z += z2part[(int64_t)t * n + i];
        T oi = sigmoid_out(z);
        o[i] = oi;
        if (y) {
            T e = oi - y[i];
            d2[i] = c * e * oi * (T(1) - oi);
            se = (double)e * (double)e;
        } else if (dLdo) {
            d2[i] = dLdo[i] * oi * (T(1) - oi);
        }
    }
    if (ssep) {
        se = warp_sum(se);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w];
            ssep[blockIdx.x] = s;
        }
    }
}

// d2 = dLdo * o (1 - o) from saved outputs (autograd backward).
template <typename T>
__global__ void k_d2_upstream(int64_t n, const T *__restrict__ o, const T *__restrict__ dLdo, T *__restrict__ d2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d2[i] = dLdo[i] * o[i] * (T(1) - o[i]);
}

// Gradient partials over one chunk of rows (Sec. 2.2 backpropagation):
//   d1 = d2 w2 f'(h);  part[c] W1-slot (j, k) = sum_rows d1 X;
//   b1-slot = sum d1;  w2-slot = sum d2 h;  b2-slot = sum d2.
// grid: x = unit tiles, y = input tiles, z = chunks.
template <typename T, typename TX, int ACT>
__global__ void __launch_bounds__(NTH) k_bwd_grad(int D, int H, int64_t n, int64_t CH, const TX *__restrict__ X,
                                                  const T *__restrict__ w2, const T *__restrict__ hid,
                                                  const T *__restrict__ d2, T *__restrict__ part) {
    __shared__ T Ds[TK][TJ + 1];
    __shared__ T Xs[TK][64 + 1];
    __shared__ T red_b1[4][TJ];
    __shared__ T red_w2[4][TJ];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int j0 = blockIdx.x * TJ, k0 = blockIdx.y * 64;
    const int64_t c = blockIdx.z;
    const int64_t r0 = c * CH, r1 = min(n, r0 + CH);
    const int64_t P = (int64_t)(D + 2) * H + 1;
    const bool do_bias = (blockIdx.y == 0);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    T gb1 = T(0), gw2 = T(0);  // for unit j0 + (tid & 63)
    const int jl = tid & 63;
    const T w2j = (j0 + jl < H) ? w2[j0 + jl] : T(0);

    for (int64_t rs = r0; rs < r1; rs += TK) {
#pragma unroll
        for (int r = 0; r < (TK * TJ) / NTH; ++r) {
            int e = tid + r * NTH, s = e / TJ, j = e % TJ;  // j == jl
            int64_t row = rs + s;
            T d1 = T(0);
            if (row < r1 && j0 + j < H) {
                T h = hid[row * H + j0 + j];
                T dd = d2[row];
                d1 = dd * w2j * Act<ACT>::df(h);
                if (do_bias) {
                    gb1 += d1;
                    gw2 = fma(dd, h, gw2);
                }
            }
            Ds[s][j] = d1;
            int kk = e % 64;
            Xs[s][kk] = (row < r1 && k0 + kk < D) ? ldx<T, TX>(X, row * D + k0 + kk) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < TK; ++s) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ds[s][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Xs[s][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) acc[i][kk] = fma(a[i], b[kk], acc[i][kk]);
        }
        __syncthreads();
    }
    T *pc = part + c * P;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int j = j0 + ty * 4 + i;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            int k = k0 + tx * 4 + kk;
            if (j < H && k < D) pc[(int64_t)j * D + k] = acc[i][kk];
        }
    }
    if (do_bias) {
        red_b1[tid >> 6][jl] = gb1;
        red_w2[tid >> 6][jl] = gw2;
        __syncthreads();
        if (tid < TJ && j0 + tid < H) {
            T sb = red_b1[0][tid], sw = red_w2[0][tid];
            for (int q = 1; q < 4; ++q) {
                sb += red_b1[q][tid];
                sw += red_w2[q][tid];
            }
            pc[(int64_t)H * D + j0 + tid] = sb;
            pc[(int64_t)H * D + H + j0 + tid] = sw;
        }
        if (blockIdx.x == 0 && tid < 32) {
            T s = T(0);
            for (int64_t row = r0 + tid; row < r1; row += 32) s += d2[row];
            s = warp_sum(s);
            if (tid == 0) pc[P - 1] = s;
        }
    }
}

// g[p] = sum over chunks c = 0..C-1 of part[c][p], scattered to the four
// gradient arrays.
template <typename T>
__global__ void k_reduce_partials(int D, int H, int C, const T *__restrict__ part, T *gW1, T *gb1, T *gw2,
                                  T *gb2) {
    const int64_t P = (int64_t)(D + 2) * H + 1;
    const int64_t HD = (int64_t)H * D;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    T g = T(0);
    for (int c = 0; c < C; ++c) g += part[(int64_t)c * P + p];
    if (p < HD) gW1[p] = g;
    else if (p < HD + H) gb1[p - HD] = g;
    else if (p < HD + 2 * H) gw2[p - HD - H] = g;
    else gb2[0] = g;
}

// Fixed-order FP64 sum of `m` partials (one block), scaled, into *out.
__global__ void k_sum_doubles(int64_t m, const double *__restrict__ v, double scale, double *out, int *status) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += 256) s += v[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        t *= scale;
        *out = t;
        if (status && !isfinite(t)) atomicOr(status, ST_NONFINITE);
    }
}

// gX = d1 W1 on a 64-row x 64-input tile, d1 recomputed from hid, d2, w2.
template <typename T, int ACT>
__global__ void __launch_bounds__(NTH) k_bwd_input(int D, int H, int64_t n, const T *__restrict__ W1,
                                                   const T *__restrict__ w2, const T *__restrict__ hid,
                                                   const T *__restrict__ d2, T *__restrict__ gX) {
    __shared__ T Ds[TK][TS + 1];   // [j][row]
    __shared__ T Ws[TK][64 + 1];   // [j][k]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t s0 = (int64_t)blockIdx.x * TS;
    const int k0 = blockIdx.y * 64;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int j0 = 0; j0 < H; j0 += TK) {
#pragma unroll
        for (int r = 0; r < (TK * TS) / NTH; ++r) {
            int e = tid + r * NTH;
            int s = e / TK, j = e % TK;
            int64_t row = s0 + s;
            T d1 = T(0);
            if (row < n && j0 + j < H) d1 = d2[row] * w2[j0 + j] * Act<ACT>::df(hid[row * H + j0 + j]);
            Ds[j][s] = d1;
            int jw = e / 64, k = e % 64;
            Ws[jw][k] = (j0 + jw < H && k0 + k < D) ? W1[(int64_t)(j0 + jw) * D + k0 + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TK; ++j) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ds[j][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Ws[j][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) acc[i][kk] = fma(a[i], b[kk], acc[i][kk]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t row = s0 + ty * 4 + i;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            int k = k0 + tx * 4 + kk;
            if (row < n && k < D) gX[row * D + k] = acc[i][kk];
        }
    }
}

template <typename T>
__global__ void k_update(int64_t m, T lr, T *__restrict__ w, const T *__restrict__ g) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) w[i] -= lr * g[i];
}

template <typename T>
__global__ void k_gnorm_partial(int64_t P, const T *__restrict__ g, double *part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x; p < P; p += (int64_t)gridDim.x * 256) {
        double v = (double)g[p];
        s += v * v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_sqrt_sum(int m, const double *part, double *out) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t += part[i];
        *out = sqrt(t);
    }
}

__global__ void k_accum(double *dst, const double *src, int first) {
    if (threadIdx.x == 0) *dst = (first ? 0.0 : *dst) + *src;
}

template <typename T>
__global__ void k_labels(int64_t n, const T *__restrict__ o, int8_t *__restrict__ lab) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lab[i] = (o[i] >= T(0.5)) ? 1 : 0;
}

// ---------------------------------------------------------------- dispatch

template <typename T, typename TX>
cudaError_t forward_t(int act, int D, int H, int64_t n, const void *X, const void *W1, const void *b1,
                      const void *w2, const void *b2, void *hid, void *o, const void *y, const void *dLdo,
                      double c, const PlainWork &w, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dim3 g1((unsigned)cdiv(n, TS), (unsigned)cdiv(H, TJ));
    if (act == MLP_ACT_TANH)
        k_fwd_hidden<T, TX, MLP_ACT_TANH><<<g1, NTH, 0, st>>>(D, H, n, (const TX *)X, (const T *)W1,
                                                               (const T *)b1, (const T *)w2, (T *)hid,
                                                               (T *)w.z2part);
    else
        k_fwd_hidden<T, TX, MLP_ACT_SIGMOID><<<g1, NTH, 0, st>>>(D, H, n, (const TX *)X, (const T *)W1,
                                                                  (const T *)b1, (const T *)w2, (T *)hid,
                                                                  (T *)w.z2part);
    k_fwd_output<T><<<(unsigned)cdiv(n, 256), 256, 0, st>>>((int)cdiv(H, TJ), n, (const T *)w.z2part,
                                                            (const T *)b2, (T *)o, (const T *)y,
                                                            (const T *)dLdo, (T)c, (T *)w.d2,
                                                            (y != nullptr) ? w.ssep : nullptr);
    return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t backward_t(int act, int D, int H, int64_t n, const void *X, const void *W1, const void *w2,
                       const void *hid, void *gW1, void *gb1, void *gw2, void *gb2, void *gX, double *loss,
                       double c_loss, int *status, const PlainWork &w, cudaStream_t st) {
    const int64_t P = (int64_t)(D + 2) * H + 1;
    if (n == 0) {
        cudaMemsetAsync(gW1, 0, sizeof(T) * (size_t)H * D, st);
        cudaMemsetAsync(gb1, 0, sizeof(T) * (size_t)H, st);
        cudaMemsetAsync(gw2, 0, sizeof(T) * (size_t)H, st);
        cudaMemsetAsync(gb2, 0, sizeof(T), st);
        if (loss) cudaMemsetAsync(loss, 0, sizeof(double), st);
        return cudaGetLastError();
    }
    dim3 g2((unsigned)cdiv(H, TJ), (unsigned)cdiv(D, 64), (unsigned)w.C);
    if (act == MLP_ACT_TANH)
        k_bwd_grad<T, TX, MLP_ACT_TANH><<<g2, NTH, 0, st>>>(D, H, n, w.CH, (const TX *)X, (const T *)w2,
                                                             (const T *)hid, (const T *)w.d2, (T *)w.part);
    else
        k_bwd_grad<T, TX, MLP_ACT_SIGMOID><<<g2, NTH, 0, st>>>(D, H, n, w.CH, (const TX *)X, (const T *)w2,
                                                                (const T *)hid, (const T *)w.d2, (T *)w.part);
    k_reduce_partials<T><<<(unsigned)cdiv(P, 256), 256, 0, st>>>(D, H, w.C, (const T *)w.part, (T *)gW1,
                                                                 (T *)gb1, (T *)gw2, (T *)gb2);
    if (loss) k_sum_doubles<<<1, 256, 0, st>>>(cdiv(n, 256), w.ssep, 0.5 * c_loss, loss, status);
    if (gX) {
        dim3 g3((unsigned)cdiv(n, TS), (unsigned)cdiv(D, 64));
        if (act == MLP_ACT_TANH)
            k_bwd_input<T, MLP_ACT_TANH><<<g3, NTH, 0, st>>>(D, H, n, (const T *)W1, (const T *)w2,
                                                             (const T *)hid, (const T *)w.d2, (T *)gX);
        else
            k_bwd_input<T, MLP_ACT_SIGMOID><<<g3, NTH, 0, st>>>(D, H, n, (const T *)W1, (const T *)w2,
                                                                (const T *)hid, (const T *)w.d2, (T *)gX);
    }
    return cudaGetLastError();
}

template <typename T> size_t tsize() { return sizeof(T); }

}  // namespace

size_t plain_workspace_bytes(int prec, int D, int H, int64_t n, int sms) {
    PlainWork w;
    plain_workspace_carve(nullptr, prec, D, H, n, sms, &w);
    return (size_t)(uintptr_t)w.part + (size_t)w.C * ((size_t)(D + 2) * H + 1) *
                                           (prec == MLP_FP64 ? sizeof(double) : sizeof(float));
}

void plain_workspace_carve(void *base, int prec, int D, int H, int64_t n, int sms, PlainWork *w) {
    size_t es = (prec == MLP_FP64) ? sizeof(double) : sizeof(float);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    int64_t nn = n > 0 ? n : 1;
    int tiles = (int)(cdiv(H, TJ) * cdiv(D, 64));
    // Enough row chunks for about two blocks per SM, at least 16 rows each.
    int64_t C = cdiv(2 * (int64_t)sms, tiles);
    C = C < 1 ? 1 : C;
    int64_t maxC = cdiv(nn, TK);
    if (C > maxC) C = maxC;
    int64_t CH = cdiv(cdiv(nn, C), TK) * TK;
    C = cdiv(nn, CH);
    size_t off = 0;
    char *b = (char *)base;
    w->z2part = b + off;
    off = al(off + es * (size_t)cdiv(H, TJ) * (size_t)nn);
    w->d2 = b + off;
    off = al(off + es * (size_t)nn);
    w->ssep = (double *)(b + off);
    off = al(off + sizeof(double) * (size_t)cdiv(nn, 256));
    w->part = b + off;
    w->C = (int)C;
    w->CH = CH;
}

cudaError_t plain_forward(int prec, int act, int D, int H, int64_t n, const void *X, const void *W1,
                          const void *b1, const void *w2, const void *b2, void *hid, void *o, const void *y,
                          const void *dLdo, double c, const PlainWork &w, cudaStream_t st) {
    if (prec == MLP_FP64)
        return forward_t<double, double>(act, D, H, n, X, W1, b1, w2, b2, hid, o, y, dLdo, c, w, st);
    if (prec == MLP_BF16)
        return forward_t<float, uint16_t>(act, D, H, n, X, W1, b1, w2, b2, hid, o, y, dLdo, c, w, st);
    return forward_t<float, float>(act, D, H, n, X, W1, b1, w2, b2, hid, o, y, dLdo, c, w, st);
}

cudaError_t plain_backward(int prec, int act, int D, int H, int64_t n, const void *X, const void *W1,
                           const void *w2, const void *hid, void *gW1, void *gb1, void *gw2, void *gb2,
                           void *gX, double *loss, double c_loss, int *status, const PlainWork &w,
                           cudaStream_t st) {
    if (prec == MLP_FP64)
        return backward_t<double, double>(act, D, H, n, X, W1, w2, hid, gW1, gb1, gw2, gb2, gX, loss, c_loss,
                                          status, w, st);
    if (prec == MLP_BF16)
        return backward_t<float, uint16_t>(act, D, H, n, X, W1, w2, hid, gW1, gb1, gw2, gb2, gX, loss, c_loss,
                                           status, w, st);
    return backward_t<float, float>(act, D, H, n, X, W1, w2, hid, gW1, gb1, gw2, gb2, gX, loss, c_loss, status,
                                    w, st);
}

cudaError_t plain_d2_upstream(int prec, int64_t n, const void *o, const void *dLdo, void *d2, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (prec == MLP_FP64)
        k_d2_upstream<double><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, (const double *)o, (const double *)dLdo,
                                                                      (double *)d2);
    else
        k_d2_upstream<float><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, (const float *)o, (const float *)dLdo,
                                                                     (float *)d2);
    return cudaGetLastError();
}

cudaError_t plain_update(int prec, int D, int H, double lr, void *W1, void *b1, void *w2, void *b2,
                         const void *gW1, const void *gb1, const void *gw2, const void *gb2, cudaStream_t st) {
    int64_t HD = (int64_t)H * D;
    if (prec == MLP_FP64) {
        k_update<double><<<(unsigned)cdiv(HD, 256), 256, 0, st>>>(HD, lr, (double *)W1, (const double *)gW1);
        k_update<double><<<(unsigned)cdiv(H, 256), 256, 0, st>>>(H, lr, (double *)b1, (const double *)gb1);
        k_update<double><<<(unsigned)cdiv(H, 256), 256, 0, st>>>(H, lr, (double *)w2, (const double *)gw2);
        k_update<double><<<1, 32, 0, st>>>(1, lr, (double *)b2, (const double *)gb2);
    } else {
        float l = (float)lr;
        k_update<float><<<(unsigned)cdiv(HD, 256), 256, 0, st>>>(HD, l, (float *)W1, (const float *)gW1);
        k_update<float><<<(unsigned)cdiv(H, 256), 256, 0, st>>>(H, l, (float *)b1, (const float *)gb1);
        k_update<float><<<(unsigned)cdiv(H, 256), 256, 0, st>>>(H, l, (float *)w2, (const float *)gw2);
        k_update<float><<<1, 32, 0, st>>>(1, l, (float *)b2, (const float *)gb2);
    }
    return cudaGetLastError();
}

cudaError_t plain_gnorm(int prec, int64_t P, const void *g, double *scratch64, double *out, cudaStream_t st) {
    // Two fixed-order levels: 64 block partials in scratch64, then one serial sum.
    if (prec == MLP_FP64) k_gnorm_partial<double><<<64, 256, 0, st>>>(P, (const double *)g, scratch64);
    else k_gnorm_partial<float><<<64, 256, 0, st>>>(P, (const float *)g, scratch64);
    k_sqrt_sum<<<1, 32, 0, st>>>(64, scratch64, out);
    return cudaGetLastError();
}

cudaError_t plain_accum(double *dst, const double *src, int first, cudaStream_t st) {
    k_accum<<<1, 32, 0, st>>>(dst, src, first);
    return cudaGetLastError();
}

cudaError_t plain_labels(int prec, int64_t n, const void *o, int8_t *labels, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (prec == MLP_FP64) k_labels<double><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, (const double *)o, labels);
    else k_labels<float><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, (const float *)o, labels);
    return cudaGetLastError();
}

}  // namespace mlp
