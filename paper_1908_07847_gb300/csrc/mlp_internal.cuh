// Internal declarations shared by the library's translation units.
// The method: one-hidden-layer feed-forward network, sigmoid (Eq. 1) or tanh
// hidden units, sigmoid output, squared-error backpropagation and gradient
// descent without momentum (Sec. 2.2 of arXiv 1908.07847).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_gb300.h"

namespace mlp {

// Device status bits (mlp_net::status).
constexpr int ST_TIMEOUT = 1;
constexpr int ST_NONFINITE = 2;
constexpr int ST_BADLAUNCH = 4;   // a kernel found its launch shape wrong and did nothing

// A cross-block wait gives up after this many nanoseconds.
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;

// ---------------------------------------------------------------- activations

// Eq. 1, sigmoid(x) = 1 / (1 + e^-x), in FP32 from hardware approximations:
//   t = 2^(-|x| log2 e) in (0, 1]: the product |x| log2 e is split into
//     hi + lo (Cody and Waite's split-constant argument reduction, with the
//     exact product error from one fused multiply-add), 2^-hi comes from the
//     ex2.approx instruction and 2^-lo ~ 1 - lo ln 2 corrects it;
//   r = 1 / (1 + t) from rcp.approx refined by one Newton-Raphson step;
//   sigmoid(x) = r for x >= 0 and t r for x < 0 (so that nothing overflows).
// Maximum relative error about 4e-7 (ex2.approx's error dominates); the tests
// bound it against FP64.
__device__ __forceinline__ float sigmoid_f32(float x) {
    const float L2E_HI = 1.44269502162933349609375f;      // log2(e) rounded to float
    const float L2E_LO = 1.925963033500011079e-8f;        // log2(e) - L2E_HI
    const float LN2 = 0.693147180559945309f;
    float a = fabsf(x);
    a = a > 104.0f ? 104.0f : a;  // 2^-150 is already 0; NaN passes through
    const float hi = a * L2E_HI;
    const float lo = fmaf(a, L2E_LO, fmaf(a, L2E_HI, -hi));
    float t;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(-hi));
    t = fmaf(t, -lo * LN2, t);
    const float d = 1.0f + t;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    r = fmaf(r, fmaf(-d, r, 1.0f), r);
    return x >= 0.0f ? r : t * r;
}

template <int ACT> struct Act;

// Eq. 1 sigmoid; derivative through the value: s (1 - s).
template <> struct Act<MLP_ACT_SIGMOID> {
    static __device__ __forceinline__ float f(float x) { return sigmoid_f32(x); }
    static __device__ __forceinline__ double f(double x) { return 1.0 / (1.0 + exp(-x)); }
    static __device__ __forceinline__ float df(float v) { return v * (1.0f - v); }
    static __device__ __forceinline__ double df(double v) { return v * (1.0 - v); }
};

// tanh (Sec. 2.2 names it as the other traditional activation); 1 - t^2.
template <> struct Act<MLP_ACT_TANH> {
    static __device__ __forceinline__ float f(float x) { return tanhf(x); }
    static __device__ __forceinline__ double f(double x) { return tanh(x); }
    static __device__ __forceinline__ float df(float v) { return 1.0f - v * v; }
    static __device__ __forceinline__ double df(double v) { return 1.0 - v * v; }
};

__device__ __forceinline__ float sigmoid_out(float x) { return sigmoid_f32(x); }
__device__ __forceinline__ double sigmoid_out(double x) { return 1.0 / (1.0 + exp(-x)); }

// ------------------------------------------------------------- element loads

// X element as the arithmetic type T: float from float, float from bf16 bits,
// double from double.
template <typename T, typename TX> __device__ __forceinline__ T ldx(const TX *p, int64_t i);
template <> __device__ __forceinline__ float ldx<float, float>(const float *p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ double ldx<double, double>(const double *p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ float ldx<float, uint16_t>(const uint16_t *p, int64_t i) {
    return __uint_as_float(((uint32_t)p[i]) << 16);
}

// ------------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) {
    return *(const volatile int *)p;
}

// 4-byte asynchronous global -> shared copy (all copies of a thread stay in
// flight until cp_async_wait_all).
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}
// 16-byte asynchronous global -> shared copy that bypasses L1 (both addresses
// 16-byte aligned).
__device__ __forceinline__ void cp_async16_cg(void *smem_dst, const void *gmem_src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Grid-wide barrier for kernels launched cooperatively (all blocks resident).
// `bar` is a 64-bit arrival counter that only ever grows; the host passes the
// value it had when the launch started (it knows how many arrivals every
// launch adds), and the k-th barrier of the launch waits until the counter
// reaches base + k * nblocks.  The wait gives up after WAIT_LIMIT_NS, or as
// soon as another block has recorded a failure, and then returns false after
// recording ST_TIMEOUT.
__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, unsigned long long target, int *status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1ull);
        unsigned long long t0 = global_ns();
        int ok = 1;
        while (ld_acquire(bar) < target) {
            if (ld_volatile(status) & ST_TIMEOUT) { ok = 0; break; }
            if (global_ns() - t0 > WAIT_LIMIT_NS) {
                atomicOr(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------ plain-path launchers
// Generic kernels for any D and H (FP32, FP64; BF16 inputs with FP32 math).
// All return cudaGetLastError() of their launches.

struct PlainWork {
    // device scratch, sized by plain_workspace_bytes()
    void *z2part;   // [ceil(H/64)] x n   (T)
    void *d2;       // n                   (T)
    double *ssep;   // ceil(n/256)
    void *part;     // C x P               (T)
    int C;          // number of sample chunks for gradient partials
    int64_t CH;     // rows per chunk
};

size_t plain_workspace_bytes(int prec, int D, int H, int64_t n, int sms);
void plain_workspace_carve(void *base, int prec, int D, int H, int64_t n, int sms, PlainWork *w);

// hid may be NULL.  When y != NULL also writes d2 = c (o - y) o (1 - o) and the
// per-block squared-error partials; when dLdo != NULL writes d2 = dLdo o (1-o).
cudaError_t plain_forward(int prec, int act, int D, int H, int64_t n, const void *X,
                          const void *W1, const void *b1, const void *w2, const void *b2,
                          void *hid, void *o, const void *y, const void *dLdo, double c,
                          const PlainWork &w, cudaStream_t st);

// Gradient partials and their fixed-order reduction into gW1, gb1, gw2, gb2.
// Needs hid and d2 from plain_forward.  loss (may be NULL) = 0.5 c_loss sse.
// gX (may be NULL) = d1 W1.
cudaError_t plain_backward(int prec, int act, int D, int H, int64_t n, const void *X,
                           const void *W1, const void *w2, const void *hid,
                           void *gW1, void *gb1, void *gw2, void *gb2, void *gX,
                           double *loss, double c_loss, int *status,
                           const PlainWork &w, cudaStream_t st);

// w <- w - lr g over the four parameter arrays.
cudaError_t plain_update(int prec, int D, int H, double lr, void *W1, void *b1, void *w2,
                         void *b2, const void *gW1, const void *gb1, const void *gw2,
                         const void *gb2, cudaStream_t st);

// ||g||_2 in FP64 (fixed order) written to *out; scratch64 holds 64 doubles.
cudaError_t plain_gnorm(int prec, int64_t P, const void *g_packed, double *scratch64, double *out,
                        cudaStream_t st);

// d2 = dLdo o (1 - o) into w.d2 (autograd backward).
cudaError_t plain_d2_upstream(int prec, int64_t n, const void *o, const void *dLdo, void *d2, cudaStream_t st);

// *dst = (first ? 0 : *dst) + *src (one thread).
cudaError_t plain_accum(double *dst, const double *src, int first, cudaStream_t st);

// labels[i] = o_i >= 0.5
cudaError_t plain_labels(int prec, int64_t n, const void *o, int8_t *labels, cudaStream_t st);

// ------------------------------------------------------- fused-path launcher

struct FusedScratch {
    long long *acc;           // 3 x (P + 1) fixed-point gradient accumulators
    unsigned long long *bar;  // barrier arrival counter
};

// Host-side view of the scratch state when the next launch starts: the
// counter's value and which accumulator buffer is first (the other two are 0).
struct FusedCounters {
    unsigned long long bar = 0;
    int rot = 0;
};

// True if the fused cooperative kernel supports this shape.
bool fused_supported(int D, int H);
// Scratch bytes for the fused kernel at its largest grid.
size_t fused_scratch_bytes(int D, int H, int sms);
void fused_scratch_carve(void *base, int D, int H, int sms, FusedScratch *s);

// Trains in place on the packed FP32 params [W1, b1, w2, b2].
// `ctr` is advanced by the arrivals the launches add.
cudaError_t fused_train(int act, int D, int H, int64_t n, const float *X, const float *y,
                        float *params, float lr, int loss_mean, int epochs, int64_t mb,
                        double *loss_hist, double *gnorm_hist, int *status,
                        const FusedScratch &s, FusedCounters *ctr, int rows_per_block,
                        int skip_block, cudaStream_t st, int *grid_used);

// ------------------------------------------------------ batched-path launcher

// One network of a batch, as the kernel reads it (device memory).
struct BatchNet {
    const float *X;      // n x D rows
    const float *y;      // n labels
    float *params;       // packed [W1, b1, w2, b2], trained in place
    double *loss_hist;   // [epochs] or NULL
    double *gnorm_hist;  // [epochs] or NULL
    int64_t n;
    int32_t H;
    int32_t pad;
};

int batched_max_H();
int batched_max_D();
void batched_smem_layout(int D, int Hmax, int *part_floats, int *wm_floats, size_t *bytes);

// Kernel shapes of the FP32 many-nets launch (the tuning knob of a plan).
constexpr int BATCH_SHAPE_U1 = 0;      // one hidden unit a lane, blocks of 8 warps, two per SM
constexpr int BATCH_SHAPE_U2_RB1 = 1;  // two units a lane, blocks of 4 warps, two per SM, one row in flight
constexpr int BATCH_SHAPE_U2_RB2 = 2;  // the same with two rows in flight (D = 33 only)
constexpr int BATCH_SHAPE_TILED128 = 3; // register-tiled products, passes of up to 128 rows
constexpr int BATCH_SHAPE_TILED64 = 4;  // register-tiled products, passes of 64 rows (less shared memory)
constexpr int BATCH_SHAPE_TILED32 = 5;  // register-tiled products, passes of 32 rows
constexpr int BATCH_SHAPE_U2_3B = 6;    // two units a lane, three blocks per SM (D = 33 only)
bool batched_shape_supported(int D, int shape);
cudaError_t batched_train(int act, int D, int Hmax, int64_t nmax, const BatchNet *nets_dev, const int *order_dev,
                          int n_nets, int epochs, float lr, int loss_mean, int *status, int shape, cudaStream_t st);
bool batched_tiled_supported(int D, int Hmax);
size_t batched_tiled_smem(int D, int Hmax, int ncap, int hcap);
cudaError_t batched_train_tiled(int act, int D, int Hmax, int64_t nmax, const BatchNet *nets_dev,
                                const int *order_dev, int n_nets, int epochs, float lr, int loss_mean, int *status,
                                int hcap_max, cudaStream_t st);
cudaError_t batched_train_u2(int act, int D, int Hmax, const BatchNet *nets_dev, const int *order_dev, int n_nets,
                             int epochs, float lr, int loss_mean, int *status, int rb, cudaStream_t st);
bool batched_u2_supported(int D, int rb);

// ------------------------------------------- bf16 tensor-core (tcgen05) path

bool tc_supported(int D, int H);
size_t tc_desc_bytes();
size_t tc_tmap_bytes();
cudaError_t tc_encode_map(void *map, const void *X, int D, int64_t n);
void tc_fill_desc(void *desc, const void *tmap_dev, const float *y, float *params, double *loss_hist,
                  double *gnorm_hist, int64_t n, int H);
cudaError_t tc_batched_train(const void *descs_dev, const int *order_dev, int n_nets, int D, int epochs, float lr,
                             int loss_mean, int act, int *status, int *next, cudaStream_t st);

// One wide network (H = 256..2048, a multiple of 256) trained by clusters of
// H/256 blocks; scratch of tc_cluster_scratch_bytes(), all zero before the first
// launch (the counters in *ctr then zero too).
bool tc_cluster_supported(int D, int H);
size_t tc_cluster_scratch_bytes(int D, int H);
int tc_cluster_max_clusters(int H);
// gnorm_hist (may be NULL) needs gn_part, (H/256 + 1) x epochs doubles of
// device scratch.  A device that refuses the cooperative cluster launch makes
// the call fail with that launch's error.
cudaError_t tc_cluster_train(const void *X, const float *y, float *params, int D, int H, int64_t n, int epochs,
                             int64_t mb, float lr, int loss_mean, int act, double *loss_hist, double *gnorm_hist,
                             double *gn_part, int *status, void *scratch, int max_clusters, FusedCounters *ctr,
                             cudaStream_t st);

int device_sm_count();

// Records msg as the calling thread's last error (mlp_last_error) and returns s.
mlp_status set_error(mlp_status s, const char *msg);

}  // namespace mlp
