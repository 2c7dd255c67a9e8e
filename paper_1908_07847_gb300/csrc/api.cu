// C ABI of the training library (declarations and contracts in mlp_gb300.h).
// Host code only: argument checks, handle-owned memory, kernel dispatch.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <algorithm>
#include <vector>

#include "mlp_internal.cuh"

struct mlp_net {
    mlp_config cfg;
    int device;
    int sms;
    size_t esz;       // bytes per master weight (4 or 8)
    int64_t P;        // (D + 2) H + 1
    void *params;     // packed master weights [W1, b1, w2, b2]
    void *grads;      // packed gradients
    int *status;      // device status word
    double *dtmp;     // 64 doubles of reduction scratch + 1 step loss
    void *pw = nullptr;   // plain workspace
    size_t pw_cap = 0;
    void *hid = nullptr;  // n x H activations (plain path)
    size_t hid_cap = 0;
    void *obuf = nullptr; // n outputs
    size_t obuf_cap = 0;
    void *fs = nullptr;   // fused-kernel scratch
    size_t fs_cap = 0;
    void *xstage = nullptr, *ystage = nullptr;  // mlp_train_host staging
    size_t xstage_cap = 0, ystage_cap = 0;
    double *lstage = nullptr;
    size_t lstage_cap = 0;
    double *gnp = nullptr;    // per-epoch gradient-norm partials (tensor-core cluster path)
    size_t gnp_cap = 0;
    int skip_block = -1;
    int rows_per_block = 32;
    int max_clusters = 1 << 30;   // cap on clusters of the tensor-core kernel
    mlp::FusedCounters ctr;   // fused-kernel counter values at the next launch
};

namespace {

thread_local std::string g_err;

mlp_status fail(mlp_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

mlp_status cuda_fail(cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(MLP_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(MLP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// Makes the handle's device current for the scope of a call, then restores.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// The tensor-core kernels address rows with 32-bit TMA coordinates and count a
// launch's tiles (and derive their barrier phases) in 32-bit integers.
bool tc_fits_32bit(int64_t n, int64_t epochs) {
    const int64_t tiles = (n + 127) / 128;
    return n <= (int64_t)INT32_MAX - 127 && epochs * tiles <= (int64_t)INT32_MAX;
}

// The device address of page-locked host memory, or NULL for pageable memory.
const void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

mlp_status grow(void **p, size_t *cap, size_t need, const char *what) {
    if (need <= *cap && *p) return MLP_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = need < 256 ? 256 : need;
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(MLP_ENOMEM, "cannot allocate %zu bytes for %s", want, what);
    }
    *cap = want;
    return MLP_OK;
}

size_t x_elem_bytes(int prec) { return prec == MLP_FP64 ? 8 : (prec == MLP_BF16 ? 2 : 4); }

char *W1p(mlp_t h) { return (char *)h->params; }
char *b1p(mlp_t h) { return (char *)h->params + h->esz * (size_t)h->cfg.H * h->cfg.D; }
char *w2p(mlp_t h) { return b1p(h) + h->esz * (size_t)h->cfg.H; }
char *b2p(mlp_t h) { return w2p(h) + h->esz * (size_t)h->cfg.H; }
char *gW1p(mlp_t h) { return (char *)h->grads; }
char *gb1p(mlp_t h) { return (char *)h->grads + h->esz * (size_t)h->cfg.H * h->cfg.D; }
char *gw2p(mlp_t h) { return gb1p(h) + h->esz * (size_t)h->cfg.H; }
char *gb2p(mlp_t h) { return gw2p(h) + h->esz * (size_t)h->cfg.H; }

mlp_status ensure_plain(mlp_t h, int64_t n, bool need_hid, mlp::PlainWork *w) {
    const int prec = h->cfg.prec, D = h->cfg.D, H = h->cfg.H;
    mlp_status s = grow(&h->pw, &h->pw_cap, mlp::plain_workspace_bytes(prec, D, H, n, h->sms), "workspace");
    if (s) return s;
    mlp::plain_workspace_carve(h->pw, prec, D, H, n, h->sms, w);
    s = grow(&h->obuf, &h->obuf_cap, h->esz * (size_t)(n > 0 ? n : 1), "outputs");
    if (s) return s;
    if (need_hid) {
        s = grow(&h->hid, &h->hid_cap, h->esz * (size_t)(n > 0 ? n : 1) * (size_t)H, "activations");
        if (s) return s;
    }
    return MLP_OK;
}

double loss_scale(int loss_mean, int64_t n) { return loss_mean ? (n > 0 ? 1.0 / (double)n : 0.0) : 1.0; }

// One plain-path gradient evaluation into the handle's packed gradient buffer
// (or caller pointers); loss (may be NULL) = 0.5 * c_loss * sse.
mlp_status plain_grad(mlp_t h, const void *X, const void *y, int64_t n, void *gW1, void *gb1, void *gw2,
                      void *gb2, double *loss, double c_loss, cudaStream_t st) {
    mlp::PlainWork w;
    mlp_status s = ensure_plain(h, n, true, &w);
    if (s) return s;
    const double c = loss_scale(h->cfg.loss_mean, n);
    CK(mlp::plain_forward(h->cfg.prec, h->cfg.act, h->cfg.D, h->cfg.H, n, X, W1p(h), b1p(h), w2p(h), b2p(h),
                          h->hid, h->obuf, y, nullptr, c, w, st),
       "forward kernels");
    CK(mlp::plain_backward(h->cfg.prec, h->cfg.act, h->cfg.D, h->cfg.H, n, X, W1p(h), w2p(h), h->hid, gW1, gb1,
                           gw2, gb2, nullptr, loss, c_loss, h->status, w, st),
       "backward kernels");
    return MLP_OK;
}

mlp_status check_handle(mlp_t h) {
    if (!h) return fail(MLP_EINVAL, "null handle");
    return MLP_OK;
}

}  // namespace

// Records the message of a failure in a translation unit of its own.
mlp_status noalloc_fail(mlp_status s, const char *msg) { return fail(s, "%s", msg); }

namespace mlp {
mlp_status set_error(mlp_status s, const char *msg) { return fail(s, "%s", msg); }

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}
}  // namespace mlp

extern "C" {

const char *mlp_last_error(void) { return g_err.c_str(); }

const char *mlp_version(void) { return "mlp_gb300 1.0 (sm_103a)"; }

mlp_status mlp_create(const mlp_config *cfg, mlp_t *out) {
    if (!cfg || !out) return fail(MLP_EINVAL, "mlp_create: null argument");
    *out = nullptr;
    if (cfg->D < 1 || cfg->D > 4096) return fail(MLP_EINVAL, "mlp_create: D=%d out of 1..4096", cfg->D);
    if (cfg->H < 1 || cfg->H > 65536) return fail(MLP_EINVAL, "mlp_create: H=%d out of 1..65536", cfg->H);
    if (cfg->prec < MLP_FP32 || cfg->prec > MLP_FP64) return fail(MLP_EINVAL, "mlp_create: bad precision");
    if (cfg->act != MLP_ACT_SIGMOID && cfg->act != MLP_ACT_TANH) return fail(MLP_EINVAL, "mlp_create: bad act");
    if (!(cfg->lr == cfg->lr)) return fail(MLP_EINVAL, "mlp_create: lr is NaN");
    mlp_t h = new (std::nothrow) mlp_net();
    if (!h) return fail(MLP_ENOMEM, "mlp_create: host allocation");
    h->cfg = *cfg;
    h->cfg.loss_mean = cfg->loss_mean ? 1 : 0;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(MLP_ECUDA, "mlp_create: no CUDA device");
    }
    h->sms = mlp::device_sm_count();
    h->esz = cfg->prec == MLP_FP64 ? 8 : 4;
    h->P = (int64_t)(cfg->D + 2) * cfg->H + 1;
    size_t pb = h->esz * (size_t)h->P;
    size_t need = 2 * ((pb + 255) & ~(size_t)255) + 256 + 66 * sizeof(double);
    char *base = nullptr;
    if (cudaMalloc((void **)&base, need) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(MLP_ENOMEM, "mlp_create: cannot allocate %zu bytes", need);
    }
    h->params = base;
    h->grads = base + ((pb + 255) & ~(size_t)255);
    h->status = (int *)(base + 2 * ((pb + 255) & ~(size_t)255));
    h->dtmp = (double *)((char *)h->status + 256);
    if (cudaMemset(base, 0, need) != cudaSuccess) {
        cudaFree(base);
        delete h;
        return fail(MLP_ECUDA, "mlp_create: memset failed");
    }
    *out = h;
    return MLP_OK;
}

void mlp_destroy(mlp_t h) {
    if (!h) return;
    DeviceScope ds(h->device);
    cudaFree(h->params);
    if (h->pw) cudaFree(h->pw);
    if (h->hid) cudaFree(h->hid);
    if (h->obuf) cudaFree(h->obuf);
    if (h->fs) cudaFree(h->fs);
    if (h->xstage) cudaFree(h->xstage);
    if (h->ystage) cudaFree(h->ystage);
    if (h->lstage) cudaFree(h->lstage);
    if (h->gnp) cudaFree(h->gnp);
    delete h;
}

mlp_status mlp_set_weights(mlp_t h, const void *W1, const void *b1, const void *w2, const void *b2) {
    if (check_handle(h)) return MLP_EINVAL;
    if (!W1 || !b1 || !w2 || !b2) return fail(MLP_EINVAL, "mlp_set_weights: null pointer");
    DeviceScope ds(h->device);
    const size_t HD = (size_t)h->cfg.H * h->cfg.D, Hs = (size_t)h->cfg.H;
    CK(cudaMemcpy(W1p(h), W1, h->esz * HD, cudaMemcpyHostToDevice), "mlp_set_weights");
    CK(cudaMemcpy(b1p(h), b1, h->esz * Hs, cudaMemcpyHostToDevice), "mlp_set_weights");
    CK(cudaMemcpy(w2p(h), w2, h->esz * Hs, cudaMemcpyHostToDevice), "mlp_set_weights");
    CK(cudaMemcpy(b2p(h), b2, h->esz, cudaMemcpyHostToDevice), "mlp_set_weights");
    return MLP_OK;
}

mlp_status mlp_get_weights(mlp_t h, void *W1, void *b1, void *w2, void *b2) {
    if (check_handle(h)) return MLP_EINVAL;
    if (!W1 || !b1 || !w2 || !b2) return fail(MLP_EINVAL, "mlp_get_weights: null pointer");
    DeviceScope ds(h->device);
    const size_t HD = (size_t)h->cfg.H * h->cfg.D, Hs = (size_t)h->cfg.H;
    CK(cudaDeviceSynchronize(), "mlp_get_weights");
    CK(cudaMemcpy(W1, W1p(h), h->esz * HD, cudaMemcpyDeviceToHost), "mlp_get_weights");
    CK(cudaMemcpy(b1, b1p(h), h->esz * Hs, cudaMemcpyDeviceToHost), "mlp_get_weights");
    CK(cudaMemcpy(w2, w2p(h), h->esz * Hs, cudaMemcpyDeviceToHost), "mlp_get_weights");
    CK(cudaMemcpy(b2, b2p(h), h->esz, cudaMemcpyDeviceToHost), "mlp_get_weights");
    return MLP_OK;
}

mlp_status mlp_weights_device(mlp_t h, void **p) {
    if (check_handle(h)) return MLP_EINVAL;
    if (!p) return fail(MLP_EINVAL, "mlp_weights_device: null pointer");
    *p = h->params;
    return MLP_OK;
}

mlp_status mlp_forward(mlp_t h, const void *X, int64_t n, void *o, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (n < 0 || (n > 0 && (!X || !o))) return fail(MLP_EINVAL, "mlp_forward: bad arguments");
    if (n == 0) return MLP_OK;
    DeviceScope ds(h->device);
    mlp::PlainWork w;
    mlp_status s = ensure_plain(h, n, false, &w);
    if (s) return s;
    CK(mlp::plain_forward(h->cfg.prec, h->cfg.act, h->cfg.D, h->cfg.H, n, X, W1p(h), b1p(h), w2p(h), b2p(h),
                          nullptr, o, nullptr, nullptr, 0.0, w, (cudaStream_t)stream),
       "mlp_forward");
    return MLP_OK;
}

mlp_status mlp_backward(mlp_t h, const void *X, const void *y, int64_t n, void *gW1, void *gb1, void *gw2,
                        void *gb2, double *loss, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (n < 0 || !gW1 || !gb1 || !gw2 || !gb2 || (n > 0 && (!X || !y)))
        return fail(MLP_EINVAL, "mlp_backward: bad arguments");
    DeviceScope ds(h->device);
    return plain_grad(h, X, y, n, gW1, gb1, gw2, gb2, loss, loss_scale(h->cfg.loss_mean, n),
                      (cudaStream_t)stream);
}

mlp_status mlp_update(mlp_t h, const void *gW1, const void *gb1, const void *gw2, const void *gb2,
                      void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (!gW1 || !gb1 || !gw2 || !gb2) return fail(MLP_EINVAL, "mlp_update: null gradient");
    DeviceScope ds(h->device);
    CK(mlp::plain_update(h->cfg.prec, h->cfg.D, h->cfg.H, (double)h->cfg.lr, W1p(h), b1p(h), w2p(h), b2p(h), gW1,
                         gb1, gw2, gb2, (cudaStream_t)stream),
       "mlp_update");
    return MLP_OK;
}

mlp_status mlp_step_plain(mlp_t h, const void *X, const void *y, int64_t n, double *loss, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (n < 0 || (n > 0 && (!X || !y))) return fail(MLP_EINVAL, "mlp_step_plain: bad arguments");
    DeviceScope ds(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    mlp_status s = plain_grad(h, X, y, n, gW1p(h), gb1p(h), gw2p(h), gb2p(h), loss,
                              loss_scale(h->cfg.loss_mean, n), st);
    if (s) return s;
    CK(mlp::plain_update(h->cfg.prec, h->cfg.D, h->cfg.H, (double)h->cfg.lr, W1p(h), b1p(h), w2p(h), b2p(h),
                         gW1p(h), gb1p(h), gw2p(h), gb2p(h), st),
       "mlp_step_plain update");
    return MLP_OK;
}

mlp_status mlp_train_epochs(mlp_t h, const void *X, const void *y, int64_t n, int32_t epochs, int64_t minibatch,
                            double *loss_hist, double *gnorm_hist, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (n < 0 || epochs < 0 || (n > 0 && (!X || !y))) return fail(MLP_EINVAL, "mlp_train_epochs: bad arguments");
    if (epochs == 0) return MLP_OK;
    DeviceScope ds(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (loss_hist) CK(cudaMemsetAsync(loss_hist, 0, sizeof(double) * epochs, st), "mlp_train_epochs");
        if (gnorm_hist) CK(cudaMemsetAsync(gnorm_hist, 0, sizeof(double) * epochs, st), "mlp_train_epochs");
        return MLP_OK;
    }
    const int D = h->cfg.D, H = h->cfg.H;
    if (h->cfg.prec == MLP_FP32 && mlp::fused_supported(D, H)) {
        void *before = h->fs;
        mlp_status s = grow(&h->fs, &h->fs_cap, mlp::fused_scratch_bytes(D, H, h->sms), "fused scratch");
        if (s) return s;
        mlp::FusedScratch fsc;
        mlp::fused_scratch_carve(h->fs, D, H, h->sms, &fsc);
        // A fresh buffer starts with zero accumulators and counter.
        if (h->fs != before) {
            CK(cudaMemsetAsync(h->fs, 0, h->fs_cap, st), "fused scratch reset");
            h->ctr = mlp::FusedCounters();
        }
        CK(mlp::fused_train(h->cfg.act, D, H, n, (const float *)X, (const float *)y, (float *)h->params,
                            h->cfg.lr, h->cfg.loss_mean, epochs, minibatch, loss_hist, gnorm_hist, h->status,
                            fsc, &h->ctr, h->rows_per_block, h->skip_block, st, nullptr),
           "fused training kernel");
        return MLP_OK;
    }
    if (h->cfg.prec == MLP_BF16 && mlp::tc_cluster_supported(D, H)) {
        if (!tc_fits_32bit(n, epochs))
            return fail(MLP_EINVAL, "mlp_train_epochs: more than 2^31 - 128 rows, or epochs x tiles beyond 2^31");
        void *before = h->fs;
        mlp_status s = grow(&h->fs, &h->fs_cap, mlp::tc_cluster_scratch_bytes(D, H), "cluster scratch");
        if (s) return s;
        if (h->fs != before) {
            CK(cudaMemsetAsync(h->fs, 0, h->fs_cap, st), "cluster scratch reset");
            h->ctr = mlp::FusedCounters();
        }
        if (gnorm_hist) {
            s = grow((void **)&h->gnp, &h->gnp_cap, sizeof(double) * (size_t)(H / 256 + 1) * epochs, "norm scratch");
            if (s) return s;
        }
        cudaError_t e = mlp::tc_cluster_train(X, (const float *)y, (float *)h->params, D, H, n, epochs, minibatch,
                                              h->cfg.lr, h->cfg.loss_mean, h->cfg.act, loss_hist, gnorm_hist, h->gnp,
                                              h->status, h->fs, h->max_clusters, &h->ctr, st);
        if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
            cudaGetLastError();
            return fail(MLP_EUNSUPPORTED, "tensor-core cluster kernel: the device refused its cooperative cluster "
                                          "launch (%s)", cudaGetErrorString(e));
        }
        CK(e, "tensor-core cluster kernel");
        return MLP_OK;
    }
    // Plain path, one step at a time.
    const int64_t mbs = (minibatch <= 0 || minibatch >= n) ? n : minibatch;
    const double C = loss_scale(h->cfg.loss_mean, n);
    const size_t xb = x_elem_bytes(h->cfg.prec) * (size_t)D;
    for (int e = 0; e < epochs; ++e) {
        int first = 1;
        for (int64_t b0 = 0; b0 < n; b0 += mbs) {
            const int64_t m = (n - b0) < mbs ? (n - b0) : mbs;
            mlp_status s = plain_grad(h, (const char *)X + xb * b0, (const char *)y + h->esz * b0, m, gW1p(h),
                                      gb1p(h), gw2p(h), gb2p(h), h->dtmp + 64, C, st);
            if (s) return s;
            if (gnorm_hist && b0 + mbs >= n)
                CK(mlp::plain_gnorm(h->cfg.prec, h->P, h->grads, h->dtmp, gnorm_hist + e, st), "gnorm");
            CK(mlp::plain_update(h->cfg.prec, D, H, (double)h->cfg.lr, W1p(h), b1p(h), w2p(h), b2p(h), gW1p(h),
                                 gb1p(h), gw2p(h), gb2p(h), st),
               "update");
            if (loss_hist) CK(mlp::plain_accum(loss_hist + e, h->dtmp + 64, first, st), "loss");
            first = 0;
        }
    }
    return MLP_OK;
}

mlp_status mlp_train_path(mlp_t h, int64_t n, int64_t minibatch, int32_t *path) {
    if (check_handle(h)) return MLP_EINVAL;
    if (!path || n < 0) return fail(MLP_EINVAL, "mlp_train_path: bad arguments");
    (void)minibatch;   // every path takes any mini-batch size
    const int D = h->cfg.D, H = h->cfg.H;
    if (h->cfg.prec == MLP_FP32 && mlp::fused_supported(D, H)) *path = MLP_PATH_FUSED;
    else if (h->cfg.prec == MLP_BF16 && mlp::tc_cluster_supported(D, H)) *path = MLP_PATH_TC_CLUSTER;
    else *path = MLP_PATH_PLAIN;
    return MLP_OK;
}

mlp_status mlp_train_host(mlp_t h, const void *X_host, const void *y_host, int64_t n, int32_t epochs,
                          int64_t minibatch, double *loss_hist_host, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (n < 0 || epochs < 0 || (n > 0 && (!X_host || !y_host)))
        return fail(MLP_EINVAL, "mlp_train_host: bad arguments");
    DeviceScope ds(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (epochs == 1 && n > 0 && h->cfg.prec == MLP_FP32 && mlp::fused_supported(h->cfg.D, h->cfg.H)) {
        // One epoch of the fused kernel reads every row once: page-locked host
        // buffers are read where they are, through the device's mapping of them
        // (over NVLink-C2C on a Grace-Blackwell node), and the loss is written
        // straight back, instead of staging copies that only add their latency.
        // The plain path reads X once per tile of hidden units and the bf16 paths
        // load it by TMA from device memory: those always stage.
        const void *Xm = mapped_host(X_host), *ym = mapped_host(y_host);
        double *lm = loss_hist_host ? (double *)mapped_host(loss_hist_host) : nullptr;
        if (Xm && ym && (!loss_hist_host || lm)) {
            mlp_status s = mlp_train_epochs(h, Xm, ym, n, 1, minibatch, lm, nullptr, stream);
            if (s) return s;
            CK(cudaStreamSynchronize(st), "mlp_train_host sync");
            return MLP_OK;
        }
    }
    const size_t xb = x_elem_bytes(h->cfg.prec) * (size_t)h->cfg.D * (size_t)n;
    const size_t yb = h->esz * (size_t)n;
    mlp_status s = grow(&h->xstage, &h->xstage_cap, xb, "X staging");
    if (s) return s;
    s = grow(&h->ystage, &h->ystage_cap, yb, "y staging");
    if (s) return s;
    s = grow((void **)&h->lstage, &h->lstage_cap, sizeof(double) * (size_t)(epochs > 0 ? epochs : 1), "loss staging");
    if (s) return s;
    if (n > 0) {
        CK(cudaMemcpyAsync(h->xstage, X_host, xb, cudaMemcpyHostToDevice, st), "mlp_train_host copy X");
        CK(cudaMemcpyAsync(h->ystage, y_host, yb, cudaMemcpyHostToDevice, st), "mlp_train_host copy y");
    }
    s = mlp_train_epochs(h, h->xstage, h->ystage, n, epochs, minibatch, h->lstage, nullptr, stream);
    if (s) return s;
    if (loss_hist_host && epochs > 0)
        CK(cudaMemcpyAsync(loss_hist_host, h->lstage, sizeof(double) * epochs, cudaMemcpyDeviceToHost, st),
           "mlp_train_host copy loss");
    CK(cudaStreamSynchronize(st), "mlp_train_host sync");
    return MLP_OK;
}

mlp_status mlp_predict(mlp_t h, const void *X, int64_t n, int8_t *labels, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    if (n < 0 || (n > 0 && (!X || !labels))) return fail(MLP_EINVAL, "mlp_predict: bad arguments");
    if (n == 0) return MLP_OK;
    DeviceScope ds(h->device);
    mlp::PlainWork w;
    mlp_status s = ensure_plain(h, n, false, &w);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    CK(mlp::plain_forward(h->cfg.prec, h->cfg.act, h->cfg.D, h->cfg.H, n, X, W1p(h), b1p(h), w2p(h), b2p(h),
                          nullptr, h->obuf, nullptr, nullptr, 0.0, w, st),
       "mlp_predict forward");
    CK(mlp::plain_labels(h->cfg.prec, n, h->obuf, labels, st), "mlp_predict labels");
    return MLP_OK;
}

mlp_status mlp_check(mlp_t h, void *stream) {
    if (check_handle(h)) return MLP_EINVAL;
    DeviceScope ds(h->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream), "mlp_check sync");
    int st = 0;
    CK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "mlp_check read");
    CK(cudaMemset(h->status, 0, sizeof(int)), "mlp_check clear");
    if (st & mlp::ST_TIMEOUT) {
        // The failed launch left its barrier counters part-way: restart them.
        if (h->fs) {
            CK(cudaMemset(h->fs, 0, h->fs_cap), "mlp_check reset");
            h->ctr = mlp::FusedCounters();
        }
        return fail(MLP_ETIMEOUT, "a cross-block wait gave up");
    }
    if (st & mlp::ST_BADLAUNCH) return fail(MLP_ECUDA, "a kernel was launched without its cluster shape");
    if (st & mlp::ST_NONFINITE) return fail(MLP_ENONFINITE, "a loss was not finite");
    return MLP_OK;
}

mlp_status mlp_debug_skip_block(mlp_t h, int32_t skip_block) {
    if (check_handle(h)) return MLP_EINVAL;
    h->skip_block = skip_block < 0 ? -1 : skip_block;
    return MLP_OK;
}

mlp_status mlp_set_rows_per_block(mlp_t h, int32_t rows) {
    if (check_handle(h)) return MLP_EINVAL;
    if (rows < 1) return fail(MLP_EINVAL, "mlp_set_rows_per_block: rows must be >= 1");
    h->rows_per_block = rows;
    return MLP_OK;
}

mlp_status mlp_set_clusters(mlp_t h, int32_t clusters) {
    if (check_handle(h)) return MLP_EINVAL;
    if (clusters < 0) return fail(MLP_EINVAL, "mlp_set_clusters: clusters must be >= 0");
    h->max_clusters = clusters == 0 ? (1 << 30) : clusters;
    return MLP_OK;
}

mlp_status mlp_cluster_limit(int32_t H, int32_t *clusters) {
    if (!clusters || H < 256 || H > 2048 || H % 256 != 0)
        return fail(MLP_EINVAL, "mlp_cluster_limit: H must be a multiple of 256 in 256..2048");
    *clusters = mlp::tc_cluster_max_clusters(H);
    return MLP_OK;
}

mlp_status mlp_workspace_bytes(int32_t prec, int32_t D, int32_t H, int64_t n, uint64_t *bytes) {
    if (!bytes || D < 1 || H < 1 || n < 0 || prec < MLP_FP32 || prec > MLP_FP64)
        return fail(MLP_EINVAL, "mlp_workspace_bytes: bad arguments");
    *bytes = mlp::plain_workspace_bytes(prec, D, H, n, mlp::device_sm_count());
    return MLP_OK;
}

static mlp_status check_w(const char *fn, int32_t prec, int32_t act, int32_t D, int32_t H, int64_t n,
                          uint64_t ws_bytes, const void *ws) {
    if (prec != MLP_FP32 && prec != MLP_FP64) return fail(MLP_EINVAL, "%s: prec must be FP32 or FP64", fn);
    if (act != MLP_ACT_SIGMOID && act != MLP_ACT_TANH) return fail(MLP_EINVAL, "%s: bad act", fn);
    if (D < 1 || H < 1 || n < 0) return fail(MLP_EINVAL, "%s: bad shape", fn);
    uint64_t need = mlp::plain_workspace_bytes(prec, D, H, n, mlp::device_sm_count());
    if (n > 0 && (!ws || ws_bytes < need))
        return fail(MLP_EINVAL, "%s: workspace of %llu bytes needed", fn, (unsigned long long)need);
    if (((uintptr_t)ws & 255) != 0) return fail(MLP_EINVAL, "%s: workspace not 256-byte aligned", fn);
    return MLP_OK;
}

mlp_status mlp_forward_w(int32_t prec, int32_t act, int32_t D, int32_t H, int64_t n, const void *X,
                         const void *W1, const void *b1, const void *w2, const void *b2, void *hid, void *o,
                         void *workspace, uint64_t workspace_bytes, void *stream) {
    mlp_status s = check_w("mlp_forward_w", prec, act, D, H, n, workspace_bytes, workspace);
    if (s) return s;
    if (n > 0 && (!X || !W1 || !b1 || !w2 || !b2 || !o)) return fail(MLP_EINVAL, "mlp_forward_w: null pointer");
    if (n == 0) return MLP_OK;
    mlp::PlainWork w;
    mlp::plain_workspace_carve(workspace, prec, D, H, n, mlp::device_sm_count(), &w);
    CK(mlp::plain_forward(prec, act, D, H, n, X, W1, b1, w2, b2, hid, o, nullptr, nullptr, 0.0, w,
                          (cudaStream_t)stream),
       "mlp_forward_w");
    return MLP_OK;
}

mlp_status mlp_backward_w(int32_t prec, int32_t act, int32_t D, int32_t H, int64_t n, const void *X,
                          const void *W1, const void *w2, const void *hid, const void *o, const void *dLdo,
                          void *gW1, void *gb1, void *gw2, void *gb2, void *gX, void *workspace,
                          uint64_t workspace_bytes, void *stream) {
    mlp_status s = check_w("mlp_backward_w", prec, act, D, H, n, workspace_bytes, workspace);
    if (s) return s;
    if (!gW1 || !gb1 || !gw2 || !gb2 || (n > 0 && (!X || !W1 || !w2 || !hid || !o || !dLdo)))
        return fail(MLP_EINVAL, "mlp_backward_w: null pointer");
    mlp::PlainWork w;
    mlp::plain_workspace_carve(workspace, prec, D, H, n, mlp::device_sm_count(), &w);
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0) CK(mlp::plain_d2_upstream(prec, n, o, dLdo, w.d2, st), "mlp_backward_w d2");
    CK(mlp::plain_backward(prec, act, D, H, n, X, W1, w2, hid, gW1, gb1, gw2, gb2, gX, nullptr, 0.0, nullptr, w,
                           st),
       "mlp_backward_w");
    return MLP_OK;
}

}  // extern "C"

struct mlp_batch {
    int device;
    int prec, act, D, Hmax, n_nets;
    float lr;
    int loss_mean;
    void *mem;                 // one allocation: nets (or tensor-core descriptors and maps), order, status
    mlp::BatchNet *nets;
    void *tc_descs;
    int *order;
    int *status;
    int64_t max_tiles;         // BF16: the most 128-row tiles of any net
    // mlp_batch_create_host: device copies of every net's data, host layout
    void *owned = nullptr;
    char *xd = nullptr;
    float *yd = nullptr, *pd = nullptr;
    double *ld = nullptr;
    size_t x_bytes = 0, y_bytes = 0, p_bytes = 0;
    int max_epochs = 0;
    int shape = mlp::BATCH_SHAPE_U1;   // FP32 kernel shape (mlp_batch_set_shape)
    int64_t nmax = 0;                   // FP32: the most rows of any net
};

// BF16 plan: per-net TMA tensor maps and descriptors for the tcgen05 kernel.
static mlp_status batch_create_tc(int32_t act, int32_t D, const mlp_net_desc *nets, int32_t n_nets, float lr,
                                  int32_t loss_mean, mlp_batch_t *out) {
    std::vector<double> cost(n_nets);
    for (int t = 0; t < n_nets; ++t) {
        const mlp_net_desc &d = nets[t];
        if (!mlp::tc_supported(D, d.H))
            return fail(MLP_EINVAL, "mlp_batch_create: BF16 needs D %% 8 == 0, 8 <= D <= 56 and H in {128, 256} "
                                    "(net %d: D=%d H=%d)", t, D, d.H);
        if (d.n < 0 || !d.params || (d.n > 0 && (!d.X || !d.y)))
            return fail(MLP_EINVAL, "mlp_batch_create: net %d has a null buffer or n < 0", t);
        if (((uintptr_t)d.X & 15) != 0) return fail(MLP_EINVAL, "mlp_batch_create: net %d X not 16-byte aligned", t);
        if (!tc_fits_32bit(d.n, 1)) return fail(MLP_EINVAL, "mlp_batch_create: net %d has more than 2^31 - 128 rows", t);
        cost[t] = (double)d.n * d.H;
    }
    std::vector<int> order(n_nets);
    for (int t = 0; t < n_nets; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    mlp_batch_t b = new (std::nothrow) mlp_batch();
    if (!b) return fail(MLP_ENOMEM, "mlp_batch_create: host allocation");
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return fail(MLP_ECUDA, "mlp_batch_create: no device");
    }
    b->prec = MLP_BF16;
    b->act = act;
    b->D = D;
    b->Hmax = 256;
    b->n_nets = n_nets;
    b->lr = lr;
    b->loss_mean = loss_mean ? 1 : 0;
    b->nets = nullptr;
    b->max_tiles = 0;
    for (int t = 0; t < n_nets; ++t) b->max_tiles = std::max<int64_t>(b->max_tiles, (nets[t].n + 127) / 128);
    const size_t N1 = (size_t)(n_nets > 0 ? n_nets : 1);
    const size_t mb = (mlp::tc_tmap_bytes() + 127) & ~(size_t)127;
    const size_t db = mlp::tc_desc_bytes();   // the kernel reads them as an array: stride = sizeof
    const size_t maps = ((mb * N1) + 255) & ~(size_t)255;
    const size_t descs = ((db * N1) + 255) & ~(size_t)255;
    const size_t ords = ((sizeof(int) * N1) + 255) & ~(size_t)255;
    if (cudaMalloc(&b->mem, maps + descs + ords + 256) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(MLP_ENOMEM, "mlp_batch_create: device allocation");
    }
    char *base = (char *)b->mem;
    b->tc_descs = base + maps;
    b->order = (int *)(base + maps + descs);
    b->status = (int *)(base + maps + descs + ords);   // status, and 64 bytes on the net counter
    std::vector<unsigned char> hmaps(mb * N1, 0), hdescs(db * N1, 0);
    for (int t = 0; t < n_nets; ++t) {
        const mlp_net_desc &d = nets[t];
        cudaError_t e = mlp::tc_encode_map(hmaps.data() + mb * t, d.X, D, d.n);
        if (e != cudaSuccess) {
            cudaFree(b->mem);
            delete b;
            return fail(MLP_ECUDA, "mlp_batch_create: tensor map of net %d: %s", t, cudaGetErrorString(e));
        }
        mlp::tc_fill_desc(hdescs.data() + db * t, base + mb * t, d.y, d.params, d.loss_hist, d.gnorm_hist, d.n,
                          d.H);
    }
    cudaError_t e = cudaSuccess;
    if (n_nets > 0) {
        e = cudaMemcpy(base, hmaps.data(), mb * n_nets, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->tc_descs, hdescs.data(), db * n_nets, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->order, order.data(), sizeof(int) * n_nets, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(b->mem);
        delete b;
        return cuda_fail(e, "mlp_batch_create");
    }
    *out = b;
    return MLP_OK;
}

extern "C" {

mlp_status mlp_batch_create(int32_t prec, int32_t act, int32_t D, const mlp_net_desc *nets, int32_t n_nets,
                            float lr, int32_t loss_mean, mlp_batch_t *out) {
    if (!out) return fail(MLP_EINVAL, "mlp_batch_create: null out");
    *out = nullptr;
    if (prec != MLP_FP32 && prec != MLP_BF16) return fail(MLP_EUNSUPPORTED, "mlp_batch_create: FP32 or BF16 only");
    if (act != MLP_ACT_SIGMOID && act != MLP_ACT_TANH) return fail(MLP_EINVAL, "mlp_batch_create: bad act");
    if (n_nets < 0 || (n_nets > 0 && !nets)) return fail(MLP_EINVAL, "mlp_batch_create: bad net list");
    if (prec == MLP_BF16) return batch_create_tc(act, D, nets, n_nets, lr, loss_mean, out);
    if (D < 1 || D > mlp::batched_max_D()) return fail(MLP_EINVAL, "mlp_batch_create: D=%d out of 1..64", D);
    int Hmax = 1;
    int64_t nmax = 0;
    std::vector<mlp::BatchNet> host(n_nets);
    std::vector<double> cost(n_nets);
    for (int t = 0; t < n_nets; ++t) {
        const mlp_net_desc &d = nets[t];
        if (d.H < 1 || d.H > mlp::batched_max_H())
            return fail(MLP_EINVAL, "mlp_batch_create: net %d has H=%d out of 1..128", t, d.H);
        if (d.n < 0 || !d.params || (d.n > 0 && (!d.X || !d.y)))
            return fail(MLP_EINVAL, "mlp_batch_create: net %d has a null buffer or n < 0", t);
        Hmax = d.H > Hmax ? d.H : Hmax;
        nmax = d.n > nmax ? d.n : nmax;
        host[t] = {(const float *)d.X, d.y, d.params, d.loss_hist, d.gnorm_hist, d.n, d.H, 0};
        // lanes busy per row: a power-of-two segment up to 32, else 32 per 32 units
        int lanes = d.H <= 32 ? 4 : 32 * ((d.H + 31) / 32);
        while (d.H <= 32 && lanes < d.H) lanes <<= 1;
        cost[t] = (double)d.n * lanes;
    }
    std::vector<int> order(n_nets);
    for (int t = 0; t < n_nets; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    mlp_batch_t b = new (std::nothrow) mlp_batch();
    if (!b) return fail(MLP_ENOMEM, "mlp_batch_create: host allocation");
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return fail(MLP_ECUDA, "mlp_batch_create: no device");
    }
    b->prec = MLP_FP32;
    b->tc_descs = nullptr;
    b->act = act;
    b->D = D;
    b->Hmax = Hmax;
    b->nmax = nmax;
    b->n_nets = n_nets;
    b->lr = lr;
    b->loss_mean = loss_mean ? 1 : 0;
    const size_t nb = ((sizeof(mlp::BatchNet) * (size_t)(n_nets > 0 ? n_nets : 1)) + 255) & ~(size_t)255;
    const size_t ob = ((sizeof(int) * (size_t)(n_nets > 0 ? n_nets : 1)) + 255) & ~(size_t)255;
    if (cudaMalloc(&b->mem, nb + ob + 256) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(MLP_ENOMEM, "mlp_batch_create: device allocation");
    }
    b->nets = (mlp::BatchNet *)b->mem;
    b->order = (int *)((char *)b->mem + nb);
    b->status = (int *)((char *)b->mem + nb + ob);
    cudaError_t e = cudaSuccess;
    if (n_nets > 0) {
        e = cudaMemcpy(b->nets, host.data(), sizeof(mlp::BatchNet) * n_nets, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->order, order.data(), sizeof(int) * n_nets, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(b->mem);
        delete b;
        return cuda_fail(e, "mlp_batch_create");
    }
    *out = b;
    return MLP_OK;
}

mlp_status mlp_batch_run(mlp_batch_t b, int32_t epochs, void *stream) {
    if (!b) return fail(MLP_EINVAL, "mlp_batch_run: null plan");
    if (epochs < 0) return fail(MLP_EINVAL, "mlp_batch_run: epochs < 0");
    DeviceScope ds(b->device);
    if (b->prec == MLP_BF16) {
        if ((int64_t)epochs * b->max_tiles > (int64_t)INT32_MAX)
            return fail(MLP_EINVAL, "mlp_batch_run: epochs x tiles of the largest net beyond 2^31; split the epochs");
        CK(mlp::tc_batched_train(b->tc_descs, b->order, b->n_nets, b->D, epochs, b->lr, b->loss_mean, b->act,
                                 b->status, b->status + 16, (cudaStream_t)stream),
           "tensor-core batched training kernel");
        return MLP_OK;
    }
    CK(mlp::batched_train(b->act, b->D, b->Hmax, b->nmax, b->nets, b->order, b->n_nets, epochs, b->lr,
                          b->loss_mean, b->status, b->shape, (cudaStream_t)stream),
       "batched training kernel");
    return MLP_OK;
}

mlp_status mlp_batch_set_shape(mlp_batch_t b, int32_t shape) {
    if (!b) return fail(MLP_EINVAL, "mlp_batch_set_shape: null plan");
    if (b->prec != MLP_FP32) return fail(MLP_EUNSUPPORTED, "mlp_batch_set_shape: FP32 plans only");
    if (!mlp::batched_shape_supported(b->D, shape))
        return fail(MLP_EINVAL, "mlp_batch_set_shape: shape %d does not take D = %d", shape, b->D);
    b->shape = shape;
    return MLP_OK;
}

mlp_status mlp_batch_get_shape(mlp_batch_t b, int32_t *shape) {
    if (!b || !shape) return fail(MLP_EINVAL, "mlp_batch_get_shape: null argument");
    *shape = b->prec == MLP_FP32 ? b->shape : -1;
    return MLP_OK;
}

mlp_status mlp_batch_check(mlp_batch_t b, void *stream) {
    if (!b) return fail(MLP_EINVAL, "mlp_batch_check: null plan");
    DeviceScope ds(b->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream), "mlp_batch_check sync");
    int st = 0;
    CK(cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost), "mlp_batch_check read");
    CK(cudaMemset(b->status, 0, sizeof(int)), "mlp_batch_check clear");
    if (st & mlp::ST_TIMEOUT) return fail(MLP_ETIMEOUT, "a wait inside the training kernel gave up");
    if (st & mlp::ST_NONFINITE) return fail(MLP_ENONFINITE, "a net's loss was not finite");
    return MLP_OK;
}

void mlp_batch_destroy(mlp_batch_t b) {
    if (!b) return;
    DeviceScope ds(b->device);
    cudaFree(b->mem);
    if (b->owned) cudaFree(b->owned);
    delete b;
}

mlp_status mlp_batch_create_host(int32_t prec, int32_t act, int32_t D, const int32_t *H, const int64_t *n,
                                 int32_t n_nets, int32_t max_epochs, float lr, int32_t loss_mean, mlp_batch_t *out) {
    if (!out) return fail(MLP_EINVAL, "mlp_batch_create_host: null out");
    *out = nullptr;
    if (prec != MLP_FP32 && prec != MLP_BF16) return fail(MLP_EUNSUPPORTED, "mlp_batch_create_host: FP32 or BF16 only");
    if (n_nets < 0 || (n_nets > 0 && (!H || !n)) || max_epochs < 0 || D < 1)
        return fail(MLP_EINVAL, "mlp_batch_create_host: bad arguments");
    const size_t xe = prec == MLP_BF16 ? 2 : 4;
    size_t rows = 0, params = 0;
    for (int t = 0; t < n_nets; ++t) {
        if (n[t] < 0 || H[t] < 1) return fail(MLP_EINVAL, "mlp_batch_create_host: net %d has n < 0 or H < 1", t);
        rows += (size_t)n[t];
        params += (size_t)(D + 2) * H[t] + 1;
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t xb = rows * D * xe, yb = rows * sizeof(float), pb = params * sizeof(float);
    const size_t lb = (size_t)n_nets * max_epochs * sizeof(double);
    void *mem = nullptr;
    if (cudaMalloc(&mem, al(xb) + al(yb) + al(pb) + al(lb) + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(MLP_ENOMEM, "mlp_batch_create_host: cannot allocate the device copies");
    }
    char *xd = (char *)mem;
    float *yd = (float *)(xd + al(xb));
    float *pd = (float *)((char *)yd + al(yb));
    double *ld = (double *)((char *)pd + al(pb));
    std::vector<mlp_net_desc> descs(n_nets);
    size_t r0 = 0, p0 = 0;
    for (int t = 0; t < n_nets; ++t) {
        descs[t].H = H[t];
        descs[t].n = n[t];
        descs[t].X = xd + r0 * D * xe;
        descs[t].y = yd + r0;
        descs[t].params = pd + p0;
        descs[t].loss_hist = max_epochs > 0 ? ld + (size_t)t * max_epochs : nullptr;
        descs[t].gnorm_hist = nullptr;
        r0 += (size_t)n[t];
        p0 += (size_t)(D + 2) * H[t] + 1;
    }
    mlp_batch_t b = nullptr;
    mlp_status s = mlp_batch_create(prec, act, D, descs.data(), n_nets, lr, loss_mean, &b);
    if (s) {
        cudaFree(mem);
        return s;
    }
    b->owned = mem;
    b->xd = xd;
    b->yd = yd;
    b->pd = pd;
    b->ld = ld;
    b->x_bytes = xb;
    b->y_bytes = yb;
    b->p_bytes = pb;
    b->max_epochs = max_epochs;
    *out = b;
    return MLP_OK;
}

mlp_status mlp_batch_run_host(mlp_batch_t b, const void *X_host, const float *y_host, const float *params_in_host,
                              float *params_out_host, double *loss_hist_host, int32_t epochs, void *stream) {
    if (!b) return fail(MLP_EINVAL, "mlp_batch_run_host: null plan");
    if (!b->owned) return fail(MLP_EINVAL, "mlp_batch_run_host: the plan was not made by mlp_batch_create_host");
    if (epochs < 0 || epochs > b->max_epochs)
        return fail(MLP_EINVAL, "mlp_batch_run_host: epochs %d outside 0..%d", epochs, b->max_epochs);
    if ((b->x_bytes && !X_host) || (b->y_bytes && !y_host) || (b->p_bytes && (!params_in_host || !params_out_host)))
        return fail(MLP_EINVAL, "mlp_batch_run_host: null host buffer");
    DeviceScope ds(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (b->x_bytes) CK(cudaMemcpyAsync(b->xd, X_host, b->x_bytes, cudaMemcpyHostToDevice, st), "copy X in");
    if (b->y_bytes) CK(cudaMemcpyAsync(b->yd, y_host, b->y_bytes, cudaMemcpyHostToDevice, st), "copy y in");
    if (b->p_bytes) CK(cudaMemcpyAsync(b->pd, params_in_host, b->p_bytes, cudaMemcpyHostToDevice, st), "copy weights in");
    mlp_status s = mlp_batch_run(b, epochs, stream);
    if (s) return s;
    if (b->p_bytes)
        CK(cudaMemcpyAsync(params_out_host, b->pd, b->p_bytes, cudaMemcpyDeviceToHost, st), "copy weights out");
    if (loss_hist_host && epochs > 0 && b->n_nets > 0)
        CK(cudaMemcpy2DAsync(loss_hist_host, sizeof(double) * epochs, b->ld, sizeof(double) * b->max_epochs,
                             sizeof(double) * epochs, b->n_nets, cudaMemcpyDeviceToHost, st),
           "copy losses out");
    return mlp_batch_check(b, stream);
}

mlp_status mlp_batch_train(int32_t prec, int32_t act, int32_t D, const mlp_net_desc *nets, int32_t n_nets,
                           int32_t epochs, float lr, int32_t loss_mean, void *stream) {
    mlp_batch_t b = nullptr;
    mlp_status s = mlp_batch_create(prec, act, D, nets, n_nets, lr, loss_mean, &b);
    if (s) return s;
    s = mlp_batch_run(b, epochs, stream);
    if (s == MLP_OK) s = mlp_batch_check(b, stream);
    mlp_batch_destroy(b);
    return s;
}

}  // extern "C"
