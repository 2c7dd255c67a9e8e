/*
 * mlp_gb300.h -- C ABI of the GB300 (sm_103a) training library for the
 * one-hidden-layer feed-forward network of Ramroach et al., "CUDA optimized
 * Neural Network predicts blood glucose control from quantified joint mobility
 * and anthropometrics" (arXiv 1908.07847).
 *
 * The method (Sec. 2.2 and Eq. 1 of the paper):
 *   forward    z1 = X W1^T + b1,  h = f(z1),  z2 = h w2 + b2,  o = sigmoid(z2)
 *              with sigmoid(x) = 1 / (1 + e^-x) (Eq. 1) and f = sigmoid (or tanh,
 *              the other activation Sec. 2.2 names);
 *   error      the difference o - y between outputs and true values (Sec. 2.2);
 *              loss E = (c/2) sum_i (o_i - y_i)^2, c = 1/n (loss_mean = 1) or 1;
 *   backward   d2 = dE/do * o (1 - o),  d1 = (d2 w2^T) .* f'(h),
 *              gW1 = d1^T X, gb1 = sum_i d1, gw2 = h^T d2, gb2 = sum_i d2;
 *   update     gradient descent without momentum, w <- w - lr g (Sec. 2.2,
 *              lr = 0.1 in the paper);
 *   classify   label = 1 iff o >= 0.5 (Sec. 2.2: the test rows are classified).
 *
 * Layouts (Sec. 2.2: the input is one flat array of rows x columns, each
 * layer's weights one flat array of hidden x columns):
 *   X   n x D row-major; element type float (MLP_FP32), bfloat16 bits as
 *       uint16_t (MLP_BF16; padding columns must hold 0) or double (MLP_FP64).
 *   y   n labels, float (double for MLP_FP64), normally 0 or 1.
 *   W1  H x D row-major (neuron j's D incoming weights contiguous), b1 [H],
 *       w2 [H], b2 [1]; float for MLP_FP32 / MLP_BF16 (FP32 master weights),
 *       double for MLP_FP64.  Packed parameter vector order, where one is used:
 *       [W1, b1, w2, b2], (D + 2) H + 1 values.
 *   o   n outputs, float (double for MLP_FP64).
 *
 * Conventions for every call:
 *   - Pointers named *_host are host memory; every other data pointer is device
 *     memory on the current CUDA device.  The caller owns every buffer it
 *     passes; the library only borrows it for the duration of the call.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     asynchronous on that stream unless they read or write host memory; those
 *     synchronise the stream before returning.
 *   - Every call returns an mlp_status and never aborts the process.  On
 *     MLP_EINVAL nothing has been launched and no output has been written.  The
 *     message of the last failure on the calling thread is in mlp_last_error().
 *   - Kernels that wait on one another across thread blocks give up after about
 *     one second; they then record MLP_ETIMEOUT in the handle's device status,
 *     which mlp_check() returns.  Until mlp_check() has read it, further fused
 *     training launches on that handle return without doing anything.
 *     Non-finite losses record MLP_ENONFINITE.
 *   - n = 0 is valid: outputs of size n are untouched, gradients are zero,
 *     an update with zero gradients leaves the weights unchanged.
 */
#ifndef MLP_GB300_H
#define MLP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlp_net *mlp_t;

typedef enum {
    MLP_OK = 0,
    MLP_EINVAL = 1,       /* bad argument (null pointer, size, precision) */
    MLP_ENOMEM = 2,       /* device or host allocation failed */
    MLP_ECUDA = 3,        /* a CUDA runtime call failed */
    MLP_ETIMEOUT = 4,     /* a cross-block wait gave up (see mlp_check) */
    MLP_ENONFINITE = 5,   /* a loss became NaN or infinite (see mlp_check) */
    MLP_EUNSUPPORTED = 6  /* valid request that this build does not implement */
} mlp_status;

typedef enum { MLP_FP32 = 0, MLP_BF16 = 1, MLP_FP64 = 2 } mlp_precision;
typedef enum { MLP_ACT_SIGMOID = 0, MLP_ACT_TANH = 1 } mlp_activation;

/* Network shape and training constants (Sec. 2.2). */
typedef struct {
    int32_t D;         /* inputs per row, 1..4096 */
    int32_t H;         /* hidden units, 1..65536 */
    float lr;          /* learning rate (the paper uses 0.1) */
    int32_t loss_mean; /* 1: c = 1/n (mean squared error / 2); 0: c = 1 */
    int32_t prec;      /* mlp_precision of X and of the arithmetic */
    int32_t act;       /* mlp_activation of the hidden layer */
} mlp_config;

/* Create a network on the current device.  The handle owns its FP32 (FP64 for
 * MLP_FP64) master weights, initialised to zero, and its scratch buffers.
 * Returns MLP_EINVAL for an out-of-range field, MLP_ENOMEM if the weights
 * cannot be allocated. */
mlp_status mlp_create(const mlp_config *cfg, mlp_t *out);

/* Free the handle and everything it owns.  NULL is ignored. */
void mlp_destroy(mlp_t net);

/* Copy weights from / to host memory (W1 H x D row-major, b1 [H], w2 [H],
 * b2 [1]; float, or double for MLP_FP64).  Synchronous. */
mlp_status mlp_set_weights(mlp_t net, const void *W1_host, const void *b1_host,
                           const void *w2_host, const void *b2_host);
mlp_status mlp_get_weights(mlp_t net, void *W1_host, void *b1_host,
                           void *w2_host, void *b2_host);

/* Device address of the handle's packed weights [W1, b1, w2, b2] (valid until
 * mlp_destroy). */
mlp_status mlp_weights_device(mlp_t net, void **params_dev);

/* Forward pass (Sec. 2.2, Eq. 1) with the handle's weights: writes o [n]. */
mlp_status mlp_forward(mlp_t net, const void *X, int64_t n, void *o, void *stream);

/* Squared-error gradients at the handle's weights (Sec. 2.2 backpropagation):
 * writes gW1 [H x D], gb1 [H], gw2 [H], gb2 [1] (float; double for MLP_FP64)
 * and, if loss != NULL, the FP64 loss E on the device.  Does not update. */
mlp_status mlp_backward(mlp_t net, const void *X, const void *y, int64_t n,
                        void *gW1, void *gb1, void *gw2, void *gb2,
                        double *loss, void *stream);

/* Gradient-descent step w <- w - lr g with caller-supplied gradients
 * (Sec. 2.2, no momentum). */
mlp_status mlp_update(mlp_t net, const void *gW1, const void *gb1,
                      const void *gw2, const void *gb2, void *stream);

/* Exchange step of data-parallel training of one network across ranks.  The
 * gradient of a mini-batch (Sec. 2.2) is a sum over its rows, so ranks that
 * each hold a shard of the rows compute summed (loss_mean = 0) gradients and
 * every rank then adds all ranks' vectors in rank order:
 *   out[i] = scale * (((parts[0][i] + parts[1][i]) + parts[2][i]) + ...)
 * with parts an nparts x len row-major device array of floats (rank p's flat
 * gradient [gW1, gb1, gw2, gb2] at parts + p * len) and out a device array of
 * len floats (not overlapping parts); scale is 1/m for the mean loss over a
 * mini-batch of m rows, else 1.  If loss_parts (nparts device doubles: each
 * rank's summed shard loss) is given, *loss_acc (one device double) is
 * increased by loss_scale times their rank-order sum; loss_parts and loss_acc
 * are both given or both NULL.  Asynchronous on `stream`; the same inputs give
 * the same bits on every rank.  MLP_EINVAL for nparts < 1, len < 0 or missing
 * pointers. */
mlp_status mlp_grad_sum(const float *parts, const double *loss_parts,
                        int32_t nparts, int64_t len, float scale,
                        double loss_scale, float *out, double *loss_acc,
                        void *stream);

/* One training step by the plain path: separate forward, output, gradient,
 * reduction and update kernels with the hidden activations materialised in
 * device memory.  Same result as one full-batch epoch of mlp_train_epochs. */
mlp_status mlp_step_plain(mlp_t net, const void *X, const void *y, int64_t n,
                          double *loss, void *stream);

/* Train `epochs` epochs (Sec. 2.2, Fig. 2).  minibatch <= 0 or >= n is full-batch
 * gradient descent (one update per epoch); otherwise each epoch visits
 * contiguous slices of `minibatch` rows in order with one update per slice
 * (the last slice may be shorter; minibatch = 1 is online backpropagation).
 * loss_hist [epochs] (device, may be NULL) receives (C/2) sum_i (o_i - y_i)^2
 * with o_i taken when row i was visited (C = 1/n or 1), accumulated in FP64;
 * gnorm_hist [epochs] (device, may be NULL) the FP64 2-norm of the last
 * update's gradient.  Paths, by precision and shape:
 *   MLP_FP32, D <= 64, H <= 128: one fused cooperative kernel per call
 *     (forward, backward, cross-block reduction and update per step);
 *   MLP_BF16 (sigmoid or tanh), D % 8 == 0, 8 <= D <= 48, H a multiple of
 *     256 up to 2048: one tensor-core (tcgen05) kernel per call, blocks
 *     in clusters of H/256 that share z2 through distributed shared memory,
 *     bf16 operands (W1, h and the hidden deltas rounded to bf16, FP32
 *     accumulation and FP32 master weights); X must be 16-byte aligned,
 *     n < 2^31 - 127 and epochs x ceil(n / 128) < 2^31 (else MLP_EINVAL);
 *     the gradient norm, if asked for, is taken from the summed FP32 gradient
 *     in FP64 by a second small kernel; a device that refuses the cooperative
 *     cluster launch gives MLP_EUNSUPPORTED;
 *   everything else: the plain path, one step at a time (FP32 arithmetic on
 *     bf16 inputs for MLP_BF16).
 * The tensor-core kernel records MLP_ECUDA through mlp_check if it ever finds
 * itself launched without its cluster shape. */
mlp_status mlp_train_epochs(mlp_t net, const void *X, const void *y, int64_t n,
                            int32_t epochs, int64_t minibatch, double *loss_hist,
                            double *gnorm_hist, void *stream);

/* Which path mlp_train_epochs takes for this handle and these sizes, so that
 * a caller can tell a shape that leaves the fast kernels (the plain path runs
 * several kernels a step and is about 10x slower) before training:
 * MLP_PATH_FUSED (the fused FP32 kernel), MLP_PATH_TC_CLUSTER (the bf16
 * tensor-core cluster kernel) or MLP_PATH_PLAIN.  No device work. */
typedef enum { MLP_PATH_FUSED = 0, MLP_PATH_TC_CLUSTER = 1, MLP_PATH_PLAIN = 2 } mlp_path;
mlp_status mlp_train_path(mlp_t net, int64_t n, int64_t minibatch, int32_t *path);

/* mlp_train_epochs on host buffers: copies X and y to device staging memory
 * owned by the handle, trains, and copies the loss history back to
 * loss_hist_host (may be NULL).  Synchronous.  A one-epoch call that takes the
 * fused FP32 kernel (D <= 64, H <= 128), with all buffers page-locked
 * (cudaHostAlloc, pinned tensors), skips the staging: the kernel reads X and y
 * through the device's mapping of that memory and writes the loss there. */
mlp_status mlp_train_host(mlp_t net, const void *X_host, const void *y_host,
                          int64_t n, int32_t epochs, int64_t minibatch,
                          double *loss_hist_host, void *stream);

/* Classification (Sec. 2.2): labels[i] = 1 iff o_i >= 0.5, else 0. */
mlp_status mlp_predict(mlp_t net, const void *X, int64_t n, int8_t *labels, void *stream);

/* Synchronise `stream`, then return and clear the handle's device status:
 * MLP_OK, MLP_ETIMEOUT or MLP_ENONFINITE. */
mlp_status mlp_check(mlp_t net, void *stream);

/*
 * Handle-free forms on caller-owned weights, for automatic differentiation
 * frameworks.  prec is MLP_FP32 or MLP_FP64 (all of X, weights, hid, o, dLdo
 * and gradients are then float or double).  Both need a caller-owned device
 * workspace of at least mlp_workspace_bytes(prec, D, H, n) bytes (256-byte
 * aligned); it is scratch for the duration of the call only, so calls that
 * may overlap on the GPU need separate workspaces.
 *   mlp_forward_w: writes hid [n x H] (if not NULL) and o [n].
 *   mlp_backward_w: backpropagates an arbitrary upstream gradient dLdo [n]
 *     (Sec. 2.2 chain rule) using the saved hid [n x H] and o [n]; writes gW1,
 *     gb1, gw2, gb2 and, if gX != NULL, gX [n x D] = d1 W1.
 */
mlp_status mlp_workspace_bytes(int32_t prec, int32_t D, int32_t H, int64_t n, uint64_t *bytes);
mlp_status mlp_forward_w(int32_t prec, int32_t act, int32_t D, int32_t H, int64_t n,
                         const void *X, const void *W1, const void *b1,
                         const void *w2, const void *b2, void *hid, void *o,
                         void *workspace, uint64_t workspace_bytes, void *stream);
mlp_status mlp_backward_w(int32_t prec, int32_t act, int32_t D, int32_t H, int64_t n,
                          const void *X, const void *W1, const void *w2,
                          const void *hid, const void *o, const void *dLdo,
                          void *gW1, void *gb1, void *gw2, void *gb2, void *gX,
                          void *workspace, uint64_t workspace_bytes, void *stream);

/* Test hook for the failure path of cross-block waits: when skip_block >= 0,
 * that block of the next fused training launches returns before its first
 * barrier, so the other blocks give up after about one second and the launch
 * records MLP_ETIMEOUT (read it with mlp_check).  -1 restores normal runs. */
mlp_status mlp_debug_skip_block(mlp_t net, int32_t skip_block);

/* Rows per block of the fused training kernel (tuning knob, default 32).  When
 * a step's rows fit one block, the launch is a single block that sums and
 * updates on chip (no cross-block accumulator or barrier); the result follows
 * the same fixed-point rounding of the gradient as a multi-block launch. */
mlp_status mlp_set_rows_per_block(mlp_t net, int32_t rows);

/* Thread-block clusters of the bf16 wide-network kernel (MLP_PATH_TC_CLUSTER;
 * tuning knob, no counterpart in the paper).  Each mini-batch's 128-row tiles
 * are dealt round-robin to K clusters of H/256 blocks, and at the end of every
 * step the K clusters' gradient slices are summed in cluster order: more
 * clusters give each fewer tiles but add partial slices to the sum.
 * mlp_set_clusters caps K at `clusters` (>= 1; 0 restores the default, the
 * most clusters the device keeps resident at once, which is also the upper
 * limit; K never exceeds the tiles of a step).  Results for different K agree
 * within the bf16 bars but not bit for bit (the sum order follows K).
 * mlp_cluster_limit writes that device limit for hidden width H (a multiple of
 * 256, at most 2048) on the current device to *clusters (1 if the occupancy
 * query fails). */
mlp_status mlp_set_clusters(mlp_t net, int32_t clusters);
mlp_status mlp_cluster_limit(int32_t H, int32_t *clusters);

/*
 * Many independent networks trained in one launch (the paper trains its male
 * and female subsets as separate networks, Sec. 2.1; here any number, each with
 * its own H and n).  All nets share D, the activation, lr, the loss scaling and
 * full-batch gradient descent (Sec. 2.2).  Each descriptor names device memory:
 * X (n x D row-major, float), y (n floats), params (the net's packed weights
 * [W1 (H x D), b1, w2, b2], float, trained in place), loss_hist (epochs
 * doubles, may be NULL; receives the loss before each epoch's update) and
 * gnorm_hist (epochs doubles, may be NULL; receives the 2-norm of the gradient
 * each epoch's update applied, summed in FP64 in a fixed order: the convergence
 * check beside the loss).
 * Limits of this build: MLP_FP32 (FP32 X): D <= 64, H <= 128; n is unbounded
 * (rows beyond 256 are streamed from device memory each epoch).  MLP_BF16
 * (bf16 X, 16-byte aligned, padding columns zero; FP32 master weights,
 * tcgen05 tensor cores, one block per net): sigmoid or tanh, D % 8 == 0,
 * 8 <= D <= 56, H = 128 or 256, n < 2^31 - 127 per net, and in one
 * mlp_batch_run epochs x ceil(n / 128) < 2^31 for the largest net (MLP_EINVAL
 * otherwise).
 */
typedef struct {
    int32_t H;
    int64_t n;
    const void *X;
    const float *y;
    float *params;
    double *loss_hist;
    double *gnorm_hist;
} mlp_net_desc;

typedef struct mlp_batch *mlp_batch_t;

/* Validate the descriptors (read on the host), copy them to device memory
 * owned by the plan, ordered by cost, largest first.  The buffers they name
 * must stay valid while the plan is run. */
mlp_status mlp_batch_create(int32_t prec, int32_t act, int32_t D,
                            const mlp_net_desc *nets, int32_t n_nets, float lr,
                            int32_t loss_mean, mlp_batch_t *out);

/* Train every net of the plan for `epochs` epochs: one kernel launch, no
 * allocation and no host synchronisation, so it can be captured in a CUDA
 * graph.  Each loss_hist must hold `epochs` doubles.  A plan runs one launch
 * at a time: two launches of the same plan that overlap on the GPU train the
 * same weights and, for MLP_BF16 plans, share the counter through which the
 * plan's blocks take their nets (a small memset before the kernel, on
 * `stream`, zeroes it). */
mlp_status mlp_batch_run(mlp_batch_t b, int32_t epochs, void *stream);

/* Synchronise `stream`, then return and clear the plan's device status
 * (MLP_OK or MLP_ENONFINITE). */
mlp_status mlp_batch_check(mlp_batch_t b, void *stream);

/* Kernel shape of an FP32 plan's launches, a tuning knob (autotune.py times
 * the shapes a plan allows and keeps the fastest).  Every shape runs the same
 * method and meets the same FP32 bars against the oracle; a given shape is
 * bitwise reproducible, two shapes differ by the order of their FP32 sums.
 *   0  one hidden unit a lane, blocks of 8 warps, two per SM (any D <= 64);
 *   1  two hidden units a lane (each row word read from shared memory feeds
 *      two multiply-adds), blocks of 4 warps, two per SM, one row in flight
 *      per lane (D <= 36);
 *   2  as 1 with two rows in flight per lane (D = 33, the paper's markers);
 *   3  register-tiled products (each thread a 4 x 4 tile of the forward and
 *      of the weight gradient, all sums in registers), blocks of 4 warps,
 *      rows in chunks of up to 128 (D <= 36);
 *   4  as 3 with chunks of 64 rows (less shared memory, more blocks an SM);
 *   5  as 3 with chunks of 32 rows;
 *   6  as 1 at three blocks an SM (registers capped at 168 a thread; D = 33).
 * A new FP32 plan has shape 0.  set: MLP_EINVAL for a shape the plan's D
 * does not take, MLP_EUNSUPPORTED for a BF16 plan.  get: -1 for BF16 plans. */
mlp_status mlp_batch_set_shape(mlp_batch_t b, int32_t shape);
mlp_status mlp_batch_get_shape(mlp_batch_t b, int32_t *shape);

/* Free the plan (not the buffers its descriptors name).  NULL is ignored. */
void mlp_batch_destroy(mlp_batch_t b);

/* mlp_batch_create + mlp_batch_run + mlp_batch_check + mlp_batch_destroy.
 * Synchronous. */
mlp_status mlp_batch_train(int32_t prec, int32_t act, int32_t D,
                           const mlp_net_desc *nets, int32_t n_nets,
                           int32_t epochs, float lr, int32_t loss_mean,
                           void *stream);

/*
 * Many-nets training on host buffers: the end-to-end form of mlp_batch_run,
 * for callers whose data live in host memory.  mlp_batch_create_host makes a
 * plan that owns device memory for every net's rows, labels, weights and
 * histories, laid out as on the host: all nets' rows one net after another
 * (net t's n[t] x D rows follow net t-1's), their labels likewise, the packed
 * weights [W1, b1, w2, b2] of (D + 2) H[t] + 1 floats one net after another,
 * and n_nets x max_epochs doubles of loss history.  H and n are host arrays of
 * n_nets entries; the limits are mlp_batch_create's.  Every
 * mlp_batch_run_host call then copies X_host (float for MLP_FP32, bfloat16
 * bits for MLP_BF16), y_host and params_in_host to the device, trains
 * `epochs` (<= max_epochs) epochs in one launch, and copies the trained
 * weights to params_out_host (may equal params_in_host) and, if
 * loss_hist_host is not NULL, the losses to it as n_nets x epochs doubles.
 * Synchronous; returns the plan's status as mlp_batch_check does.  Page-locked
 * host buffers make the copies asynchronous DMA; pageable ones work, slower.
 * mlp_batch_run_host on a plan from mlp_batch_create returns MLP_EINVAL.
 */
mlp_status mlp_batch_create_host(int32_t prec, int32_t act, int32_t D,
                                 const int32_t *H, const int64_t *n,
                                 int32_t n_nets, int32_t max_epochs, float lr,
                                 int32_t loss_mean, mlp_batch_t *out);
mlp_status mlp_batch_run_host(mlp_batch_t b, const void *X_host,
                              const float *y_host, const float *params_in_host,
                              float *params_out_host, double *loss_hist_host,
                              int32_t epochs, void *stream);

/*
 * Fused training (as mlp_train_epochs, without the gradient norm) on
 * caller-owned weights, allocating no device memory.  It is for callers that
 * cannot call cudaMalloc: a framework that hands out every byte of device
 * memory from its own pool (an allocation beside the pool fails or fragments
 * it), or a real-time loop that must not block on the allocator, whose
 * cudaMalloc and cudaFree synchronise the device.  The paper has no
 * counterpart; it is a property of this library's interface.
 *
 * The kernel's scratch (fixed-point gradient accumulators, a barrier counter
 * and a status word) lives in one statically sized device array of 203,520
 * bytes that every GPU which loads this library holds until the process exits.
 * Hence the limits D <= 64 and H <= 128; larger networks are rejected with
 * MLP_EINVAL.  Every call uses that one array and clears it on `stream` before
 * its kernel runs, so calls that overlap on the GPU (from two streams or two
 * threads) race with each other and must be ordered by the caller.  Every
 * call looks up the array's device address with the device current (no
 * allocation; the address can change after cudaDeviceReset).  The first call
 * on a device, and the first call with each new combination of activation,
 * input-width class (D up to 8, 16, 36, 48, 64) and hidden-width class (H up
 * to 32, 64, 128), may load that kernel's device code and set its
 * shared-memory attribute; make those first calls before any stream capture.
 *
 * X (n x D), y (n), params (packed [W1, b1, w2, b2], 16-byte aligned, trained
 * in place) and loss_hist (epochs doubles, may be NULL) are device memory.
 * status_out (device int32, may be NULL) receives 0, or the bit 1 if a
 * cross-block wait gave up, or the bit 2 if the loss was not finite.
 */
mlp_status mlp_train_fused_noalloc(int32_t act, int32_t D, int32_t H, int64_t n,
                                   const float *X, const float *y, float *params,
                                   float lr, int32_t loss_mean, int32_t epochs,
                                   int64_t minibatch, double *loss_hist,
                                   int32_t *status_out, void *stream);

/* Z-score normalisation of the feature table (Sec. 2.2 normalises the data
 * before training; the reading: per-column mean and population standard
 * deviation of the first n_fit rows, the training rows, applied to all n rows;
 * a column with zero deviation maps to 0), fused with the conversion to the
 * layout the training calls read.
 *   X      n x D float, row-major (device); must not overlap Y.
 *   Y      n x D_out (D_out >= D) of out_prec: MLP_FP32 (float) or MLP_BF16
 *          (bfloat16 bits, round to nearest even); columns D..D_out-1 are 0,
 *          so a bf16 output with D_out = 48 is the padded input of the
 *          tensor-core paths.
 *   mean, sdev  D doubles each (device): the statistics used.
 *   workspace   device scratch of at least mlp_zscore_workspace_bytes(D).
 * The statistics are FP64 sums in a fixed order (bitwise reproducible); the
 * normalisation is FP32, ((x - m_hi) - m_lo) * (1/s) with the mean split
 * into two floats.  n = 0 does nothing.  MLP_EINVAL: a NULL pointer, D < 1,
 * D_out < D, n_fit outside 1..n, a bad precision or a short workspace;
 * MLP_EUNSUPPORTED: D > 4096.  Asynchronous on `stream`. */
mlp_status mlp_zscore_workspace_bytes(int32_t D, uint64_t *bytes);
mlp_status mlp_zscore(const float *X, int64_t n, int32_t D, int64_t n_fit,
                      int32_t out_prec, int32_t D_out, void *Y, double *mean,
                      double *sdev, void *workspace, uint64_t workspace_bytes,
                      void *stream);

/* Diagnostic, not part of the method: measured rates of the FP32 FMA pipe and
 * of the special-function unit for tanh.approx.f32 and ex2.approx.f32, in
 * instructions per second over the whole current device (CUDA-event timed
 * register-only kernels, about 10 ms).  The benchmark states its ALU and SFU
 * roofline peaks from these.  MLP_EINVAL for a NULL pointer, MLP_ENOMEM /
 * MLP_ECUDA if the 4 x SMs x 512-word buffer or a launch fails. */
mlp_status mlp_unit_rates(double *ffma_per_s, double *tanh_per_s, double *ex2_per_s);

/* Message of the last failure on the calling thread ("" if none). */
const char *mlp_last_error(void);

/* Library version string. */
const char *mlp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLP_GB300_H */
