/*
 * FP64 CPU oracle for the one-hidden-layer feed-forward network trained by
 * backpropagation and gradient descent (Ramroach, Dhanoo, Cockburn, Joshi,
 * "CUDA optimized Neural Network predicts blood glucose control from
 * quantified joint mobility and anthropometrics", arXiv 1908.07847).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, serial reference
 * that the CUDA path is checked against.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.  It shares no code, header or constant with the CUDA library.
 *
 * What the paper fixes and what this file reads into it:
 *   - Sec. 2.2: a multi-layer perceptron, every neuron of a layer connected to
 *     every neuron of the adjacent layers, one hidden layer (Abstract), trained
 *     by gradient descent through backpropagation.
 *   - Eq. 1: the logistic sigmoid 1 / (1 + e^-x).  Used on the hidden units and
 *     (reading: the paper calls the sigmoid suitable for classification and the
 *     task is binary) on the single output unit.  tanh, named in Sec. 2.2 as
 *     the other traditional activation, is available for the hidden units.
 *   - Sec. 2.2: learning rate 0.1, no momentum: w <- w - lr * g.
 *   - Sec. 2.2 / Fig. 2: after each feed-forward pass the difference between
 *     outputs and true values drives the backpropagation step.  Reading: the
 *     loss is the squared error E = (c/2) * sum_i (o_i - y_i)^2 with c = 1/n
 *     (mean, default) or c = 1 (sum); the output error is o - y.
 *   - Sec. 2.2: the input is one flat float array of rows x columns (row-major
 *     X[i*D + k]); each layer's weights are one flat array of
 *     hidden x columns (W1[j*D + k]: neuron j's incoming weights contiguous).
 *   - Reading: biases b1 (per hidden unit) and b2 (output) are present.
 *   - Reading: full-batch gradient descent (one update per pass over all
 *     training rows); a mini-batch of m contiguous rows is the same step on
 *     each slice in order (m = 1 is online backpropagation).
 *   - Sec. 2.2: after training, test rows are classified; reading: class 1
 *     iff o >= 0.5.
 *
 * Samples are visited in increasing index and every sum is accumulated in
 * that order, in double precision, with no blocking or reordering.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ACT_SIGMOID 0
#define ORC_ACT_TANH 1

/* Eq. 1: sigmoid(x) = 1 / (1 + e^-x). */
double orc_sigmoid(double x)
{
    return 1.0 / (1.0 + exp(-x));
}

/* Hidden-unit activation (Sec. 2.2: logistic sigmoid or hyperbolic tangent). */
static double orc_hidden_act(int act, double z)
{
    if (act == ORC_ACT_TANH)
        return tanh(z);
    return orc_sigmoid(z);
}

/* Derivative of the hidden activation written through its value v = f(z):
 * sigmoid' = v (1 - v), tanh' = 1 - v^2. */
static double orc_hidden_act_deriv(int act, double v)
{
    if (act == ORC_ACT_TANH)
        return 1.0 - v * v;
    return v * (1.0 - v);
}

/*
 * Feed-forward pass for one sample (Sec. 2.2): every hidden neuron j takes the
 * weighted sum of all inputs plus its bias and applies the activation; the
 * output neuron takes the weighted sum of all hidden outputs plus its bias and
 * applies the sigmoid (Eq. 1).  h receives the H hidden outputs; returns o.
 */
static double orc_forward_one(int D, int H, const double *x, const double *W1,
                              const double *b1, const double *w2, double b2,
                              int act, double *h)
{
    double z2 = b2;
    for (int j = 0; j < H; ++j) {
        double z1 = b1[j];
        for (int k = 0; k < D; ++k)
            z1 += x[k] * W1[(long)j * D + k];
        h[j] = orc_hidden_act(act, z1);
        z2 += h[j] * w2[j];
    }
    return orc_sigmoid(z2);
}

/*
 * Forward pass over n samples (Sec. 2.2, Eq. 1).  X is n x D row-major,
 * W1 is H x D row-major.  hid (n x H, may be NULL) receives the hidden
 * outputs, o (n) the network outputs.
 */
void orc_forward(int D, int H, long n, const double *X, const double *W1,
                 const double *b1, const double *w2, double b2, int act,
                 double *hid, double *o)
{
    double *h = (double *)malloc(sizeof(double) * (size_t)(H > 0 ? H : 1));
    for (long i = 0; i < n; ++i) {
        o[i] = orc_forward_one(D, H, X + i * D, W1, b1, w2, b2, act, h);
        if (hid)
            for (int j = 0; j < H; ++j)
                hid[i * H + j] = h[j];
    }
    free(h);
}

/*
 * Backpropagation (Sec. 2.2) for an arbitrary upstream gradient dLdo[i] of a
 * scalar loss with respect to each output o_i.  Chain rule through the
 * network, sample by sample in increasing i:
 *   output delta   d2_i    = dLdo_i * o_i (1 - o_i)            (sigmoid output)
 *   hidden delta   d1_ij   = d2_i * w2_j * f'(h_ij)
 *   gw2_j  = sum_i d2_i h_ij          gb2   = sum_i d2_i
 *   gW1_jk = sum_i d1_ij X_ik         gb1_j = sum_i d1_ij
 *   gX_ik  = sum_j d1_ij W1_jk        (only if gX != NULL)
 * All gradient outputs are overwritten.
 */
void orc_backward(int D, int H, long n, const double *X, const double *W1,
                  const double *b1, const double *w2, double b2, int act,
                  const double *dLdo, double *gW1, double *gb1, double *gw2,
                  double *gb2, double *gX)
{
    double *h = (double *)malloc(sizeof(double) * (size_t)(H > 0 ? H : 1));
    memset(gW1, 0, sizeof(double) * (size_t)H * (size_t)D);
    memset(gb1, 0, sizeof(double) * (size_t)H);
    memset(gw2, 0, sizeof(double) * (size_t)H);
    *gb2 = 0.0;
    if (gX)
        memset(gX, 0, sizeof(double) * (size_t)n * (size_t)D);
    for (long i = 0; i < n; ++i) {
        const double *x = X + i * D;
        double o = orc_forward_one(D, H, x, W1, b1, w2, b2, act, h);
        double d2 = dLdo[i] * o * (1.0 - o);
        *gb2 += d2;
        for (int j = 0; j < H; ++j) {
            gw2[j] += d2 * h[j];
            double d1 = d2 * w2[j] * orc_hidden_act_deriv(act, h[j]);
            gb1[j] += d1;
            for (int k = 0; k < D; ++k) {
                gW1[(long)j * D + k] += d1 * x[k];
                if (gX)
                    gX[i * D + k] += d1 * W1[(long)j * D + k];
            }
        }
    }
    free(h);
}

/*
 * Gradient of the squared-error loss E = (c/2) sum_i (o_i - y_i)^2 over n
 * samples (Sec. 2.2: the difference between outputs and true values drives
 * backpropagation), c = 1/n if loss_mean else 1 (c = 0 when n = 0).  The
 * upstream gradient is dE/do_i = c (o_i - y_i).  Writes the gradients and
 * returns the sum of squared errors sum_i (o_i - y_i)^2.
 */
double orc_mse_gradients(int D, int H, long n, const double *X, const double *y,
                         const double *W1, const double *b1, const double *w2,
                         double b2, int act, int loss_mean, double *gW1,
                         double *gb1, double *gw2, double *gb2)
{
    double c = loss_mean ? (n > 0 ? 1.0 / (double)n : 0.0) : 1.0;
    double *o = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dLdo = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_forward(D, H, n, X, W1, b1, w2, b2, act, NULL, o);
    double sse = 0.0;
    for (long i = 0; i < n; ++i) {
        double e = o[i] - y[i];
        sse += e * e;
        dLdo[i] = c * e;
    }
    orc_backward(D, H, n, X, W1, b1, w2, b2, act, dLdo, gW1, gb1, gw2, gb2, NULL);
    free(o);
    free(dLdo);
    return sse;
}

/* Gradient-descent update, no momentum (Sec. 2.2): w <- w - lr * g. */
void orc_update(int D, int H, double lr, double *W1, double *b1, double *w2,
                double *b2, const double *gW1, const double *gb1,
                const double *gw2, double gb2)
{
    for (long p = 0; p < (long)H * D; ++p)
        W1[p] -= lr * gW1[p];
    for (int j = 0; j < H; ++j) {
        b1[j] -= lr * gb1[j];
        w2[j] -= lr * gw2[j];
    }
    *b2 -= lr * gb2;
}

/* Euclidean norm of the full gradient vector (convergence check). */
static double orc_grad_norm(int D, int H, const double *gW1, const double *gb1,
                            const double *gw2, double gb2)
{
    double s = 0.0;
    for (long p = 0; p < (long)H * D; ++p)
        s += gW1[p] * gW1[p];
    for (int j = 0; j < H; ++j)
        s += gb1[j] * gb1[j] + gw2[j] * gw2[j];
    s += gb2 * gb2;
    return sqrt(s);
}

/*
 * Training loop (Sec. 2.2, Fig. 2): for each epoch, for each contiguous batch
 * of `minibatch` rows in order (the whole set when minibatch <= 0 or >= n):
 * feed forward, backpropagate the squared-error gradient, update with lr.
 * The weights are updated in place.
 *   loss_hist[e]  (may be NULL) = (C/2) sum_i (o_i - y_i)^2 with o_i taken when
 *                 row i was visited in epoch e (before that batch's update),
 *                 C = 1/n if loss_mean else 1.
 *   gnorm_hist[e] (may be NULL) = ||g||_2 of the last update of epoch e.
 */
void orc_train(int D, int H, long n, const double *X, const double *y,
               double *W1, double *b1, double *w2, double *b2, int act,
               int loss_mean, double lr, int epochs, long minibatch,
               double *loss_hist, double *gnorm_hist)
{
    long mb = (minibatch <= 0 || minibatch >= n) ? n : minibatch;
    double *gW1 = (double *)malloc(sizeof(double) * (size_t)((long)H * D + 1));
    double *gb1 = (double *)malloc(sizeof(double) * (size_t)(H + 1));
    double *gw2 = (double *)malloc(sizeof(double) * (size_t)(H + 1));
    double gb2 = 0.0;
    for (int e = 0; e < epochs; ++e) {
        double sse = 0.0, gn = 0.0;
        long start = 0;
        do {
            long m = n - start < mb ? n - start : mb;
            sse += orc_mse_gradients(D, H, m, X + start * D, y + start, W1, b1,
                                     w2, *b2, act, loss_mean, gW1, gb1, gw2,
                                     &gb2);
            gn = orc_grad_norm(D, H, gW1, gb1, gw2, gb2);
            orc_update(D, H, lr, W1, b1, w2, b2, gW1, gb1, gw2, gb2);
            start += m;
        } while (start < n);
        if (loss_hist)
            loss_hist[e] = 0.5 * sse * (loss_mean ? (n > 0 ? 1.0 / (double)n : 0.0) : 1.0);
        if (gnorm_hist)
            gnorm_hist[e] = gn;
    }
    free(gW1);
    free(gb1);
    free(gw2);
}

/* Classification of rows after training (Sec. 2.2): class 1 iff o >= 0.5. */
void orc_predict(int D, int H, long n, const double *X, const double *W1,
                 const double *b1, const double *w2, double b2, int act,
                 signed char *label)
{
    double *o = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_forward(D, H, n, X, W1, b1, w2, b2, act, NULL, o);
    for (long i = 0; i < n; ++i)
        label[i] = o[i] >= 0.5 ? 1 : 0;
    free(o);
}

/*
 * Many independent networks (the paper's separately trained male and female
 * subsets, Sec. 2.1, generalised to any number of nets).  Net t has D[t]
 * inputs, H[t] hidden units and n[t] rows; its rows start at X_all + x_off[t]
 * (n[t] x D[t]) and y_all + y_off[t]; its parameters are packed at
 * P_all + p_off[t] as [W1 (H x D), b1 (H), w2 (H), b2 (1)] and are trained in
 * place by orc_train.  loss_all[t * epochs + e] receives net t's loss history.
 * Nets are independent; `threads` > 1 spreads them over host cores.
 */
void orc_batch_train(int n_nets, const int *Ds, const int *Hs, const long *ns,
                     const double *X_all, const long *x_off, const double *y_all,
                     const long *y_off, double *P_all, const long *p_off,
                     int act, int loss_mean, double lr, int epochs,
                     long minibatch, double *loss_all, int threads)
{
    (void)threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
    for (int t = 0; t < n_nets; ++t) {
        int D = Ds[t], H = Hs[t];
        double *P = P_all + p_off[t];
        double *W1 = P, *b1 = P + (long)H * D, *w2 = b1 + H, *b2 = w2 + H;
        orc_train(D, H, ns[t], X_all + x_off[t], y_all + y_off[t], W1, b1, w2,
                  b2, act, loss_mean, lr, epochs, minibatch,
                  loss_all ? loss_all + (long)t * epochs : NULL, NULL);
    }
}

/*
 * Sec. 2.2: the data are normalised before training (the paper does not say
 * how).  Reading: z-score per column with statistics of the training rows
 * only (the first n_fit rows): mean_j = (1/n_fit) sum_i X[i][j], the
 * population deviation s_j = sqrt((1/n_fit) sum_i (X[i][j] - mean_j)^2), and
 * Y[i][j] = (X[i][j] - mean_j) / s_j for every row i < n, or 0 where s_j = 0
 * (a constant column carries no information).  Sums in increasing row order.
 */
void orc_zscore(long n, int D, long n_fit, const double *X, double *mean, double *sdev, double *Y)
{
    for (int j = 0; j < D; ++j) {
        double s = 0.0;
        for (long i = 0; i < n_fit; ++i) s += X[i * D + j];
        const double m = s / (double)n_fit;
        double q = 0.0;
        for (long i = 0; i < n_fit; ++i) {
            const double d = X[i * D + j] - m;
            q += d * d;
        }
        const double sd = sqrt(q / (double)n_fit);
        mean[j] = m;
        sdev[j] = sd;
        for (long i = 0; i < n; ++i) Y[i * D + j] = sd > 0.0 ? (X[i * D + j] - m) / sd : 0.0;
    }
}
