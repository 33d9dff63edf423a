/*
 * mlp.c -- the learned leaf decoder (a project extension; the paper only
 * cites NeuralVDB as related work in Section 2.3, where inference is too slow
 * for real time).  The paper prints nothing for it to be compared with, so
 * it is pinned to calculus instead (finite differences, closed-form networks,
 * Adam's steps in closed form).
 *
 * Network (shared by all leaves): input x = (u, v, w, z_0 .. z_15), with
 * (u, v, w) = the voxel's position in its 8^3 leaf divided by 7 and z the
 * leaf's latent; h1 = relu(W1 x + b1) (32), h2 = relu(W2 h1 + b2) (32),
 * y = w3 . h2 + b3.  y predicts the leaf's normalized value
 * (v - offset) / scale; the decoded value is offset + scale * y.
 * Parameters, in this order: W1 (32 x 19, row major), b1 (32), W2 (32 x 32),
 * b2 (32), w3 (32), b3 (1) -- 1729 values.  Loss: mean squared error of y.
 * Optimizer: Adam (Kingma and Ba, 2015).
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define IN 19
#define HID 32
#define NPAR (HID * IN + HID + HID * HID + HID + HID + 1)

int or_mlp_num_params(void) { return NPAR; }

static void forward_one(const double* p, const double* x, double h1[HID], double h2[HID], double* y)
{
    const double* W1 = p;
    const double* b1 = W1 + HID * IN;
    const double* W2 = b1 + HID;
    const double* b2 = W2 + HID * HID;
    const double* w3 = b2 + HID;
    const double* b3 = w3 + HID;
    for (int i = 0; i < HID; ++i) {
        double a = b1[i];
        for (int k = 0; k < IN; ++k) a += W1[i * IN + k] * x[k];
        h1[i] = a > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < HID; ++i) {
        double a = b2[i];
        for (int k = 0; k < HID; ++k) a += W2[i * HID + k] * h1[k];
        h2[i] = a > 0.0 ? a : 0.0;
    }
    double o = b3[0];
    for (int k = 0; k < HID; ++k) o += w3[k] * h2[k];
    *y = o;
}

void or_mlp_forward(const double* params, const double* inputs, int64_t n, double* out)
{
    double h1[HID], h2[HID];
    for (int64_t s = 0; s < n; ++s) forward_one(params, inputs + s * IN, h1, h2, out + s);
}

/* loss = mean over the n samples of (y - target)^2; gradients of the loss
 * with respect to every parameter and every input (the latent gradients are
 * the input gradients' last 16 columns) */
double or_mlp_loss_grad(const double* params, const double* inputs, const double* targets, int64_t n,
                        double* grad_params, double* grad_inputs)
{
    const double* W1 = params;
    const double* W2 = W1 + HID * IN + HID;
    const double* w3 = W2 + HID * HID + HID;
    double* gW1 = grad_params;
    double* gb1 = gW1 + HID * IN;
    double* gW2 = gb1 + HID;
    double* gb2 = gW2 + HID * HID;
    double* gw3 = gb2 + HID;
    double* gb3 = gw3 + HID;
    memset(grad_params, 0, sizeof(double) * NPAR);
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        const double* x = inputs + s * IN;
        double h1[HID], h2[HID], y;
        forward_one(params, x, h1, h2, &y);
        double e = y - targets[s];
        loss += e * e;
        double dy = 2.0 * e / (double)n;
        double dh2[HID], dh1[HID];
        gb3[0] += dy;
        for (int k = 0; k < HID; ++k) {
            gw3[k] += dy * h2[k];
            dh2[k] = h2[k] > 0.0 ? dy * w3[k] : 0.0;      /* relu' (0 at 0) */
        }
        for (int i = 0; i < HID; ++i) {
            gb2[i] += dh2[i];
            for (int k = 0; k < HID; ++k) gW2[i * HID + k] += dh2[i] * h1[k];
        }
        for (int k = 0; k < HID; ++k) {
            double a = 0.0;
            for (int i = 0; i < HID; ++i) a += W2[i * HID + k] * dh2[i];
            dh1[k] = h1[k] > 0.0 ? a : 0.0;
        }
        for (int i = 0; i < HID; ++i) {
            gb1[i] += dh1[i];
            for (int k = 0; k < IN; ++k) gW1[i * IN + k] += dh1[i] * x[k];
        }
        if (grad_inputs) {
            for (int k = 0; k < IN; ++k) {
                double a = 0.0;
                for (int i = 0; i < HID; ++i) a += W1[i * IN + k] * dh1[i];
                grad_inputs[s * IN + k] = a;
            }
        }
    }
    return loss / (double)n;
}

/* one Adam step (bias-corrected moments; `step` counts from 1) */
void or_adam_step(double* params, const double* grads, double* m, double* v, int64_t n, int64_t step,
                  double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grads[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grads[i] * grads[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        params[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* The precision of the GPU's tensor-core evaluation, written out: inputs,
 * weights and the two hidden activations rounded to bfloat16 (round to
 * nearest even, the minifloat routine of encode.c with 8 exponent and 7
 * fraction bits), sums and biases exact (FP64 here, FP32 accumulation on the
 * GPU), output y in full precision. */
float or_round_bf16(float x) { return or_round_minifloat(x, 8, 7, 127, 0); }

static double bf(double x) { return (double)or_round_bf16((float)x); }

void or_mlp_forward_bf16(const double* params, const double* inputs, int64_t n, double* out)
{
    const double* W1 = params;
    const double* b1 = W1 + HID * IN;
    const double* W2 = b1 + HID;
    const double* b2 = W2 + HID * HID;
    const double* w3 = b2 + HID;
    const double* b3 = w3 + HID;
    for (int64_t s = 0; s < n; ++s) {
        const double* x = inputs + s * IN;
        double h1[HID], h2[HID];
        for (int i = 0; i < HID; ++i) {
            double a = 0.0;
            for (int k = 0; k < IN; ++k) a += bf(W1[i * IN + k]) * bf(x[k]);
            a = (double)(float)a + (double)(float)b1[i];
            h1[i] = bf(a > 0.0 ? a : 0.0);
        }
        for (int i = 0; i < HID; ++i) {
            double a = 0.0;
            for (int k = 0; k < HID; ++k) a += bf(W2[i * HID + k]) * h1[k];
            a = (double)(float)a + (double)(float)b2[i];
            h2[i] = bf(a > 0.0 ? a : 0.0);
        }
        double o = 0.0;
        for (int k = 0; k < HID; ++k) o += bf(w3[k]) * h2[k];
        out[s] = (double)(float)o + (double)(float)b3[0];
    }
}

/* A neural leaf: the leaf's (scale, offset) are those of its FP16 payload
 * (range and minimum of the source values, or_quantize_leaf), its latent is
 * stored in bfloat16 (the precision the network reads it in, so one rounding
 * of the trained FP32 value), and voxel n = a + 8b + 64c decodes to
 * offset + scale * clamp(y, 0, 1) with y the network at (a/7, b/7, c/7, z)
 * evaluated in the tensor cores' precision (or_mlp_forward_bf16); the FP32
 * result is the rounding of that exact value. */
void or_learned_leaf(const double* params, const float latent[16], const float src[512], float out[512])
{
    float q[512], scale, offset;
    or_quantize_leaf(src, OR_FP16, q, &scale, &offset);
    double x[512 * IN], y[512];
    for (int n = 0; n < 512; ++n) {
        x[n * IN + 0] = (double)(float)((double)(n & 7) / 7.0);
        x[n * IN + 1] = (double)(float)((double)((n >> 3) & 7) / 7.0);
        x[n * IN + 2] = (double)(float)((double)(n >> 6) / 7.0);
        for (int c = 0; c < 16; ++c) x[n * IN + 3 + c] = (double)latent[c];   /* rounded to bf16 in the forward */
    }
    or_mlp_forward_bf16(params, x, 512, y);
    for (int n = 0; n < 512; ++n) {
        double yc = y[n] < 0.0 ? 0.0 : (y[n] > 1.0 ? 1.0 : y[n]);
        out[n] = (float)((double)offset + (double)scale * yc);
    }
}

/* The training gradient at the tensor cores' precision: the loss of the bf16
 * forward above (inputs, weights and hidden activations rounded to bf16, w3
 * and h2 rounded to bf16 in the output sum), differentiated with the backward
 * operands that feed a multiply also rounded to bf16: dh2 = relu'(a2) dy
 * bf(w3) and dh1 = relu'(a1) (bf(W2)^T bf(dh2)); weight gradients
 * gW2 = sum bf(dh2) bf(h1)^T, gW1 = sum bf(dh1) bf(x)^T, gw3 = sum dy bf(h2);
 * bias gradients from the unrounded dh1, dh2, dy; input gradients
 * bf(W1)^T bf(dh1).  Sums exact (FP64); FP32 values rounded where the GPU
 * holds them in FP32 (pre-activations, dy, dh2, dh1). */
double or_mlp_loss_grad_bf16(const double* params, const double* inputs, const double* targets, int64_t n,
                             double* grad_params, double* grad_inputs)
{
    const double* W1 = params;
    const double* b1 = W1 + HID * IN;
    const double* W2 = b1 + HID;
    const double* b2 = W2 + HID * HID;
    const double* w3 = b2 + HID;
    const double* b3 = w3 + HID;
    double* gW1 = grad_params;
    double* gb1 = gW1 + HID * IN;
    double* gW2 = gb1 + HID;
    double* gb2 = gW2 + HID * HID;
    double* gw3 = gb2 + HID;
    double* gb3 = gw3 + HID;
    memset(grad_params, 0, sizeof(double) * NPAR);
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        const double* x = inputs + s * IN;
        double xb[IN], a1[HID], h1b[HID], a2[HID], h2b[HID];
        for (int k = 0; k < IN; ++k) xb[k] = bf(x[k]);
        for (int i = 0; i < HID; ++i) {
            double a = 0.0;
            for (int k = 0; k < IN; ++k) a += bf(W1[i * IN + k]) * xb[k];
            a1[i] = (double)(float)((double)(float)a + (double)(float)b1[i]);
            h1b[i] = bf(a1[i] > 0.0 ? a1[i] : 0.0);
        }
        for (int i = 0; i < HID; ++i) {
            double a = 0.0;
            for (int k = 0; k < HID; ++k) a += bf(W2[i * HID + k]) * h1b[k];
            a2[i] = (double)(float)((double)(float)a + (double)(float)b2[i]);
            h2b[i] = bf(a2[i] > 0.0 ? a2[i] : 0.0);
        }
        double o = 0.0;
        for (int k = 0; k < HID; ++k) o += bf(w3[k]) * h2b[k];
        double y = (double)(float)((double)(float)o + (double)(float)b3[0]);
        double e = y - targets[s];
        loss += e * e;
        double dy = (double)(float)(2.0 * e / (double)n);
        double dh2[HID], dh1[HID];
        gb3[0] += dy;
        for (int k = 0; k < HID; ++k) {
            gw3[k] += dy * h2b[k];
            dh2[k] = a2[k] > 0.0 ? (double)(float)(dy * bf(w3[k])) : 0.0;
        }
        for (int i = 0; i < HID; ++i) {
            gb2[i] += dh2[i];
            for (int k = 0; k < HID; ++k) gW2[i * HID + k] += bf(dh2[i]) * h1b[k];
        }
        for (int k = 0; k < HID; ++k) {
            double a = 0.0;
            for (int i = 0; i < HID; ++i) a += bf(W2[i * HID + k]) * bf(dh2[i]);
            dh1[k] = a1[k] > 0.0 ? (double)(float)a : 0.0;
        }
        for (int i = 0; i < HID; ++i) {
            gb1[i] += dh1[i];
            for (int k = 0; k < IN; ++k) gW1[i * IN + k] += bf(dh1[i]) * xb[k];
        }
        if (grad_inputs) {
            for (int k = 0; k < IN; ++k) {
                double a = 0.0;
                for (int i = 0; i < HID; ++i) a += bf(W1[i * IN + k]) * bf(dh1[i]);
                grad_inputs[s * IN + k] = a;
            }
        }
    }
    return loss / (double)n;
}
