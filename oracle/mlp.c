/*
 * mlp.c -- FP64 reference of the small network that can stand in for the
 * QED tables (test infrastructure: the reference the GPU network's
 * gradients are checked against).  Architecture 2 -> 64 -> 64 -> 64 -> 2 with SiLU on the hidden
 * layers, parameters packed as
 *   W0[64][2] b0[64] W1[64][64] b1[64] W2[64][64] b2[64] W3[2][64] b3[2]
 * Loss: L = (1/n) sum_i sum_o (y_io - t_io)^2.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

#define H 64
#define NI 2
#define NO 2

static const long OFF_W0 = 0, OFF_B0 = H * NI, OFF_W1 = H * NI + H, OFF_B1 = H * NI + H + H * H,
                  OFF_W2 = H * NI + 2 * H + H * H, OFF_B2 = H * NI + 2 * H + 2 * H * H,
                  OFF_W3 = H * NI + 3 * H + 2 * H * H, OFF_B3 = H * NI + 3 * H + 2 * H * H + NO * H;

long or_mlp_nparams(void) { return OFF_B3 + NO; }

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double dsilu(double z)
{
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* one sample: pre-activations z1..z3, activations a1..a3, outputs y */
static void fwd1(const double *P, const double *x, double *z, double *a, double *y)
{
    for (int j = 0; j < H; j++) {
        double s = P[OFF_B0 + j];
        for (int k = 0; k < NI; k++) s += P[OFF_W0 + j * NI + k] * x[k];
        z[j] = s;
        a[j] = silu(s);
    }
    const long W[2] = {OFF_W1, OFF_W2}, B[2] = {OFF_B1, OFF_B2};
    for (int l = 0; l < 2; l++) {
        for (int j = 0; j < H; j++) {
            double s = P[B[l] + j];
            for (int k = 0; k < H; k++) s += P[W[l] + j * H + k] * a[l * H + k];
            z[(l + 1) * H + j] = s;
            a[(l + 1) * H + j] = silu(s);
        }
    }
    for (int o = 0; o < NO; o++) {
        double s = P[OFF_B3 + o];
        for (int k = 0; k < H; k++) s += P[OFF_W3 + o * H + k] * a[2 * H + k];
        y[o] = s;
    }
}

void or_mlp_forward(const double *P, long n, const double *in, double *out)
{
    double z[3 * H], a[3 * H];
    for (long i = 0; i < n; i++) fwd1(P, &in[NI * i], z, a, &out[NO * i]);
}

/* loss and its gradient with respect to every parameter (backpropagation) */
double or_mlp_loss_grad(const double *P, long n, const double *in, const double *tgt, double *G)
{
    long np = or_mlp_nparams();
    memset(G, 0, (size_t)np * sizeof(double));
    double z[3 * H], a[3 * H], y[NO], dy[NO], d3[H], d2[H], d1[H];
    double loss = 0.0;
    for (long i = 0; i < n; i++) {
        const double *x = &in[NI * i];
        fwd1(P, x, z, a, y);
        for (int o = 0; o < NO; o++) {
            double e = y[o] - tgt[NO * i + o];
            loss += e * e / (double)n;
            dy[o] = 2.0 * e / (double)n;
        }
        /* output layer */
        for (int o = 0; o < NO; o++) {
            G[OFF_B3 + o] += dy[o];
            for (int k = 0; k < H; k++) G[OFF_W3 + o * H + k] += dy[o] * a[2 * H + k];
        }
        for (int k = 0; k < H; k++) {
            double s = 0.0;
            for (int o = 0; o < NO; o++) s += dy[o] * P[OFF_W3 + o * H + k];
            d3[k] = s * dsilu(z[2 * H + k]);
        }
        /* layer 2: z3 = W2 a2 + b2 */
        for (int j = 0; j < H; j++) {
            G[OFF_B2 + j] += d3[j];
            for (int k = 0; k < H; k++) G[OFF_W2 + j * H + k] += d3[j] * a[H + k];
        }
        for (int k = 0; k < H; k++) {
            double s = 0.0;
            for (int j = 0; j < H; j++) s += d3[j] * P[OFF_W2 + j * H + k];
            d2[k] = s * dsilu(z[H + k]);
        }
        /* layer 1: z2 = W1 a1 + b1 */
        for (int j = 0; j < H; j++) {
            G[OFF_B1 + j] += d2[j];
            for (int k = 0; k < H; k++) G[OFF_W1 + j * H + k] += d2[j] * a[k];
        }
        for (int k = 0; k < H; k++) {
            double s = 0.0;
            for (int j = 0; j < H; j++) s += d2[j] * P[OFF_W1 + j * H + k];
            d1[k] = s * dsilu(z[k]);
        }
        /* layer 0: z1 = W0 x + b0 */
        for (int j = 0; j < H; j++) {
            G[OFF_B0 + j] += d1[j];
            for (int k = 0; k < NI; k++) G[OFF_W0 + j * NI + k] += d1[j] * x[k];
        }
    }
    return loss;
}
