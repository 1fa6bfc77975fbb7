/*
 * mlp_oracle.c -- FP64 CPU oracle of the learned pre-screen network (test infrastructure only).
 *
 * The pre-screen surrogate is an ensemble member of shape d -> H -> H -> 2 with the exact
 * GELU activation g(z) = z Phi(z) (Phi via erfc), predicting (mu, log sigma) of the GP
 * posterior in standardised units.  Loss for a batch of B rows:
 *     L = (1 / (2B)) sum_b sum_j (o_bj - t_bj)^2.
 * Parameter layout (one network, contiguous):
 *     W1 [d x H] (in-major), b1 [H], W2 [H x H], b2 [H], W3 [H x 2], b3 [2].
 * Forward:  z1 = x W1 + b1, h1 = g(z1), z2 = h1 W2 + b2, h2 = g(z2), o = h2 W3 + b3.
 * Backward (plain chain rule):
 *     dO = (o - t) / B;  dW3 = h2^T dO;  db3 = sum_b dO;  dh2 = dO W3^T;  dz2 = dh2 g'(z2);
 *     dW2 = h1^T dz2;  db2 = sum_b dz2;  dh1 = dz2 W2^T;  dz1 = dh1 g'(z1);
 *     dW1 = x^T dz1;  db1 = sum_b dz1;   g'(z) = Phi(z) + z phi(z).
 * Ensemble of E networks (the pre-screen's score of a candidate):
 *     mu_e = o_e0 n1 + n0,  sigma_e = exp(o_e1 n3 + n2)   (n = target mean/sd of mu, log sigma)
 *     mu_bar = (1/E) sum_e mu_e,  sigma_bar^2 = (1/E) sum_e sigma_e^2 + (1/E) sum_e (mu_e - mu_bar)^2
 *     (the variance of the equal-weight mixture of the members), ei = EI(mu_bar, sigma_bar).
 * Pins: tests/test_oracle_mlp.py checks the forward against numpy matrix products, the
 * GELU against scipy's normal CDF, every gradient against central finite differences, and
 * the ensemble against the one-member case, identical members, and the two-member closed
 * form sigma_bar^2 = (s1^2 + s2^2)/2 + ((m1 - m2)/2)^2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double MLP_PI = 3.14159265358979323846;

double orc_gelu(double z) { return z * 0.5 * erfc(-z / sqrt(2.0)); }

static double gelu_grad(double z)
{
    return 0.5 * erfc(-z / sqrt(2.0)) + z * exp(-0.5 * z * z) / sqrt(2.0 * MLP_PI);
}

/* o [B x 2]; z1, h1, z2, h2 [B x H] are written when non-NULL (activations for backward). */
void orc_mlp_forward(const double *x, int B, int d, int H, const double *W1, const double *b1, const double *W2,
                     const double *b2, const double *W3, const double *b3, double *z1, double *z2, double *h2_out,
                     double *o)
{
    double *Z1 = z1 ? z1 : (double *)malloc(sizeof(double) * (size_t)B * H);
    double *Z2 = z2 ? z2 : (double *)malloc(sizeof(double) * (size_t)B * H);
    double *H1 = (double *)malloc(sizeof(double) * (size_t)H);
    double *H2 = (double *)malloc(sizeof(double) * (size_t)H);
    for (int b = 0; b < B; ++b) {
        for (int j = 0; j < H; ++j) {
            double s = b1[j];
            for (int k = 0; k < d; ++k) s += x[(size_t)b * d + k] * W1[(size_t)k * H + j];
            Z1[(size_t)b * H + j] = s;
            H1[j] = orc_gelu(s);
        }
        for (int j = 0; j < H; ++j) {
            double s = b2[j];
            for (int k = 0; k < H; ++k) s += H1[k] * W2[(size_t)k * H + j];
            Z2[(size_t)b * H + j] = s;
            H2[j] = orc_gelu(s);
            if (h2_out) h2_out[(size_t)b * H + j] = H2[j];
        }
        for (int j = 0; j < 2; ++j) {
            double s = b3[j];
            for (int k = 0; k < H; ++k) s += H2[k] * W3[(size_t)k * 2 + j];
            o[(size_t)b * 2 + j] = s;
        }
    }
    if (!z1) free(Z1);
    if (!z2) free(Z2);
    free(H1);
    free(H2);
}

/* Gradients of L for one batch.  Returns L; writes dW1 .. db3 (same layout as the weights). */
double orc_mlp_backward(const double *x, int B, int d, int H, const double *W1, const double *b1, const double *W2,
                        const double *b2, const double *W3, const double *b3, const double *t, double *dW1,
                        double *db1, double *dW2, double *db2, double *dW3, double *db3, double *loss_out)
{
    double *Z1 = (double *)malloc(sizeof(double) * (size_t)B * H);
    double *Z2 = (double *)malloc(sizeof(double) * (size_t)B * H);
    double *H2 = (double *)malloc(sizeof(double) * (size_t)B * H);
    double *O = (double *)malloc(sizeof(double) * (size_t)B * 2);
    orc_mlp_forward(x, B, d, H, W1, b1, W2, b2, W3, b3, Z1, Z2, H2, O);
    memset(dW1, 0, sizeof(double) * (size_t)d * H);
    memset(db1, 0, sizeof(double) * (size_t)H);
    memset(dW2, 0, sizeof(double) * (size_t)H * H);
    memset(db2, 0, sizeof(double) * (size_t)H);
    memset(dW3, 0, sizeof(double) * (size_t)H * 2);
    memset(db3, 0, sizeof(double) * 2);
    double L = 0.0;
    double *dz2 = (double *)malloc(sizeof(double) * (size_t)H);
    double *dz1 = (double *)malloc(sizeof(double) * (size_t)H);
    for (int b = 0; b < B; ++b) {
        double dO[2];
        for (int j = 0; j < 2; ++j) {
            const double e = O[(size_t)b * 2 + j] - t[(size_t)b * 2 + j];
            L += 0.5 * e * e / B;
            dO[j] = e / B;
            db3[j] += dO[j];
        }
        for (int k = 0; k < H; ++k) {
            const double h2 = H2[(size_t)b * H + k];
            dW3[(size_t)k * 2 + 0] += h2 * dO[0];
            dW3[(size_t)k * 2 + 1] += h2 * dO[1];
            const double dh2 = dO[0] * W3[(size_t)k * 2 + 0] + dO[1] * W3[(size_t)k * 2 + 1];
            dz2[k] = dh2 * gelu_grad(Z2[(size_t)b * H + k]);
            db2[k] += dz2[k];
        }
        for (int k = 0; k < H; ++k) {
            const double h1 = orc_gelu(Z1[(size_t)b * H + k]);
            double dh1 = 0.0;
            for (int j = 0; j < H; ++j) {
                dW2[(size_t)k * H + j] += h1 * dz2[j];
                dh1 += dz2[j] * W2[(size_t)k * H + j];
            }
            dz1[k] = dh1 * gelu_grad(Z1[(size_t)b * H + k]);
            db1[k] += dz1[k];
        }
        for (int k = 0; k < d; ++k)
            for (int j = 0; j < H; ++j) dW1[(size_t)k * H + j] += x[(size_t)b * d + k] * dz1[j];
    }
    free(Z1); free(Z2); free(H2); free(O); free(dz2); free(dz1);
    if (loss_out) *loss_out = L;
    return L;
}

double orc_ei(double mu, double sigma, double tau, double xi);

/* theta: E x P (one network after another); X: B x d; norm4 = {n0, n1, n2, n3}.
 * Outputs B values each (any may be NULL). */
void orc_mlp_ensemble(const double *theta, int E, const double *X, int B, int d, int H, const double *norm4,
                      double tau, double xi, double *mu_bar, double *sigma_bar, double *ei)
{
    const size_t P = (size_t)d * H + H + (size_t)H * H + H + 2 * (size_t)H + 2;
    double *o = (double *)malloc(sizeof(double) * (size_t)E * B * 2);
    for (int e = 0; e < E; ++e) {
        const double *th = theta + (size_t)e * P;
        const double *W1 = th, *b1 = W1 + (size_t)d * H, *W2 = b1 + H, *b2 = W2 + (size_t)H * H, *W3 = b2 + H,
                     *b3 = W3 + 2 * (size_t)H;
        orc_mlp_forward(X, B, d, H, W1, b1, W2, b2, W3, b3, NULL, NULL, NULL, o + (size_t)e * B * 2);
    }
    for (int b = 0; b < B; ++b) {
        double m = 0.0, v = 0.0, s2 = 0.0;
        for (int e = 0; e < E; ++e) m += o[((size_t)e * B + b) * 2] * norm4[1] + norm4[0];
        m /= E;
        for (int e = 0; e < E; ++e) {
            const double mu = o[((size_t)e * B + b) * 2] * norm4[1] + norm4[0];
            const double sg = exp(o[((size_t)e * B + b) * 2 + 1] * norm4[3] + norm4[2]);
            v += (mu - m) * (mu - m);
            s2 += sg * sg;
        }
        const double sb = sqrt(s2 / E + v / E);
        if (mu_bar) mu_bar[b] = m;
        if (sigma_bar) sigma_bar[b] = sb;
        if (ei) ei[b] = orc_ei(m, sb, tau, xi);
    }
    free(o);
}
