/*
 * mle_oracle.c -- FP64 CPU oracle of the GP log marginal likelihood and its gradient
 * (test infrastructure only: the tests, the smoke check and the bench's CPU-baseline leg may
 * load it; it shares no code with the CUDA path).
 *
 * For y ~ N(0, K), K = s2 m(r_ij) + sn2 I with the Matern-5/2 ARD shape m (the model of the
 * fit), following Rasmussen & Williams, "Gaussian Processes for Machine Learning" (2006):
 *   LML = -1/2 y^T alpha - sum_i log L_ii - n/2 log(2 pi)            (eq. 2.30, Alg. 2.1)
 *   dLML/dtheta_j = 1/2 tr((alpha alpha^T - K^-1) dK/dtheta_j)       (eq. 5.9)
 * over theta = (log l_1 .. log l_d, log s2, log sn2), where for r^2 = sum_k ((x_k - x'_k)/l_k)^2
 *   dK/dlog l_k = s2 (5/3) (1 + sqrt5 r) exp(-sqrt5 r) ((x_k - x'_k)/l_k)^2
 *   dK/dlog s2  = s2 m(r),            dK/dlog sn2 = sn2 I.
 * alpha and L come from the oracle's fit (textbook Cholesky, refined alpha); K^-1 is formed
 * column by column by forward and back substitution.
 * Pins: tests/test_oracle_mle.py checks the LML and the gradient against scikit-learn's
 * GaussianProcessRegressor and the gradient against central differences of this LML.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int orc_gp_fit(const double *X, const double *y, int n, int d, const double *ls, double s2, double sn2,
               double *K, double *L, double *alpha);
void orc_forward(const double *L, int n, const double *b, double *x);
void orc_backward_t(const double *L, int n, const double *b, double *x);

int orc_lml_grad(const double *X, const double *y, int n, int d, const double *ls, double s2, double sn2,
                 double *lml, double *grad)
{
    const size_t nn = (size_t)n * n;
    double *K = (double *)malloc(sizeof(double) * nn);
    double *L = (double *)malloc(sizeof(double) * nn);
    double *Ki = (double *)malloc(sizeof(double) * nn);
    double *alpha = (double *)malloc(sizeof(double) * (size_t)n);
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *col = (double *)malloc(sizeof(double) * (size_t)n);
    int st = orc_gp_fit(X, y, n, d, ls, s2, sn2, K, L, alpha);
    if (st) {
        free(K); free(L); free(Ki); free(alpha); free(e); free(z); free(col);
        return st;
    }
    double quad = 0.0, logdet = 0.0;
    for (int i = 0; i < n; ++i) {
        quad += y[i] * alpha[i];
        logdet += log(L[(size_t)i * n + i]);
    }
    *lml = -0.5 * quad - logdet - 0.5 * n * log(2.0 * 3.14159265358979323846);
    for (int j = 0; j < n; ++j) {  /* column j of K^-1 */
        memset(e, 0, sizeof(double) * (size_t)n);
        e[j] = 1.0;
        orc_forward(L, n, e, z);
        orc_backward_t(L, n, z, col);
        for (int i = 0; i < n; ++i) Ki[(size_t)i * n + j] = col[i];
    }
    for (int q = 0; q < d + 2; ++q) grad[q] = 0.0;
    const double sq5 = sqrt(5.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double w = alpha[i] * alpha[k] - Ki[(size_t)i * n + k];
            double r2 = 0.0;
            for (int q = 0; q < d; ++q) {
                const double t = (X[(size_t)i * d + q] - X[(size_t)k * d + q]) / ls[q];
                r2 += t * t;
            }
            const double r = sqrt(r2);
            const double ex = exp(-sq5 * r);
            const double c = s2 * (5.0 / 3.0) * (1.0 + sq5 * r) * ex;
            for (int q = 0; q < d; ++q) {
                const double t = (X[(size_t)i * d + q] - X[(size_t)k * d + q]) / ls[q];
                grad[q] += 0.5 * w * c * t * t;
            }
            grad[d] += 0.5 * w * s2 * (1.0 + sq5 * r + (5.0 / 3.0) * r2) * ex;
            if (i == k) grad[d + 1] += 0.5 * w * sn2;
        }
    free(K); free(L); free(Ki); free(alpha); free(e); free(z); free(col);
    return 0;
}
