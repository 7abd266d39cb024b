/*
 * FP64 CPU oracle for the Gaussian kernel matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition that the
 * GPU path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library itself never
 * does.  It shares no code, header or constant with the CUDA sources.
 *
 * Definition followed (Sec. 1, Eqs. 1-3 of the paper, and the weighted-sum
 * form of the product in Sec. 3.1 "Fast matrix-vector products"):
 *
 *     y_r = sum_j exp(-||x_r - x_j||^2 / (2 sigma^2)) q_j + gamma q_r
 *
 * written out as a direct double loop in double precision.  Rows may be a
 * subset of the points (for large N); every row still sums over all N sources.
 * The loop over rows is split across OpenMP threads; the order of the sum over
 * sources inside one row is the plain j = 0..N-1 order.
 *
 * The Matern kernel of Sec. 6.1 has its own two functions below.
 *
 * Parity: pinned by the closed forms and invariants in tests/test_oracle_mvp.py
 * (Gaussian) and tests/test_oracle_matern.py (Matern).
 */
#include <math.h>
#include <stdint.h>

/*
 * X: N x d row-major (double); Q: N x m column-major (double);
 * rows: nrows indices into 0..N-1, or NULL for all rows (nrows = N);
 * Y: nrows x m column-major output.
 */
void oracle_mvp(const double* X, int64_t N, int d, double sigma, double gamma,
                const double* Q, int m, const int64_t* rows, int64_t nrows,
                double* Y)
{
    const double two_sigma2 = 2.0 * sigma * sigma;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        const double* xi = X + i * d;
        for (int c = 0; c < m; ++c) {
            const double* q = Q + (int64_t)c * N;
            double acc = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                const double* xj = X + j * d;
                double dist2 = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double diff = xi[k] - xj[k];
                    dist2 += diff * diff;
                }
                acc += exp(-dist2 / two_sigma2) * q[j];
            }
            Y[(int64_t)c * nrows + r] = acc + gamma * q[i];
        }
    }
}

/*
 * Rectangular product for prediction (Eqs. GPR_mean / Kriging): targets Xt
 * (Nt x d) against sources Xs (Ns x d), no diagonal term.
 *   y_t = sum_j exp(-||xt_t - xs_j||^2 / (2 sigma^2)) q_j
 */
void oracle_mvp_rect(const double* Xt, int64_t Nt, const double* Xs, int64_t Ns,
                     int d, double sigma, const double* q, double* y)
{
    const double two_sigma2 = 2.0 * sigma * sigma;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < Nt; ++t) {
        const double* xt = Xt + t * d;
        double acc = 0.0;
        for (int64_t j = 0; j < Ns; ++j) {
            const double* xj = Xs + j * d;
            double dist2 = 0.0;
            for (int k = 0; k < d; ++k) {
                const double diff = xt[k] - xj[k];
                dist2 += diff * diff;
            }
            acc += exp(-dist2 / two_sigma2) * q[j];
        }
        y[t] = acc;
    }
}

/*
 * Matern kernel of Sec. 6.1 (Eq. MaternKernel, smoothness 3/2), with the
 * length scale h in the role sigma has for the Gaussian:
 *
 *     k(x_i, x_j) = (1 + sqrt(3) d_ij) exp(-sqrt(3) d_ij),
 *     d_ij = ||x_i - x_j|| / h,
 *
 * and the same weighted sums as above:
 *     y_r = sum_j k(x_r, x_j) q_j + gamma q_r           (square, Eq. 3)
 *     y_t = sum_j k(xt_t, xs_j) q_j                      (rectangular)
 */
static double matern32(const double* a, const double* b, int d, double h)
{
    double dist2 = 0.0;
    for (int k = 0; k < d; ++k) {
        const double diff = a[k] - b[k];
        dist2 += diff * diff;
    }
    const double t = sqrt(3.0) * sqrt(dist2) / h;
    return (1.0 + t) * exp(-t);
}

void oracle_mvp_matern(const double* X, int64_t N, int d, double h, double gamma,
                       const double* Q, int m, const int64_t* rows, int64_t nrows,
                       double* Y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        const double* xi = X + i * d;
        for (int c = 0; c < m; ++c) {
            const double* q = Q + (int64_t)c * N;
            double acc = 0.0;
            for (int64_t j = 0; j < N; ++j) acc += matern32(xi, X + j * d, d, h) * q[j];
            Y[(int64_t)c * nrows + r] = acc + gamma * q[i];
        }
    }
}

void oracle_mvp_rect_matern(const double* Xt, int64_t Nt, const double* Xs, int64_t Ns,
                            int d, double h, const double* q, double* y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < Nt; ++t) {
        double acc = 0.0;
        for (int64_t j = 0; j < Ns; ++j) acc += matern32(Xt + t * d, Xs + j * d, d, h) * q[j];
        y[t] = acc;
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
