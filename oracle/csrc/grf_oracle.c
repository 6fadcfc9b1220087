/*
 * FP64 reference of the spectral field sum and of its per-mode adjoint sums.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; the CUDA library never links it.
 *
 * Field (Icardi et al., arXiv 2212.10961, Sec. 4.1, Eq. DiscreteFT, real
 * reading with amplitudes and phases):
 *     Y(x_i) = mu + sum_{j=0}^{N-1} A_j cos(2 pi r_ij),
 *     r_ij = t_ij - rint(t_ij),  t_ij = sum_c a_jc x_ic + psi_j  (turns).
 * Modes are summed in ascending j, each cell on its own; cells are spread
 * over OpenMP threads, which does not change any result.
 *
 * Adjoint sums (derivative of the same sum), per mode j, over cells in
 * ascending i:
 *     S_cos[j]    = sum_i g_i cos(2 pi r_ij)
 *     S_sin[j]    = sum_i g_i sin(2 pi r_ij)
 *     S_sinx[j,c] = sum_i g_i sin(2 pi r_ij) x_ic
 *
 * Layout: x is row-major (M, d); a is row-major (N, d).  Plain C99 + libm.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static double reduced_phase(const double *x, const double *a, double psi, int d)
{
    double t = psi;
    for (int c = 0; c < d; ++c)
        t += a[c] * x[c];
    return t - rint(t);
}

int oracle_synth(int64_t m, int d, const double *x, int64_t n, const double *a,
                 const double *amp, const double *psi, double mu, double *y)
{
    if (m < 0 || n < 0 || d < 1 || d > 3)
        return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j)
            acc += amp[j] * cos(TWO_PI * reduced_phase(x + i * d, a + j * d, psi[j], d));
        y[i] = mu + acc;
    }
    return 0;
}

int oracle_mode_sums(int64_t m, int d, const double *x, const double *g, int64_t n,
                     const double *a, const double *psi, double *s_cos, double *s_sin,
                     double *s_sinx)
{
    if (m < 0 || n < 0 || d < 1 || d > 3)
        return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        double sc = 0.0, ss = 0.0, sx[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < m; ++i) {
            double th = TWO_PI * reduced_phase(x + i * d, a + j * d, psi[j], d);
            double gs = g[i] * sin(th);
            sc += g[i] * cos(th);
            ss += gs;
            for (int c = 0; c < d; ++c)
                sx[c] += gs * x[i * d + c];
        }
        s_cos[j] = sc;
        s_sin[j] = ss;
        for (int c = 0; c < d; ++c)
            s_sinx[j * d + c] = sx[c];
    }
    return 0;
}
