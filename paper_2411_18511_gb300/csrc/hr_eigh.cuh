// hr_eigh.cuh -- eigen-decomposition of a small Hermitian matrix by cyclic
// Jacobi rotations (Jacobi 1846; the complex form as in Golub and Van Loan,
// Matrix Computations, Sec. 8.5): A = V diag(w) V^+.  Each rotation zeroes
// one off-diagonal pair (p, q): a phase on column q makes A_pq real, then a
// real plane rotation with t = sgn(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (A_qq - A_pp) / (2 |A_pq|), annihilates it.  Native FP64; used per
// site on the 4 x 4 chiral blocks of the clover term.  Plain C++ as well as
// CUDA (HR_HD), so that the host can check it.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define HR_HD __host__ __device__
#else
#define HR_HD
#endif

namespace hr {

struct zd {
    double re, im;
};

// A (Hermitian, overwritten), V the eigenvectors (columns), w the eigenvalues
template <int N> HR_HD inline void jacobi_eigh(zd (&A)[N][N], zd (&V)[N][N], double (&w)[N])
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) V[i][j] = {i == j ? 1.0 : 0.0, 0.0};
    double scale = 0.0;
    for (int i = 0; i < N; ++i) scale += A[i][i].re * A[i][i].re;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q) off += A[p][q].re * A[p][q].re + A[p][q].im * A[p][q].im;
        if (off <= 1e-34 * (scale + off) || off == 0.0) break;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q) {
                const double r = std::sqrt(A[p][q].re * A[p][q].re + A[p][q].im * A[p][q].im);
                if (r == 0.0) continue;
                // phase e = A_pq / r; U = diag(..., conj(e) at q, ...) R
                const zd e = {A[p][q].re / r, A[p][q].im / r};
                const double tau = (A[q][q].re - A[p][p].re) / (2.0 * r);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // U_pp = c, U_pq = s, U_qp = -s conj(e), U_qq = c conj(e)
                const zd upp = {c, 0.0}, upq = {s, 0.0}, uqp = {-s * e.re, s * e.im}, uqq = {c * e.re, -c * e.im};
                auto mul = [](zd x, zd y) { return zd{x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re}; };
                auto add = [](zd x, zd y) { return zd{x.re + y.re, x.im + y.im}; };
                auto cj = [](zd x) { return zd{x.re, -x.im}; };
                for (int k = 0; k < N; ++k) { // columns: A U, V U
                    const zd akp = A[k][p], akq = A[k][q];
                    A[k][p] = add(mul(akp, upp), mul(akq, uqp));
                    A[k][q] = add(mul(akp, upq), mul(akq, uqq));
                    const zd vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = add(mul(vkp, upp), mul(vkq, uqp));
                    V[k][q] = add(mul(vkp, upq), mul(vkq, uqq));
                }
                for (int k = 0; k < N; ++k) { // rows: U^+ (A U)
                    const zd apk = A[p][k], aqk = A[q][k];
                    A[p][k] = add(mul(cj(upp), apk), mul(cj(uqp), aqk));
                    A[q][k] = add(mul(cj(upq), apk), mul(cj(uqq), aqk));
                }
                A[p][q] = A[q][p] = {0.0, 0.0};
                A[p][p].im = A[q][q].im = 0.0;
            }
    }
    for (int i = 0; i < N; ++i) w[i] = A[i][i].re;
}

} // namespace hr
