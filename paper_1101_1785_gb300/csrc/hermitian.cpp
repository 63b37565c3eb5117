// Spectral functions for the observables of Sec. 5.2 (von Neumann entropy, fidelity) on reduced
// density matrices, which the GPU partial trace brings to the host (2^k x 2^k, k <= 6).
#include "hermitian.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace qcw {

using cd = std::complex<double>;

// Cyclic Jacobi: for each off-diagonal pair (p, q) with a_pq = r e^{i phi}, the unitary
// U = diag(1, e^{-i phi}) G on coordinates (p, q), G the plane rotation by
// theta = atan2(2 r, a_pp - a_qq) / 2, makes (U^dagger A U)_pq = 0 (the phase turns a_pq into r,
// G diagonalises the real 2 x 2 block).  Sweeps repeat until the off-diagonal part is below
// 1e-15 of the matrix norm (quadratic convergence: a handful of sweeps).
void herm_eig(const cd *A_in, int N, double *w, cd *V)
{
    std::vector<cd> A(A_in, A_in + (size_t)N * N);
    std::vector<cd> U;
    if (V) {
        U.assign((size_t)N * N, cd(0, 0));
        for (int i = 0; i < N; i++) U[(size_t)i * N + i] = 1.0;
    }
    double norm = 0;
    for (const cd &x : A) norm += std::norm(x);
    norm = std::sqrt(norm);
    for (int sweep = 0; sweep < 100 && norm > 0; sweep++) {
        double off = 0;
        for (int p = 0; p < N; p++)
            for (int q = p + 1; q < N; q++) off += std::norm(A[(size_t)p * N + q]);
        if (std::sqrt(2 * off) <= 1e-15 * norm) break;
        for (int p = 0; p < N; p++)
            for (int q = p + 1; q < N; q++) {
                const cd apq = A[(size_t)p * N + q];
                const double r = std::abs(apq);
                if (r == 0) continue;
                const cd e = std::conj(apq / r);  // e^{-i phi}
                const double th = 0.5 * std::atan2(2 * r, A[(size_t)p * N + p].real() - A[(size_t)q * N + q].real());
                const double c = std::cos(th), s = std::sin(th);
                const cd upp = c, upq = -s, uqp = e * s, uqq = e * c;
                for (int k = 0; k < N; k++) {  // A <- A U
                    const cd akp = A[(size_t)k * N + p], akq = A[(size_t)k * N + q];
                    A[(size_t)k * N + p] = akp * upp + akq * uqp;
                    A[(size_t)k * N + q] = akp * upq + akq * uqq;
                }
                for (int k = 0; k < N; k++) {  // A <- U^dagger A
                    const cd apk = A[(size_t)p * N + k], aqk = A[(size_t)q * N + k];
                    A[(size_t)p * N + k] = std::conj(upp) * apk + std::conj(uqp) * aqk;
                    A[(size_t)q * N + k] = std::conj(upq) * apk + std::conj(uqq) * aqk;
                }
                A[(size_t)p * N + q] = A[(size_t)q * N + p] = 0.0;
                A[(size_t)p * N + p] = A[(size_t)p * N + p].real();
                A[(size_t)q * N + q] = A[(size_t)q * N + q].real();
                if (V)
                    for (int k = 0; k < N; k++) {  // U_acc <- U_acc U
                        const cd vkp = U[(size_t)k * N + p], vkq = U[(size_t)k * N + q];
                        U[(size_t)k * N + p] = vkp * upp + vkq * uqp;
                        U[(size_t)k * N + q] = vkp * upq + vkq * uqq;
                    }
            }
    }
    std::vector<int> idx(N);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(),
              [&](int a, int b) { return A[(size_t)a * N + a].real() < A[(size_t)b * N + b].real(); });
    for (int i = 0; i < N; i++) w[i] = A[(size_t)idx[i] * N + idx[i]].real();
    if (V)
        for (int k = 0; k < N; k++)
            for (int i = 0; i < N; i++) V[(size_t)k * N + i] = U[(size_t)k * N + idx[i]];
}

double entropy_bits(const double *w, int N)
{
    double s = 0;
    for (int i = 0; i < N; i++)
        if (w[i] > 1e-15) s -= w[i] * std::log2(w[i]);
    return s;
}

double fidelity_root(const cd *rho, const cd *sigma, int N)
{
    std::vector<double> mu(N), nu(N);
    std::vector<cd> V((size_t)N * N), S((size_t)N * N, cd(0, 0)), T((size_t)N * N), M((size_t)N * N);
    herm_eig(sigma, N, mu.data(), V.data());
    for (int a = 0; a < N; a++)  // sqrt(sigma) = V diag(sqrt mu) V^dagger
        for (int b = 0; b < N; b++) {
            cd x = 0;
            for (int i = 0; i < N; i++)
                x += V[(size_t)a * N + i] * std::sqrt(std::max(mu[i], 0.0)) * std::conj(V[(size_t)b * N + i]);
            S[(size_t)a * N + b] = x;
        }
    for (int a = 0; a < N; a++)  // T = sqrt(sigma) rho
        for (int b = 0; b < N; b++) {
            cd x = 0;
            for (int i = 0; i < N; i++) x += S[(size_t)a * N + i] * rho[(size_t)i * N + b];
            T[(size_t)a * N + b] = x;
        }
    for (int a = 0; a < N; a++)  // M = T sqrt(sigma), made exactly Hermitian
        for (int b = 0; b < N; b++) {
            cd x = 0;
            for (int i = 0; i < N; i++) x += T[(size_t)a * N + i] * S[(size_t)i * N + b];
            M[(size_t)a * N + b] = x;
        }
    for (int a = 0; a < N; a++)
        for (int b = a; b < N; b++) {
            const cd h = 0.5 * (M[(size_t)a * N + b] + std::conj(M[(size_t)b * N + a]));
            M[(size_t)a * N + b] = h;
            M[(size_t)b * N + a] = std::conj(h);
        }
    herm_eig(M.data(), N, nu.data(), nullptr);
    double f = 0;
    for (int i = 0; i < N; i++) f += std::sqrt(std::max(nu[i], 0.0));
    return f;
}

}  // namespace qcw
