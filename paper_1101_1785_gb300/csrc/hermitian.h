// Host-side spectral functions of small Hermitian matrices (reduced density matrices of at most
// a few qubits): eigenvalues, von Neumann entropy and fidelity.  Plain C++, no CUDA.
#pragma once
#include <complex>

namespace qcw {

// Eigenvalues (ascending) of the complex Hermitian N x N matrix A (row-major) into w[N] and, if
// V is not null, the eigenvectors as the columns of V (row-major N x N, unitary).
void herm_eig(const std::complex<double> *A, int N, double *w, std::complex<double> *V);

// -sum_i w_i log2 w_i over the positive eigenvalues w_i (entries below 1e-15 count as 0).
double entropy_bits(const double *w, int N);

// Tr sqrt(sqrt(sigma) rho sqrt(sigma)) for Hermitian positive semidefinite N x N rho and sigma
// (row-major); negative rounding residue in the spectra counts as 0.
double fidelity_root(const std::complex<double> *rho, const std::complex<double> *sigma, int N);

}  // namespace qcw
