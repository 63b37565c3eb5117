// Test-only C shim around the library's host spectral functions (hermitian.cpp).
#include <complex>
#include <vector>

#include "hermitian.h"

extern "C" void shim_herm_eig(const double *a_c128, int n, double *w, double *v_c128)
{
    qcw::herm_eig(reinterpret_cast<const std::complex<double> *>(a_c128), n, w,
                  reinterpret_cast<std::complex<double> *>(v_c128));
}

extern "C" double shim_entropy_bits(const double *w, int n) { return qcw::entropy_bits(w, n); }

extern "C" double shim_fidelity(const double *rho_c128, const double *sigma_c128, int n)
{
    return qcw::fidelity_root(reinterpret_cast<const std::complex<double> *>(rho_c128),
                              reinterpret_cast<const std::complex<double> *>(sigma_c128), n);
}
