/* qcw CPU oracle (test infrastructure only): declarations of oracle/qcw_oracle.c.
 * rho buffers are 2^n x 2^n row-major interleaved complex128; matrices are row-major
 * interleaved complex128.  Qubit q is the paper's qubit i_s = q + 1 (Sec. 2.3). */
#ifndef QCW_ORACLE_H
#define QCW_ORACLE_H

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EZEROPROB (-3)

int orc_apply_unitary(double *rho, int n, const double *u, const int *qubits, int k,
                      const int *controls, int ncontrols);
int orc_apply_kraus(double *rho, int n, const double *kraus, int nkraus, const int *qubits, int k);
int orc_apply_vec(double *psi, int n, const double *u, const int *qubits, int k,
                  const int *controls, int ncontrols);
void orc_trace(const double *rho, int n, double *re, double *im);
double orc_purity(const double *rho, int n);
void orc_probabilities(const double *rho, int n, double *p1);
int orc_measure(double *rho, int n, int qubit, int forced, double u, int *outcome, double *prob);
int orc_partial_trace(const double *rho, int n, const int *keep, int nkeep, double *out);
/* Tr[P rho] for the Pauli string P = (x)_j sigma_{paulis[j]} on qubits[j] (1 = X, 2 = Y, 3 = Z;
 * distinct qubits), identity elsewhere: the polarisation vectors and spin correlation tensor
 * of Sec. 5.2 are such traces.  out = {Re, Im}. */
int orc_pauli_expectation(const double *rho, int n, const int *qubits, const int *paulis, int k, double *out);
int orc_set_threads(int nthreads);

#endif
