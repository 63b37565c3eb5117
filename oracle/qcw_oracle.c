/*
 * qcw CPU oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow complex128 restatement of what the QCWAVE density-matrix path computes
 * (Tabakin & Julia-Diaz, "QCWAVE - a Mathematica quantum computer simulation update").
 * Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or table with the CUDA library.
 *
 * Conventions
 *   - An n-qubit basis label is n = sum_i q_i 2^(n_q - i) (Sec. 2.3, Eq. staten): the
 *     paper's qubit i_s is API qubit q = i_s - 1, and its "stride" is 2^(n-1-q)
 *     (Sec. 3.1, text after Eq. resmat1).
 *   - rho is a 2^n x 2^n row-major array of interleaved complex128 (re, im) pairs.
 *   - A k-qubit operator is a 2^k x 2^k row-major complex128 matrix whose index is the
 *     binary number (q_{s1} q_{s2} ... q_{sk}) of the struck qubits in the order given,
 *     which for k = 2 is the quartet order n00, n01, n10, n11 of Eq. resmat2.
 *
 * Parity status: every function below is pinned by tests/test_oracle_pins.py.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "qcw_oracle.h"

typedef double _Complex cplx;

#define ORC_MAXK 6

/* Stride of API qubit q in an n-qubit label (Eq. staten; n1 = n0 + 2^(n_q - i_s)). */
static long orc_stride(int n, int q) { return 1L << (n - 1 - q); }

static int orc_check_qubits(int n, const int *qs, int k, const int *ctrl, int nc)
{
    if (n < 1 || n > 20 || k < 1 || k > ORC_MAXK || nc < 0 || k + nc > n) return ORC_EINVAL;
    long seen = 0;
    for (int j = 0; j < k + nc; j++) {
        int q = j < k ? qs[j] : ctrl[j - k];
        if (q < 0 || q >= n) return ORC_EINVAL;
        if (seen & (1L << q)) return ORC_EINVAL;
        seen |= 1L << q;
    }
    return ORC_OK;
}

/* Offsets of the 2^k members of a group ("pair", "quartet", "octet", ...) relative to its
 * member n_{0...0}: member i has struck qubit j equal to bit (k-1-j) of i (Sec. 3.2). */
static void orc_group_offsets(int n, const int *qs, int k, long *offs, long *tmask)
{
    int m = 1 << k;
    *tmask = 0;
    for (int j = 0; j < k; j++) *tmask |= orc_stride(n, qs[j]);
    for (int i = 0; i < m; i++) {
        long o = 0;
        for (int j = 0; j < k; j++)
            if ((i >> (k - 1 - j)) & 1) o += orc_stride(n, qs[j]);
        offs[i] = o;
    }
}

static long orc_ctrl_mask(int n, const int *ctrl, int nc)
{
    long cm = 0;
    for (int j = 0; j < nc; j++) cm |= orc_stride(n, ctrl[j]);
    return cm;
}

/* Eq. resmat1 / resmat2 (and their k-qubit analogue, Sec. 3.3) on the group whose
 * members sit at base + offs[i]*inc of the array v:  C~_i = sum_j W_ij C_j,
 * with W = U, or W = conj(U) when conj_u is set. */
static void orc_group_update(cplx *v, long base, long inc, const long *offs, int k,
                             const cplx *U, int conj_u)
{
    int m = 1 << k;
    cplx in[1 << ORC_MAXK];
    for (int i = 0; i < m; i++) in[i] = v[base + offs[i] * inc];
    for (int i = 0; i < m; i++) {
        cplx s = 0;
        for (int j = 0; j < m; j++) {
            cplx w = conj_u ? conj(U[i * m + j]) : U[i * m + j];
            s += w * in[j];
        }
        v[base + offs[i] * inc] = s;
    }
}

/* rho <- U rho: every column of rho is an amplitude vector (Sec. 3.1, Eq. resmat1); the
 * groups (Pick1/Pick2 of Sec. 4) run over the row label.  With controls, a group is
 * updated only when every control qubit is 1 in its row label. */
static void orc_left(cplx *rho, int n, const cplx *U, const int *qs, int k, const int *ctrl, int nc)
{
    long dim = 1L << n, offs[1 << ORC_MAXK], tmask;
    long cm = orc_ctrl_mask(n, ctrl, nc);
    orc_group_offsets(n, qs, k, offs, &tmask);
#pragma omp parallel for schedule(static)
    for (long n0 = 0; n0 < dim; n0++) {
        if (n0 & tmask) continue;
        if ((n0 & cm) != cm) continue;
        for (long c = 0; c < dim; c++) orc_group_update(rho, n0 * dim + c, dim, offs, k, U, 0);
    }
}

/* rho <- rho U^dagger: (rho U^dagger)[r, c] = sum_c' conj(U[c, c']) rho[r, c'], i.e. every
 * row of rho is an amplitude vector acted on by conj(U); groups run over the column label. */
static void orc_right(cplx *rho, int n, const cplx *U, const int *qs, int k, const int *ctrl, int nc)
{
    long dim = 1L << n, offs[1 << ORC_MAXK], tmask;
    long cm = orc_ctrl_mask(n, ctrl, nc);
    orc_group_offsets(n, qs, k, offs, &tmask);
#pragma omp parallel for schedule(static)
    for (long r = 0; r < dim; r++) {
        for (long n0 = 0; n0 < dim; n0++) {
            if (n0 & tmask) continue;
            if ((n0 & cm) != cm) continue;
            orc_group_update(rho, r * dim + n0, 1, offs, k, U, 1);
        }
    }
}

int orc_apply_unitary(double *rho, int n, const double *u, const int *qubits, int k,
                      const int *controls, int ncontrols)
{
    int st = orc_check_qubits(n, qubits, k, controls, ncontrols);
    if (st) return st;
    orc_left((cplx *)rho, n, (const cplx *)u, qubits, k, controls, ncontrols);
    orc_right((cplx *)rho, n, (const cplx *)u, qubits, k, controls, ncontrols);
    return ORC_OK;
}

/* Eq. rhoE2: rho_f = sum_n K_n rho_0 K_n^dagger, each term by the sweeps above. */
int orc_apply_kraus(double *rho, int n, const double *kraus, int nkraus, const int *qubits, int k)
{
    int st = orc_check_qubits(n, qubits, k, NULL, 0);
    if (st) return st;
    if (nkraus < 1) return ORC_EINVAL;
    long nel = 1L << (2 * n);
    long msz = 1L << (2 * k);
    cplx *acc = calloc((size_t)nel, sizeof(cplx));
    cplx *tmp = malloc((size_t)nel * sizeof(cplx));
    if (!acc || !tmp) { free(acc); free(tmp); return ORC_ENOMEM; }
    for (int t = 0; t < nkraus; t++) {
        const cplx *K = (const cplx *)kraus + t * msz;
        memcpy(tmp, rho, (size_t)nel * sizeof(cplx));
        orc_left(tmp, n, K, qubits, k, NULL, 0);
        orc_right(tmp, n, K, qubits, k, NULL, 0);
#pragma omp parallel for schedule(static)
        for (long e = 0; e < nel; e++) acc[e] += tmp[e];
    }
    memcpy(rho, acc, (size_t)nel * sizeof(cplx));
    free(acc);
    free(tmp);
    return ORC_OK;
}

/* Op1 / Op2 / Op3 on a state vector psi (Sec. 3.1-3.3): psi <- U psi. */
int orc_apply_vec(double *psi, int n, const double *u, const int *qubits, int k,
                  const int *controls, int ncontrols)
{
    int st = orc_check_qubits(n, qubits, k, controls, ncontrols);
    if (st) return st;
    long dim = 1L << n, offs[1 << ORC_MAXK], tmask;
    long cm = orc_ctrl_mask(n, controls, ncontrols);
    orc_group_offsets(n, qubits, k, offs, &tmask);
    for (long n0 = 0; n0 < dim; n0++) {
        if (n0 & tmask) continue;
        if ((n0 & cm) != cm) continue;
        orc_group_update((cplx *)psi, n0, 1, offs, k, (const cplx *)u, 0);
    }
    return ORC_OK;
}

/* Tr rho (Sec. 5.2: Tr[rho] = 1 for a state). */
void orc_trace(const double *rho, int n, double *re, double *im)
{
    long dim = 1L << n;
    const cplx *p = (const cplx *)rho;
    cplx s = 0;
    for (long i = 0; i < dim; i++) s += p[i * dim + i];
    *re = creal(s);
    *im = cimag(s);
}

/* Purity as the sum of |rho_ij|^2, equal to Tr[rho . rho] (Sec. 5.2.3) for Hermitian rho. */
double orc_purity(const double *rho, int n)
{
    long nel = 1L << (2 * n);
    const cplx *p = (const cplx *)rho;
    double s = 0;
    for (long e = 0; e < nel; e++) s += creal(p[e]) * creal(p[e]) + cimag(p[e]) * cimag(p[e]);
    return s;
}

/* p1[q] = sum over labels r with q_r = 1 of Re rho_rr. */
void orc_probabilities(const double *rho, int n, double *p1)
{
    long dim = 1L << n;
    const cplx *p = (const cplx *)rho;
    for (int q = 0; q < n; q++) {
        double s = 0;
        long st = orc_stride(n, q);
        for (long r = 0; r < dim; r++)
            if (r & st) s += creal(p[r * dim + r]);
        p1[q] = s;
    }
}

/* Projective measurement of one qubit: p_m = sum_{r: q(r) = m} Re rho_rr; the outcome is
 * `forced` when it is 0 or 1, else 0 iff u < p_0; rho <- P_m rho P_m / p_m.
 * p_m < 1e-12 leaves rho unchanged and returns ORC_EZEROPROB. */
int orc_measure(double *rho, int n, int qubit, int forced, double u, int *outcome, double *prob)
{
    if (n < 1 || qubit < 0 || qubit >= n || forced < -1 || forced > 1) return ORC_EINVAL;
    long dim = 1L << n, st = orc_stride(n, qubit);
    cplx *p = (cplx *)rho;
    double p0 = 0, p1 = 0;
    for (long r = 0; r < dim; r++) {
        if (r & st) p1 += creal(p[r * dim + r]);
        else p0 += creal(p[r * dim + r]);
    }
    int m = forced >= 0 ? forced : (u < p0 ? 0 : 1);
    double pm = m ? p1 : p0;
    *outcome = m;
    *prob = pm;
    if (!(pm >= 1e-12)) return ORC_EZEROPROB;
    long want = m ? st : 0;
    for (long r = 0; r < dim; r++)
        for (long c = 0; c < dim; c++) {
            cplx *e = &p[r * dim + c];
            if ((r & st) == want && (c & st) == want) *e = *e / pm;
            else *e = 0;
        }
    return ORC_OK;
}

/* Reduced density matrix of the kept qubits (listed in ascending order; the first kept
 * qubit is the most significant bit of the result): rho_A[a, a'] = sum_b rho[(a b), (a' b)]. */
int orc_partial_trace(const double *rho, int n, const int *keep, int nkeep, double *out)
{
    if (n < 1 || nkeep < 0 || nkeep > n) return ORC_EINVAL;
    for (int j = 0; j < nkeep; j++) {
        if (keep[j] < 0 || keep[j] >= n) return ORC_EINVAL;
        if (j && keep[j] <= keep[j - 1]) return ORC_EINVAL;
    }
    int trc[32], ntr = 0;
    for (int q = 0; q < n; q++) {
        int kept = 0;
        for (int j = 0; j < nkeep; j++) kept |= keep[j] == q;
        if (!kept) trc[ntr++] = q;
    }
    long dim = 1L << n, da = 1L << nkeep, db = 1L << ntr;
    const cplx *p = (const cplx *)rho;
    cplx *o = (cplx *)out;
    for (long a = 0; a < da; a++)
        for (long a2 = 0; a2 < da; a2++) {
            cplx s = 0;
            for (long b = 0; b < db; b++) {
                long r = 0, c = 0;
                for (int j = 0; j < nkeep; j++) {
                    if ((a >> (nkeep - 1 - j)) & 1) r |= orc_stride(n, keep[j]);
                    if ((a2 >> (nkeep - 1 - j)) & 1) c |= orc_stride(n, keep[j]);
                }
                for (int j = 0; j < ntr; j++)
                    if ((b >> (ntr - 1 - j)) & 1) {
                        r |= orc_stride(n, trc[j]);
                        c |= orc_stride(n, trc[j]);
                    }
                s += p[r * dim + c];
            }
            o[a * da + a2] = s;
        }
    (void)dim;
    return ORC_OK;
}

// One Pauli matrix entry sigma_p[a][b] (p = 0: identity).
static cplx pauli_entry(int p, int a, int b)
{
    switch (p) {
    case 0: return a == b ? 1.0 : 0.0;
    case 1: return a != b ? 1.0 : 0.0;
    case 2: return a == b ? 0.0 : (a == 0 ? -I : I);
    case 3: return a == b ? (a == 0 ? 1.0 : -1.0) : 0.0;
    }
    return 0.0;
}

int orc_pauli_expectation(const double *rho, int n, const int *qubits, const int *paulis, int k, double *out)
{
    if (n < 1 || k < 0 || k > n) return ORC_EINVAL;
    int pq[32] = {0};  // Pauli index per qubit
    for (int j = 0; j < k; j++) {
        if (qubits[j] < 0 || qubits[j] >= n || paulis[j] < 1 || paulis[j] > 3) return ORC_EINVAL;
        if (pq[qubits[j]]) return ORC_EINVAL;
        pq[qubits[j]] = paulis[j];
    }
    long dim = 1L << n;
    const cplx *p = (const cplx *)rho;
    cplx s = 0;
    // Tr[P rho] = sum_r sum_c P[r][c] rho[c][r], P[r][c] the product over qubits of sigma[r_q][c_q]
    for (long r = 0; r < dim; r++)
        for (long c = 0; c < dim; c++) {
            cplx f = 1.0;
            for (int q = 0; q < n && f != 0.0; q++) {
                const long st = orc_stride(n, q);
                f *= pauli_entry(pq[q], (r & st) != 0, (c & st) != 0);
            }
            if (f != 0.0) s += f * p[c * dim + r];
        }
    out[0] = creal(s);
    out[1] = cimag(s);
    return ORC_OK;
}

int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
