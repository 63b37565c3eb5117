// Test-only C shim around the fusion planner (host code of the library): plans an op list and
// returns the phases it produced, so that a CPU test can replay them against the oracle.
#include <cstring>
#include <vector>

#include "planner.h"

using namespace qcw;

extern "C" int planner_phases(int n, int kmax, int search, int nops, const int *kind, const int *k, const int *qubits,
                              const double *mats, const long long *mat_off, int max_phases, int *phase_pass,
                              int *phase_nq, int *phase_q, int *phase_product, double *phase_S, int *pass_nq)
{
    std::vector<QOp> ops(nops);
    for (int i = 0; i < nops; i++) {
        QOp &o = ops[i];
        o.kind = kind[i];
        o.k = k[i];
        o.ncontrols = 0;
        for (int j = 0; j < o.k; j++) o.qubits[j] = qubits[2 * i + j];
        const int dim = o.kind == 0 ? (1 << o.k) : (1 << (2 * o.k));
        o.m.resize((size_t)dim * dim);
        for (int t = 0; t < dim * dim; t++)
            o.m[t] = c128(mats[2 * (mat_off[i] + t)], mats[2 * (mat_off[i] + t) + 1]);
    }
    std::vector<PassPlan> plan =
        plan_passes(ops, 0, ops.size(), n, kmax, false, static_cast<PassSearch>(search));
    int np = 0;
    for (size_t p = 0; p < plan.size(); p++) {
        pass_nq[p] = (int)plan[p].Q.size();
        for (const PhasePlan &ph : plan[p].phases) {
            if (np >= max_phases) return -1;
            phase_pass[np] = (int)p;
            phase_nq[np] = ph.nq;
            phase_product[np] = ph.product ? 1 : 0;
            phase_q[2 * np] = ph.qa;
            phase_q[2 * np + 1] = ph.qb;
            for (size_t t = 0; t < ph.S.size() && t < 256; t++) {
                phase_S[512 * (size_t)np + 2 * t] = ph.S[t].real();
                phase_S[512 * (size_t)np + 2 * t + 1] = ph.S[t].imag();
            }
            np++;
        }
    }
    return np * 1000 + (int)plan.size();
}

// Pass / phase structure of the count-only plan (used by the fusion-width search) against the
// full plan of the same ops: returns the number of mismatching fields (0 when they agree).
extern "C" int planner_count_only_mismatch(int n, int kmax, int search, int nops, const int *kind, const int *k,
                                           const int *qubits, const double *mats, const long long *mat_off)
{
    std::vector<QOp> ops(nops);
    for (int i = 0; i < nops; i++) {
        QOp &o = ops[i];
        o.kind = kind[i];
        o.k = k[i];
        o.ncontrols = 0;
        for (int j = 0; j < o.k; j++) o.qubits[j] = qubits[2 * i + j];
        const int dim = o.kind == 0 ? (1 << o.k) : (1 << (2 * o.k));
        o.m.resize((size_t)dim * dim);
        for (int t = 0; t < dim * dim; t++)
            o.m[t] = c128(mats[2 * (mat_off[i] + t)], mats[2 * (mat_off[i] + t) + 1]);
    }
    const PassSearch ps = static_cast<PassSearch>(search);
    const std::vector<PassPlan> a = plan_passes(ops, 0, ops.size(), n, kmax, false, ps);
    const std::vector<PassPlan> b = plan_passes(ops, 0, ops.size(), n, kmax, true, ps);
    int bad = a.size() != b.size();
    for (size_t p = 0; p < a.size() && p < b.size(); p++) {
        bad += a[p].Q != b[p].Q;
        bad += a[p].nops != b[p].nops;
        bad += a[p].phases.size() != b[p].phases.size();
        for (size_t i = 0; i < a[p].phases.size() && i < b[p].phases.size(); i++) {
            const PhasePlan &x = a[p].phases[i], &y = b[p].phases[i];
            bad += x.nq != y.nq || x.product != y.product || x.qa != y.qa || x.qb != y.qb || x.nops != y.nops;
            bad += !y.S.empty();
        }
    }
    return bad;
}

// Tile plan (descriptors and packed coefficients) of ops[0, nops) for an n-qubit register, as
// the fused kernels receive it.  Per phase: kind (1 one-qubit, 2 two-qubit, 3 product), tile
// positions (4), coefficient offset; per pass: TB and tile bits (16).  Returns the number of
// phases, or -1 if an output array is too small.
#include "tile.h"

extern "C" int tile_plan(int n, int kmax, int search, int herm, int tbmax, int nops, const int *kind, const int *k,
                         const int *qubits, const double *mats, const long long *mat_off, int max_phases,
                         int *phase_kind, int *phase_pos, int *phase_coef, int *phase_pass, int max_passes,
                         int *pass_tb, int *pass_tbits, int max_coefs, float *coefs, int *ncoefs)
{
    std::vector<QOp> ops(nops);
    for (int i = 0; i < nops; i++) {
        QOp &o = ops[i];
        o.kind = kind[i];
        o.k = k[i];
        o.ncontrols = 0;
        for (int j = 0; j < o.k; j++) o.qubits[j] = qubits[2 * i + j];
        const int dim = o.kind == 0 ? (1 << o.k) : (1 << (2 * o.k));
        o.m.resize((size_t)dim * dim);
        for (int t = 0; t < dim * dim; t++)
            o.m[t] = c128(mats[2 * (mat_off[i] + t)], mats[2 * (mat_off[i] + t) + 1]);
    }
    TilePlan tp;
    append_tile_plan(plan_passes(ops, 0, ops.size(), n, kmax, false, static_cast<PassSearch>(search)),
                     n, tbmax, tp, herm != 0);
    if ((int)tp.phases.size() > max_phases || (int)tp.passes.size() > max_passes || (int)tp.coefs.size() > max_coefs)
        return -1;
    for (size_t p = 0; p < tp.passes.size(); p++) {
        pass_tb[p] = tp.passes[p].TB;
        for (int j = 0; j < 16; j++) pass_tbits[16 * p + j] = tp.passes[p].tbits[j];
        for (int ph = 0; ph < tp.passes[p].nphase; ph++) phase_pass[tp.passes[p].phase0 + ph] = (int)p;
    }
    for (size_t i = 0; i < tp.phases.size(); i++) {
        phase_kind[i] = tp.phases[i].nq;
        for (int j = 0; j < 4; j++) phase_pos[4 * i + j] = tp.phases[i].pos[j];
        phase_coef[i] = tp.phases[i].coef;
    }
    for (size_t i = 0; i < tp.coefs.size(); i++) {
        coefs[2 * i] = tp.coefs[i].x;
        coefs[2 * i + 1] = tp.coefs[i].y;
    }
    *ncoefs = (int)tp.coefs.size();
    return (int)tp.phases.size();
}

// Real Pauli-basis transfer matrix of a one- or two-qubit superoperator S (complex128,
// interleaved, 4^k x 4^k row-major) as the plain kernels k_super1 / k_super2 receive it.
extern "C" void pauli_transfer_k(int k, const double *S, double *R)
{
    const int D = 1 << (2 * k);
    std::vector<c128> s((size_t)D * D);
    for (int t = 0; t < D * D; t++) s[t] = c128(S[2 * t], S[2 * t + 1]);
    if (k == 1) {
        double r[4][4];
        pauli_transfer1(s.data(), r);
        for (int i = 0; i < 16; i++) R[i] = r[i / 4][i % 4];
    } else {
        double r[16][16];
        pauli_transfer(s, r);
        for (int i = 0; i < 256; i++) R[i] = r[i / 16][i % 16];
    }
}
