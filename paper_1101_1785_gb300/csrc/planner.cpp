// Fusion planner (host, complex128).
//
// Pass packing is a greedy scan with commutation: an operation joins the current pass when
// the union of touched qubits stays within kmax and it shares no qubit with an earlier
// operation that was left out (operations on disjoint qubits commute, so moving it ahead of
// those is exact).  Inside a pass the same scan with a two-qubit limit forms phases, and the
// operations of a phase are multiplied into one superoperator on the phase's qubits.
//
// Superoperator index convention: for phase qubits (a, b), e = 4 R + C with
// R = 2 r_a + r_b (row bits) and C = 2 c_a + c_b (column bits); for one qubit e = 2 r + c.
#include "planner.h"

#include <algorithm>

namespace qcw {

std::vector<c128> unitary_superop(const std::vector<c128> &u, int k)
{
    int d = 1 << k, D = d * d;
    std::vector<c128> s((size_t)D * D);
    for (int r2 = 0; r2 < d; r2++)
        for (int c2 = 0; c2 < d; c2++)
            for (int r = 0; r < d; r++)
                for (int c = 0; c < d; c++)
                    s[(size_t)(r2 * d + c2) * D + (r * d + c)] = u[r2 * d + r] * std::conj(u[c2 * d + c]);
    return s;
}

// S_phase <- S_op (lifted to the phase qubits) * S_phase.
// Phase bits of an index e: for nq == 2, r_a = bit 3, r_b = bit 2, c_a = bit 1, c_b = bit 0;
// for nq == 1, r_a = bit 1, c_a = bit 0.
static void fold_op(PhasePlan &ph, const QOp &op)
{
    const int nq = ph.nq, D = 1 << (2 * nq);
    const int k = op.k, dk = 1 << k, Dk = dk * dk;
    const std::vector<c128> sop = op.kind == 0 ? unitary_superop(op.m, k) : op.m;
    // slot of each op qubit in the phase (0 = a, 1 = b)
    int slot[2];
    for (int j = 0; j < k; j++) slot[j] = op.qubits[j] == ph.qa ? 0 : 1;
    auto rbit = [&](int e, int s) { return nq == 2 ? (e >> (3 - s)) & 1 : (e >> 1) & 1; };
    auto cbit = [&](int e, int s) { return nq == 2 ? (e >> (1 - s)) & 1 : e & 1; };
    // projection of a phase index onto the op's local index, and the mask of "other" bits
    auto op_index = [&](int e) {
        int R = 0, C = 0;
        for (int j = 0; j < k; j++) {
            R |= rbit(e, slot[j]) << (k - 1 - j);
            C |= cbit(e, slot[j]) << (k - 1 - j);
        }
        return R * dk + C;
    };
    int opmask = 0;  // phase-index bits that belong to the op
    for (int j = 0; j < k; j++) {
        if (nq == 2) opmask |= (1 << (3 - slot[j])) | (1 << (1 - slot[j]));
        else opmask |= 3;
    }
    std::vector<c128> out((size_t)D * D, c128(0, 0));
    for (int e2 = 0; e2 < D; e2++) {
        int o2 = op_index(e2);
        for (int e1 = 0; e1 < D; e1++) {
            if ((e1 & ~opmask) != (e2 & ~opmask)) continue;
            c128 w = sop[(size_t)o2 * Dk + op_index(e1)];
            if (w == c128(0, 0)) continue;
            const c128 *src = &ph.S[(size_t)e1 * D];
            c128 *dst = &out[(size_t)e2 * D];
            for (int e0 = 0; e0 < D; e0++) dst[e0] += w * src[e0];
        }
    }
    ph.S.swap(out);
    ph.nops++;
}

static void identity(std::vector<c128> &s, int D)
{
    s.assign((size_t)D * D, c128(0, 0));
    for (int i = 0; i < D; i++) s[(size_t)i * D + i] = 1.0;
}

static unsigned qmask(const QOp &op)
{
    unsigned m = 0;
    for (int j = 0; j < op.k; j++) m |= 1u << op.qubits[j];
    return m;
}

static int popc(unsigned x) { return __builtin_popcount(x); }

std::vector<PassPlan> plan_passes(const std::vector<QOp> &ops, size_t begin, size_t end, int n, int kmax)
{
    std::vector<PassPlan> passes;
    std::vector<size_t> rem;
    for (size_t i = begin; i < end; i++) rem.push_back(i);
    const unsigned all = n >= 32 ? ~0u : ((1u << n) - 1u);
    while (!rem.empty()) {
        unsigned Q = 0, blocked = 0;
        std::vector<size_t> chosen, rest;
        for (size_t idx = 0; idx < rem.size(); idx++) {
            size_t i = rem[idx];
            unsigned S = qmask(ops[i]);
            if (blocked == all) {  // every qubit is held by a skipped op: nothing more can join
                rest.insert(rest.end(), rem.begin() + idx, rem.end());
                break;
            }
            if (S & blocked) {
                rest.push_back(i);
                blocked |= S;
            } else if (popc(Q | S) <= kmax) {
                Q |= S;
                chosen.push_back(i);
            } else {
                rest.push_back(i);
                blocked |= S;
            }
        }
        PassPlan pp;
        pp.nops = (int)chosen.size();
        for (int q = 0; q < n; q++)
            if (Q & (1u << q)) pp.Q.push_back(q);
        // phases of at most two qubits
        std::vector<size_t> prem = chosen;
        while (!prem.empty()) {
            unsigned P = 0, pblocked = 0;
            std::vector<size_t> pch, prest;
            for (size_t i : prem) {
                unsigned S = qmask(ops[i]);
                if (S & pblocked) {
                    prest.push_back(i);
                    pblocked |= S;
                } else if (popc(P | S) <= 2) {
                    P |= S;
                    pch.push_back(i);
                } else {
                    prest.push_back(i);
                    pblocked |= S;
                }
            }
            PhasePlan ph;
            ph.nq = popc(P);
            ph.qa = ph.qb = -1;
            for (int q = 0; q < n; q++)
                if (P & (1u << q)) {
                    if (ph.qa < 0) ph.qa = q;
                    else ph.qb = q;
                }
            ph.nops = 0;
            identity(ph.S, 1 << (2 * ph.nq));
            for (size_t i : pch) fold_op(ph, ops[i]);
            pp.phases.push_back(std::move(ph));
            prem.swap(prest);
        }
        passes.push_back(std::move(pp));
        rem.swap(rest);
    }
    return passes;
}

}  // namespace qcw
