// Fusion planner: packs a queue of one- and two-qubit operations (unitaries and channel
// superoperators) into passes over rho, each touching at most k qubits, and each pass into
// phases of at most two qubits whose operations are composed into one superoperator.
#pragma once
#include <complex>
#include <vector>

#include "qcw_internal.h"

namespace qcw {

struct PhasePlan {
    int nq;                 // 1 or 2
    bool product = false;   // nq == 2 with no two-qubit op: S = S_a (x) S_b
    int qa, qb;             // phase qubits (qb = -1 when nq == 1)
    std::vector<c128> S;    // composed superoperator: 4x4 (nq = 1), 16x16 (nq = 2),
                            // or S_a then S_b, 4x4 each (product)
    int nops;               // operations folded into S
};

struct PassPlan {
    std::vector<int> Q;           // qubits the pass touches (ascending)
    std::vector<PhasePlan> phases;
    int nops;
};

// How a pass's qubit set is chosen.  ORDER: grow it from the remaining operations in order.
// BEST: among all kmax-qubit sets, the one that absorbs the most remaining operations (C(n,
// kmax) candidates per pass; about a third fewer passes on random circuits, for host time that
// suits plans that are cached and replayed).
// BEAM: the sequence of kmax-qubit sets chosen by a beam search (the kBeamWidth partial
// sequences that leave the fewest operations, each extended by its kBeamBranch most absorbing
// sets) instead of one greedy choice per pass; it finds shorter pass sequences where a greedy
// choice strands operations that then need passes of their own.
enum class PassSearch { ORDER, BEST, BEAM };

// Plan ops[begin, end) (all with k <= 2 and no controls) for an n-qubit register.  With
// count_only the pass / phase structure is produced without composing the superoperators.
std::vector<PassPlan> plan_passes(const std::vector<QOp> &ops, size_t begin, size_t end, int n, int kmax,
                                  bool count_only = false, PassSearch search = PassSearch::ORDER);

}  // namespace qcw
