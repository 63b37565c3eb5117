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

// Native superoperator of an op (4x4 for one qubit, 16x16 for two), index (R, C) with the
// op's qubits in its own order; unitaries become U (x) conj(U).
static void op_superop(const QOp &op, c128 *out)
{
    if (op.kind != 0) {
        for (size_t i = 0; i < op.m.size(); i++) out[i] = op.m[i];
        return;
    }
    const int d = 1 << op.k, D = d * d;
    const c128 *u = op.m.data();
    for (int r2 = 0; r2 < d; r2++)
        for (int c2 = 0; c2 < d; c2++)
            for (int r = 0; r < d; r++)
                for (int c = 0; c < d; c++) out[(r2 * d + c2) * D + (r * d + c)] = u[r2 * d + r] * std::conj(u[c2 * d + c]);
}

// Phase accumulator: S (D x D, D = 4^nq) kept as split real / imaginary rows so that
// S <- A S is a set of length-D row AXPYs that the compiler vectorises.  Runs of consecutive
// ops on the same qubit list are first multiplied at their native size and lifted once.
struct PhaseAcc {
    int nq = 0, qa = -1, qb = -1, D = 0;
    double Sr[256], Si[256];
    // pending run
    int rk = 0, rq[2] = {-1, -1};
    c128 run[256];
    bool has_run = false;

    void start(int nq_, int a, int b)
    {
        nq = nq_;
        qa = a;
        qb = b;
        D = 1 << (2 * nq);
        for (int i = 0; i < D * D; i++) Sr[i] = Si[i] = 0;
        for (int i = 0; i < D; i++) Sr[i * D + i] = 1.0;
        has_run = false;
    }

    // S <- lift(A) * S for a native superoperator A on qubits q[0..k-1].
    void lift(const c128 *A, int k, const int *q)
    {
        const int dk = 1 << k, Dk = dk * dk;
        int slot[2] = {0, 0};
        for (int j = 0; j < k; j++) slot[j] = q[j] == qa ? 0 : 1;
        // phase index bits: nq == 2: r_a = 3, r_b = 2, c_a = 1, c_b = 0; nq == 1: r = 1, c = 0
        auto rbitpos = [&](int s) { return nq == 2 ? 3 - s : 1; };
        auto cbitpos = [&](int s) { return nq == 2 ? 1 - s : 0; };
        int opmask = 0;
        for (int j = 0; j < k; j++) opmask |= (1 << rbitpos(slot[j])) | (1 << cbitpos(slot[j]));
        int oi[16];  // op-local index of every phase index
        for (int e = 0; e < D; e++) {
            int R = 0, C = 0;
            for (int j = 0; j < k; j++) {
                R |= ((e >> rbitpos(slot[j])) & 1) << (k - 1 - j);
                C |= ((e >> cbitpos(slot[j])) & 1) << (k - 1 - j);
            }
            oi[e] = R * dk + C;
        }
        double Nr[256], Ni[256];
        for (int e2 = 0; e2 < D; e2++) {
            double *nr = Nr + e2 * D, *ni = Ni + e2 * D;
            for (int c = 0; c < D; c++) nr[c] = ni[c] = 0;
            for (int e1 = 0; e1 < D; e1++) {
                if ((e1 & ~opmask) != (e2 & ~opmask)) continue;
                const c128 w = A[oi[e2] * Dk + oi[e1]];
                const double wr = w.real(), wi = w.imag();
                if (wr == 0 && wi == 0) continue;
                const double *sr = Sr + e1 * D, *si = Si + e1 * D;
                for (int c = 0; c < D; c++) {
                    nr[c] += wr * sr[c] - wi * si[c];
                    ni[c] += wr * si[c] + wi * sr[c];
                }
            }
        }
        for (int i = 0; i < D * D; i++) {
            Sr[i] = Nr[i];
            Si[i] = Ni[i];
        }
    }

    void flush()
    {
        if (has_run) lift(run, rk, rq);
        has_run = false;
    }

    void add(const QOp &op)
    {
        c128 A[256];
        op_superop(op, A);
        const bool same = has_run && rk == op.k && rq[0] == op.qubits[0] && (op.k == 1 || rq[1] == op.qubits[1]);
        if (same) {  // run <- A * run at native size
            const int Dk = 1 << (2 * op.k);
            c128 T[256];
            for (int i = 0; i < Dk; i++)
                for (int j = 0; j < Dk; j++) {
                    c128 acc = 0;
                    for (int l = 0; l < Dk; l++) acc += A[i * Dk + l] * run[l * Dk + j];
                    T[i * Dk + j] = acc;
                }
            for (int i = 0; i < Dk * Dk; i++) run[i] = T[i];
            return;
        }
        flush();
        rk = op.k;
        rq[0] = op.qubits[0];
        rq[1] = op.k > 1 ? op.qubits[1] : -1;
        for (int i = 0; i < (1 << (4 * op.k)); i++) run[i] = A[i];
        has_run = true;
    }

    void result(std::vector<c128> &out)
    {
        flush();
        out.resize((size_t)D * D);
        for (int i = 0; i < D * D; i++) out[i] = c128(Sr[i], Si[i]);
    }
};

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

// All subsets of the n qubits with exactly k members, as masks.
static std::vector<unsigned> subsets_of_size(int n, int k)
{
    std::vector<unsigned> out;
    if (k > n) return out;
    unsigned s = (1u << k) - 1u;
    const unsigned limit = n >= 32 ? 0u : 1u << n;
    while (s < limit || (limit == 0 && s != 0)) {
        out.push_back(s);
        const unsigned c = s & (0u - s), r = s + c;  // next subset of the same size (Gosper)
        if (r == 0) break;
        s = (((r ^ s) >> 2) / c) | r;
    }
    return out;
}

// Operations of rem a pass on qubit set Q can take: an operation joins when its qubits lie in Q
// and no skipped earlier operation shares a qubit with it (they commute past the skipped ones).
static size_t absorbable(const std::vector<unsigned> &masks, unsigned Q)
{
    unsigned blocked = 0;
    size_t taken = 0;
    for (unsigned S : masks) {
        if ((S & ~Q) || (S & blocked)) blocked |= S;
        else taken++;
    }
    return taken;
}

// Beam search over pass sequences (PassSearch::BEAM): returns the candidate set of every pass
// of the shortest sequence found that absorbs all operations (masks in order).  A partial
// sequence's remaining operations are what the absorb rule leaves; partial sequences are ranked
// by how many remain, and identical remainders are kept once.
constexpr int kBeamWidth = 64;
constexpr int kBeamBranch = 12;

static std::vector<unsigned> beam_pass_sets(const std::vector<unsigned> &masks, const std::vector<unsigned> &cand)
{
    struct Node {
        std::vector<unsigned> rem;
        std::vector<unsigned> seq;
    };
    std::vector<Node> beam(1);
    beam[0].rem = masks;
    for (;;) {
        std::vector<Node> next;
        for (const Node &nd : beam) {
            // the kBeamBranch most absorbing candidate sets (ties: the earlier candidate)
            std::vector<std::pair<size_t, size_t>> score;  // (absorbed, candidate index)
            score.reserve(cand.size());
            for (size_t c = 0; c < cand.size(); c++) score.emplace_back(absorbable(nd.rem, cand[c]), c);
            const size_t nb = std::min<size_t>(kBeamBranch, score.size());
            std::partial_sort(score.begin(), score.begin() + nb, score.end(),
                              [](const std::pair<size_t, size_t> &a, const std::pair<size_t, size_t> &b) {
                                  return a.first != b.first ? a.first > b.first : a.second < b.second;
                              });
            for (size_t j = 0; j < nb; j++) {
                if (score[j].first == 0) break;
                const unsigned Q = cand[score[j].second];
                Node ch;
                ch.seq = nd.seq;
                ch.seq.push_back(Q);
                unsigned blocked = 0;
                for (unsigned S : nd.rem) {
                    if ((S & ~Q) || (S & blocked)) {
                        blocked |= S;
                        ch.rem.push_back(S);
                    }
                }
                if (ch.rem.empty()) return ch.seq;
                next.push_back(std::move(ch));
            }
        }
        if (next.empty()) return {};  // nothing absorbs anything: the caller's greedy choice handles it
        std::stable_sort(next.begin(), next.end(),
                         [](const Node &a, const Node &b) { return a.rem.size() < b.rem.size(); });
        beam.clear();
        for (Node &ch : next) {
            bool dup = false;
            for (const Node &kept : beam)
                if (kept.rem == ch.rem) {
                    dup = true;
                    break;
                }
            if (!dup) beam.push_back(std::move(ch));
            if ((int)beam.size() == kBeamWidth) break;
        }
    }
}

std::vector<PassPlan> plan_passes(const std::vector<QOp> &ops, size_t begin, size_t end, int n, int kmax,
                                  bool count_only, PassSearch search)
{
    PhaseAcc acc;
    std::vector<PassPlan> passes;
    std::vector<size_t> rem;
    for (size_t i = begin; i < end; i++) rem.push_back(i);
    const unsigned all = n >= 32 ? ~0u : ((1u << n) - 1u);
    const std::vector<unsigned> cand = search != PassSearch::ORDER ? subsets_of_size(n, kmax < n ? kmax : n)
                                                                   : std::vector<unsigned>();
    std::vector<unsigned> masks, seq;
    if (search == PassSearch::BEAM && !cand.empty()) {
        for (size_t i : rem) masks.push_back(qmask(ops[i]));
        seq = beam_pass_sets(masks, cand);
    }
    size_t npass = 0;
    while (!rem.empty()) {
        unsigned Q = 0, blocked = 0;
        std::vector<size_t> chosen, rest;
        if (!cand.empty()) {
            masks.clear();
            for (size_t i : rem) masks.push_back(qmask(ops[i]));
            if (npass < seq.size()) {
                Q = seq[npass];
            } else {
                size_t best = 0;
                for (unsigned C : cand) {
                    const size_t t = absorbable(masks, C);
                    if (t > best) {
                        best = t;
                        Q = C;
                    }
                }
            }
            for (size_t idx = 0; idx < rem.size(); idx++) {
                const unsigned S = masks[idx];
                if ((S & ~Q) || (S & blocked)) {
                    rest.push_back(rem[idx]);
                    blocked |= S;
                } else {
                    chosen.push_back(rem[idx]);
                }
            }
            unsigned used = 0;  // the qubits the taken operations touch
            for (size_t i : chosen) used |= qmask(ops[i]);
            Q = used;
        } else {
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
        }
        npass++;
        PassPlan pp;
        pp.nops = (int)chosen.size();
        for (int q = 0; q < n; q++)
            if (Q & (1u << q)) pp.Q.push_back(q);
        // Phases of at most two qubits, anchored on the two-qubit operations.  Walking the
        // pass's operations in order: a two-qubit op on (a, b) joins the last phase of a if
        // that phase is also the last of b (same pair), else opens a phase that also takes the
        // single-qubit ops on a and b not yet placed (all earlier, commuting with everything
        // between); a single-qubit op on q joins the last phase touching q (no later phase
        // touches q, so it commutes past them) or waits for q's first two-qubit op.  Qubits
        // with no two-qubit op in the pass pair up into product phases (one left over: a
        // one-qubit phase), placed first: they share no qubit with the other phases.
        struct Grp {
            unsigned P;
            std::vector<size_t> ops;
            bool linked;
        };
        std::vector<Grp> grp;
        int last[32];
        std::vector<size_t> pend[32];
        for (int q = 0; q < 32; q++) last[q] = -1;
        for (size_t i : chosen) {
            const QOp &op = ops[i];
            if (op.k == 1) {
                const int q = op.qubits[0];
                if (last[q] >= 0) grp[last[q]].ops.push_back(i);
                else pend[q].push_back(i);
                continue;
            }
            const int a = op.qubits[0], b = op.qubits[1];
            if (last[a] >= 0 && last[a] == last[b]) {
                grp[last[a]].ops.push_back(i);
                continue;
            }
            Grp g{(1u << a) | (1u << b), {}, true};
            g.ops.insert(g.ops.end(), pend[a].begin(), pend[a].end());
            g.ops.insert(g.ops.end(), pend[b].begin(), pend[b].end());
            g.ops.push_back(i);
            pend[a].clear();
            pend[b].clear();
            last[a] = last[b] = (int)grp.size();
            grp.push_back(std::move(g));
        }
        std::vector<Grp> order;
        int lone = -1;
        for (int q = 0; q < n; q++) {
            if (pend[q].empty()) continue;
            if (lone < 0) {
                lone = q;
                continue;
            }
            Grp g{(1u << lone) | (1u << q), pend[lone], false};
            g.ops.insert(g.ops.end(), pend[q].begin(), pend[q].end());
            order.push_back(std::move(g));
            lone = -1;
        }
        if (lone >= 0) order.push_back(Grp{1u << lone, pend[lone], false});
        for (Grp &g : grp) order.push_back(std::move(g));
        for (const Grp &g : order) {
            const unsigned P = g.P;
            const std::vector<size_t> &pch = g.ops;
            PhasePlan ph;
            ph.nq = popc(P);
            ph.qa = ph.qb = -1;
            for (int q = 0; q < n; q++)
                if (P & (1u << q)) {
                    if (ph.qa < 0) ph.qa = q;
                    else ph.qb = q;
                }
            ph.nops = (int)pch.size();
            ph.product = ph.nq == 2 && !g.linked;
            if (count_only) {
                identity(ph.S, 0);
            } else if (ph.product) {
                // ops on different qubits commute: compose each qubit's ops on their own
                std::vector<c128> sa, sb;
                for (int side = 0; side < 2; side++) {
                    const int qq = side == 0 ? ph.qa : ph.qb;
                    acc.start(1, qq, -1);
                    for (size_t i : pch)
                        if (ops[i].qubits[0] == qq) acc.add(ops[i]);
                    acc.result(side == 0 ? sa : sb);
                }
                ph.S = sa;
                ph.S.insert(ph.S.end(), sb.begin(), sb.end());
            } else {
                acc.start(ph.nq, ph.qa, ph.qb);
                for (size_t i : pch) acc.add(ops[i]);
                acc.result(ph.S);
            }
            pp.phases.push_back(std::move(ph));
        }
        passes.push_back(std::move(pp));
        rem.swap(rest);
    }
    return passes;
}

}  // namespace qcw
