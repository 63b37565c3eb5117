// Host side of the tile descriptors: tile bit selection and packing of planner output.
#include "tile.h"

#include <algorithm>

namespace qcw {

size_t tile_smem_bytes(int TB, int L)
{
    return ((size_t)8 << TB) + 8 * ((((size_t)1 << (TB - L)) | 1) + 1) + 256 * sizeof(float2);
}

// Tile bits of a pass: rows and columns of Q, then the lowest column bits until tbmax bits
// (or all column bits are in).
static void tile_layout(const std::vector<int> &Q, int n, int tbmax, FPass &fp, bool herm)
{
    uint64_t in = 0;
    for (int q : Q) {
        in |= 1ull << (n - 1 - q);
        in |= 1ull << (2 * n - 1 - q);
    }
    int want = tbmax < 2 * n ? tbmax : 2 * n;
    if (herm) {  // add whole qubits, lowest first: column bit v and row bit n + v together
        want &= ~1;
        for (int v = 0; v < n && __builtin_popcountll(in) < want; v++) in |= (1ull << v) | (1ull << (n + v));
    } else {
        for (int v = 0; v < n && __builtin_popcountll(in) < want; v++) in |= 1ull << v;
    }
    fp.herm = herm ? 1 : 0;
    int tb = 0, ob = 0;
    for (int v = 0; v < 2 * n; v++) {
        if (in & (1ull << v)) fp.tbits[tb++] = (int8_t)v;
        else fp.obits[ob++] = (int8_t)v;
    }
    fp.TB = tb;
    fp.nother = ob;
    int L = 0;
    while (L < tb && fp.tbits[L] == L) L++;
    fp.L = L;
}

static int tile_pos(const FPass &fp, int vbit)
{
    for (int j = 0; j < fp.TB; j++)
        if (fp.tbits[j] == vbit) return j;
    return -1;
}

// Two-qubit phases run in a Pauli basis (see tile_phase2).  Per qubit of the phase, with its
// row and column bits (r, c), the device maps the members (b00, b01, b10, b11) to
// (I, X, D, Z) = (b00 + b11, b01 + b10, b01 - b10, b00 - b11) and back with
// (b00, b01, b10, b11) = (I + Z, X + D, X - D, I - Z); I, X, Z and i D are 2x the Pauli
// coefficients tr(P b) of the 2x2 block.  Member e = 8 r_a + 4 r_b + 2 c_a + c_b keeps its bit
// positions: Pauli index bits (2 r + c) per qubit.
// Transfer-matrix entries below this are FP64 rounding residue of exact zeros (the entries of
// a map of unit-norm operators are O(1)); they are stored as 0 so that, for instance, the trace
// row of a trace-preserving map is exactly (2^-k, 0, ...).
constexpr double kTransferZero = 1e-14;

static void pauli_fwd(c128 *x)
{
    for (int e2 = 0; e2 < 2; e2++)
        for (int e0 = 0; e0 < 2; e0++) {
            const int i = 4 * e2 + e0;
            const c128 b00 = x[i], b01 = x[i + 2], b10 = x[i + 8], b11 = x[i + 10];
            x[i] = b00 + b11, x[i + 2] = b01 + b10, x[i + 8] = b01 - b10, x[i + 10] = b00 - b11;
        }
    for (int e3 = 0; e3 < 2; e3++)
        for (int e1 = 0; e1 < 2; e1++) {
            const int i = 8 * e3 + 2 * e1;
            const c128 b00 = x[i], b01 = x[i + 1], b10 = x[i + 4], b11 = x[i + 5];
            x[i] = b00 + b11, x[i + 1] = b01 + b10, x[i + 4] = b01 - b10, x[i + 5] = b00 - b11;
        }
}

static void pauli_inv(c128 *w)
{
    for (int e3 = 0; e3 < 2; e3++)
        for (int e1 = 0; e1 < 2; e1++) {
            const int i = 8 * e3 + 2 * e1;
            const c128 I = w[i], X = w[i + 1], D = w[i + 4], Z = w[i + 5];
            w[i] = I + Z, w[i + 1] = X + D, w[i + 4] = X - D, w[i + 5] = I - Z;
        }
    for (int e2 = 0; e2 < 2; e2++)
        for (int e0 = 0; e0 < 2; e0++) {
            const int i = 4 * e2 + e0;
            const c128 I = w[i], X = w[i + 2], D = w[i + 8], Z = w[i + 10];
            w[i] = I + Z, w[i + 2] = X + D, w[i + 8] = X - D, w[i + 10] = I - Z;
        }
}

// Pauli index with an odd number of D components: there the Pauli coefficient is i D.
static bool pauli_odd(int e) { return (((e >> 3) & 1) && !((e >> 1) & 1)) != (((e >> 2) & 1) && !(e & 1)); }

// Real transfer matrix R of a two-qubit superoperator S (16 x 16, S[e][f], row-major) for the
// device's order of operations: u = fwd(x); v_f = i u_f on odd indices (u_f elsewhere);
// c = R v; w_e = -i c_e on odd indices (c_e elsewhere); x' = inv(w) = S x.  Since
// inv(fwd(x)) = 4 x, R = (1/16) d fwd(S inv(.)) conj(d) with d = i on odd indices.  R is real
// because S preserves Hermiticity (every gate and channel does): in the Hermitian Pauli basis
// its matrix is real, and the d factors turn D into the Y coefficient.
void pauli_transfer(const std::vector<c128> &S, double R[16][16])
{
    c128 M[16][16];
    for (int f = 0; f < 16; f++) {
        c128 col[16] = {};
        col[f] = 1.0;
        pauli_inv(col);  // column f of inv
        c128 sc[16];
        for (int e = 0; e < 16; e++) {
            c128 acc = 0;
            for (int g = 0; g < 16; g++) acc += S[(size_t)e * 16 + g] * col[g];
            sc[e] = acc;
        }
        pauli_fwd(sc);
        for (int e = 0; e < 16; e++) M[e][f] = sc[e];
    }
    for (int e = 0; e < 16; e++)
        for (int f = 0; f < 16; f++) {
            c128 z = M[e][f] / 16.0;
            if (pauli_odd(e)) z *= c128(0, 1);
            if (pauli_odd(f)) z *= c128(0, -1);
            R[e][f] = std::abs(z.real()) < kTransferZero ? 0.0 : z.real();
        }
}

// One qubit: members (b00, b01, b10, b11) -> (I, X, D, Z) by the same butterflies; the real
// 4 x 4 transfer matrix of a one-qubit superoperator S (S[e][f], e = 2 r + c) for the device's
// v = (I, X, i D, Z), c = R v, w = (c_I, c_X, -i c_D, c_Z), x' = butterflies(w) = S x is
// R = (1/4) d fwd(S fwd(.)) conj(d), d = i on D.
static void pauli1_fwd(c128 *x)
{
    const c128 a = x[0], b = x[1], c = x[2], d = x[3];
    x[0] = a + d, x[1] = b + c, x[2] = b - c, x[3] = a - d;
}

void pauli_transfer1(const c128 *S, double R[4][4])
{
    for (int f = 0; f < 4; f++) {
        c128 col[4] = {};
        col[f] = 1.0;
        pauli1_fwd(col);
        c128 sc[4];
        for (int e = 0; e < 4; e++) {
            c128 acc = 0;
            for (int g = 0; g < 4; g++) acc += S[4 * e + g] * col[g];
            sc[e] = acc;
        }
        pauli1_fwd(sc);
        for (int e = 0; e < 4; e++) {
            c128 z = sc[e] / 4.0;
            if (e == 2) z *= c128(0, 1);
            if (f == 2) z *= c128(0, -1);
            R[e][f] = std::abs(z.real()) < kTransferZero ? 0.0 : z.real();
        }
    }
}

static void push_transfer1(const c128 *S, std::vector<float2> &out)
{
    double R[4][4];
    pauli_transfer1(S, R);
    for (int e = 0; e < 4; e++)
        for (int f = 0; f < 4; f++) out.push_back(make_float2((float)R[e][f], (float)R[e][f]));
}

// Hermitian passes: enumeration order of the tile bits outside a phase (positions pos[0..np)).
// The first bits are the ones whose shared-memory bank pairs (bits 0..3 of herm_phys) are
// linearly independent, so that the 32 groups a warp handles at once spread over all 16
// bank pairs (8 when bit 0 is a phase bit); the rest follow in ascending order.
static void herm_group_order(const FPass &fp, FPhase &f, int np)
{
    unsigned in_phase = 0;
    for (int a = 0; a < np; a++) in_phase |= 1u << f.pos[a];
    int order[16], no = 0;
    unsigned basis[4];
    int nb = 0;
    bool taken[16] = {};
    for (int b = 0; b < fp.TB && nb < 4; b++) {
        if (in_phase & (1u << b)) continue;
        unsigned v = herm_phys(1u << b) & 15u;
        for (int i = 0; i < nb; i++) v = std::min(v, v ^ basis[i]);
        if (!v) continue;
        basis[nb++] = v;
        order[no++] = b;
        taken[b] = true;
    }
    for (int b = 0; b < fp.TB; b++)
        if (!(in_phase & (1u << b)) && !taken[b]) order[no++] = b;
    for (int i = 0; i < no && i < 12; i++) f.opos[i] = (int8_t)order[i];
}

void append_tile_plan(const std::vector<PassPlan> &plan, int n, int tbmax, TilePlan &out, bool herm)
{
    for (const PassPlan &pp : plan) {
        FPass fp{};
        tile_layout(pp.Q, n, tbmax, fp, herm);
        fp.nphase = (int)pp.phases.size();
        fp.phase0 = (int)out.phases.size();
        for (const PhasePlan &ph : pp.phases) {
            FPhase f{};
            f.nq = ph.nq == 1 ? PH_ONE : ph.product ? PH_PRODUCT : PH_TWO;
            f.coef = (int)out.coefs.size();
            if (ph.nq == 2) {
                f.pos[0] = (int8_t)tile_pos(fp, 2 * n - 1 - ph.qa);
                f.pos[1] = (int8_t)tile_pos(fp, 2 * n - 1 - ph.qb);
                f.pos[2] = (int8_t)tile_pos(fp, n - 1 - ph.qa);
                f.pos[3] = (int8_t)tile_pos(fp, n - 1 - ph.qb);
                if (ph.product) out.nphasep++;
                else out.nphase2++;
            } else {
                f.pos[0] = (int8_t)tile_pos(fp, 2 * n - 1 - ph.qa);
                f.pos[1] = (int8_t)tile_pos(fp, n - 1 - ph.qa);
                out.nphase1++;
            }
            if (herm) herm_group_order(fp, f, ph.nq == 2 ? 4 : 2);
            if (ph.S.empty()) {
                // structure-only plan (width search): no coefficients
            } else if (f.nq == PH_TWO) {
                double R[16][16];
                pauli_transfer(ph.S, R);
                for (int in = 0; in < 16; in++)
                    for (int pr = 0; pr < 8; pr++)
                        out.coefs.push_back(make_float2((float)R[2 * pr][in], (float)R[2 * pr + 1][in]));
            } else if (f.nq == PH_PRODUCT) {
                push_transfer1(ph.S.data(), out.coefs);
                push_transfer1(ph.S.data() + 16, out.coefs);
            } else {
                push_transfer1(ph.S.data(), out.coefs);
            }
            out.phases.push_back(f);
        }
        out.passes.push_back(fp);
        out.smem.push_back(tile_smem_bytes(fp.TB, fp.L));
    }
}

}  // namespace qcw
