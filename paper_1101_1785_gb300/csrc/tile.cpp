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
                for (int in = 0; in < 16; in++)
                    for (int pr = 0; pr < 8; pr++) {
                        const c128 a = ph.S[(size_t)(2 * pr) * 16 + in], b = ph.S[(size_t)(2 * pr + 1) * 16 + in];
                        out.coefs.push_back(make_float2((float)a.real(), (float)b.real()));
                        out.coefs.push_back(make_float2((float)a.imag(), (float)b.imag()));
                    }
            } else {
                for (const c128 &z : ph.S) out.coefs.push_back(make_float2((float)z.real(), (float)z.imag()));
            }
            out.phases.push_back(f);
        }
        out.passes.push_back(fp);
        out.smem.push_back(tile_smem_bytes(fp.TB, fp.L));
    }
}

}  // namespace qcw
