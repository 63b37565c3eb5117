// Device side of a fused pass over one tile: cp.async load into shared memory, the pass's
// phases applied in place, write-back.  Used by k_fused_pass (one tile per CTA) and by the
// batched persistent kernel (a CTA walks all tiles of all passes of one circuit).
//
// A phase is a composed superoperator on one or two qubits of the pass.  A two-qubit phase
// gathers 16-element groups (the row quartet x column quartet of Sec. 3.2 for the phase's
// qubits), a one-qubit phase 4-element groups (row pair x column pair, Sec. 3.1); each
// group is multiplied by the phase superoperator and scattered back.  Groups of one phase
// are disjoint, so no atomics are needed.
#pragma once
#include "qcw_device.cuh"
#include "tile.h"

namespace qcw {

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned ins0u(unsigned x, int p)
{
    unsigned lo = x & ((1u << p) - 1u);
    return ((x ^ lo) << 1) | lo;
}

// Packed FP32 (two lanes per register pair): d = a * b + c element-wise.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;\n" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;\n" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ float2 unpack2(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;\n" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ unsigned long long pack2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};\n" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

// Coefficient pairs A = (Re S[2p][f], Re S[2p+1][f]) and B = (Im S[2p][f], Im S[2p+1][f]) at a
// 32-bit shared address plus an immediate offset; volatile so that the compiler re-reads them
// (one broadcast per warp) instead of hoisting a phase's 256 coefficients into registers.
template <int OFF>
__device__ __forceinline__ void lds_coef(unsigned addr, unsigned long long &A, unsigned long long &B)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2+%3];\n" : "=l"(A), "=l"(B) : "r"(addr), "n"(OFF));
}

// Coefficient pairs OFF / 8 and OFF / 8 + 1 of input f: from shared memory (PRM false, S a
// shared-memory array, sf its 32-bit address plus 64 f) or by plain loads from S (PRM true: S
// points into the kernel's parameter block, read through the constant cache).
template <bool PRM, int OFF>
__device__ __forceinline__ void coef_pairs(const float2 *__restrict__ S, unsigned sf, int f, unsigned long long &A,
                                           unsigned long long &B)
{
    if (PRM) {
        const unsigned long long *p = reinterpret_cast<const unsigned long long *>(S) + 8 * f + OFF / 8;
        A = p[0];
        B = p[1];
    } else {
        lds_coef<OFF>(sf, A, B);
    }
}

// Shared-memory offset of the first member of group g of a phase (members then differ by the
// phase deltas).  SWZ (Hermitian passes, swizzled tile): g's bits go to the phase's outside
// bits in the order opos lists them and the result is mapped by herm_phys; otherwise they go
// to the outside bits in ascending order (insert a zero at each sorted phase position).
template <bool SWZ, int NPOS>
__device__ __forceinline__ unsigned group_base(unsigned g, const FPhase &F, const int (&p)[NPOS], int nout)
{
    if (SWZ) {
        unsigned b = 0;
#pragma unroll
        for (int i = 0; i < 12; i++)
            if (i < nout) b |= ((g >> i) & 1u) << F.opos[i];
        return herm_phys(b);
    }
    unsigned b = g;
#pragma unroll
    for (int a = 0; a < NPOS; a++) b = ins0u(b, p[a]);
    return b;
}

// Logical (unswizzled) tile index of the first member of group g of a Hermitian-pass phase.
__device__ __forceinline__ unsigned group_logical(unsigned g, const FPhase &F, int nout)
{
    unsigned b = 0;
#pragma unroll
    for (int i = 0; i < 12; i++)
        if (i < nout) b |= ((g >> i) & 1u) << F.opos[i];
    return b;
}

// Half storage (Hermitian passes): members whose tile element (er, ec) has
// (er >> s) < (ec >> s) were copied from the mirror tile and must be conjugated when the
// pass's first phase reads them; s = 6 turns this off.  Flips the sign of the imaginary half.
__device__ __forceinline__ unsigned long long conj_if(unsigned long long x, unsigned logical, int s)
{
    const bool c = (logical >> (6 + s)) < ((logical & 63u) >> s);
    return c ? x ^ 0x8000000000000000ull : x;
}

// The same test for the 16 members of a two-qubit group: R = er >> s and C = ec >> s of a
// member are the group base's plus the contributions of the member's phase bits that fall in
// the top region (positions pos[0], pos[1] are row bits, pos[2], pos[3] column bits).
struct ConjTop {
    unsigned ra, rb, ca, cb;  // top-region contribution of each phase position
};

__device__ __forceinline__ ConjTop conj_top(const FPhase &F, int s)
{
    auto top = [&](int pos, bool row) -> unsigned {
        const int sh = row ? 6 + s : s;
        if (row ? pos < 6 : pos >= 6) return 0u;
        return pos >= sh ? 1u << (pos - sh) : 0u;
    };
    return ConjTop{top(F.pos[0], true), top(F.pos[1], true), top(F.pos[2], false), top(F.pos[3], false)};
}

__device__ __forceinline__ void conj_group16(unsigned long long (&x)[16], unsigned logical_base, int s, const ConjTop &T)
{
    const unsigned R0 = logical_base >> (6 + s), C0 = (logical_base & 63u) >> s;
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const unsigned R = R0 | ((e & 8) ? T.ra : 0u) | ((e & 4) ? T.rb : 0u);
        const unsigned C = C0 | ((e & 2) ? T.ca : 0u) | ((e & 1) ? T.cb : 0u);
        if (R < C) x[e] ^= 0x8000000000000000ull;
    }
}

template <bool SWZ>
__device__ __forceinline__ unsigned member_delta(int pos)
{
    return SWZ ? herm_phys(1u << pos) : 1u << pos;
}

__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;\n" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Pauli index (two bits per qubit, as the member index) with an odd number of D components.
__host__ __device__ constexpr bool pauli_odd_idx(int e)
{
    return (((e >> 3) & 1) && !((e >> 1) & 1)) != (((e >> 2) & 1) && !(e & 1));
}

// Butterflies on one qubit of a 16-member group (packed complex), in place: the members
// (b00, b01, b10, b11) of the qubit's (row, column) bits at offsets (0, S2, S1, S1 + S2) from
// O become (b00 + b11, b01 + b10, b01 - b10, b00 - b11) = (I, X, D, Z).  Applied twice this
// gives 2x the input, so the same butterflies also return from (I, X, D, Z).
template <int S1, int S2, int O>
__device__ __forceinline__ void pauli_quad(unsigned long long (&x)[16])
{
    const unsigned long long a = x[O], b = x[O + S2], c = x[O + S1], d = x[O + S1 + S2];
    x[O] = fadd2(a, d);
    x[O + S2] = fadd2(b, c);
    x[O + S1] = fsub2(b, c);
    x[O + S1 + S2] = fsub2(a, d);
}

// Both qubits of a two-qubit phase: qubit a on bits (e3, e1), qubit b on bits (e2, e0).
__device__ __forceinline__ void pauli_butterflies(unsigned long long (&x)[16])
{
    pauli_quad<8, 2, 0>(x), pauli_quad<8, 2, 1>(x), pauli_quad<8, 2, 4>(x), pauli_quad<8, 2, 5>(x);
    pauli_quad<4, 1, 0>(x), pauli_quad<4, 1, 2>(x), pauli_quad<4, 1, 8>(x), pauli_quad<4, 1, 10>(x);
}

// Two-qubit phase on every 16-member group (the row quartet x column quartet of Sec. 3.2 for
// the phase's qubits), x' = S x, computed in the Pauli basis of the two qubits: forward
// butterflies (additions only), v = the Pauli coefficients (i on the members with an odd
// number of D components), c = R v with R the real transfer matrix (one packed FMA per
// coefficient: R[e][f] times the real and imaginary parts of v_f, two outputs per register
// pair), back to the butterfly basis (-i on the odd members) and inverse butterflies.  Half
// the multiply-adds of the complex 16 x 16 product, and half the coefficient bytes.
// Member offsets combine by XOR: without the swizzle they are disjoint bits, with it the map
// is linear.
// G groups per thread (g, g + NT, ...) share every coefficient load.
template <int G, int NT = kTileThreads, bool SWZ = false, bool PRM = false>
__device__ __forceinline__ void tile_phase2(float2 *__restrict__ tile, int TB, const FPhase &F,
                                            const float2 *__restrict__ S, int conj_s = 6)
{
    const unsigned d0 = member_delta<SWZ>(F.pos[0]), d1 = member_delta<SWZ>(F.pos[1]),
                   d2 = member_delta<SWZ>(F.pos[2]), d3 = member_delta<SWZ>(F.pos[3]);
    int p[4] = {F.pos[0], F.pos[1], F.pos[2], F.pos[3]};
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = a + 1; b < 4; b++)
            if (p[b] < p[a]) { int t = p[a]; p[a] = p[b]; p[b] = t; }
    const unsigned ng = 1u << (TB - 4);
    const unsigned sbase = smem_u32(S);
    unsigned long long *t64 = reinterpret_cast<unsigned long long *>(tile);
    auto member = [&](int e) {
        return ((e & 8) ? d0 : 0u) ^ ((e & 4) ? d1 : 0u) ^ ((e & 2) ? d2 : 0u) ^ ((e & 1) ? d3 : 0u);
    };
    for (unsigned g0 = threadIdx.x; g0 < ng; g0 += G * NT) {
        unsigned base[G];
        unsigned long long x[G][16];
#pragma unroll
        for (int j = 0; j < G; j++) {
            unsigned bl = 0;
            if (SWZ) {
                bl = group_logical(g0 + j * NT, F, TB - 4);
                base[j] = herm_phys(bl);
            } else {
                base[j] = group_base<SWZ>(g0 + j * NT, F, p, TB - 4);
            }
#pragma unroll
            for (int e = 0; e < 16; e++) x[j][e] = t64[base[j] ^ member(e)];
            if (SWZ && conj_s < 6) conj_group16(x[j], bl, conj_s, conj_top(F, conj_s));
            pauli_butterflies(x[j]);
        }
        unsigned long long R[G][8], I[G][8];
#pragma unroll
        for (int j = 0; j < G; j++)
#pragma unroll
            for (int q = 0; q < 8; q++) R[j][q] = I[j][q] = 0ull;
#pragma unroll
        for (int f = 0; f < 16; f++) {
            unsigned long long xr[G], xi[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const float2 u = unpack2(x[j][f]);
                xr[j] = pauli_odd_idx(f) ? pack2(-u.y, -u.y) : pack2(u.x, u.x);
                xi[j] = pauli_odd_idx(f) ? pack2(u.x, u.x) : pack2(u.y, u.y);
            }
            const unsigned sf = sbase + 64u * (unsigned)f;  // input f: 8 pairs x 8 bytes
#define QCW_PAULI_PAIRS(Q)                                 \
    {                                                      \
        unsigned long long A, B;                           \
        coef_pairs<PRM, 8 * (Q)>(S, sf, f, A, B);          \
        _Pragma("unroll") for (int j = 0; j < G; j++)      \
        {                                                  \
            R[j][(Q)] = ffma2(A, xr[j], R[j][(Q)]);        \
            I[j][(Q)] = ffma2(A, xi[j], I[j][(Q)]);        \
            R[j][(Q) + 1] = ffma2(B, xr[j], R[j][(Q) + 1]); \
            I[j][(Q) + 1] = ffma2(B, xi[j], I[j][(Q) + 1]); \
        }                                                  \
    }
            QCW_PAULI_PAIRS(0) QCW_PAULI_PAIRS(2) QCW_PAULI_PAIRS(4) QCW_PAULI_PAIRS(6)
#undef QCW_PAULI_PAIRS
        }
#pragma unroll
        for (int j = 0; j < G; j++) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const float2 re = unpack2(R[j][q]), im = unpack2(I[j][q]);
                x[j][2 * q] = pauli_odd_idx(2 * q) ? pack2(im.x, -re.x) : pack2(re.x, im.x);
                x[j][2 * q + 1] = pauli_odd_idx(2 * q + 1) ? pack2(im.y, -re.y) : pack2(re.y, im.y);
            }
            pauli_butterflies(x[j]);
#pragma unroll
            for (int e = 0; e < 16; e++) t64[base[j] ^ member(e)] = x[j][e];
        }
    }
}

// One qubit in the Pauli basis, on the quartet of x at (O, O + S2, O + S1, O + S1 + S2) after
// the butterflies (I, X, D, Z): v = (I, X, i D, Z), c = R v with R the qubit's real 4 x 4
// transfer matrix (coefficients as duplicated pairs (R[e][f], R[e][f]), row-major), back to
// (c_I, c_X, -i c_D, c_Z) for the inverse butterflies.
template <int S1, int S2, int O>
__device__ __forceinline__ void pauli_apply4(unsigned long long (&x)[16], const unsigned long long (&r)[16])
{
    const float2 d = unpack2(x[O + S1]);
    const unsigned long long v[4] = {x[O], x[O + S2], pack2(-d.y, d.x), x[O + S1 + S2]};
    unsigned long long c[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        c[e] = 0ull;
#pragma unroll
        for (int f = 0; f < 4; f++) c[e] = ffma2(r[4 * e + f], v[f], c[e]);
    }
    const float2 cd = unpack2(c[2]);
    x[O] = c[0];
    x[O + S2] = c[1];
    x[O + S1] = pack2(cd.y, -cd.x);
    x[O + S1 + S2] = c[3];
}

// One-qubit phase on every (row pair x column pair) group, in the Pauli basis of the qubit:
// butterflies, the real 4 x 4 transfer matrix, butterflies back.
template <int NT = kTileThreads, bool SWZ = false>
__device__ __forceinline__ void tile_phase1(float2 *__restrict__ tile, int TB, const FPhase &F,
                                            const float2 *__restrict__ S, int conj_s = 6)
{
    const int pr = F.pos[0], pc = F.pos[1];
    const int p[2] = {pr < pc ? pr : pc, pr < pc ? pc : pr};
    const unsigned dr = member_delta<SWZ>(pr), dc = member_delta<SWZ>(pc);
    const unsigned long long *S64 = reinterpret_cast<const unsigned long long *>(S);
    unsigned long long r[16];
#pragma unroll
    for (int i = 0; i < 16; i++) r[i] = S64[i];
    unsigned long long *t64 = reinterpret_cast<unsigned long long *>(tile);
    const unsigned ng = 1u << (TB - 2);
    for (unsigned g = threadIdx.x; g < ng; g += NT) {
        const unsigned b = group_base<SWZ>(g, F, p, TB - 2);
        unsigned long long x[16];  // members 00, 01, 10, 11 in slots 0, 1, 2, 3 (S1 = 2, S2 = 1)
        x[0] = t64[b], x[1] = t64[b ^ dc], x[2] = t64[b ^ dr], x[3] = t64[b ^ dr ^ dc];
        if (SWZ && conj_s < 6) {
            const unsigned bl = group_logical(g, F, TB - 2), lr = 1u << pr, lc = 1u << pc;
            x[0] = conj_if(x[0], bl, conj_s), x[1] = conj_if(x[1], bl | lc, conj_s);
            x[2] = conj_if(x[2], bl | lr, conj_s), x[3] = conj_if(x[3], bl | lr | lc, conj_s);
        }
        pauli_quad<2, 1, 0>(x);
        pauli_apply4<2, 1, 0>(x, r);
        pauli_quad<2, 1, 0>(x);
        t64[b] = x[0], t64[b ^ dc] = x[1], t64[b ^ dr] = x[2], t64[b ^ dr ^ dc] = x[3];
    }
}

// Product phase: two one-qubit superoperators (S_a on (r_a, c_a) and S_b on (r_b, c_b); they
// commute) on every 16-member group, in one shared-memory round trip and in the Pauli basis:
// butterflies on both qubits, R_a on every quartet of qubit a, R_b on every quartet of qubit
// b, butterflies back.  Member index e = 8 r_a + 4 r_b + 2 c_a + c_b.
template <int NT = kTileThreads, bool SWZ = false>
__device__ __forceinline__ void tile_phase_prod(float2 *__restrict__ tile, int TB, const FPhase &F,
                                                const float2 *__restrict__ S, int conj_s = 6)
{
    const unsigned d0 = member_delta<SWZ>(F.pos[0]), d1 = member_delta<SWZ>(F.pos[1]),
                   d2 = member_delta<SWZ>(F.pos[2]), d3 = member_delta<SWZ>(F.pos[3]);
    int p[4] = {F.pos[0], F.pos[1], F.pos[2], F.pos[3]};
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = a + 1; b < 4; b++)
            if (p[b] < p[a]) { int t = p[a]; p[a] = p[b]; p[b] = t; }
    const unsigned long long *S64 = reinterpret_cast<const unsigned long long *>(S);
    unsigned long long *t64 = reinterpret_cast<unsigned long long *>(tile);
    auto member = [&](int e) {
        return ((e & 8) ? d0 : 0u) ^ ((e & 4) ? d1 : 0u) ^ ((e & 2) ? d2 : 0u) ^ ((e & 1) ? d3 : 0u);
    };
    const unsigned ng = 1u << (TB - 4);
    for (unsigned g = threadIdx.x; g < ng; g += NT) {
        const unsigned base = group_base<SWZ>(g, F, p, TB - 4);
        unsigned long long x[16];
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = t64[base ^ member(e)];
        if (SWZ && conj_s < 6) conj_group16(x, group_logical(g, F, TB - 4), conj_s, conj_top(F, conj_s));
        pauli_butterflies(x);
        unsigned long long r[16];
#pragma unroll
        for (int i = 0; i < 16; i++) r[i] = S64[i];
        pauli_apply4<8, 2, 0>(x, r), pauli_apply4<8, 2, 1>(x, r), pauli_apply4<8, 2, 4>(x, r),
            pauli_apply4<8, 2, 5>(x, r);
#pragma unroll
        for (int i = 0; i < 16; i++) r[i] = S64[16 + i];
        pauli_apply4<4, 1, 0>(x, r), pauli_apply4<4, 1, 2>(x, r), pauli_apply4<4, 1, 8>(x, r),
            pauli_apply4<4, 1, 10>(x, r);
        pauli_butterflies(x);
#pragma unroll
        for (int e = 0; e < 16; e++) t64[base ^ member(e)] = x[e];
    }
}

// Apply one phase whose coefficients are at S (shared or global memory).
// PRM: S points into the kernel parameter block (see coef_pairs); that caller (the
// warp-specialised pass) has the registers for two groups per thread in two-qubit phases, which
// halves the coefficient reads and doubles the independent work per thread.
// conj_s < 6: half-storage conjugation of the members read (see conj_if), on a pass's first phase.
template <int NT = kTileThreads, bool UNROLL = true, bool SWZ = false, bool PRM = false>
__device__ __forceinline__ void tile_apply_phase(float2 *__restrict__ tile, int TB, const FPhase &F,
                                                 const float2 *__restrict__ S, int conj_s = 6)
{
    if (F.nq == PH_TWO) {
        if (PRM) tile_phase2<2, NT, SWZ, PRM>(tile, TB, F, S, conj_s);
        else tile_phase2<1, NT, SWZ, PRM>(tile, TB, F, S, conj_s);
    } else if (F.nq == PH_PRODUCT) {
        tile_phase_prod<NT, SWZ>(tile, TB, F, S, conj_s);
    } else {
        tile_phase1<NT, SWZ>(tile, TB, F, S, conj_s);
    }
}

// Shared-memory carve-up for a pass: tile | high-offset table | one superoperator.
struct TileSmem {
    float2 *tile;
    uint64_t *hoff;
    float2 *S;
};

__device__ __forceinline__ TileSmem tile_smem(unsigned char *smem, int TB, int L)
{
    TileSmem t;
    t.tile = reinterpret_cast<float2 *>(smem);
    t.hoff = reinterpret_cast<uint64_t *>(t.tile + (1u << TB));
    t.S = reinterpret_cast<float2 *>(t.hoff + ((1u << (TB - L)) | 1u) + 1u);  // 16-byte aligned
    return t;
}

// Offsets (relative to the tile base) of the 2^(TB-L) contiguous runs of a tile.
template <int NT>
__device__ __forceinline__ void tile_hoff_nt(const FPass &P, uint64_t *hoff)
{
    const int TB = P.TB, L = P.L;
    for (unsigned i = threadIdx.x; i < (1u << (TB - L)); i += NT) {
        uint64_t o = 0;
        for (int j = 0; j < TB - L; j++) o |= (uint64_t)((i >> j) & 1u) << P.tbits[L + j];
        hoff[i] = o;
    }
}

__device__ __forceinline__ void tile_hoff(const FPass &P, uint64_t *hoff)
{
    const int TB = P.TB, L = P.L;
    for (unsigned i = threadIdx.x; i < (1u << (TB - L)); i += kTileThreads) {
        uint64_t o = 0;
        for (int j = 0; j < TB - L; j++) o |= (uint64_t)((i >> j) & 1u) << P.tbits[L + j];
        hoff[i] = o;
    }
}

__device__ __forceinline__ uint64_t tile_base(const FPass &P, uint64_t tile)
{
    uint64_t base = 0;
    for (int j = 0; j < P.nother; j++) base |= ((tile >> j) & 1ull) << P.obits[j];
    return base;
}

// Bring tile `t` of pass P into shared memory (or, with init, write |0..0><0..0| there: the
// element of global index 0 is tile index 0 of tile 0).  Expects sm.hoff filled for P.
__device__ __forceinline__ void tile_load(const float2 *__restrict__ rho, const FPass &P, uint64_t t, const TileSmem &sm,
                                          bool init)
{
    const int TB = P.TB, L = P.L;
    const unsigned nvec = 1u << (TB - 1);
    if (init) {
        float4 *t4 = reinterpret_cast<float4 *>(sm.tile);
        for (unsigned v = threadIdx.x; v < nvec; v += kTileThreads)
            t4[v] = (t == 0 && v == 0) ? make_float4(1.f, 0.f, 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const uint64_t base = tile_base(P, t);
        const unsigned lmask = (1u << L) - 1u;
        for (unsigned v = threadIdx.x; v < nvec; v += kTileThreads) {
            unsigned e = 2 * v;
            cp_async16(&sm.tile[e], rho + base + sm.hoff[e >> L] + (e & lmask));
        }
        cp_async_wait_all();
    }
    __syncthreads();
}

// Apply the phases of pass P to the tile in shared memory (coefficients staged per phase).
__device__ __forceinline__ void tile_phases(const FPass &P, const FPhase *__restrict__ phases,
                                            const float2 *__restrict__ coefs, const TileSmem &sm)
{
    const int TB = P.TB;
    for (int ph = 0; ph < P.nphase; ph++) {
        const FPhase F = phases[P.phase0 + ph];
        const int ncoef = phase_coefs(F.nq);
        for (int i = threadIdx.x; i < ncoef; i += kTileThreads) sm.S[i] = coefs[F.coef + i];
        __syncthreads();
        tile_apply_phase(sm.tile, TB, F, sm.S);
        __syncthreads();
    }
}

template <int NT, bool SWZ = false>
__device__ __forceinline__ void tile_store_nt(float2 *__restrict__ rho, const FPass &P, uint64_t t,
                                              const float2 *__restrict__ tile, const uint64_t *__restrict__ hoff)
{
    const int TB = P.TB, L = P.L;
    const uint64_t base = tile_base(P, t);
    const unsigned nvec = 1u << (TB - 1);
    const unsigned lmask = (1u << L) - 1u;
    const float4 *t4 = reinterpret_cast<const float4 *>(tile);
    for (unsigned v = threadIdx.x; v < nvec; v += NT) {
        unsigned e = 2 * v;
        *reinterpret_cast<float4 *>(rho + base + hoff[e >> L] + (e & lmask)) = t4[SWZ ? herm_phys(e) >> 1 : v];
    }
}

__device__ __forceinline__ void tile_store(float2 *__restrict__ rho, const FPass &P, uint64_t t, const TileSmem &sm)
{
    const int TB = P.TB, L = P.L;
    const uint64_t base = tile_base(P, t);
    const unsigned nvec = 1u << (TB - 1);
    const unsigned lmask = (1u << L) - 1u;
    const float4 *t4 = reinterpret_cast<const float4 *>(sm.tile);
    for (unsigned v = threadIdx.x; v < nvec; v += kTileThreads) {
        unsigned e = 2 * v;
        *reinterpret_cast<float4 *>(rho + base + sm.hoff[e >> L] + (e & lmask)) = t4[v];
    }
}

// Load tile `t` of pass P, apply its phases, store it.  Expects sm.hoff filled for P and a
// __syncthreads() after that; the caller synchronises before reusing shared memory.
__device__ __forceinline__ void tile_process(float2 *__restrict__ rho, const FPass &P, uint64_t t,
                                             const FPhase *__restrict__ phases, const float2 *__restrict__ coefs,
                                             const TileSmem &sm, bool init = false)
{
    tile_load(rho, P, t, sm, init);
    tile_phases(P, phases, coefs, sm);
    tile_store(rho, P, t, sm);
}

// ------------------------------------------------------------------ mbarriers (CTA scope)
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Arrive on `bar` once every cp.async this thread issued before has landed (the barrier's
// expected count includes this arrival).
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` of `bar` to complete, giving up after `limit` polls
// (each failed poll also sleeps ~256 ns); returns whether the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit)
{
    for (unsigned it = 0;; it++) {
        if (mbar_test(bar, parity)) return true;
        if (it >= limit) return false;
        __nanosleep(256);
    }
}

// AND of `pred` over the `count` threads that take part in named barrier `id` (also a
// barrier among them).
__device__ __forceinline__ bool bar_and(int id, int count, bool pred)
{
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

}  // namespace qcw
