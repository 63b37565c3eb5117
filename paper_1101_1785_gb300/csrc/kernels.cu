// Plain (one launch per operation) kernels of the qcw library and the FP64 readouts.
//
// Every evolution kernel is one HBM pass over rho: it gathers the members of one group
// (a pair of row labels x a pair of column labels for a one-qubit operation, Sec. 3.1;
// quartet x quartet for two qubits, Sec. 3.2), applies the update and scatters it back.
// Threads take consecutive groups, so a warp reads consecutive column labels (coalesced);
// when no struck bit is bit 0, each thread takes two neighbouring groups and moves them
// as float4.
#include "qcw_device.cuh"
#include "qcw_internal.h"

namespace qcw {

static inline unsigned grid_for(uint64_t items, int threads, int nsm)
{
    uint64_t g = (items + threads - 1) / threads;
    uint64_t cap = (uint64_t)nsm * 32ull;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// --------------------------------------------------------------------- one-qubit gate
// X = [[x00, x01], [x10, x11]] (row bit, column bit).  Rows: X <- U X (Eq. resmat1 on every
// column).  Columns: X <- X U^dagger (Eq. resmat1 with conj(U) on every row).
__device__ __forceinline__ void gate1_quartet(const Gate1Params &p, bool rok, bool cok, float2 &x00,
                                              float2 &x01, float2 &x10, float2 &x11)
{
    if (rok) {
        float2 y00 = make_float2(0, 0), y01 = y00, y10 = y00, y11 = y00;
        cfma(y00, p.u[0], x00); cfma(y00, p.u[1], x10);
        cfma(y10, p.u[2], x00); cfma(y10, p.u[3], x10);
        cfma(y01, p.u[0], x01); cfma(y01, p.u[1], x11);
        cfma(y11, p.u[2], x01); cfma(y11, p.u[3], x11);
        x00 = y00; x01 = y01; x10 = y10; x11 = y11;
    }
    if (cok) {
        float2 z00 = make_float2(0, 0), z01 = z00, z10 = z00, z11 = z00;
        cfmac(z00, p.u[0], x00); cfmac(z00, p.u[1], x01);
        cfmac(z01, p.u[2], x00); cfmac(z01, p.u[3], x01);
        cfmac(z10, p.u[0], x10); cfmac(z10, p.u[1], x11);
        cfmac(z11, p.u[2], x10); cfmac(z11, p.u[3], x11);
        x00 = z00; x01 = z01; x10 = z10; x11 = z11;
    }
}

// pc == 0: the column pair is adjacent (one float4 per row).
__global__ void k_gate1_lsb(float2 *__restrict__ rho, uint64_t nq, Gate1Params p)
{
    const uint64_t dr = 1ull << p.pr;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nq;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = insert0(insert0(t, 0), p.pr);
        float4 a = *reinterpret_cast<const float4 *>(rho + g);
        float4 b = *reinterpret_cast<const float4 *>(rho + g + dr);
        float2 x00 = make_float2(a.x, a.y), x01 = make_float2(a.z, a.w);
        float2 x10 = make_float2(b.x, b.y), x11 = make_float2(b.z, b.w);
        gate1_quartet(p, (g & p.cmask_r) == p.cmask_r, (g & p.cmask_c) == p.cmask_c, x00, x01, x10, x11);
        *reinterpret_cast<float4 *>(rho + g) = make_float4(x00.x, x00.y, x01.x, x01.y);
        *reinterpret_cast<float4 *>(rho + g + dr) = make_float4(x10.x, x10.y, x11.x, x11.y);
    }
}

// pc >= 1: thread s takes quartets 2s and 2s+1, which sit at labels g and g+1.
__global__ void k_gate1_vec(float2 *__restrict__ rho, uint64_t npairs, Gate1Params p)
{
    const uint64_t dc = 1ull << p.pc, dr = 1ull << p.pr;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < npairs;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = insert0(insert0(2 * s, p.pc), p.pr);
        float4 a = *reinterpret_cast<const float4 *>(rho + g);
        float4 b = *reinterpret_cast<const float4 *>(rho + g + dc);
        float4 c = *reinterpret_cast<const float4 *>(rho + g + dr);
        float4 d = *reinterpret_cast<const float4 *>(rho + g + dr + dc);
        bool rok = (g & p.cmask_r) == p.cmask_r;
        bool cok0 = (g & p.cmask_c) == p.cmask_c;
        bool cok1 = ((g + 1) & p.cmask_c) == p.cmask_c;
        float2 x00 = make_float2(a.x, a.y), x01 = make_float2(b.x, b.y);
        float2 x10 = make_float2(c.x, c.y), x11 = make_float2(d.x, d.y);
        float2 w00 = make_float2(a.z, a.w), w01 = make_float2(b.z, b.w);
        float2 w10 = make_float2(c.z, c.w), w11 = make_float2(d.z, d.w);
        gate1_quartet(p, rok, cok0, x00, x01, x10, x11);
        gate1_quartet(p, rok, cok1, w00, w01, w10, w11);
        *reinterpret_cast<float4 *>(rho + g) = make_float4(x00.x, x00.y, w00.x, w00.y);
        *reinterpret_cast<float4 *>(rho + g + dc) = make_float4(x01.x, x01.y, w01.x, w01.y);
        *reinterpret_cast<float4 *>(rho + g + dr) = make_float4(x10.x, x10.y, w10.x, w10.y);
        *reinterpret_cast<float4 *>(rho + g + dr + dc) = make_float4(x11.x, x11.y, w11.x, w11.y);
    }
}

void launch_gate1(const Gate1Params &p, float2 *rho, int n, int nsm, cudaStream_t s)
{
    uint64_t nq = 1ull << (2 * n - 2);
    const int th = 256;
    if (p.pc == 0) {
        k_gate1_lsb<<<grid_for(nq, th, nsm), th, 0, s>>>(rho, nq, p);
    } else {
        k_gate1_vec<<<grid_for(nq / 2, th, nsm), th, 0, s>>>(rho, nq / 2, p);
    }
}

// --------------------------------------------------------------------- 16-member groups
// Shared by the two-qubit gate and the two-qubit superoperator: X[i][j] with i the local
// row index and j the local column index, both 2*q(q1) + q(q2) (Eq. resmat2 order).
template <int V>
__device__ __forceinline__ void load16(const float2 *__restrict__ rho, uint64_t g, const uint64_t *offr,
                                       const uint64_t *offc, float2 (&x)[V][16])
{
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float2 *a = rho + g + offr[i] + offc[j];
            if (V == 2) {
                float4 v = *reinterpret_cast<const float4 *>(a);
                x[0][4 * i + j] = make_float2(v.x, v.y);
                x[V - 1][4 * i + j] = make_float2(v.z, v.w);
            } else {
                x[0][4 * i + j] = *a;
            }
        }
}

template <int V>
__device__ __forceinline__ void store16(float2 *__restrict__ rho, uint64_t g, const uint64_t *offr,
                                        const uint64_t *offc, const float2 (&x)[V][16])
{
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float2 *a = rho + g + offr[i] + offc[j];
            if (V == 2) {
                *reinterpret_cast<float4 *>(a) =
                    make_float4(x[0][4 * i + j].x, x[0][4 * i + j].y, x[V - 1][4 * i + j].x, x[V - 1][4 * i + j].y);
            } else {
                *a = x[0][4 * i + j];
            }
        }
}

__device__ __forceinline__ uint64_t group_base(uint64_t t, const int *pos)
{
    return insert0(insert0(insert0(insert0(t, pos[0]), pos[1]), pos[2]), pos[3]);
}

template <int V>
__global__ void k_gate2(float2 *__restrict__ rho, uint64_t nitems, Gate2Params p)
{
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nitems;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = group_base(V * s, p.pos);
        float2 x[V][16];
        load16<V>(rho, g, p.off_r, p.off_c, x);
#pragma unroll
        for (int v = 0; v < V; v++) {
            uint64_t gv = g + v;
            bool rok = (gv & p.cmask_r) == p.cmask_r;
            bool cok = (gv & p.cmask_c) == p.cmask_c;
            if (rok) {  // X <- V X
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    float2 y[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        y[i] = make_float2(0, 0);
#pragma unroll
                        for (int l = 0; l < 4; l++) cfma(y[i], p.u[4 * i + l], x[v][4 * l + j]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; i++) x[v][4 * i + j] = y[i];
                }
            }
            if (cok) {  // X <- X V^dagger
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    float2 y[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        y[j] = make_float2(0, 0);
#pragma unroll
                        for (int l = 0; l < 4; l++) cfmac(y[j], p.u[4 * j + l], x[v][4 * i + l]);
                    }
#pragma unroll
                    for (int j = 0; j < 4; j++) x[v][4 * i + j] = y[j];
                }
            }
        }
        store16<V>(rho, g, p.off_r, p.off_c, x);
    }
}

void launch_gate2(const Gate2Params &p, float2 *rho, int n, int nsm, cudaStream_t s)
{
    uint64_t ng = 1ull << (2 * n - 4);
    const int th = 128;
    if (p.pos[0] == 0) {
        k_gate2<1><<<grid_for(ng, th, nsm), th, 0, s>>>(rho, ng, p);
    } else {
        k_gate2<2><<<grid_for(ng / 2, th, nsm), th, 0, s>>>(rho, ng / 2, p);
    }
}

// Pauli-basis butterflies on one qubit of a 16-member group (members (b00, b01, b10, b11) at
// O, O + S2, O + S1, O + S1 + S2 become (b00 + b11, b01 + b10, b01 - b10, b00 - b11)); applied
// twice they give 2x the input.
template <int S1, int S2, int O>
__device__ __forceinline__ void pquad(float2 (&x)[16])
{
    const float2 a = x[O], b = x[O + S2], c = x[O + S1], d = x[O + S1 + S2];
    x[O] = make_float2(a.x + d.x, a.y + d.y);
    x[O + S2] = make_float2(b.x + c.x, b.y + c.y);
    x[O + S1] = make_float2(b.x - c.x, b.y - c.y);
    x[O + S1 + S2] = make_float2(a.x - d.x, a.y - d.y);
}

// Both qubits of the group: qubit 1 on member bits (3, 1), qubit 2 on (2, 0).
__device__ __forceinline__ void pbutterflies(float2 (&x)[16])
{
    pquad<8, 2, 0>(x), pquad<8, 2, 1>(x), pquad<8, 2, 4>(x), pquad<8, 2, 5>(x);
    pquad<4, 1, 0>(x), pquad<4, 1, 2>(x), pquad<4, 1, 8>(x), pquad<4, 1, 10>(x);
}

// Member index with an odd number of D components (bit pattern (row, col) = (0, 1) on a qubit).
__host__ __device__ constexpr bool podd(int e)
{
    return (((e >> 3) & 1) && !((e >> 1) & 1)) != (((e >> 2) & 1) && !(e & 1));
}

// Two-qubit superoperator on a 16-member group (Eq. rhoE2 as S = sum_k K (x) conj K), applied in
// the Pauli basis of the two qubits: butterflies, v = the coefficients (times i where odd),
// c = R v with the real transfer matrix R, -i back where odd, butterflies again.  For a
// trace-preserving S the first row of R is exactly (1/4, 0, ..., 0): the trace then changes
// only by the rounding of the butterflies, with either sign, not by the rounding of S's
// entries, whose sign is the same at every application (a drift that grows with the number of
// channels).  Half the multiply-adds of the complex 16 x 16 product as well.
template <int V>
__global__ void k_super2(float2 *__restrict__ rho, uint64_t nitems, Super2Params p)
{
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nitems;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = group_base(V * s, p.pos);
        float2 x[V][16];
        load16<V>(rho, g, p.off_r, p.off_c, x);
        float2 y[V][16];
#pragma unroll
        for (int v = 0; v < V; v++) {
            pbutterflies(x[v]);
#pragma unroll
            for (int f = 0; f < 16; f++)
                if (podd(f)) x[v][f] = make_float2(-x[v][f].y, x[v][f].x);
        }
#pragma unroll
        for (int e = 0; e < 16; e++) {
#pragma unroll
            for (int v = 0; v < V; v++) y[v][e] = make_float2(0, 0);
#pragma unroll
            for (int f = 0; f < 16; f++) {
                const float c = p.r[16 * e + f];
#pragma unroll
                for (int v = 0; v < V; v++) {
                    y[v][e].x = fmaf(c, x[v][f].x, y[v][e].x);
                    y[v][e].y = fmaf(c, x[v][f].y, y[v][e].y);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; v++) {
#pragma unroll
            for (int e = 0; e < 16; e++)
                if (podd(e)) y[v][e] = make_float2(y[v][e].y, -y[v][e].x);
            pbutterflies(y[v]);
        }
        store16<V>(rho, g, p.off_r, p.off_c, y);
    }
}

void launch_super2(const Super2Params &p, float2 *rho, int n, int nsm, cudaStream_t s)
{
    uint64_t ng = 1ull << (2 * n - 4);
    const int th = 128;
    if (p.pos[0] == 0) {
        k_super2<1><<<grid_for(ng, th, nsm), th, 0, s>>>(rho, ng, p);
    } else {
        k_super2<2><<<grid_for(ng / 2, th, nsm), th, 0, s>>>(rho, ng / 2, p);
    }
}

// --------------------------------------------------------------------- monomial two-qubit gates
// A gate with one entry u_i of modulus 1 per row, at column sigma(i), and entries among
// 1, -1, i, -i (CNOT, CZ, SWAP, iSWAP): (U rho U^dagger)_ij = u_i conj(u_j) rho_sigma(i)sigma(j),
// a permutation of each 16-member group with exact sign / quarter-turn factors -- a pure data
// movement (no rounding at all, so the trace is kept exactly), one read and one write of rho.
template <int V>
__global__ void k_mono2(float2 *__restrict__ rho, uint64_t nitems, Mono2Params p)
{
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nitems;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = group_base(V * s, p.pos);
        float2 x[V][16];
        load16<V>(rho, g, p.src_r, p.src_c, x);  // x[4 i + j] = the input member (sigma(i), sigma(j))
#pragma unroll
        for (int v = 0; v < V; v++)
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const float2 a = x[v][e], f = p.ph[e];
                x[v][e] = make_float2(f.x * a.x - f.y * a.y, f.x * a.y + f.y * a.x);
            }
        store16<V>(rho, g, p.off_r, p.off_c, x);
    }
}

void launch_mono2(const Mono2Params &p, float2 *rho, int n, int nsm, cudaStream_t s)
{
    uint64_t ng = 1ull << (2 * n - 4);
    const int th = 128;
    if (p.pos[0] == 0) {
        k_mono2<1><<<grid_for(ng, th, nsm), th, 0, s>>>(rho, ng, p);
    } else {
        k_mono2<2><<<grid_for(ng / 2, th, nsm), th, 0, s>>>(rho, ng / 2, p);
    }
}

// --------------------------------------------------------------------- one-qubit channel
// Superoperator S = sum_k K (x) conj(K) (Eq. rhoE2; a gate is S = U (x) conj U) on the quartet
// (x00, x01, x10, x11), e = 2*row+col, in the Pauli basis of the qubit: (I, X, D, Z) =
// (x00 + x11, x01 + x10, x01 - x10, x00 - x11), v = (I, X, i D, Z), c = R v with the real
// transfer matrix R, (c_I, c_X, -i c_D, c_Z) through the same butterflies gives S x.  A
// trace-preserving S has the first row of R exactly (1/2, 0, 0, 0), so the trace sees only the
// butterflies' rounding (either sign), not the fixed-sign rounding of S's entries.
__device__ __forceinline__ void super1_quartet(const Super1Params &p, float2 (&x)[4])
{
    const float2 v[4] = {make_float2(x[0].x + x[3].x, x[0].y + x[3].y),
                         make_float2(x[1].x + x[2].x, x[1].y + x[2].y),
                         make_float2(x[2].y - x[1].y, x[1].x - x[2].x),  // i (x01 - x10)
                         make_float2(x[0].x - x[3].x, x[0].y - x[3].y)};
    float2 c[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        c[e] = make_float2(0, 0);
#pragma unroll
        for (int f = 0; f < 4; f++) {
            c[e].x = fmaf(p.r[4 * e + f], v[f].x, c[e].x);
            c[e].y = fmaf(p.r[4 * e + f], v[f].y, c[e].y);
        }
    }
    const float2 d = make_float2(c[2].y, -c[2].x);  // -i c_D
    x[0] = make_float2(c[0].x + c[3].x, c[0].y + c[3].y);
    x[1] = make_float2(c[1].x + d.x, c[1].y + d.y);
    x[2] = make_float2(c[1].x - d.x, c[1].y - d.y);
    x[3] = make_float2(c[0].x - c[3].x, c[0].y - c[3].y);
}

__global__ void k_super1_lsb(float2 *__restrict__ rho, uint64_t nq, Super1Params p)
{
    const uint64_t dr = 1ull << p.pr;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nq;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = insert0(insert0(t, 0), p.pr);
        float4 a = *reinterpret_cast<const float4 *>(rho + g);
        float4 b = *reinterpret_cast<const float4 *>(rho + g + dr);
        float2 x[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y), make_float2(b.z, b.w)};
        super1_quartet(p, x);
        *reinterpret_cast<float4 *>(rho + g) = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
        *reinterpret_cast<float4 *>(rho + g + dr) = make_float4(x[2].x, x[2].y, x[3].x, x[3].y);
    }
}

__global__ void k_super1_vec(float2 *__restrict__ rho, uint64_t npairs, Super1Params p)
{
    const uint64_t dc = 1ull << p.pc, dr = 1ull << p.pr;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < npairs;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = insert0(insert0(2 * s, p.pc), p.pr);
        float4 a = *reinterpret_cast<const float4 *>(rho + g);
        float4 b = *reinterpret_cast<const float4 *>(rho + g + dc);
        float4 c = *reinterpret_cast<const float4 *>(rho + g + dr);
        float4 d = *reinterpret_cast<const float4 *>(rho + g + dr + dc);
        float2 x[4] = {make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y), make_float2(d.x, d.y)};
        float2 w[4] = {make_float2(a.z, a.w), make_float2(b.z, b.w), make_float2(c.z, c.w), make_float2(d.z, d.w)};
        super1_quartet(p, x);
        super1_quartet(p, w);
        *reinterpret_cast<float4 *>(rho + g) = make_float4(x[0].x, x[0].y, w[0].x, w[0].y);
        *reinterpret_cast<float4 *>(rho + g + dc) = make_float4(x[1].x, x[1].y, w[1].x, w[1].y);
        *reinterpret_cast<float4 *>(rho + g + dr) = make_float4(x[2].x, x[2].y, w[2].x, w[2].y);
        *reinterpret_cast<float4 *>(rho + g + dr + dc) = make_float4(x[3].x, x[3].y, w[3].x, w[3].y);
    }
}

void launch_super1(const Super1Params &p, float2 *rho, int n, int nsm, cudaStream_t s)
{
    uint64_t nq = 1ull << (2 * n - 2);
    const int th = 256;
    if (p.pc == 0) {
        k_super1_lsb<<<grid_for(nq, th, nsm), th, 0, s>>>(rho, nq, p);
    } else {
        k_super1_vec<<<grid_for(nq / 2, th, nsm), th, 0, s>>>(rho, nq / 2, p);
    }
}

// --------------------------------------------------------------------- k-qubit gate, one side
// Row side: every column is an amplitude vector and each group of 2^k row labels gets
// U (Sec. 3.3 generalised).  Column side: every row, groups of column labels, conj(U).
// Threads take consecutive labels of the other side so that a warp stays coalesced.
template <int K>
__global__ void k_gatek_side(float2 *__restrict__ rho, uint64_t ngroups, GateKParams p)
{
    constexpr int M = 1 << K;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < ngroups;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = t;
#pragma unroll
        for (int j = 0; j < K; j++) g = insert0(g, p.pos[j]);
        float2 x[M];
#pragma unroll
        for (int i = 0; i < M; i++) x[i] = rho[g + p.off[i]];
#pragma unroll
        for (int i = 0; i < M; i++) {
            float2 y = make_float2(0, 0);
#pragma unroll
            for (int l = 0; l < M; l++) cfma(y, p.u[M * i + l], x[l]);
            rho[g + p.off[i]] = y;
        }
    }
}

void launch_gatek_side(const GateKParams &p, float2 *rho, int n, int nsm, cudaStream_t s)
{
    uint64_t ng = 1ull << (2 * n - p.k);
    const int th = 128;
    unsigned gr = grid_for(ng, th, nsm);
    switch (p.k) {
    case 1: k_gatek_side<1><<<gr, th, 0, s>>>(rho, ng, p); break;
    case 2: k_gatek_side<2><<<gr, th, 0, s>>>(rho, ng, p); break;
    case 3: k_gatek_side<3><<<gr, th, 0, s>>>(rho, ng, p); break;
    case 4: k_gatek_side<4><<<gr, th, 0, s>>>(rho, ng, p); break;
    default: k_gatek_side<5><<<gr, th, 0, s>>>(rho, ng, p); break;
    }
}

// acc += x, element-wise (Kraus sums over more than two qubits).
__global__ void k_accumulate(float4 *__restrict__ acc, const float4 *__restrict__ x, uint64_t n4)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n4;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const float4 a = acc[t], b = x[t];
        acc[t] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
}

void launch_accumulate(float2 *acc, const float2 *x, int n, int nsm, cudaStream_t s)
{
    const uint64_t n4 = (1ull << (2 * n)) / 2;
    k_accumulate<<<grid_for(n4, 256, nsm), 256, 0, s>>>(reinterpret_cast<float4 *>(acc),
                                                        reinterpret_cast<const float4 *>(x), n4);
}

// --------------------------------------------------------------------- state set-up
// |0..0><0..0|.  lower (half storage: only r >= c is current): element pairs wholly above the
// diagonal are left alone (n is the register size).
__global__ void k_zero_state(float4 *__restrict__ rho4, uint64_t n4, int n, int lower)
{
    const uint64_t cmask = (1ull << n) - 1;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n4;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t g = 2 * t;
        if (lower && (g & cmask) > (g >> n)) continue;
        rho4[t] = t == 0 ? make_float4(1.f, 0.f, 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

void launch_zero_state(float2 *rho, int n, bool lower, int nsm, cudaStream_t s)
{
    uint64_t n4 = (1ull << (2 * n)) / 2;
    k_zero_state<<<grid_for(n4, 256, nsm), 256, 0, s>>>(reinterpret_cast<float4 *>(rho), n4, n, lower ? 1 : 0);
}

__global__ void k_c128_to_c64(const double2 *__restrict__ src, float2 *__restrict__ dst, uint64_t cnt)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (uint64_t)gridDim.x * blockDim.x) {
        double2 v = src[t];
        dst[t] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_c64_to_c128(const float2 *__restrict__ src, double2 *__restrict__ dst, uint64_t cnt)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (uint64_t)gridDim.x * blockDim.x) {
        float2 v = src[t];
        dst[t] = make_double2(v.x, v.y);
    }
}

void launch_c128_to_c64(const double2 *src, float2 *dst, size_t count, int nsm, cudaStream_t s)
{
    k_c128_to_c64<<<grid_for(count, 256, nsm), 256, 0, s>>>(src, dst, count);
}

void launch_c64_to_c128(const float2 *src, double2 *dst, size_t count, int nsm, cudaStream_t s)
{
    k_c64_to_c128<<<grid_for(count, 256, nsm), 256, 0, s>>>(src, dst, count);
}

// --------------------------------------------------------------------- FP64 readouts
// Reductions accumulate per thread, fold each warp with shuffles, each block through
// shared memory into `partials[block][v]`, and a one-block kernel adds the partials in
// block order: a fixed tree, so the result does not depend on scheduling.
constexpr int RED_THREADS = 256;
constexpr int MAXV = QCW_MAX_QUBITS + 2;

int reduce_blocks(int nsm) { return nsm * 4; }
int launches_per_reduce() { return 2; }

template <int NV>
__device__ __forceinline__ void block_store(double (&acc)[NV], int nv, double *partials)
{
    __shared__ double sh[RED_THREADS / 32][MAXV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        if (v < nv) {
            double s = warp_sum(acc[v]);
            if (lane == 0) sh[w][v] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0;
        for (int j = 0; j < RED_THREADS / 32; j++) s += sh[j][threadIdx.x];
        partials[(size_t)blockIdx.x * nv + threadIdx.x] = s;
    }
}

__global__ void k_fold(const double *__restrict__ partials, int nblocks, int nv, double *__restrict__ out)
{
    // one warp per value; lanes stride over blocks, then a fixed shuffle tree
    int v = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < nblocks; b += 32) s += partials[(size_t)b * nv + v];
    s = warp_sum(s);
    if (threadIdx.x == 0) out[v] = s;
}

// Diagonal: out[0] = sum Re rho_ii, out[1] = sum Im rho_ii, out[2+q] = sum over labels with
// qubit q = 1 of Re rho_ii.
__global__ void __launch_bounds__(RED_THREADS) k_diag(const float2 *__restrict__ rho, int n, double *partials)
{
    const uint64_t dim = 1ull << n;
    double acc[MAXV];
#pragma unroll
    for (int v = 0; v < MAXV; v++) acc[v] = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float2 d = rho[i * dim + i];
        double re = d.x;
        acc[0] += re;
        acc[1] += d.y;
#pragma unroll
        for (int q = 0; q < QCW_MAX_QUBITS; q++)
            if (q < n && ((i >> (n - 1 - q)) & 1)) acc[2 + q] += re;
    }
    block_store<MAXV>(acc, n + 2, partials);
}

void launch_diag_reduce(const float2 *rho, int n, double *partials, double *out, int nblocks,
                        cudaStream_t s)
{
    uint64_t dim = 1ull << n;
    uint64_t need = (dim + RED_THREADS - 1) / RED_THREADS;
    int nb = (int)(need < (uint64_t)nblocks ? need : (uint64_t)nblocks);
    k_diag<<<nb, RED_THREADS, 0, s>>>(rho, n, partials);
    k_fold<<<n + 2, 32, 0, s>>>(partials, nb, n + 2, out);
}

// Purity: sum |rho_ij|^2.  Squares and short sums in FP32 (8 elements), totals in FP64.
__global__ void __launch_bounds__(RED_THREADS) k_purity(const float4 *__restrict__ rho4, uint64_t n4, double *partials)
{
    double acc[1] = {0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (; t + 3 * stride < n4; t += 4 * stride) {
        float4 a = rho4[t], b = rho4[t + stride], c = rho4[t + 2 * stride], d = rho4[t + 3 * stride];
        float s = a.x * a.x;
        s = fmaf(a.y, a.y, s); s = fmaf(a.z, a.z, s); s = fmaf(a.w, a.w, s);
        s = fmaf(b.x, b.x, s); s = fmaf(b.y, b.y, s); s = fmaf(b.z, b.z, s); s = fmaf(b.w, b.w, s);
        s = fmaf(c.x, c.x, s); s = fmaf(c.y, c.y, s); s = fmaf(c.z, c.z, s); s = fmaf(c.w, c.w, s);
        s = fmaf(d.x, d.x, s); s = fmaf(d.y, d.y, s); s = fmaf(d.z, d.z, s); s = fmaf(d.w, d.w, s);
        acc[0] += (double)s;
    }
    for (; t < n4; t += stride) {
        float4 a = rho4[t];
        float s = a.x * a.x;
        s = fmaf(a.y, a.y, s); s = fmaf(a.z, a.z, s); s = fmaf(a.w, a.w, s);
        acc[0] += (double)s;
    }
    block_store<1>(acc, 1, partials);
}

void launch_purity(const float2 *rho, int n, double *partials, double *out, int nblocks, cudaStream_t s)
{
    uint64_t n4 = (1ull << (2 * n)) / 2;
    uint64_t need = (n4 + RED_THREADS - 1) / RED_THREADS;
    int nb = (int)(need < (uint64_t)nblocks ? need : (uint64_t)nblocks);
    k_purity<<<nb, RED_THREADS, 0, s>>>(reinterpret_cast<const float4 *>(rho), n4, partials);
    k_fold<<<1, 32, 0, s>>>(partials, nb, 1, out);
}

// Purity of a Hermitian rho from its lower triangle: sum_r |rho_rr|^2 + 2 sum_{r > c} |rho_rc|^2.
// Blocks take rows in turn; the threads of a block read the row's element pairs (2p, 2p + 1)
// with 2p <= r contiguously, four in flight, weighting the diagonal pair at the end.
__global__ void __launch_bounds__(RED_THREADS) k_purity_lower(const float4 *__restrict__ rho4, int n, double *partials)
{
    double acc[1] = {0};
    const uint64_t dim = 1ull << n, half = dim >> 1;
    for (uint64_t r = blockIdx.x; r < dim; r += gridDim.x) {
        const float4 *row = rho4 + r * half;
        const uint64_t np = r / 2 + 1;  // pairs with 2p <= r
        const uint64_t full = r / 2;    // pairs 0 .. full - 1 lie strictly below the diagonal
        float s = 0.f;
        uint64_t p = threadIdx.x;
        for (; p + 3 * RED_THREADS < full; p += 4 * RED_THREADS) {
            const float4 a = row[p], b = row[p + RED_THREADS], c = row[p + 2 * RED_THREADS], d = row[p + 3 * RED_THREADS];
            s = fmaf(a.x, a.x, s); s = fmaf(a.y, a.y, s); s = fmaf(a.z, a.z, s); s = fmaf(a.w, a.w, s);
            s = fmaf(b.x, b.x, s); s = fmaf(b.y, b.y, s); s = fmaf(b.z, b.z, s); s = fmaf(b.w, b.w, s);
            s = fmaf(c.x, c.x, s); s = fmaf(c.y, c.y, s); s = fmaf(c.z, c.z, s); s = fmaf(c.w, c.w, s);
            s = fmaf(d.x, d.x, s); s = fmaf(d.y, d.y, s); s = fmaf(d.z, d.z, s); s = fmaf(d.w, d.w, s);
        }
        for (; p < full; p += RED_THREADS) {
            const float4 a = row[p];
            s = fmaf(a.x, a.x, s); s = fmaf(a.y, a.y, s); s = fmaf(a.z, a.z, s); s = fmaf(a.w, a.w, s);
        }
        float sdiag = 0.f;
        if (threadIdx.x == 0) {  // pair 'full' holds the diagonal element (and one below it if r is odd)
            const float4 a = row[full];
            const float e0 = fmaf(a.x, a.x, a.y * a.y), e1 = fmaf(a.z, a.z, a.w * a.w);
            sdiag = (r & 1) ? fmaf(2.f, e0, e1) : e0;
        }
        (void)np;
        acc[0] += 2.0 * (double)s + (double)sdiag;
    }
    block_store<1>(acc, 1, partials);
}

// Tr[P rho] = sum_r P[r][r ^ f] rho[r ^ f][r] for a Pauli string P with flip mask f (its X and
// Y qubits' label bits): P[r][r ^ f] = (-1)^(Z qubits set in r) i^(2 (Y qubits set in r) - #Y)
// (sigma_y[0][1] = -i, sigma_y[1][0] = i).  rho[r ^ f][r] is read from the lower triangle
// (conjugated when r ^ f < r), so half storage needs no completion.  One term after the other,
// each thread sums its rows in FP64, then a fixed tree per block: partials[block][term].
__global__ void __launch_bounds__(RED_THREADS) k_pauli_expect(const float2 *__restrict__ rho, int n,
                                                              const __grid_constant__ PauliTerms T,
                                                              double *__restrict__ partials)
{
    __shared__ double sh[RED_THREADS / 32];
    const uint64_t dim = 1ull << n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = 0; s < T.count; s++) {
        const uint64_t flip = T.flip[s], ym = T.ym[s], zm = T.zm[s];
        const int ny = T.ny[s];
        double acc = 0;
        for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < dim;
             r += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t t = r ^ flip;
            float2 z = t >= r ? rho[t * dim + r] : rho[r * dim + t];
            if (t < r) z.y = -z.y;
            const int k = (2 * __popcll(r & ym) - ny) & 3;
            float v = k == 0 ? z.x : k == 1 ? -z.y : k == 2 ? -z.x : z.y;
            if (__popcll(r & zm) & 1) v = -v;
            acc += (double)v;
        }
        acc = warp_sum(acc);
        if (lane == 0) sh[w] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int j = 0; j < RED_THREADS / 32; j++) t += sh[j];
            partials[(size_t)blockIdx.x * T.count + s] = t;
        }
        __syncthreads();
    }
}

void launch_pauli_expect(const float2 *rho, int n, const PauliTerms &T, double *partials, int max_partials,
                         double *out, cudaStream_t s)
{
    const uint64_t dim = 1ull << n;
    const uint64_t need = (dim + RED_THREADS - 1) / RED_THREADS;
    uint64_t nb = (uint64_t)max_partials / (uint64_t)T.count;
    if (nb > need) nb = need;
    if (nb < 1) nb = 1;
    k_pauli_expect<<<(unsigned)nb, RED_THREADS, 0, s>>>(rho, n, T, partials);
    k_fold<<<T.count, 32, 0, s>>>(partials, (int)nb, T.count, out);
}

// out[0] = the sum of nblocks partials (fixed tree).
void launch_fold(const double *partials, int nblocks, double *out, cudaStream_t s)
{
    k_fold<<<1, 32, 0, s>>>(partials, nblocks, 1, out);
}

void launch_purity_lower(const float2 *rho, int n, double *partials, double *out, int nblocks, cudaStream_t s)
{
    const uint64_t dim = 1ull << n;
    int nb = (int)(dim < (uint64_t)nblocks ? dim : (uint64_t)nblocks);
    k_purity_lower<<<nb, RED_THREADS, 0, s>>>(reinterpret_cast<const float4 *>(rho), n, partials);
    k_fold<<<1, 32, 0, s>>>(partials, nb, 1, out);
}

// Complete rho from its lower triangle: rho[r][c] = conj(rho[c][r]) for r < c.  32 x 32 blocks:
// block (I, J), I <= J, reads the lower block (J, I) into shared memory and writes its
// conjugate transpose (only r < c inside diagonal blocks).  Loads and stores run along rows.
__global__ void __launch_bounds__(256) k_symmetrize(float2 *__restrict__ rho, int n)
{
    __shared__ float2 sh[32][33];
    const uint64_t dim = 1ull << n;
    const unsigned nb = (unsigned)(dim >> 5);
    const uint64_t nblk = (uint64_t)nb * (nb + 1) / 2;
    for (uint64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        // blk -> (I, J), I <= J, blk = J (J + 1) / 2 + I
        uint64_t J = (uint64_t)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
        while ((J + 1) * (J + 2) / 2 <= blk) J++;
        while (J * (J + 1) / 2 > blk) J--;
        const uint64_t I = blk - J * (J + 1) / 2;
        for (unsigned y = threadIdx.y; y < 32; y += 8) sh[y][threadIdx.x] = rho[(J * 32 + y) * dim + I * 32 + threadIdx.x];
        __syncthreads();
        for (unsigned y = threadIdx.y; y < 32; y += 8) {
            const uint64_t r = I * 32 + y, c = J * 32 + threadIdx.x;
            if (r < c) {
                const float2 v = sh[threadIdx.x][y];
                rho[r * dim + c] = make_float2(v.x, -v.y);
            }
        }
        __syncthreads();
    }
}

__global__ void k_symmetrize_small(float2 *__restrict__ rho, int n)
{
    const unsigned dim = 1u << n;
    for (unsigned e = threadIdx.x; e < dim * dim; e += blockDim.x) {
        const unsigned r = e >> n, c = e & (dim - 1);
        if (r < c) {
            const float2 v = rho[(size_t)c * dim + r];
            rho[e] = make_float2(v.x, -v.y);
        }
    }
}

void launch_symmetrize(float2 *rho, int n, int nsm, cudaStream_t s)
{
    if (n < 5) {
        k_symmetrize_small<<<1, 256, 0, s>>>(rho, n);
        return;
    }
    const uint64_t nb = 1ull << (n - 5), nblk = nb * (nb + 1) / 2;
    const uint64_t cap = (uint64_t)nsm * 8;
    k_symmetrize<<<(unsigned)(nblk < cap ? nblk : cap), dim3(32, 8), 0, s>>>(rho, n);
}

// Projector and renormalisation: keep (r, c) with qubit bit == m on both sides, times scale;
// every other element becomes 0 (read only when kept).  lower (half storage: only r >= c is
// current): element pairs wholly above the diagonal are left alone (n is the register size).
__global__ void k_project(float4 *__restrict__ rho4, uint64_t npairs, int pc, int pr, int m, float scale, int n,
                          int lower)
{
    const uint64_t cmask = (1ull << n) - 1;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < npairs;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = 2 * t;
        if (lower && (g & cmask) > (g >> n)) continue;
        bool rk = (int)((g >> pr) & 1) == m;
        bool k0 = rk && (int)((g >> pc) & 1) == m;
        bool k1 = rk && (int)(((g + 1) >> pc) & 1) == m;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k0 || k1) {
            float4 a = rho4[t];
            if (k0) { v.x = a.x * scale; v.y = a.y * scale; }
            if (k1) { v.z = a.z * scale; v.w = a.w * scale; }
        }
        rho4[t] = v;
    }
}

void launch_project(float2 *rho, int n, int qubit, int m, float scale, bool lower, int nsm, cudaStream_t s)
{
    uint64_t npairs = (1ull << (2 * n)) / 2;
    int pc = n - 1 - qubit, pr = 2 * n - 1 - qubit;
    k_project<<<grid_for(npairs, 256, nsm), 256, 0, s>>>(reinterpret_cast<float4 *>(rho), npairs, pc, pr, m, scale,
                                                         n, lower ? 1 : 0);
}

// Element (r, c) of rho; with lower (half storage) the upper triangle is taken from its mirror.
__device__ __forceinline__ float2 pt_elem(const float2 *__restrict__ rho, uint64_t dim, uint64_t r, uint64_t c,
                                          int lower)
{
    if (lower && r < c) {
        const float2 v = rho[c * dim + r];
        return make_float2(v.x, -v.y);
    }
    return rho[r * dim + c];
}

// Partial trace: out[a][a'] = sum_b rho[(a b), (a' b)] in FP64.
__global__ void __launch_bounds__(RED_THREADS) k_ptrace_block(const float2 *__restrict__ rho, PTParams p, double2 *out)
{
    const uint64_t dim = 1ull << p.n;
    const uint64_t da = 1ull << p.nkeep, db = 1ull << p.ntr;
    for (uint64_t o = blockIdx.x; o < da * da; o += gridDim.x) {
        uint64_t a = o / da, a2 = o % da;
        uint64_t r0 = 0, c0 = 0;
        for (int j = 0; j < p.nkeep; j++) {
            int bit = p.nkeep - 1 - j;
            r0 |= ((a >> bit) & 1ull) << p.kpos[j];
            c0 |= ((a2 >> bit) & 1ull) << p.kpos[j];
        }
        double acc[2] = {0, 0};
        for (uint64_t b = threadIdx.x; b < db; b += blockDim.x) {
            uint64_t off = 0;
            for (int j = 0; j < p.ntr; j++) off |= ((b >> (p.ntr - 1 - j)) & 1ull) << p.tpos[j];
            const float2 v = pt_elem(rho, dim, r0 | off, c0 | off, p.lower);
            acc[0] += v.x;
            acc[1] += v.y;
        }
        __shared__ double sh[RED_THREADS / 32][2];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        double s0 = warp_sum(acc[0]), s1 = warp_sum(acc[1]);
        if (lane == 0) { sh[w][0] = s0; sh[w][1] = s1; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0, t1 = 0;
            for (int j = 0; j < RED_THREADS / 32; j++) { t0 += sh[j][0]; t1 += sh[j][1]; }
            out[o] = make_double2(t0, t1);
        }
        __syncthreads();
    }
}

__global__ void k_ptrace_thread(const float2 *__restrict__ rho, PTParams p, double2 *out)
{
    const uint64_t dim = 1ull << p.n;
    const uint64_t da = 1ull << p.nkeep, db = 1ull << p.ntr;
    for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < da * da;
         o += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = o / da, a2 = o % da;
        uint64_t r0 = 0, c0 = 0;
        for (int j = 0; j < p.nkeep; j++) {
            int bit = p.nkeep - 1 - j;
            r0 |= ((a >> bit) & 1ull) << p.kpos[j];
            c0 |= ((a2 >> bit) & 1ull) << p.kpos[j];
        }
        double sr = 0, si = 0;
        for (uint64_t b = 0; b < db; b++) {
            uint64_t off = 0;
            for (int j = 0; j < p.ntr; j++) off |= ((b >> (p.ntr - 1 - j)) & 1ull) << p.tpos[j];
            const float2 v = pt_elem(rho, dim, r0 | off, c0 | off, p.lower);
            sr += v.x;
            si += v.y;
        }
        out[o] = make_double2(sr, si);
    }
}

void launch_partial_trace(const float2 *rho, const PTParams &p, double2 *out, int nsm, cudaStream_t s)
{
    uint64_t nout = 1ull << (2 * p.nkeep);
    if (p.ntr >= 8) {
        unsigned gb = (unsigned)(nout < (uint64_t)nsm * 8 ? nout : (uint64_t)nsm * 8);
        k_ptrace_block<<<gb, RED_THREADS, 0, s>>>(rho, p, out);
    } else {
        k_ptrace_thread<<<grid_for(nout, 256, nsm), 256, 0, s>>>(rho, p, out);
    }
}

}  // namespace qcw
