// Pass / phase descriptors shared by the fused-pass kernel and the batched persistent
// kernel, and the host routine that turns planner output into them.
//
// A pass touches a qubit set Q.  Its tile is the set of 2^TB elements whose flat indices
// differ only in the "tile bits": the row and column bits of Q plus the lowest column bits
// (contiguous runs of 2^L elements).  The other 2n - TB bits enumerate the tiles.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include <vector>

#include "planner.h"

namespace qcw {

struct FPass {
    int TB;            // tile bits
    int L;             // tile bits 0..L-1 are virtual bits 0..L-1 (contiguous run)
    int nother;        // 2n - TB
    int nphase;
    int phase0;        // first phase in the phase array
    int herm;          // symmetric tile: the same qubits' row and column bits (Hermitian kernel)
    int8_t tbits[16];  // virtual bit of tile bit j (ascending)
    int8_t obits[40];  // virtual bits outside the tile (ascending)
};

enum : int { PH_ONE = 1, PH_TWO = 2, PH_PRODUCT = 3 };

struct FPhase {
    int nq;            // PH_ONE (4x4), PH_TWO (16x16) or PH_PRODUCT (two 4x4: S_a then S_b)
    int coef;          // offset of the superoperator(s) in the coefficient array (float2 units)
    int8_t pos[4];     // tile positions of (r_a, r_b, c_a, c_b); (r_a, c_a) for PH_ONE
    int8_t opos[12];   // Hermitian passes: the tile bits outside the phase, in the order the
                       // group index enumerates them (the first five vary across a warp)
    int pad[2];
};

// Shared-memory position of tile element e in a Hermitian pass: bits 1..3 of e are XORed with
// a linear function of bits 4..11, bit 0 and bits 4.. are kept, so 16-byte pairs stay whole.
// A Hermitian tile of six qubits has the column bit of tile qubit j at bit j and its row bit
// at bit j + 6; each of bits 1, 2, 3 is mixed with bits of two more qubits (bit 1 with 5, 9;
// bit 2 with 6, 10; bit 3 with 4, 7, 8, 11), so a phase on one or two qubits always leaves
// outside bits whose positions span bits 1..3 mod 16: the warp's groups then fall on distinct
// bank pairs.
__host__ __device__ inline unsigned herm_phys(unsigned e)
{
    const unsigned t = e >> 4, s = t ^ (t >> 4);
    const unsigned sw = ((s >> 1) & 3u) | (((s ^ (s >> 3)) & 1u) << 2);
    return e ^ (sw << 1);
}

// Coefficients of a phase kind, in float2 units, all real transfer matrices in the Pauli basis
// of the phase's qubits, laid out for packed FP32 arithmetic.  A two-qubit phase stores its
// 16 x 16 matrix R as pairs (R[2p][f], R[2p+1][f]) for input f and output pair p (outputs 2p,
// 2p+1), f-major (128 float2).  A one-qubit phase stores its 4 x 4 matrix as duplicated pairs
// (R[e][f], R[e][f]), row-major (16 float2); a product phase stores R_a then R_b that way.
__host__ __device__ inline int phase_coefs(int nq) { return nq == PH_TWO ? 128 : nq == PH_PRODUCT ? 32 : 16; }

constexpr int kTileThreads = 256;  // threads per CTA of the tile kernels
constexpr int kTileBitsMax = 14;   // largest tile: 2^14 complex64 = 128 KiB

// Host-side descriptor arrays for a list of passes.
struct TilePlan {
    std::vector<FPass> passes;
    std::vector<FPhase> phases;
    std::vector<float2> coefs;
    std::vector<size_t> smem;  // dynamic shared memory per pass
    int nphase2 = 0, nphase1 = 0, nphasep = 0;
};

// Append the passes of `plan` (an n-qubit register, tiles of at most tbmax bits) to `out`.
// With herm, every tile holds the row and the column bits of the same qubits (Q plus the
// lowest qubits outside Q, tbmax / 2 qubits in all), so that the conjugate transpose of a
// tile is again a tile of the pass.
void append_tile_plan(const std::vector<PassPlan> &plan, int n, int tbmax, TilePlan &out, bool herm = false);

// Real transfer matrices R of a Hermiticity-preserving superoperator S in the Pauli basis of its
// qubits, for the butterfly form the kernels apply (members to (I, X, D, Z) per qubit, i on the
// members with an odd number of D components, c = R v, -i back, the same butterflies again).
// Two qubits: S and R 16 x 16, member index 8 r_a + 4 r_b + 2 c_a + c_b; one qubit: 4 x 4,
// index 2 r + c.  For a trace-preserving S the first row of R is (1/4, 0, ...) (two qubits) or
// (1/2, 0, 0, 0) (one qubit), exact in FP32.
void pauli_transfer(const std::vector<c128> &S, double R[16][16]);
void pauli_transfer1(const c128 *S, double R[4][4]);

// Dynamic shared memory of a tile kernel for a pass with TB tile bits and an L-bit run.
size_t tile_smem_bytes(int TB, int L);

}  // namespace qcw
