// Two-qubit phases of the Hermitian pass on the 5th-generation tensor cores (tcgen05).
//
// In the Pauli basis of its two qubits a phase is a real 16 x 16 matrix R applied to every
// 16-member group of the tile (see tile_phase2): c = R v.  Stacking the groups' coefficient
// vectors as rows gives a GEMM D[M x 16] = A[M x 16] R^T, M = 2 x the groups (real and
// imaginary parts are separate rows, R being real).  Each consumer thread owns the rows of its
// groups: it writes them to tensor memory (TMEM lane = the thread), one thread issues the MMAs
// (kind::tf32, M = 128, K = 8, A read from TMEM, B = R^T from shared memory), and each thread
// reads its rows of D back.
//
// FP32 accuracy from TF32 operands (3xTF32): a = a_hi + a_lo with a_hi = a rounded to nearest
// TF32 and a_lo = a - a_hi (exact in FP32, at most 2^-11 |a|); R = R_hi + R_lo the same way,
// R_lo rounded to TF32 as well.  D = a_hi R_hi + a_lo R_hi + a_hi R_lo.  The MMA drops the low
// 13 mantissa bits of an FP32 operand (truncation); only a_lo has any, and since a_lo takes
// either sign relative to a, that error (below 2^-21 |a|) has no bias.  The dropped a_lo R_lo is
// below 2^-22 relative.  Row 0 of a trace-preserving R is (1/4, 0, ..., 0), exact in TF32, so
// the trace sees none of R's rounding (the dense complex form of the phase, whose trace
// preservation rests on cancellation among rounded entries, drifted by 2e-5 on the 14-qubit
// circuit).  B stacks R_hi and R_lo along N (N = 32): one MMA per K half gives a_hi R_hi in
// columns 0..15 and a_hi R_lo in columns 16..31, a second (N = 16) adds a_lo R_hi to columns
// 0..15; the thread sums the two halves.
//
// Tensor memory per CTA: 256 columns.  Row block rb (group j = rb / 2 of the thread, real part
// for even rb, imaginary for odd) holds a_hi in columns 32 rb + 0..15 and a_lo in 32 rb +
// 16..31, and D in columns 128 + 32 rb + 0..31.  The two groups of a thread are pipelined:
// group 1's rows are prepared while group 0's MMAs run, and group 0 is finished while group
// 1's run; each group's MMAs signal their own mbarrier.  Both groups take the same arithmetic,
// so mirror groups of a diagonal tile stay exact conjugates (rho stays exactly Hermitian).
#pragma once
#include <cstdint>

#include "tile.cuh"

namespace qcw {

// ------------------------------------------------------------------ tcgen05 primitives (inline PTX)
__device__ __forceinline__ void tmem_alloc(unsigned *slot, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// 16 consecutive 32-bit columns of the calling thread's lane (taddr's lane field must be the
// warp's first lane: 32 x (warp % 4)).
__device__ __forceinline__ void tmem_st16(unsigned taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

// D (+)= A B, kind::tf32, FP32 accumulation; A (M x 8) in tensor memory, B (8 x N) in shared
// memory through a descriptor.  Issued by one thread.
__device__ __forceinline__ void tc_mma_tf32(unsigned d_tmem, unsigned a_tmem, uint64_t b_desc, uint32_t idesc,
                                            bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"((unsigned)accumulate)
        : "memory");
}

// One arrival on `bar` once every MMA the calling thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}

// Instruction descriptor, kind::tf32: FP32 D (bits 4-5 = 1), TF32 A and B (bits 7-9, 10-12 =
// 2), both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor without swizzle: core matrices of 8 rows x 16 bytes stored
// contiguously (128 bytes); lbo = byte distance of core matrices adjacent along K, sbo = along
// M / N; bits 46-48 = 0b001 (the descriptor version).
__device__ __forceinline__ uint64_t tc_sdesc(const void *smem, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((smem_u32(smem) & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// ------------------------------------------------------------------ the phase
constexpr int kTcCols = 256;          // tensor-memory columns per CTA
constexpr int kTcBFloats = 512;       // B for both K halves: 2 x (32 rows x 8) FP32
constexpr unsigned kTcLbo = 128, kTcSbo = 256;

// Float offset of B element (row n of N = 32, column kk of K = 8) in one K half's block: core
// matrix (n / 8, kk / 4) at n / 8 x kTcSbo + kk / 4 x kTcLbo bytes, row n % 8 of 16 bytes.
__device__ __forceinline__ int tc_boff(int n, int kk)
{
    return (n >> 3) * (int)(kTcSbo / 4) + (kk >> 2) * (int)(kTcLbo / 4) + (n & 7) * 4 + (kk & 3);
}

// a rounded to the nearest TF32 value (ties away from zero; finite a): two integer operations.
__device__ __forceinline__ uint32_t tf32_round(float a)
{
    return (__float_as_uint(a) + 0x1000u) & ~0x1fffu;
}

struct TcState {
    unsigned tmem;       // tensor-memory base address (lane 0, first column)
    float *B;            // kTcBFloats, 16-byte aligned shared memory
    uint64_t *bar;       // two mbarriers (count 1), one per group of a thread
    unsigned batches;    // MMA batches completed on each barrier so far (phase parity)
};

// Two-qubit phase of a Hermitian 2^12-element tile (swizzled layout, 128 consumer threads, two
// groups per thread), coefficients R (tile_phase2's layout) in the kernel parameter block.
// conj_s < 6: half-storage conjugation on the pass's first phase (see conj_group16).  Returns
// false if an MMA batch did not complete within `limit` polls (the tile is then garbage; the
// caller reports the error).  All 128 threads must call it together.
__device__ __forceinline__ bool tile_phase2_tc(float2 *__restrict__ tile, const FPhase &F,
                                               const float2 *__restrict__ R, TcState &tc, int conj_s,
                                               unsigned limit)
{
    const unsigned tid = threadIdx.x;
    const unsigned lane_base = ((tid >> 5) * 32u) << 16;
    // B = [R_hi; R_lo]^T per K half: element (n, k) of R at row n (R_hi) and row 16 + n (R_lo)
    {
        const float2 c = R[tid];  // (R[2p][f], R[2p+1][f]), f = tid / 8, p = tid % 8
        const int f = (int)(tid >> 3), p = (int)(tid & 7u);
        float *blk = tc.B + (f >> 3) * (kTcBFloats / 2);
        const float h0 = __uint_as_float(tf32_rna(c.x)), h1 = __uint_as_float(tf32_rna(c.y));
        blk[tc_boff(2 * p, f & 7)] = h0;
        blk[tc_boff(2 * p + 1, f & 7)] = h1;
        blk[tc_boff(16 + 2 * p, f & 7)] = __uint_as_float(tf32_rna(c.x - h0));
        blk[tc_boff(16 + 2 * p + 1, f & 7)] = __uint_as_float(tf32_rna(c.y - h1));
        fence_async_smem();
    }
    const unsigned d0 = herm_phys(1u << F.pos[0]), d1 = herm_phys(1u << F.pos[1]), d2 = herm_phys(1u << F.pos[2]),
                   d3 = herm_phys(1u << F.pos[3]);
    auto member = [&](int e) {
        return ((e & 8) ? d0 : 0u) ^ ((e & 4) ? d1 : 0u) ^ ((e & 2) ? d2 : 0u) ^ ((e & 1) ? d3 : 0u);
    };
    unsigned long long *t64 = reinterpret_cast<unsigned long long *>(tile);
    const uint32_t id32 = tc_idesc_tf32(128, 32), id16 = tc_idesc_tf32(128, 16);
    unsigned base[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const unsigned bl = group_logical(tid + 128u * j, F, 8);
        base[j] = herm_phys(bl);
        unsigned long long x[16];
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = t64[base[j] ^ member(e)];
        if (conj_s < 6) conj_group16(x, bl, conj_s, conj_top(F, conj_s));
        pauli_butterflies(x);
        uint32_t hr[16], lr[16], hi[16], li[16];  // rows of v = (i on the odd Pauli indices) x
#pragma unroll
        for (int f = 0; f < 16; f++) {
            const float2 u = unpack2(x[f]);
            const float vr = pauli_odd_idx(f) ? -u.y : u.x, vi = pauli_odd_idx(f) ? u.x : u.y;
            hr[f] = tf32_round(vr), lr[f] = __float_as_uint(vr - __uint_as_float(hr[f]));
            hi[f] = tf32_round(vi), li[f] = __float_as_uint(vi - __uint_as_float(hi[f]));
        }
        const unsigned col = 64u * j;
        tmem_st16(tc.tmem + lane_base + col, hr);
        tmem_st16(tc.tmem + lane_base + col + 16, lr);
        tmem_st16(tc.tmem + lane_base + col + 32, hi);
        tmem_st16(tc.tmem + lane_base + col + 48, li);
        tmem_wait_st();
        tc_fence_before();
        bar_sync(1, 128);  // every lane's rows (and B) are in place
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int rb = 2 * j; rb < 2 * j + 2; rb++)
#pragma unroll
                for (int kh = 0; kh < 2; kh++) {
                    const unsigned dt = tc.tmem + 128u + 32u * rb, ah = tc.tmem + 32u * rb + 8u * kh;
                    const uint64_t bd = tc_sdesc(tc.B + kh * (kTcBFloats / 2), kTcLbo, kTcSbo);
                    tc_mma_tf32(dt, ah, bd, id32, kh > 0);     // a_hi [R_hi | R_lo]
                    tc_mma_tf32(dt, ah + 16u, bd, id16, true);  // + a_lo R_hi
                }
            tc_commit(&tc.bar[j]);
        }
        __syncwarp();  // tcgen05.st / ld are warp-collective
    }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        ok &= mbar_wait(&tc.bar[j], tc.batches & 1u, limit);
        __syncwarp();
        tc_fence_after();
        uint32_t a[16], b[16], c[16], d[16];
        const unsigned col = 128u + 64u * j;
        tmem_ld16(tc.tmem + lane_base + col, a);
        tmem_ld16(tc.tmem + lane_base + col + 16, b);
        tmem_ld16(tc.tmem + lane_base + col + 32, c);
        tmem_ld16(tc.tmem + lane_base + col + 48, d);
        tmem_wait_ld();
        unsigned long long x[16];
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const float re = __uint_as_float(a[e]) + __uint_as_float(b[e]);
            const float im = __uint_as_float(c[e]) + __uint_as_float(d[e]);
            x[e] = pauli_odd_idx(e) ? pack2(im, -re) : pack2(re, im);
        }
        pauli_butterflies(x);
#pragma unroll
        for (int e = 0; e < 16; e++) t64[base[j] ^ member(e)] = x[e];
    }
    tc.batches++;
    return ok;
}

}  // namespace qcw
