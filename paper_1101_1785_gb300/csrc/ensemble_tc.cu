// Multiverse ensemble density on the 5th-generation tensor cores (tcgen05, kind::tf32, 3xTF32).
//
// rho = sum_v w_v |psi_v><psi_v| (Sec. 5.2.1, Eq. rhoE1's ensemble average) is a complex GEMM
// of rank nvec: rho = A B^H with A[r][v] = w_v psi_v[r] and B[c][v] = psi_v[c].  In real
// arithmetic, with the K index running over (v, real part) and (v, imaginary part):
//   Re rho = [Re A | Im A] [Re B | Im B]^T,   Im rho = [Re A | Im A] [-Im B | Re B]^T,
// two real GEMMs sharing their A operand.  A CTA owns a 128 x 128 tile of rho strictly below the
// diagonal (the tile above is its conjugate transpose, written from the same result); the
// 128 x 128 blocks on the diagonal are left to the FP32 kernel: the tensor cores' FP32
// accumulation drops low bits with one sign, which on the diagonal -- sums of positive terms
// w_v |psi_v[r]|^2 -- moved the trace by 2.6e-6 at 64 vectors, while the off-diagonal elements
// (either sign) keep FP32-level accuracy.  Per
// round of eight vectors (two K = 8 slabs of four) its 256 threads stage A, B1 = [Re B | Im B] and
// B2 = [-Im B | Re B] in shared memory in the no-swizzle K-major layout, each split into a TF32
// high part and the FP32 remainder (3xTF32: a_hi b_hi + a_lo b_hi + a_hi b_lo, FP32-level
// accuracy; the remainder keeps either sign, so the MMA's truncation of its low bits has no
// bias), and one thread issues twelve MMAs (M = 128, N = 128, K = 8) into two 128-column
// accumulators in tensor memory.  Rounds are double-buffered: the staging of round i + 1
// overlaps the MMAs of round i, and a buffer is refilled once the MMAs that read it have
// signalled their mbarrier; each thread loads its amplitudes one round ahead and writes its
// row of every operand slab as 16-byte pieces.  The epilogue reads each row of both
// accumulators (tensor-memory lane = row) and writes the tile (through shared memory, as
// 128-byte runs) and its mirror.
// Every wait is bounded; a wait that runs out sets *err and the CTA stops after releasing its
// tensor memory.
#include "qcw_internal.h"
#include "tc.cuh"

namespace qcw {

constexpr int kEdT = 128;                     // tile edge (MMA M and N)
constexpr int kEdV = 8;                       // vectors per round: two K = 8 slabs of four vectors each
constexpr int kEdThreads = 256;               // two threads per tile row: one per slab of the round
constexpr int kEdSlab = kEdT * 8;             // floats of one K = 8 operand slab (128 rows x 32 bytes)
constexpr int kEdStageFloats = 12 * kEdSlab;  // A_hi, A_lo, B1_hi, B1_lo, B2_hi, B2_lo, two slabs each
constexpr int kEdCols = 256;                  // tensor-memory columns: Re rho (0..127), Im rho (128..255)
constexpr unsigned kEdWaitLimit = 1u << 20;   // polls (~0.25 s with the 256 ns back-off)

// Float offset of element (row, k) of a K-major K = 8 slab: core matrices of 8 rows x 16 bytes,
// the two along K 128 bytes apart (LBO), row groups of 8 at 256 bytes (SBO), as tc_boff.
__device__ __forceinline__ int ed_off(int row, int k)
{
    return (row >> 3) * 64 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

// D (+)= A B^T, kind::tf32, both operands in shared memory (K-major descriptors).
__device__ __forceinline__ void tc_mma_tf32_ss(unsigned d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                               bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((unsigned)accumulate)
        : "memory");
}

__device__ __forceinline__ void ed_split(float x, float &hi, float &lo)
{
    hi = __uint_as_float(tf32_round(x));
    lo = x - hi;
}

__global__ void __launch_bounds__(kEdThreads) k_ens_density_tc(const float2 *__restrict__ psi, int nvec, int n,
                                                               const float *__restrict__ w,
                                                               float2 *__restrict__ rho,
                                                               unsigned *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char ed_smem[];
    float *stage = reinterpret_cast<float *>(ed_smem);  // 2 stages x kEdStageFloats
    uint64_t *bar = reinterpret_cast<uint64_t *>(stage + 2 * kEdStageFloats);  // one per stage
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 2);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (tid < 32) {
        tmem_alloc(tslot, kEdCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    const int row = tid & (kEdT - 1), half = tid >> 7;  // tile row (tensor-memory lane) and slab / column half
    const unsigned lane_base = ((unsigned)((tid >> 5) & 3) * 32u) << 16;
    const uint64_t dim = 1ull << n;
    const unsigned M = (unsigned)(dim / kEdT);
    const unsigned npairs = M * (M - 1) / 2;  // tiles strictly below the diagonal
    const int nround = (nvec + kEdV - 1) / kEdV;
    const uint32_t idesc = tc_idesc_tf32(kEdT, kEdT);
    unsigned cm0 = 0u, cm1 = 0u;  // commits issued on each stage's barrier so far (registers, not an array)
    bool ok = true;
    for (unsigned pr = blockIdx.x; ok && pr < npairs; pr += gridDim.x) {
        // pr = R (R - 1) / 2 + C with C < R
        unsigned R = (unsigned)((sqrt(8.0 * pr + 1.0) + 1.0) / 2.0);
        while (R * (R - 1) / 2 > pr) R--;
        while ((R + 1) * R / 2 <= pr) R++;
        const unsigned C = pr - R * (R - 1) / 2;
        const uint64_t r0 = (uint64_t)R * kEdT, c0 = (uint64_t)C * kEdT;
        // This thread's amplitudes of a round (its slab: vectors 8 rd + 4 half + i), loaded one
        // round ahead so that their latency overlaps the previous round's staging and MMAs.
        float2 na[4], nb[4];
        float nw[4];
        auto fetch = [&](int rd) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int v = rd * kEdV + 4 * half + i;
                na[i] = nb[i] = make_float2(0.f, 0.f);
                nw[i] = 0.f;
                if (v < nvec) {
                    const float2 *pv = psi + ((uint64_t)v << n);
                    nw[i] = w[v];
                    na[i] = pv[r0 + row];
                    nb[i] = pv[c0 + row];
                }
            }
        };
        fetch(0);
        for (int rd = 0; rd < nround; rd++) {
            float2 ca[4], cb[4];
            float cw[4];
#pragma unroll
            for (int i = 0; i < 4; i++) ca[i] = na[i], cb[i] = nb[i], cw[i] = nw[i];
            if (rd + 1 < nround) fetch(rd + 1);
            const int s = rd & 1;
            const unsigned cms = s ? cm1 : cm0;
            if (cms > 0) {  // the MMAs that last read stage s are done before it is refilled
                const bool good = tid == 0 ? mbar_wait(&bar[s], (cms - 1) & 1u, kEdWaitLimit) : true;
                ok = bar_and(1, kEdThreads, good);
                if (!ok) break;
            }
            float *st = stage + s * kEdStageFloats;
            // operand o (0 A_hi, 1 A_lo, 2 B1_hi, 3 B1_lo, 4 B2_hi, 5 B2_lo), slab ks at (2 o + ks)
            // slabs; this thread's row of its slab: K index k = i (real parts, or -Im for B2) and
            // 4 + i (imaginary parts, or Re for B2), written as two 16-byte pieces per operand
            float op[6][8];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 a = make_float2(cw[i] * ca[i].x, cw[i] * ca[i].y), b = cb[i];
                float h, l;
                ed_split(a.x, op[0][i], op[1][i]);
                ed_split(a.y, op[0][4 + i], op[1][4 + i]);
                ed_split(b.x, h, l), op[2][i] = h, op[3][i] = l, op[4][4 + i] = h, op[5][4 + i] = l;
                ed_split(b.y, h, l), op[2][4 + i] = h, op[3][4 + i] = l, op[4][i] = -h, op[5][i] = -l;
            }
#pragma unroll
            for (int o = 0; o < 6; o++)
#pragma unroll
                for (int kh = 0; kh < 2; kh++)
                    *reinterpret_cast<float4 *>(st + (2 * o + half) * kEdSlab + ed_off(row, 4 * kh)) =
                        make_float4(op[o][4 * kh], op[o][4 * kh + 1], op[o][4 * kh + 2], op[o][4 * kh + 3]);
            fence_async_smem();  // the generic-proxy writes become visible to the MMAs
            tc_fence_before();
            bar_sync(1, kEdThreads);
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 2; ks++) {
                    auto desc = [&](int o) { return tc_sdesc(st + (2 * o + ks) * kEdSlab, 128, 256); };
                    const uint64_t ah = desc(0), al = desc(1), b1h = desc(2), b1l = desc(3), b2h = desc(4),
                                   b2l = desc(5);
                    const bool acc = rd > 0 || ks > 0;
                    tc_mma_tf32_ss(tmem, ah, b1h, idesc, acc);  // Re rho
                    tc_mma_tf32_ss(tmem, al, b1h, idesc, true);
                    tc_mma_tf32_ss(tmem, ah, b1l, idesc, true);
                    tc_mma_tf32_ss(tmem + 128u, ah, b2h, idesc, acc);  // Im rho
                    tc_mma_tf32_ss(tmem + 128u, al, b2h, idesc, true);
                    tc_mma_tf32_ss(tmem + 128u, ah, b2l, idesc, true);
                }
                tc_commit(&bar[s]);
            }
            if (s) cm1++;
            else cm0++;
        }
        if (!ok) break;
        // the last round's commit covers every MMA issued before it
        {
            const int s = (nround - 1) & 1;
            const unsigned cms = s ? cm1 : cm0;
            const bool good = tid == 0 ? mbar_wait(&bar[s], (cms - 1) & 1u, kEdWaitLimit) : true;
            ok = bar_and(1, kEdThreads, good);
            if (!ok) break;
        }
        tc_fence_after();
        // The stages are free now (every MMA of the tile is done): each half of the threads
        // passes its 16-column slices of the tile's rows through a padded buffer there, so that the
        // tile's rows go out as 128-byte runs (16 threads per row) instead of one 16-byte piece per
        // thread and row.  The mirror is written straight from the registers: for one column j a
        // warp's 32 rows are 32 consecutive elements of row c0 + j.
        float2(*buf)[kEdT][17] = reinterpret_cast<float2(*)[kEdT][17]>(stage);  // [half][row][16 + pad]
        const int hl = tid & (kEdT - 1);  // this thread's index within its half
        for (int j0 = 64 * half; j0 < 64 * half + 64; j0 += 16) {  // this thread's half of the columns
            uint32_t re[16], im[16];
            tmem_ld16(tmem + lane_base + (unsigned)j0, re);
            tmem_ld16(tmem + lane_base + 128u + (unsigned)j0, im);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; j++) {
                buf[half][row][j] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
                rho[(c0 + j0 + j) * dim + r0 + row] = make_float2(__uint_as_float(re[j]), -__uint_as_float(im[j]));
            }
            bar_sync(1, kEdThreads);
#pragma unroll 4
            for (int i = 0; i < 16; i++) {  // element e = hl + 128 i of the half's 128 x 16 slice
                const int e = hl + kEdT * i, r = e >> 4, jj = e & 15;
                rho[(r0 + r) * dim + c0 + j0 + jj] = buf[half][r][jj];
            }
            bar_sync(1, kEdThreads);  // the slice is out before the next one overwrites the buffer
        }
        tc_fence_before();
        bar_sync(1, kEdThreads);  // every row is read before the next tile's first MMA overwrites it
    }
    if (!ok && tid == 0) atomicOr(err, 1u);
    // every commit's arrival has landed (after a wait that ran out, MMAs may still be in flight:
    // one more bounded wait each) before the barriers and tensor memory go away
    if (tid == 0 && cm0 > 0) mbar_wait(&bar[0], (cm0 - 1) & 1u, kEdWaitLimit);
    if (tid == 0 && cm1 > 0) mbar_wait(&bar[1], (cm1 - 1) & 1u, kEdWaitLimit);
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, kEdCols);
    }
}

// Dynamic shared memory: the two stages (48 KiB) and the barriers, rounded up to 100 KiB so that
// at most two CTAs share an SM -- two CTAs hold all 512 tensor-memory columns, and a third one's
// allocation would wait for one of them to finish.
size_t ens_density_tc_smem()
{
    const size_t need = sizeof(float) * 2 * kEdStageFloats + 2 * sizeof(uint64_t) + 16;
    const size_t two_per_sm = 100u << 10;
    return need > two_per_sm ? need : two_per_sm;
}

// Launches the tensor-core density for 2^n >= 128; returns false (nothing launched) otherwise.
bool launch_ens_density_tc(const float2 *psi, int nvec, int n, const float *w, float2 *rho, unsigned *err, int nsm,
                           cudaStream_t s)
{
    if (n < 8) return false;  // at least two 128-row blocks: one tile below the diagonal
    const size_t smem = ens_density_tc_smem();
    if (ensure_smem_attr(reinterpret_cast<const void *>(k_ens_density_tc), smem)) return false;
    const uint64_t m = (1ull << n) / kEdT, pairs = m * (m - 1) / 2;
    const uint64_t cap = (uint64_t)nsm * 2;  // two CTAs per SM (256 of the 512 tensor-memory columns each)
    k_ens_density_tc<<<(unsigned)(pairs < cap ? pairs : cap), kEdThreads, smem, s>>>(psi, nvec, n, w, rho, err);
    return true;
}

}  // namespace qcw
