// Internal declarations of the qcw library (host side): the context, kernel parameter
// blocks and the launchers implemented in the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "qcw.h"

namespace qcw {

using c128 = std::complex<double>;

// ------------------------------------------------------------------ kernel parameter blocks
// Matrices travel by value in the kernel parameter space (constant bank): every thread
// reads the same coefficient at the same time, which the constant cache broadcasts.

struct Gate1Params {
    float2 u[4];       // U row-major
    int pc, pr;        // virtual bit positions of the target's column / row bit
    uint64_t cmask_c;  // control qubits' column bits (all must be 1 for U^* on columns)
    uint64_t cmask_r;  // control qubits' row bits (all must be 1 for U on rows)
};

struct Gate2Params {
    float2 u[16];      // V row-major, index 2*q(q1) + q(q2)
    int pos[4];        // the four virtual bit positions, ascending (for insertion)
    uint64_t off_r[4]; // row offset of local row index i
    uint64_t off_c[4]; // column offset of local column index j
    uint64_t cmask_c, cmask_r;
};

struct Super1Params {
    float r[16];       // real 4x4 transfer matrix in the qubit's Pauli basis (pauli_transfer1)
    int pc, pr;
};

struct Super2Params {
    float r[256];      // real 16x16 transfer matrix in the two qubits' Pauli basis (pauli_transfer),
                       // member index e = 4*row_local + col_local = 8 r1 + 4 r2 + 2 c1 + c2
    int pos[4];
    uint64_t off_r[4], off_c[4];
};

struct Mono2Params {   // uncontrolled two-qubit gate with one entry of modulus 1 per row (CNOT, CZ, SWAP, ...)
    float2 ph[16];     // member e = 4 i + j of the output: u_i conj(u_j) (one of 1, -1, i, -i, exact)
    int pos[4];        //   times the input member (sigma(i), sigma(j))
    uint64_t off_r[4], off_c[4];    // offsets of the output members
    uint64_t src_r[4], src_c[4];    // offsets of their inputs: off_r[sigma(i)], off_c[sigma(j)]
};

struct GateKParams {   // one side (rows or columns) of a k-qubit dense gate, k <= 5
    float2 u[1024];    // U (or conj(U) for the column side), 2^k x 2^k row-major
    int k;
    int pos[5];        // ascending virtual bit positions of the struck bits on this side
    uint64_t off[32];  // offset of local index i on this side
};

struct PTParams {
    int n, nkeep, ntr;
    int lower;  // 1: only the lower triangle is current (half storage); (r, c) with r < c is read
                // as conj(rho[c][r])
    int8_t kpos[QCW_MAX_QUBITS];  // label bit of kept qubit j; j = 0 is the result's MSB
    int8_t tpos[QCW_MAX_QUBITS];  // label bit of traced qubit j
};

// ------------------------------------------------------------------ launchers (kernels.cu)
void launch_gate1(const Gate1Params &p, float2 *rho, int n, int nsm, cudaStream_t s);
void launch_gate2(const Gate2Params &p, float2 *rho, int n, int nsm, cudaStream_t s);
void launch_super1(const Super1Params &p, float2 *rho, int n, int nsm, cudaStream_t s);
void launch_super2(const Super2Params &p, float2 *rho, int n, int nsm, cudaStream_t s);
void launch_mono2(const Mono2Params &p, float2 *rho, int n, int nsm, cudaStream_t s);
void launch_gatek_side(const GateKParams &p, float2 *rho, int n, int nsm, cudaStream_t s);
void launch_zero_state(float2 *rho, int n, bool lower, int nsm, cudaStream_t s);
void launch_c128_to_c64(const double2 *src, float2 *dst, size_t count, int nsm, cudaStream_t s);
void launch_c64_to_c128(const float2 *src, double2 *dst, size_t count, int nsm, cudaStream_t s);
// Reductions write `nvals` doubles per block into partials, then fold them in block order.
int reduce_blocks(int nsm);
void launch_diag_reduce(const float2 *rho, int n, double *partials, double *out, int nblocks,
                        cudaStream_t s);
void launch_purity(const float2 *rho, int n, double *partials, double *out, int nblocks,
                   cudaStream_t s);
void launch_project(float2 *rho, int n, int qubit, int m, float scale, bool lower, int nsm, cudaStream_t s);
// Half storage: rho[r][c] = conj(rho[c][r]) for r < c (complete the matrix from its lower
// triangle), and purity from the lower triangle (2 |rho_rc|^2 below the diagonal).
void launch_symmetrize(float2 *rho, int n, int nsm, cudaStream_t s);
void launch_purity_lower(const float2 *rho, int n, double *partials, double *out, int nblocks, cudaStream_t s);
void launch_fold(const double *partials, int nblocks, double *out, cudaStream_t s);
// Multiverse density on the tensor cores (ensemble_tc.cu) for 2^n >= 128: rho = sum_v w_v
// |psi_v><psi_v|; *err gets bit 0 if a bounded wait ran out.  Returns false if not launched.
bool launch_ens_density_tc(const float2 *psi, int nvec, int n, const float *w, float2 *rho, unsigned *err, int nsm,
                           cudaStream_t s);
void launch_accumulate(float2 *acc, const float2 *x, int n, int nsm, cudaStream_t s);
// Pauli-string expectations Tr[P rho] (polarisation vectors, spin correlation tensor): per
// string the row-label masks of its X-or-Y qubits (flipped), Y qubits and Z qubits.
constexpr int kMaxPauliTerms = 3 * QCW_MAX_QUBITS;
struct PauliTerms {
    int count;
    unsigned flip[kMaxPauliTerms], ym[kMaxPauliTerms], zm[kMaxPauliTerms];
    int ny[kMaxPauliTerms];
};
// out[s] = Re Tr[P_s rho] for s < T.count (count <= 63), reading only the lower triangle.
void launch_pauli_expect(const float2 *rho, int n, const PauliTerms &T, double *partials, int max_partials,
                         double *out, cudaStream_t s);
// The purity partials of the last fused pass, if they describe the current rho.
bool fused_purity_partials(qcw_ctx *c, const double **partials, int *nblocks);
void launch_partial_trace(const float2 *rho, const PTParams &p, double2 *out, int nsm,
                          cudaStream_t s);
int launches_per_reduce();

// ------------------------------------------------------------------ queued operation
struct QOp {
    int kind;               // 0 = unitary, 1 = superoperator (channel), 2 = Kraus list (k >= 3)
    int k;                  // number of qubits (1..5)
    int qubits[5];
    int ncontrols;
    int controls[QCW_MAX_QUBITS];
    std::vector<c128> m;    // unitary 2^k x 2^k, superoperator 4^k x 4^k, or the Kraus operators
                            // (2^k x 2^k each) one after another
};

struct FusedPlan;  // planner.cpp
struct FusedRuntime;  // fused.cu

}  // namespace qcw

struct qcw_ctx {
    int n = 0;
    int dev = 0;
    int nsm = 0;
    float2 *rho = nullptr;
    bool owns_rho = false;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    int mode = QCW_MODE_PLAIN;
    bool validate = false;  // qcw_set_validation: check unitarity, Kraus trace, Hermitian states
    int fuse_k = 0;
    int fused_kernel = QCW_FUSED_KERNEL_AUTO;
    // reduction scratch: per-block partials and a small result block (+ pinned mirror)
    double *d_partials = nullptr;
    int red_blocks = 0;
    double *d_result = nullptr;
    double *h_result = nullptr;  // pinned, 64 doubles
    // staging for complex128 <-> complex64 conversion
    void *d_staging = nullptr;
    size_t staging_bytes = 0;
    // fused mode
    std::vector<qcw::QOp> queue;
    qcw::FusedRuntime *fused = nullptr;
    // bounded in-kernel waits of the fused passes: polls before giving up (0: default) and a
    // tile whose load the first CTA skips (fault injection; -1: none)
    unsigned wait_limit = 0;
    int stall_tile = -1;
    // half storage: only the lower triangle (r >= c) of rho is current (the warp-specialised
    // pass leaves it so); ensure_full completes the matrix before anything else reads it
    bool half = false;
    // Version of rho: bumped by everything that changes it.  The last fused pass of a flush
    // also sums |rho_rc|^2 over what it writes (per-CTA partials in the fused runtime);
    // purity_ver records the version those partials describe.
    // scratch copies of rho for Kraus channels on more than two qubits (allocated on first use)
    float2 *d_kacc = nullptr;
    float2 *d_ktmp = nullptr;
    unsigned long long state_ver = 1;
    unsigned long long purity_ver = 0;
    // asynchronous readouts: QCW_CHECKPOINT_SLOTS slots of kCkptVals doubles on the device and
    // in pinned host memory, the ticket each slot holds and an event marking its copy
    double *d_ckpt = nullptr;
    double *h_ckpt = nullptr;
    long long ckpt_ticket[QCW_CHECKPOINT_SLOTS];
    cudaEvent_t ckpt_ev[QCW_CHECKPOINT_SLOTS] = {};
    long long ckpt_next = 0;
    // counters
    long long launches = 0;
    long long passes = 0;
    long long timed_passes = 0;
    double pass_ms = 0;
    bool timing = false;
};

namespace qcw {
// Device word in the context's result block where kernels report a wait that ran out (bit 0:
// producer side, bit 1: consumer side).  Sticky until qcw_reset or a state load.
constexpr int kErrSlot = 63;
inline unsigned long long *device_error_word(qcw_ctx *c)
{
    return reinterpret_cast<unsigned long long *>(c->d_result + kErrSlot);
}
// fused.cu / planner.cpp entry points used by the API layer
qcw_status fused_flush(qcw_ctx *ctx);
void fused_destroy(qcw_ctx *ctx);
void fused_collect_timing(qcw_ctx *ctx);
qcw_status plain_apply(qcw_ctx *c, const QOp &op);
qcw_status ensure_full(qcw_ctx *c);
// rho is about to be overwritten from outside the queue: drop queued work, mark the storage
// full, bump the state version and clear the error word.
qcw_status begin_state_replace(qcw_ctx *c);
// Validate an op list against an n-qubit register and convert it to queued operations
// (Kraus sets become superoperators); nothing is appended on error.
qcw_status convert_ops(int n, const qcw_op *ops, int nops, const double *matrices, std::vector<QOp> &out,
                       bool validate = false);
qcw_status set_error(qcw_status st, const std::string &msg);
// Raise a kernel's max dynamic shared memory on the current device to at least `bytes`.  The
// attribute is process-wide per function and device, so it only ever grows.
qcw_status ensure_smem_attr(const void *func, size_t bytes);
qcw_status cuda_error(cudaError_t e, const char *what);
}  // namespace qcw
