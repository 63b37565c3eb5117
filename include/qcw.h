/*
 * qcw: density-matrix simulator on one GB300 (sm_103a), C ABI.
 *
 * The state is an n-qubit density matrix rho, a 2^n x 2^n complex matrix kept on the
 * device as row-major interleaved complex64 (float re, float im); element (r, c) sits at
 * offset r * 2^n + c.  A basis label is r = sum_i q_i 2^(n-1-i): API qubit i is the
 * paper's qubit i_s = i + 1 and qubit 0 is the most significant bit (Sec. 2.3,
 * Eq. staten).  Its "stride" 2^(n-1-i) is the distance between partner labels n0 and n1
 * (Sec. 3.1, Eqs. pair0 / pair1 and the text after Eq. resmat1).
 *
 * Operator matrices passed in are row-major interleaved complex128 (double re, double im)
 * on the host.  A k-qubit matrix is indexed by the binary number q_{s1} q_{s2} ... q_{sk}
 * of its qubits in the order the caller lists them; for k = 2 this is the amplitude-quartet
 * order n00, n01, n10, n11 of Eq. resmat2 (V_{ij;kl} = <i j| V |k l>).  Matrices are copied
 * during the call: the caller may free or reuse them as soon as the call returns.
 *
 * Arithmetic: gate and channel updates in FP32 complex; trace, purity, probabilities,
 * partial traces and the post-measurement scale in FP64.
 *
 * Ordering: apply calls are asynchronous on the context's CUDA stream.  Every readout
 * (trace, purity, probabilities, measure, partial trace, get_state) synchronises the
 * stream and returns host FP64 values.
 *
 * Errors: every call returns a qcw_status.  Invalid arguments (NULL pointers, qubit out of
 * range or repeated, k out of range, nkraus < 1, non-finite matrix entries) return
 * QCW_EINVAL and leave the state unchanged.  A CUDA runtime failure returns QCW_ECUDA;
 * qcw_last_error() then holds the runtime's message.
 */
#ifndef QCW_H
#define QCW_H

#include <stddef.h>

#if defined(__GNUC__)
#define QCW_API __attribute__((visibility("default")))
#else
#define QCW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qcw_ctx qcw_ctx;

typedef enum {
    QCW_OK = 0,
    QCW_EINVAL = 1,     /* bad argument; state unchanged */
    QCW_ENOMEM = 2,     /* device or host allocation failed */
    QCW_ECUDA = 3,      /* CUDA runtime error (see qcw_last_error) */
    QCW_EZEROPROB = 4,  /* measurement outcome with probability < 1e-12; state unchanged */
    QCW_ETIMEOUT = 5,   /* a bounded wait ran out */
    QCW_ENOTSUP = 6     /* size or mode not supported by this build */
} qcw_status;

/* Execution modes (qcw_set_mode). */
#define QCW_MODE_PLAIN 0 /* each apply call launches its own kernel at once */
#define QCW_MODE_FUSED 1 /* apply calls are queued; flush packs them into fused passes */

/* Largest register size: rho of 17 qubits is 128 GiB of complex64. */
#define QCW_MAX_QUBITS 17
/* Largest k accepted by qcw_apply_gate. */
#define QCW_MAX_GATE_QUBITS 5
/* Most Kraus operators in one channel: the paper's multiverse noise step (Eq. rhoE4) has
 * 1 + 2 n_p of them for n_p paths with one- and two-hit noise operators. */
#define QCW_MAX_KRAUS 64

/* --------------------------------------------------------------------- lifetime */

/* Create a context that owns a device rho of nqubits (1..QCW_MAX_QUBITS) and its own
 * non-blocking CUDA stream on the current device; rho starts as |0..0><0..0|
 * (the paper's initial state |0...0>, Sec. 4.1).  *out receives the handle. */
QCW_API qcw_status qcw_create(int nqubits, qcw_ctx **out);

/* Create a context on caller-owned memory: dev_rho points to 4^n complex64 values on the
 * current device (16-byte aligned), cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  The context never frees dev_rho or the stream; its contents are used as is. */
QCW_API qcw_status qcw_create_from_ptr(int nqubits, void *dev_rho, void *cuda_stream, qcw_ctx **out);

/* Release the context (waits for its stream).  NULL is accepted. */
QCW_API qcw_status qcw_destroy(qcw_ctx *ctx);

/* Select QCW_MODE_PLAIN or QCW_MODE_FUSED.  fuse_k (2..QCW_MAX_GATE_QUBITS, 0 = let the
 * tuner choose) bounds the number of qubits one fused pass may touch.  Switching mode
 * flushes queued work first. */
QCW_API qcw_status qcw_set_mode(qcw_ctx *ctx, int mode, int fuse_k);

/* Which kernel runs fused passes.
 *   HERM: rho is a density matrix, hence Hermitian (Sec. 5.2, rho^dagger = rho).  Tiles hold
 *     the row and column bits of the same qubits; each pass evolves the tiles on one side of
 *     the diagonal and writes the others as their conjugate transposes (half the arithmetic).
 *     A non-Hermitian matrix loaded with qcw_set_state is not preserved.  One CTA per tile.
 *   HERM_WS (and AUTO, the default): the same Hermitian pass on persistent CTAs whose
 *     producer warps load and store tiles while consumer warps evolve them, so memory traffic
 *     and arithmetic overlap; each pass reads and writes only the lower triangle r >= c of rho
 *     (a third less memory traffic), and the library completes the matrix whenever it is read
 *     as a whole.  Used for registers of 6 or more qubits (HERM below that).  Phases run on
 *     the FP32 CUDA cores.
 *   HERM_TC: HERM_WS with the two-qubit phases, dense real 16 x 16 contractions in the Pauli
 *     basis, on the tensor cores (tcgen05 TF32 MMAs with the 3xTF32 split and FP32
 *     accumulation: FP32-level accuracy).  Slower than HERM_WS on GB300 (each phase waits for
 *     its MMAs), hence not the default.
 *   TILE: one CTA per tile, no symmetry assumed.
 * Flushes queued work first. */
#define QCW_FUSED_KERNEL_AUTO 0
#define QCW_FUSED_KERNEL_TILE 1
#define QCW_FUSED_KERNEL_HERM 2
#define QCW_FUSED_KERNEL_HERM_WS 3
#define QCW_FUSED_KERNEL_HERM_TC 4
QCW_API qcw_status qcw_set_fused_kernel(qcw_ctx *ctx, int which);

/* Bounded waits inside the HERM_WS pass kernel.  Producer and consumer warps hand tiles over
 * through shared-memory barriers; each wait gives up after `polls` polls (0 restores the
 * default, about half a second or more), sets the context's error word and ends the kernel.
 * The next qcw_sync or readout then returns QCW_ETIMEOUT, and keeps doing so until qcw_reset or
 * a state load (rho is undefined after such a pass).  stall_tile >= 0 makes the first CTA skip
 * the load of its tile number stall_tile, so that its consumers' wait runs out (a test of the
 * error path without any fault); -1 turns that off.  The paper has no counterpart.
 * Flushes queued work first.  QCW_EINVAL if stall_tile < -1. */
QCW_API qcw_status qcw_set_fused_wait_limit(qcw_ctx *ctx, unsigned polls, int stall_tile);

/* Validation mode (off by default; on for every new context when the environment variable
 * QCW_VALIDATE is set to anything but 0).  When on, every apply call checks its matrices before
 * queueing anything: gates must be unitary (U^dagger U = I within 1e-6; the paper's operators
 * are unitary, Sec. 3), Kraus sets must not increase the trace (largest eigenvalue of
 * sum K^dagger K at most 1 + 1e-6; Eq. rhoE1's ensemble keeps it, trace-decreasing sets stay
 * allowed), and qcw_set_state / qcw_set_state_c64 inputs must be Hermitian with unit trace
 * (within 1e-6; Sec. 5.2) -- the default fused kernel keeps only the Hermitian part of rho.
 * Violations return QCW_EINVAL with the state unchanged.  The checks run on the host, O(4^n)
 * for a state and O(d^3) per matrix. */
QCW_API qcw_status qcw_set_validation(qcw_ctx *ctx, int on);

/* Device pointer of rho and the context's stream (borrowed; valid until destroy).  Flushes
 * queued work and completes the matrix first (the HERM_WS pass keeps only the lower triangle
 * r >= c current between readouts): the buffer holds all of rho for work ordered on the
 * returned stream until the next evolution call. */
QCW_API qcw_status qcw_get_device_state(qcw_ctx *ctx, void **dev_rho, void **cuda_stream);

/* Number of qubits of the context. */
QCW_API int qcw_nqubits(const qcw_ctx *ctx);

/* ------------------------------------------------------------------------ state */

/* rho <- |0..0><0..0|. */
QCW_API qcw_status qcw_reset(qcw_ctx *ctx);

/* rho <- host matrix: 2 * 4^n doubles, row-major interleaved complex128 (converted to
 * complex64 on the device).  The buffer may be pageable or pinned. */
QCW_API qcw_status qcw_set_state(qcw_ctx *ctx, const double *rho_c128);

/* Same from host complex64 (2 * 4^n floats), copied without conversion. */
QCW_API qcw_status qcw_set_state_c64(qcw_ctx *ctx, const float *rho_c64);

/* Host copy of rho as complex128 (2 * 4^n doubles).  Synchronises. */
QCW_API qcw_status qcw_get_state(qcw_ctx *ctx, double *rho_c128_out);

/* ------------------------------------------------------------------- evolution */

/* rho <- U rho U^dagger for a one-qubit U (2x2, 8 doubles) on `target`: the paper's
 * pair update (Sec. 3.1, Eq. resmat1) on the row label with U and on the column label
 * with conj(U).  With ncontrols > 0 the pair update happens only where every qubit in
 * controls[] is 1 (a controlled-U); controls may be NULL when ncontrols == 0. */
QCW_API qcw_status qcw_apply_gate1(qcw_ctx *ctx, const double u[8], int target, const int *controls,
                           int ncontrols);

/* rho <- V rho V^dagger for a two-qubit V (4x4, 32 doubles) on (q1, q2), index
 * 2 * q(q1) + q(q2): the amplitude-quartet update of Sec. 3.2 (Eqs. twoopB, resmat2) on
 * rows with V and on columns with conj(V).  Controls as for qcw_apply_gate1. */
QCW_API qcw_status qcw_apply_gate2(qcw_ctx *ctx, const double u[32], int q1, int q2, const int *controls,
                           int ncontrols);

/* rho <- U rho U^dagger for a k-qubit U (1 <= k <= QCW_MAX_GATE_QUBITS; 2^k x 2^k, 2 * 4^k
 * doubles) on qubits[0..k-1]: the octet update of Sec. 3.3 generalised to 2^k-member groups. */
QCW_API qcw_status qcw_apply_gate(qcw_ctx *ctx, const double *u, const int *qubits, int k);

/* rho <- sum_j K_j rho K_j^dagger (the Kraus / POVM form of the paper's ensemble average,
 * Sec. 5.2.2, Eq. rhoE2) for nkraus (1..QCW_MAX_KRAUS) operators of k (1..QCW_MAX_GATE_QUBITS) qubits,
 * stored one after another (nkraus * 2 * 4^k doubles).  Trace-decreasing sets are accepted as
 * given.  One- and two-qubit channels act as composed superoperators (and join fused passes);
 * wider ones run term by term on the plain path with two scratch copies of rho, allocated on
 * first use and kept until the context is destroyed. */
QCW_API qcw_status qcw_apply_kraus(qcw_ctx *ctx, const double *kraus, int nkraus, const int *qubits,
                           int k);

/* ---------------------------------------------------------------- multiverse ensemble */

/* The paper's own noise method (Sec. 5.2.1, Eq. rhoE1; notebooks MV1 / MV2 / MVn): an ensemble
 * of nvec state vectors ("universes"), each evolved by the one- and two-qubit operators of
 * Sec. 3 (Op1 / Op2: Eqs. resmat1, resmat2), each noise step applying one operator Omega_k per
 * vector, chosen by the caller (the random draws of the method are the caller's), and the
 * density matrix formed as rho = sum_v w_v |psi_v><psi_v|.  With every branch of every noise
 * step enumerated and sqrt(p_k) folded into the Omega_k, the result equals the Kraus-sum
 * evolution (Eq. rhoE2).  Vectors are complex64 on the device, label bit n - 1 - q for qubit q;
 * operations are asynchronous on the ensemble's own stream. */
typedef struct qcw_ensemble qcw_ensemble;
/* nvec (1..65536) vectors of nqubits (1..QCW_MAX_QUBITS), all |0..0>. */
QCW_API qcw_status qcw_ensemble_create(int nqubits, int nvec, qcw_ensemble **out);
QCW_API qcw_status qcw_ensemble_destroy(qcw_ensemble *e);
/* Load / read all vectors: nvec * 2 * 2^n doubles (complex128, vector after vector). */
QCW_API qcw_status qcw_ensemble_set(qcw_ensemble *e, const double *psi_c128);
QCW_API qcw_status qcw_ensemble_get(qcw_ensemble *e, double *psi_c128);
/* psi_v <- U psi_v for every vector: U 2 x 2 on `target` (Eq. resmat1) or 4 x 4 on (q1, q2) with
 * the quartet order 2 q(q1) + q(q2) (Eq. resmat2); row-major complex128. */
QCW_API qcw_status qcw_ensemble_apply_gate1(qcw_ensemble *e, const double u[8], int target);
QCW_API qcw_status qcw_ensemble_apply_gate2(qcw_ensemble *e, const double u[32], int q1, int q2);
/* Noise step on `target`: psi_v <- Omega_{choice[v]} psi_v, Omega_0..Omega_{nomega-1} (1..16
 * one-qubit operators, 2 x 2 complex128 each, one after another); choice (host, nvec ints in
 * 0..nomega-1) holds the caller's draws.  QCW_EINVAL on a choice out of range. */
QCW_API qcw_status qcw_ensemble_apply_noise1(qcw_ensemble *e, const double *omegas, int nomega, int target,
                                          const int *choice);
/* ctx's rho <- sum_v weights[v] |psi_v><psi_v| (weights: host, nvec doubles; FP32 sums of FP32
 * products).  ctx must have the ensemble's qubit count; its queued work is dropped as by
 * qcw_set_state.  Ordered after the ensemble's operations; asynchronous on ctx's stream. */
QCW_API qcw_status qcw_ensemble_density(qcw_ensemble *e, const double *weights, qcw_ctx *ctx);

/* One element of a circuit handed over in a single call (qcw_apply_ops). */
#define QCW_OP_GATE 0
#define QCW_OP_KRAUS 1
typedef struct {
    int kind;           /* QCW_OP_GATE or QCW_OP_KRAUS */
    int k;              /* qubits: 1..QCW_MAX_GATE_QUBITS for a gate, 1..2 for Kraus */
    int qubits[QCW_MAX_GATE_QUBITS]; /* first k entries used, paper order */
    int nkraus;         /* Kraus operators (1..QCW_MAX_KRAUS) for QCW_OP_KRAUS; ignored for gates */
    long long offset;   /* index, in doubles, of the op's first matrix in `matrices` */
} qcw_op;

/* Apply nops operations in order, exactly as the matching sequence of qcw_apply_gate /
 * qcw_apply_kraus calls would (gates: one 2^k x 2^k matrix at matrices + offset; Kraus:
 * nkraus matrices one after another).  Every op is checked before any is applied, so on
 * QCW_EINVAL nothing has changed.  Both arrays may be freed when the call returns. */
QCW_API qcw_status qcw_apply_ops(qcw_ctx *ctx, const qcw_op *ops, int nops, const double *matrices);

/* Launch queued fused work (no-op in plain mode). */
QCW_API qcw_status qcw_flush(qcw_ctx *ctx);

/* Flush and wait for the context's stream. */
QCW_API qcw_status qcw_sync(qcw_ctx *ctx);

/* ---------------------------------------------------------------------- readout */

/* Tr rho = sum_i rho_ii (FP64).  Synchronises. */
QCW_API qcw_status qcw_trace(qcw_ctx *ctx, double *re, double *im);

/* sum_ij |rho_ij|^2, which equals Tr[rho . rho] (Sec. 5.2.3) for Hermitian rho (FP64).
 * Flushes queued work first.  When the last fused pass of the latest flush was a HERM_WS /
 * HERM_TC pass and nothing has changed rho since, the value comes from sums that pass took
 * over its write-back (squares in FP32 within a tile, FP64 above; no extra read of rho);
 * otherwise rho is read.  Either way the summation order is fixed (reproducible bit for bit).
 * Synchronises. */
QCW_API qcw_status qcw_purity(qcw_ctx *ctx, double *out);

/* p1_out[i] = sum over labels r with qubit i equal to 1 of Re rho_rr, i = 0..n-1 (FP64). */
QCW_API qcw_status qcw_probabilities(qcw_ctx *ctx, double *p1_out);

/* Polarisation vectors (Sec. 5.2: the one-qubit form rho = (1 + P . sigma) / 2 with
 * P = Tr[sigma rho]): out[3 q + i] = Tr[sigma_i^(q) rho] for qubit q < n and i = 0, 1, 2 for
 * x, y, z (3 n doubles, caller-owned; FP64 sums of the FP32 elements).  Reads the lower
 * triangle only.  Flushes queued work first; synchronises. */
QCW_API qcw_status qcw_polarization(qcw_ctx *ctx, double *out);

/* Spin correlation tensor of qubits q1 != q2 (Sec. 5.2's two-qubit form):
 * out[3 i + j] = Tr[sigma_i^(q1) sigma_j^(q2) rho], i, j = x, y, z (9 doubles).  QCW_EINVAL for
 * equal or out-of-range qubits.  Flushes queued work first; synchronises. */
QCW_API qcw_status qcw_correlation(qcw_ctx *ctx, int q1, int q2, double *out);

/* von Neumann entropy S = -Tr[rho_A log2 rho_A] of the reduced state rho_A of the kept qubits
 * (Sec. 5.2; in bits, as S tends to n_q in the classical limit), keep strictly ascending,
 * 1 <= nkeep <= 6.  rho_A is the GPU partial trace (qcw_partial_trace), its eigenvalues come
 * from a host Jacobi eigensolver in FP64 (eigenvalues below 1e-15 count as 0).  Flushes queued
 * work first; synchronises. */
QCW_API qcw_status qcw_entropy(qcw_ctx *ctx, const int *keep, int nkeep, double *out);

/* Eigenvalues of the reduced state rho_A of the kept qubits, ascending, into out[2^nkeep]
 * (Sec. 5.2.3: the eigenvalues are monitored as the noise drives rho to the classical form,
 * where they all approach 1 / 2^n_q).  keep strictly ascending, 1 <= nkeep <= 6; the GPU
 * partial trace followed by the host Jacobi eigensolver in FP64, as qcw_entropy.  Flushes
 * queued work first; synchronises. */
QCW_API qcw_status qcw_eigenvalues(qcw_ctx *ctx, const int *keep, int nkeep, double *out);

/* Fidelity F = Tr sqrt(sqrt(sigma) rho_A sqrt(sigma)) (Sec. 5.2) of the reduced state of the kept
 * qubits with the caller's Hermitian positive semidefinite sigma (host complex128, 2^nkeep x
 * 2^nkeep row-major, copied during the call); 1 <= nkeep <= 6.  Same path as qcw_entropy; the
 * paper approximates F from the eigenvalues of rho . rho_0, this computes it through the
 * Hermitian form.  Synchronises. */
QCW_API qcw_status qcw_fidelity(qcw_ctx *ctx, const int *keep, int nkeep, const double *sigma_c128, double *out);

/* Asynchronous readout of the trace, purity and probabilities (the values of qcw_trace,
 * qcw_purity and qcw_probabilities, same arithmetic) at this point of the evolution, e.g.
 * every 100 gates as in the paper's noise studies (Sec. 5.2.3).  The paper has no asynchronous
 * form; it lets the host queue and plan the next operations while the GPU works.
 * qcw_checkpoint flushes queued work, enqueues the FP64 reductions and their copy to pinned
 * host memory on the context's stream, and returns at once with *ticket (0, 1, 2, ... per
 * context).  qcw_checkpoint_read waits for checkpoint `ticket` and writes
 *   out[0] = Re tr rho, out[1] = Im tr rho, out[2 + q] = P(qubit q = 1) for q < n,
 *   out[2 + n] = purity
 * (n + 3 doubles, caller-owned).  Results are kept for the last QCW_CHECKPOINT_SLOTS
 * checkpoints; reading an older or a future ticket returns QCW_EINVAL.  A fused pass whose
 * in-kernel wait ran out before the checkpoint makes the read return QCW_ETIMEOUT. */
#define QCW_CHECKPOINT_SLOTS 64
QCW_API qcw_status qcw_checkpoint(qcw_ctx *ctx, long long *ticket);
QCW_API qcw_status qcw_checkpoint_read(qcw_ctx *ctx, long long ticket, double *out);

/* Projective measurement of `qubit` (the ancilla read-out of Sec. 5.4.1; textbook form):
 * p_m = sum_{r: q(r) = m} Re rho_rr; the outcome m is `forced` when it is 0 or 1,
 * otherwise m = 0 iff u < p_0 (u: caller's uniform draw in [0, 1)).  Then
 * rho <- P_m rho P_m / p_m with the scale computed in FP64.  *outcome and *prob receive m
 * and p_m.  If p_m < 1e-12 the call returns QCW_EZEROPROB and rho is unchanged. */
QCW_API qcw_status qcw_measure(qcw_ctx *ctx, int qubit, int forced, double u, int *outcome, double *prob);

/* Reduced density matrix of the kept qubits (strictly ascending, 0 <= nkeep <= n):
 * out[a, a'] = sum_b rho[(a b), (a' b)], where the first kept qubit is the most significant
 * bit of a.  out_c128 receives 2 * 4^nkeep doubles (subsystem states of Sec. 5.2.3). */
QCW_API qcw_status qcw_partial_trace(qcw_ctx *ctx, const int *keep, int nkeep, double *out_c128);

/* Size of the fixed result array used by qcw_partial_trace_static: 4^6 complex128 entries. */
#define QCW_PT_STATIC_MAX_ENTRIES 4096

/* Partial trace that allocates nothing (the paper has no counterpart; this is a service for
 * callers that must not allocate device memory).  Some callers cannot call cudaMalloc: while
 * any thread of the process captures a CUDA graph in global mode, cudaMalloc and cudaFree are
 * not allowed; an application whose allocator already holds the whole device budget has no
 * memory to give; and cudaFree synchronises the device, which a latency-critical loop cannot
 * afford.  qcw_partial_trace takes its device result buffer from cudaMallocAsync; this variant
 * instead writes into one array of QCW_PT_STATIC_MAX_ENTRIES complex128 values (64 KiB) that
 * lives in device memory as part of the library, on every GPU that loads it, until exit.
 *
 * dev_rho: caller's device rho of nqubits (row-major complex64, the layout above); cuda_stream:
 * a cudaStream_t (NULL = legacy default stream) on the current device; keep / nkeep / out_c128
 * as for qcw_partial_trace (host output of 2 * 4^nkeep doubles).  nkeep above 6 returns
 * QCW_EINVAL ("keeps at most 6 qubits").  The call waits for its stream before returning.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture starts.  The kernel
 * writes every result entry, so nothing has to start at zero; the array keeps the last call's
 * contents.  All calls share the one array: calls whose work overlaps on the GPU (different
 * streams, or threads racing on one device) race on it and must be serialised by the caller. */
QCW_API qcw_status qcw_partial_trace_static(const void *dev_rho, int nqubits, const int *keep, int nkeep,
                                    void *cuda_stream, double *out_c128);

/* ---------------------------------------------------------------- batched circuits */

/* Many independent circuits in one launch: the paper's multiverse runs independent paths on
 * separate processors (Sec. 5.1, Sec. 5.2.1); here they share one GPU.  Circuit j has
 * nqubits[j] (1..QCW_MAX_QUBITS) qubits, starts in |0..0><0..0| and applies
 * ops[op_begin[j] .. op_begin[j+1]) (1- and 2-qubit gates and Kraus channels, matrices as in
 * qcw_apply_ops).  fuse_k (0 = chosen per circuit by the cost model, else 2..5) bounds the
 * qubits of a fused pass.  Creation plans every circuit, allocates one device arena for all
 * states and captures the whole run (one persistent kernel) in a CUDA graph on cuda_stream
 * (NULL: a non-blocking stream owned by the batch, since the legacy stream cannot be captured).  All arrays are copied; the caller may free them on return. */
typedef struct qcw_batch qcw_batch;
QCW_API qcw_status qcw_batch_create(int ncirc, const int *nqubits, const long long *op_begin, const qcw_op *ops,
                                    const double *matrices, int fuse_k, void *cuda_stream, qcw_batch **out);
/* Launch the captured graph (asynchronous).  Each run starts every circuit from |0..0><0..0|. */
QCW_API qcw_status qcw_batch_run(qcw_batch *b);
/* Wait for the last run, at most timeout_s seconds (< 0: no limit): QCW_ETIMEOUT if it is
 * still running, or if a work item's bounded dependency wait ran out inside the kernel. */
QCW_API qcw_status qcw_batch_wait(qcw_batch *b, double timeout_s);
/* Readouts of the last run (waits): p1 gets sum_j nqubits[j] values (circuit order, per qubit
 * P(q = 1)), purity and trace one value per circuit (FP64).  Any pointer may be NULL. */
QCW_API qcw_status qcw_batch_results(qcw_batch *b, double *p1, double *purity, double *trace);
/* Final rho of one circuit as host complex128 (2 * 4^n doubles). */
QCW_API qcw_status qcw_batch_get_state(qcw_batch *b, int circuit, double *rho_c128);
/* Work items, fused passes, phases and modeled SM-seconds of one run. */
QCW_API qcw_status qcw_batch_info(qcw_batch *b, long long *items, long long *passes, long long *phases,
                                  double *modeled_sm_s);
/* Diagnostics: bound every in-kernel dependency wait to `polls` polls (~128 ns each) and, when
 * stall_item >= 0, make that item wait on a counter that is never set (a host-side injected
 * fault: the wait runs out, the run ends with QCW_ETIMEOUT from qcw_batch_wait, the context
 * stays usable).  stall_item = -1 restores the normal item list. */
QCW_API qcw_status qcw_batch_set_wait_limit(qcw_batch *b, long long polls, int stall_item);
QCW_API qcw_status qcw_batch_destroy(qcw_batch *b);

/* ---------------------------------------------------------------- serving loop */

/* Continuous batching of circuit requests.  A request (1..13 qubits, op list as for
 * qcw_apply_ops) is planned when submitted and waits in FIFO order; it is admitted while the
 * summed footprint 16 * 4^n bytes of live requests stays within budget_bytes (at most
 * max_live at once); its rho stays on the device until it finishes.  Each qcw_server_step
 * waits (boundedly) for the previous step, harvests finished requests, admits waiting ones
 * and launches one engine kernel over every live request: requests whose rho fits one tile
 * finish inside the step, larger ones advance by up to passes_per_step fused passes.
 * Requests submitted while a step runs join the next one.  A request's result does not depend
 * on which other requests share its steps. */
typedef struct qcw_server qcw_server;
typedef struct {
    long long id;
    int nqubits;
    int status;        /* QCW_OK, or QCW_ETIMEOUT if a wait in its last step ran out */
    double trace;      /* Re Tr rho */
    double purity;     /* sum |rho_ij|^2 */
    double p1[QCW_MAX_QUBITS]; /* P(q = 1) for q < nqubits */
    double t_submit, t_done;   /* host steady-clock seconds */
} qcw_result;
/* cuda_stream NULL: the server creates and owns a non-blocking stream. */
QCW_API qcw_status qcw_server_create(size_t budget_bytes, int max_live, int passes_per_step, void *cuda_stream,
                                     qcw_server **out);
/* Plan and queue one request; *id receives its id.  Thread-safe with respect to qcw_server_step. */
QCW_API qcw_status qcw_server_submit(qcw_server *s, int nqubits, const qcw_op *ops, int nops, const double *matrices,
                                     long long *id);
/* One engine step (returns once the next step is launched; *launched_items may be NULL). */
QCW_API qcw_status qcw_server_step(qcw_server *s, int *launched_items);
/* Step until nothing waits or runs, at most timeout_s seconds (< 0: the server's wait limit per step). */
QCW_API qcw_status qcw_server_drain(qcw_server *s, double timeout_s);
/* Move up to max finished results (in completion order) to out; *count receives how many. */
QCW_API qcw_status qcw_server_poll(qcw_server *s, qcw_result *out, int max, int *count);
QCW_API qcw_status qcw_server_stats(qcw_server *s, long long *waiting, long long *live, long long *completed,
                                    long long *bytes_in_use);
/* Diagnostics: host wait limit per step (seconds), in-kernel dependency-wait bound (polls), and
 * with stall_next_step != 0 one item of the next step waits on a counter nothing sets (the step
 * then reports QCW_ETIMEOUT; the server stays usable). */
QCW_API qcw_status qcw_server_set_limits(qcw_server *s, double wait_limit_s, long long polls, int stall_next_step);
QCW_API qcw_status qcw_server_destroy(qcw_server *s);

/* ---------------------------------------------------------------- diagnostics */

/* Message of the last failure on this thread ("" if none). */
QCW_API const char *qcw_last_error(void);

/* Static text for a status code. */
QCW_API const char *qcw_strerror(qcw_status st);

/* Counters since creation or the last qcw_stats_reset: kernel launches of this library,
 * fused passes, and the summed device time (ms) of the fused-pass kernels when
 * timing is enabled with qcw_enable_pass_timing(ctx, 1).  Any pointer may be NULL. */
QCW_API qcw_status qcw_stats(qcw_ctx *ctx, long long *launches, long long *fused_passes,
                     double *fused_pass_ms, long long *timed_passes);
QCW_API qcw_status qcw_stats_reset(qcw_ctx *ctx);
QCW_API qcw_status qcw_enable_pass_timing(qcw_ctx *ctx, int on);

#ifdef __cplusplus
}
#endif

#endif /* QCW_H */
