// C ABI of the qcw library: argument checks, context lifetime, the plain (one launch per
// operation) path and the FP64 readouts.  The fused path lives in fused.cu / planner.cpp.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "hermitian.h"
#include "qcw_internal.h"
#include "tile.h"

using namespace qcw;

static thread_local std::string g_err;

qcw_status qcw::set_error(qcw_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

qcw_status qcw::cuda_error(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return QCW_ECUDA;
}

qcw_status qcw::ensure_smem_attr(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set[{func, dev}];
    if (bytes <= cur) return QCW_OK;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_error(e, "max dynamic shared memory attribute");
    cur = bytes;
    return QCW_OK;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);       \
    } while (0)

#define CKLAUNCH(ctx, nlaunch)                                     \
    do {                                                           \
        (ctx)->launches += (nlaunch);                              \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return cuda_error(e_, "kernel launch"); \
    } while (0)

#define CHECK_CTX(ctx)                                                             \
    do {                                                                           \
        if (!(ctx)) return set_error(QCW_EINVAL, "null context");                  \
    } while (0)

// ------------------------------------------------------------------ argument checks
static bool all_finite(const double *a, size_t cnt)
{
    for (size_t i = 0; i < cnt; i++)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// ------------------------------------------------------------------ validation (qcw_set_validation)
// The paper's gate operators are unitary (Sec. 3) and its noise ensembles keep the trace
// (Eq. rhoE1: sum of the path weights is 1); a Kraus set may also lose trace, never gain it.  A
// state is Hermitian with unit trace (Sec. 5.2).  Tolerance 1e-6 throughout.
constexpr double kValidTol = 1e-6;

static bool is_unitary(const double *u, int d)
{
    const c128 *U = reinterpret_cast<const c128 *>(u);
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) {
            c128 g = 0;  // (U^dagger U)_ij
            for (int l = 0; l < d; l++) g += std::conj(U[l * d + i]) * U[l * d + j];
            if (std::abs(g - c128(i == j ? 1.0 : 0.0, 0.0)) > kValidTol) return false;
        }
    return true;
}

// sum_j K_j^dagger K_j <= I (its largest eigenvalue at most 1 + tolerance).
static bool kraus_keeps_or_loses_trace(const double *ks, int nk, int d)
{
    const c128 *K = reinterpret_cast<const c128 *>(ks);
    std::vector<c128> M((size_t)d * d, c128(0, 0));
    for (int t = 0; t < nk; t++)
        for (int i = 0; i < d; i++)
            for (int j = 0; j < d; j++)
                for (int l = 0; l < d; l++)
                    M[(size_t)i * d + j] += std::conj(K[(size_t)t * d * d + l * d + i]) * K[(size_t)t * d * d + l * d + j];
    std::vector<double> w(d);
    herm_eig(M.data(), d, w.data(), nullptr);
    return w[d - 1] <= 1.0 + kValidTol;
}

template <typename T>
static bool is_density(const T *rho, int n)
{
    const size_t dim = (size_t)1 << n;
    double tr_re = 0, tr_im = 0;
    for (size_t i = 0; i < dim; i++) {
        tr_re += rho[2 * (i * dim + i)];
        tr_im += rho[2 * (i * dim + i) + 1];
        for (size_t j = 0; j < i; j++) {
            const T *a = rho + 2 * (i * dim + j), *b = rho + 2 * (j * dim + i);
            if (std::fabs((double)a[0] - (double)b[0]) > kValidTol || std::fabs((double)a[1] + (double)b[1]) > kValidTol)
                return false;
        }
    }
    return std::fabs(tr_re - 1.0) <= kValidTol && std::fabs(tr_im) <= kValidTol;
}

static qcw_status check_qubits(int n, const int *qs, int k, const int *ctrl, int nc)
{
    if (k < 1 || nc < 0 || k + nc > n) return set_error(QCW_EINVAL, "bad qubit count");
    if (!qs || (nc > 0 && !ctrl)) return set_error(QCW_EINVAL, "null qubit list");
    unsigned seen = 0;
    for (int j = 0; j < k + nc; j++) {
        int q = j < k ? qs[j] : ctrl[j - k];
        if (q < 0 || q >= n) return set_error(QCW_EINVAL, "qubit index out of range");
        if (seen & (1u << q)) return set_error(QCW_EINVAL, "repeated qubit");
        seen |= 1u << q;
    }
    return QCW_OK;
}

static std::vector<c128> to_c128(const double *a, size_t count)
{
    std::vector<c128> v(count);
    for (size_t i = 0; i < count; i++) v[i] = c128(a[2 * i], a[2 * i + 1]);
    return v;
}

static float2 f2(c128 z) { return make_float2((float)z.real(), (float)z.imag()); }

// Superoperator of a Kraus set on k qubits: S[(r',c'), (r,c)] = sum_j K_j[r', r] conj(K_j[c', c]),
// so that rho'_{r'c'} = sum_{rc} S rho_{rc} = sum_j (K_j rho K_j^dagger)_{r'c'} (Eq. rhoE2).
static std::vector<c128> kraus_superop(const std::vector<c128> &ks, int nk, int k)
{
    int d = 1 << k, D = d * d;
    std::vector<c128> s((size_t)D * D, c128(0, 0));
    for (int j = 0; j < nk; j++) {
        const c128 *K = ks.data() + (size_t)j * d * d;
        for (int r2 = 0; r2 < d; r2++)
            for (int c2 = 0; c2 < d; c2++)
                for (int r = 0; r < d; r++)
                    for (int c = 0; c < d; c++)
                        s[(size_t)(r2 * d + c2) * D + (r * d + c)] += K[r2 * d + r] * std::conj(K[c2 * d + c]);
    }
    return s;
}

// ------------------------------------------------------------------ plain launches
namespace qcw {

qcw_status plain_super(qcw_ctx *c, const std::vector<c128> &s, const int *qs, int k);
static std::vector<c128> gate_superop(const c128 *u, int k);

// An uncontrolled gate runs as its superoperator U (x) conj U in the Pauli basis (k_super1 /
// k_super2), which keeps the trace exactly where the complex product would let the rounding of
// U's entries move it; controlled gates act on the row and the column side separately.
qcw_status plain_gate1(qcw_ctx *c, const c128 *u, int t, const int *ctrl, int nc)
{
    const int n = c->n;
    if (nc == 0) return plain_super(c, gate_superop(u, 1), &t, 1);
    Gate1Params p{};
    for (int i = 0; i < 4; i++) p.u[i] = f2(u[i]);
    p.pc = n - 1 - t;
    p.pr = 2 * n - 1 - t;
    for (int j = 0; j < nc; j++) {
        p.cmask_c |= 1ull << (n - 1 - ctrl[j]);
        p.cmask_r |= 1ull << (2 * n - 1 - ctrl[j]);
    }
    launch_gate1(p, c->rho, n, c->nsm, c->stream);
    CKLAUNCH(c, 1);
    return QCW_OK;
}

static void quartet_layout(int n, int q1, int q2, int *pos, uint64_t *offr, uint64_t *offc)
{
    int pr1 = 2 * n - 1 - q1, pr2 = 2 * n - 1 - q2, pc1 = n - 1 - q1, pc2 = n - 1 - q2;
    int v[4] = {pc1, pc2, pr1, pr2};
    for (int a = 0; a < 4; a++)
        for (int b = a + 1; b < 4; b++)
            if (v[b] < v[a]) { int t = v[a]; v[a] = v[b]; v[b] = t; }
    for (int a = 0; a < 4; a++) pos[a] = v[a];
    for (int i = 0; i < 4; i++) {
        offr[i] = (((uint64_t)(i >> 1) & 1) << pr1) | (((uint64_t)i & 1) << pr2);
        offc[i] = (((uint64_t)(i >> 1) & 1) << pc1) | (((uint64_t)i & 1) << pc2);
    }
}

// One entry per row, at a distinct column, each exactly 1, -1, i or -i: sigma[i] = its column.
static bool monomial4(const c128 *u, int *sigma, c128 *val)
{
    bool used[4] = {false, false, false, false};
    for (int i = 0; i < 4; i++) {
        sigma[i] = -1;
        for (int j = 0; j < 4; j++) {
            const c128 z = u[4 * i + j];
            if (z == c128(0, 0)) continue;
            const bool unit = z == c128(1, 0) || z == c128(-1, 0) || z == c128(0, 1) || z == c128(0, -1);
            if (!unit || sigma[i] >= 0 || used[j]) return false;
            sigma[i] = j;
            val[i] = z;
            used[j] = true;
        }
        if (sigma[i] < 0) return false;
    }
    return true;
}

qcw_status plain_gate2(qcw_ctx *c, const c128 *u, int q1, int q2, const int *ctrl, int nc)
{
    const int n = c->n;
    int sigma[4];
    c128 val[4];
    if (nc == 0 && monomial4(u, sigma, val)) {  // CNOT, CZ, SWAP, ...: an exact permutation
        Mono2Params p{};
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) p.ph[4 * i + j] = f2(val[i] * std::conj(val[j]));
        quartet_layout(n, q1, q2, p.pos, p.off_r, p.off_c);
        for (int i = 0; i < 4; i++) {
            p.src_r[i] = p.off_r[sigma[i]];
            p.src_c[i] = p.off_c[sigma[i]];
        }
        launch_mono2(p, c->rho, n, c->nsm, c->stream);
        CKLAUNCH(c, 1);
        return QCW_OK;
    }
    if (nc == 0) {
        const int qs[2] = {q1, q2};
        return plain_super(c, gate_superop(u, 2), qs, 2);
    }
    Gate2Params p{};
    for (int i = 0; i < 16; i++) p.u[i] = f2(u[i]);
    quartet_layout(n, q1, q2, p.pos, p.off_r, p.off_c);
    for (int j = 0; j < nc; j++) {
        p.cmask_c |= 1ull << (n - 1 - ctrl[j]);
        p.cmask_r |= 1ull << (2 * n - 1 - ctrl[j]);
    }
    launch_gate2(p, c->rho, n, c->nsm, c->stream);
    CKLAUNCH(c, 1);
    return QCW_OK;
}

// k-qubit dense gate as two passes: U on the row labels, then conj(U) on the column labels.
qcw_status plain_gatek(qcw_ctx *c, const c128 *u, const int *qs, int k, float2 *target = nullptr)
{
    const int n = c->n, m = 1 << k;
    for (int side = 0; side < 2; side++) {
        GateKParams p{};
        p.k = k;
        int base = side == 0 ? 2 * n - 1 : n - 1;  // row bits, then column bits
        for (int i = 0; i < m * m; i++) p.u[i] = f2(side == 0 ? u[i] : std::conj(u[i]));
        int v[5];
        for (int j = 0; j < k; j++) v[j] = base - qs[j];
        for (int i = 0; i < m; i++) {
            uint64_t o = 0;
            for (int j = 0; j < k; j++)
                if ((i >> (k - 1 - j)) & 1) o |= 1ull << v[j];
            p.off[i] = o;
        }
        for (int a = 0; a < k; a++)
            for (int b = a + 1; b < k; b++)
                if (v[b] < v[a]) { int t = v[a]; v[a] = v[b]; v[b] = t; }
        for (int j = 0; j < k; j++) p.pos[j] = v[j];
        launch_gatek_side(p, target ? target : c->rho, n, c->nsm, c->stream);
        CKLAUNCH(c, 1);
    }
    return QCW_OK;
}

// Superoperator of a k-qubit gate: S = U (x) conj(U), index (row, column) of the group member.
static std::vector<c128> gate_superop(const c128 *u, int k)
{
    const int d = 1 << k, D = d * d;
    std::vector<c128> s((size_t)D * D);
    for (int r2 = 0; r2 < d; r2++)
        for (int c2 = 0; c2 < d; c2++)
            for (int r = 0; r < d; r++)
                for (int cc = 0; cc < d; cc++)
                    s[(size_t)(r2 * d + c2) * D + (r * d + cc)] = u[r2 * d + r] * std::conj(u[c2 * d + cc]);
    return s;
}

qcw_status plain_super(qcw_ctx *c, const std::vector<c128> &s, const int *qs, int k)
{
    const int n = c->n;
    if (k == 1) {
        Super1Params p{};
        double R[4][4];
        pauli_transfer1(s.data(), R);
        for (int i = 0; i < 16; i++) p.r[i] = (float)R[i / 4][i % 4];
        p.pc = n - 1 - qs[0];
        p.pr = 2 * n - 1 - qs[0];
        launch_super1(p, c->rho, n, c->nsm, c->stream);
    } else if (k == 2) {
        Super2Params p{};
        double R[16][16];
        pauli_transfer(s, R);
        for (int i = 0; i < 256; i++) p.r[i] = (float)R[i / 16][i % 16];
        quartet_layout(n, qs[0], qs[1], p.pos, p.off_r, p.off_c);
        launch_super2(p, c->rho, n, c->nsm, c->stream);
    } else {
        return set_error(QCW_ENOTSUP, "channels act on 1 or 2 qubits");
    }
    CKLAUNCH(c, 1);
    return QCW_OK;
}

// Half storage: the warp-specialised pass keeps only the lower triangle current; everything
// that reads the other triangle (plain kernels, the other fused kernels, state downloads, direct
// device access) completes the matrix first.  The readouts (trace, probabilities, purity, Pauli
// expectations, partial trace) and the measurement projection work on the lower triangle as it is.
qcw_status ensure_full(qcw_ctx *c)
{
    if (!c->half) return QCW_OK;
    launch_symmetrize(c->rho, c->n, c->nsm, c->stream);
    CKLAUNCH(c, 1);
    c->half = false;
    return QCW_OK;
}

// Kraus channel on k >= 3 qubits (Eq. rhoE2 term by term): acc = sum_j K_j rho K_j^dagger, each
// term on a copy of rho with the dense k-qubit side passes (K_j on the rows, conj(K_j) on the
// columns), then rho = acc.  Two scratch copies of rho stay allocated for later channels.
static qcw_status plain_kraus_list(qcw_ctx *c, const QOp &op)
{
    const size_t bytes = sizeof(float2) << (2 * c->n);
    for (float2 **b : {&c->d_kacc, &c->d_ktmp})
        if (!*b && cudaMalloc(b, bytes) != cudaSuccess) {
            cudaGetLastError();
            *b = nullptr;
            return set_error(QCW_ENOMEM, "Kraus scratch");
        }
    const size_t msz = (size_t)1 << (2 * op.k);
    const size_t nk = op.m.size() / msz;
    CK(cudaMemsetAsync(c->d_kacc, 0, bytes, c->stream));
    for (size_t j = 0; j < nk; j++) {
        CK(cudaMemcpyAsync(c->d_ktmp, c->rho, bytes, cudaMemcpyDeviceToDevice, c->stream));
        qcw_status st = plain_gatek(c, op.m.data() + j * msz, op.qubits, op.k, c->d_ktmp);
        if (st) return st;
        launch_accumulate(c->d_kacc, c->d_ktmp, c->n, c->nsm, c->stream);
        CKLAUNCH(c, 1);
    }
    CK(cudaMemcpyAsync(c->rho, c->d_kacc, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return QCW_OK;
}

qcw_status plain_apply(qcw_ctx *c, const QOp &op)
{
    c->state_ver++;
    qcw_status fs = ensure_full(c);
    if (fs) return fs;
    if (op.kind == 2) return plain_kraus_list(c, op);
    if (op.kind == 1) return plain_super(c, op.m, op.qubits, op.k);
    if (op.k == 1) return plain_gate1(c, op.m.data(), op.qubits[0], op.controls, op.ncontrols);
    if (op.k == 2) return plain_gate2(c, op.m.data(), op.qubits[0], op.qubits[1], op.controls, op.ncontrols);
    return plain_gatek(c, op.m.data(), op.qubits, op.k);
}

}  // namespace qcw

static qcw_status submit(qcw_ctx *c, QOp &&op)
{
    if (c->mode == QCW_MODE_FUSED) {
        c->queue.push_back(std::move(op));
        return QCW_OK;
    }
    return plain_apply(c, op);
}

// ------------------------------------------------------------------ lifetime
static void ctx_free(qcw_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    fused_destroy(c);
    if (c->owns_rho && c->rho) cudaFree(c->rho);
    if (c->d_partials) cudaFree(c->d_partials);
    if (c->d_result) cudaFree(c->d_result);
    if (c->h_result) cudaFreeHost(c->h_result);
    if (c->d_staging) cudaFree(c->d_staging);
    if (c->d_kacc) cudaFree(c->d_kacc);
    if (c->d_ktmp) cudaFree(c->d_ktmp);
    if (c->d_ckpt) cudaFree(c->d_ckpt);
    if (c->h_ckpt) cudaFreeHost(c->h_ckpt);
    for (cudaEvent_t e : c->ckpt_ev)
        if (e) cudaEventDestroy(e);
    if (c->owns_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static qcw_status ctx_common(qcw_ctx *c)
{
    const char *v = getenv("QCW_VALIDATE");
    c->validate = v && v[0] && v[0] != '0';
    CK(cudaGetDevice(&c->dev));
    CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev));
    c->red_blocks = reduce_blocks(c->nsm);
    if (cudaMalloc(&c->d_partials, sizeof(double) * (size_t)c->red_blocks * (QCW_MAX_QUBITS + 2)) != cudaSuccess)
        return set_error(QCW_ENOMEM, "reduction scratch");
    if (cudaMalloc(&c->d_result, 64 * sizeof(double)) != cudaSuccess) return set_error(QCW_ENOMEM, "result block");
    if (cudaMallocHost(&c->h_result, 64 * sizeof(double)) != cudaSuccess) return set_error(QCW_ENOMEM, "pinned result");
    CK(cudaMemset(c->d_result, 0, 64 * sizeof(double)));
    return QCW_OK;
}

extern "C" qcw_status qcw_create(int nqubits, qcw_ctx **out)
{
    if (!out) return set_error(QCW_EINVAL, "null out");
    *out = nullptr;
    if (nqubits < 1 || nqubits > QCW_MAX_QUBITS) return set_error(QCW_EINVAL, "nqubits out of range");
    qcw_ctx *c = new qcw_ctx();
    c->n = nqubits;
    qcw_status st = ctx_common(c);
    if (!st) {
        size_t bytes = sizeof(float2) << (2 * nqubits);
        if (cudaMalloc(&c->rho, bytes) != cudaSuccess) {
            cudaGetLastError();
            st = set_error(QCW_ENOMEM, "rho allocation");
        } else {
            c->owns_rho = true;
        }
    }
    if (!st) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_error(e, "stream");
        else c->owns_stream = true;
    }
    if (!st) st = qcw_reset(c);
    if (st) {
        ctx_free(c);
        return st;
    }
    *out = c;
    return QCW_OK;
}

extern "C" qcw_status qcw_create_from_ptr(int nqubits, void *dev_rho, void *cuda_stream, qcw_ctx **out)
{
    if (!out) return set_error(QCW_EINVAL, "null out");
    *out = nullptr;
    if (nqubits < 1 || nqubits > QCW_MAX_QUBITS) return set_error(QCW_EINVAL, "nqubits out of range");
    if (!dev_rho || (reinterpret_cast<uintptr_t>(dev_rho) & 15)) return set_error(QCW_EINVAL, "rho must be 16-byte aligned");
    qcw_ctx *c = new qcw_ctx();
    c->n = nqubits;
    c->rho = static_cast<float2 *>(dev_rho);
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    qcw_status st = ctx_common(c);
    if (st) {
        ctx_free(c);
        return st;
    }
    *out = c;
    return QCW_OK;
}

extern "C" qcw_status qcw_destroy(qcw_ctx *ctx)
{
    ctx_free(ctx);
    return QCW_OK;
}

extern "C" int qcw_nqubits(const qcw_ctx *ctx) { return ctx ? ctx->n : -1; }

extern "C" qcw_status qcw_set_validation(qcw_ctx *ctx, int on)
{
    CHECK_CTX(ctx);
    ctx->validate = on != 0;
    return QCW_OK;
}

extern "C" qcw_status qcw_set_fused_kernel(qcw_ctx *ctx, int which)
{
    CHECK_CTX(ctx);
    if (which < QCW_FUSED_KERNEL_AUTO || which > QCW_FUSED_KERNEL_HERM_TC) return set_error(QCW_EINVAL, "bad kernel choice");
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    ctx->fused_kernel = which;
    return QCW_OK;
}

extern "C" qcw_status qcw_get_device_state(qcw_ctx *ctx, void **dev_rho, void **cuda_stream)
{
    CHECK_CTX(ctx);
    qcw_status st = fused_flush(ctx);
    if (!st) st = ensure_full(ctx);
    if (st) return st;
    if (dev_rho) *dev_rho = ctx->rho;
    if (cuda_stream) *cuda_stream = ctx->stream;
    ctx->state_ver++;  // the caller may write rho
    return QCW_OK;
}

extern "C" qcw_status qcw_set_mode(qcw_ctx *ctx, int mode, int fuse_k)
{
    CHECK_CTX(ctx);
    if (mode != QCW_MODE_PLAIN && mode != QCW_MODE_FUSED) return set_error(QCW_EINVAL, "bad mode");
    if (fuse_k != 0 && (fuse_k < 2 || fuse_k > QCW_MAX_GATE_QUBITS)) return set_error(QCW_EINVAL, "bad fuse_k");
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    ctx->mode = mode;
    ctx->fuse_k = fuse_k;
    return QCW_OK;
}

// ------------------------------------------------------------------ state
// A fused pass whose in-kernel wait ran out left rho undefined: the error word stays set (and
// readouts fail) until the state is replaced.
static qcw_status clear_error_word(qcw_ctx *c)
{
    CK(cudaMemsetAsync(device_error_word(c), 0, sizeof(unsigned long long), c->stream));
    return QCW_OK;
}

static qcw_status check_error_word(qcw_ctx *c, unsigned long long word)
{
    if (word) return set_error(QCW_ETIMEOUT, "fused pass: an in-kernel wait ran out; rho is undefined until reset");
    return QCW_OK;
}

extern "C" qcw_status qcw_set_fused_wait_limit(qcw_ctx *ctx, unsigned polls, int stall_tile)
{
    CHECK_CTX(ctx);
    if (stall_tile < -1) return set_error(QCW_EINVAL, "bad stall tile");
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    ctx->wait_limit = polls;
    ctx->stall_tile = stall_tile;
    return QCW_OK;
}

qcw_status qcw::begin_state_replace(qcw_ctx *c)
{
    c->queue.clear();
    c->half = false;
    c->state_ver++;
    return clear_error_word(c);
}

extern "C" qcw_status qcw_reset(qcw_ctx *ctx)
{
    CHECK_CTX(ctx);
    ctx->queue.clear();
    // In fused mode with the warp-specialised kernel (6 qubits and up) the next passes keep only
    // the lower triangle current anyway: write that half of |0..0><0..0| and start in half storage.
    ctx->half = ctx->mode == QCW_MODE_FUSED && ctx->n >= 6 &&
                (ctx->fused_kernel == QCW_FUSED_KERNEL_AUTO || ctx->fused_kernel == QCW_FUSED_KERNEL_HERM_WS ||
                 ctx->fused_kernel == QCW_FUSED_KERNEL_HERM_TC);
    ctx->state_ver++;
    qcw_status st = clear_error_word(ctx);
    if (st) return st;
    launch_zero_state(ctx->rho, ctx->n, ctx->half, ctx->nsm, ctx->stream);
    CKLAUNCH(ctx, 1);
    return QCW_OK;
}

static const size_t kStageElems = (size_t)1 << 22;  // 4 Mi complex128 = 64 MiB per chunk

static qcw_status ensure_staging(qcw_ctx *c)
{
    if (c->d_staging) return QCW_OK;
    size_t bytes = kStageElems * sizeof(double2);
    if (cudaMalloc(&c->d_staging, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(QCW_ENOMEM, "staging buffer");
    }
    c->staging_bytes = bytes;
    return QCW_OK;
}

extern "C" qcw_status qcw_set_state(qcw_ctx *ctx, const double *rho_c128)
{
    CHECK_CTX(ctx);
    if (!rho_c128) return set_error(QCW_EINVAL, "null state");
    if (ctx->validate && !is_density(rho_c128, ctx->n))
        return set_error(QCW_EINVAL, "state is not Hermitian with unit trace (validation)");
    qcw_status st = ensure_staging(ctx);
    if (st) return st;
    ctx->queue.clear();
    ctx->half = false;
    ctx->state_ver++;
    st = clear_error_word(ctx);
    if (st) return st;
    size_t total = (size_t)1 << (2 * ctx->n);
    for (size_t off = 0; off < total; off += kStageElems) {
        size_t cnt = total - off < kStageElems ? total - off : kStageElems;
        CK(cudaMemcpyAsync(ctx->d_staging, rho_c128 + 2 * off, cnt * sizeof(double2), cudaMemcpyHostToDevice,
                           ctx->stream));
        launch_c128_to_c64(static_cast<const double2 *>(ctx->d_staging), ctx->rho + off, cnt, ctx->nsm, ctx->stream);
        CKLAUNCH(ctx, 1);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return QCW_OK;
}

extern "C" qcw_status qcw_set_state_c64(qcw_ctx *ctx, const float *rho_c64)
{
    CHECK_CTX(ctx);
    if (!rho_c64) return set_error(QCW_EINVAL, "null state");
    if (ctx->validate && !is_density(rho_c64, ctx->n))
        return set_error(QCW_EINVAL, "state is not Hermitian with unit trace (validation)");
    ctx->queue.clear();
    ctx->half = false;
    ctx->state_ver++;
    qcw_status st = clear_error_word(ctx);
    if (st) return st;
    size_t bytes = sizeof(float2) << (2 * ctx->n);
    CK(cudaMemcpyAsync(ctx->rho, rho_c64, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return QCW_OK;
}

extern "C" qcw_status qcw_get_state(qcw_ctx *ctx, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    qcw_status st = fused_flush(ctx);
    if (!st) st = ensure_full(ctx);
    if (st) return st;
    st = ensure_staging(ctx);
    if (st) return st;
    size_t total = (size_t)1 << (2 * ctx->n);
    for (size_t off = 0; off < total; off += kStageElems) {
        size_t cnt = total - off < kStageElems ? total - off : kStageElems;
        launch_c64_to_c128(ctx->rho + off, static_cast<double2 *>(ctx->d_staging), cnt, ctx->nsm, ctx->stream);
        CKLAUNCH(ctx, 1);
        CK(cudaMemcpyAsync(out + 2 * off, ctx->d_staging, cnt * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return QCW_OK;
}

// ------------------------------------------------------------------ evolution
extern "C" qcw_status qcw_apply_gate1(qcw_ctx *ctx, const double u[8], int target, const int *controls,
                                      int ncontrols)
{
    CHECK_CTX(ctx);
    if (!u) return set_error(QCW_EINVAL, "null matrix");
    qcw_status st = check_qubits(ctx->n, &target, 1, controls, ncontrols);
    if (st) return st;
    if (!all_finite(u, 8)) return set_error(QCW_EINVAL, "non-finite matrix entry");
    if (ctx->validate && !is_unitary(u, 2)) return set_error(QCW_EINVAL, "gate is not unitary (validation)");
    QOp op;
    op.kind = 0;
    op.k = 1;
    op.qubits[0] = target;
    op.ncontrols = ncontrols;
    for (int j = 0; j < ncontrols; j++) op.controls[j] = controls[j];
    op.m = to_c128(u, 4);
    return submit(ctx, std::move(op));
}

extern "C" qcw_status qcw_apply_gate2(qcw_ctx *ctx, const double u[32], int q1, int q2, const int *controls,
                                      int ncontrols)
{
    CHECK_CTX(ctx);
    if (!u) return set_error(QCW_EINVAL, "null matrix");
    int qs[2] = {q1, q2};
    qcw_status st = check_qubits(ctx->n, qs, 2, controls, ncontrols);
    if (st) return st;
    if (!all_finite(u, 32)) return set_error(QCW_EINVAL, "non-finite matrix entry");
    if (ctx->validate && !is_unitary(u, 4)) return set_error(QCW_EINVAL, "gate is not unitary (validation)");
    QOp op;
    op.kind = 0;
    op.k = 2;
    op.qubits[0] = q1;
    op.qubits[1] = q2;
    op.ncontrols = ncontrols;
    for (int j = 0; j < ncontrols; j++) op.controls[j] = controls[j];
    op.m = to_c128(u, 16);
    return submit(ctx, std::move(op));
}

extern "C" qcw_status qcw_apply_gate(qcw_ctx *ctx, const double *u, const int *qubits, int k)
{
    CHECK_CTX(ctx);
    if (!u) return set_error(QCW_EINVAL, "null matrix");
    if (k < 1 || k > QCW_MAX_GATE_QUBITS) return set_error(QCW_EINVAL, "k out of range");
    qcw_status st = check_qubits(ctx->n, qubits, k, nullptr, 0);
    if (st) return st;
    size_t cnt = (size_t)1 << (2 * k);
    if (!all_finite(u, 2 * cnt)) return set_error(QCW_EINVAL, "non-finite matrix entry");
    if (ctx->validate && !is_unitary(u, 1 << k)) return set_error(QCW_EINVAL, "gate is not unitary (validation)");
    QOp op;
    op.kind = 0;
    op.k = k;
    for (int j = 0; j < k; j++) op.qubits[j] = qubits[j];
    op.ncontrols = 0;
    op.m = to_c128(u, cnt);
    return submit(ctx, std::move(op));
}

extern "C" qcw_status qcw_apply_kraus(qcw_ctx *ctx, const double *kraus, int nkraus, const int *qubits, int k)
{
    CHECK_CTX(ctx);
    if (!kraus) return set_error(QCW_EINVAL, "null Kraus set");
    if (k < 1 || k > QCW_MAX_GATE_QUBITS) return set_error(QCW_EINVAL, "channels act on 1 to 5 qubits");
    if (nkraus < 1 || nkraus > QCW_MAX_KRAUS) return set_error(QCW_EINVAL, "nkraus out of range");
    qcw_status st = check_qubits(ctx->n, qubits, k, nullptr, 0);
    if (st) return st;
    size_t cnt = (size_t)nkraus << (2 * k);
    if (!all_finite(kraus, 2 * cnt)) return set_error(QCW_EINVAL, "non-finite matrix entry");
    if (ctx->validate && !kraus_keeps_or_loses_trace(kraus, nkraus, 1 << k))
        return set_error(QCW_EINVAL, "Kraus set increases the trace (validation)");
    QOp op;
    op.kind = k <= 2 ? 1 : 2;
    op.k = k;
    for (int j = 0; j < k; j++) op.qubits[j] = qubits[j];
    op.ncontrols = 0;
    op.m = k <= 2 ? kraus_superop(to_c128(kraus, cnt), nkraus, k) : to_c128(kraus, cnt);
    return submit(ctx, std::move(op));
}

qcw_status qcw::convert_ops(int n, const qcw_op *ops, int nops, const double *matrices, std::vector<QOp> &out,
                            bool validate)
{
    if (nops < 0 || (nops > 0 && (!ops || !matrices))) return set_error(QCW_EINVAL, "bad op list");
    for (int i = 0; i < nops; i++) {  // validate everything first: all or nothing
        const qcw_op &o = ops[i];
        if (o.offset < 0) return set_error(QCW_EINVAL, "negative matrix offset");
        if (o.kind == QCW_OP_GATE) {
            if (o.k < 1 || o.k > QCW_MAX_GATE_QUBITS) return set_error(QCW_EINVAL, "k out of range");
            qcw_status st = check_qubits(n, o.qubits, o.k, nullptr, 0);
            if (st) return st;
            if (!all_finite(matrices + o.offset, (size_t)2 << (2 * o.k)))
                return set_error(QCW_EINVAL, "non-finite matrix entry");
            if (validate && !is_unitary(matrices + o.offset, 1 << o.k))
                return set_error(QCW_EINVAL, "gate is not unitary (validation)");
        } else if (o.kind == QCW_OP_KRAUS) {
            if (o.k < 1 || o.k > 2) return set_error(QCW_EINVAL, "channels act on 1 or 2 qubits");
            if (o.nkraus < 1 || o.nkraus > QCW_MAX_KRAUS) return set_error(QCW_EINVAL, "nkraus out of range");
            qcw_status st = check_qubits(n, o.qubits, o.k, nullptr, 0);
            if (st) return st;
            if (!all_finite(matrices + o.offset, ((size_t)2 * o.nkraus) << (2 * o.k)))
                return set_error(QCW_EINVAL, "non-finite matrix entry");
            if (validate && !kraus_keeps_or_loses_trace(matrices + o.offset, o.nkraus, 1 << o.k))
                return set_error(QCW_EINVAL, "Kraus set increases the trace (validation)");
        } else {
            return set_error(QCW_EINVAL, "bad op kind");
        }
    }
    out.reserve(out.size() + nops);
    for (int i = 0; i < nops; i++) {
        const qcw_op &o = ops[i];
        QOp op;
        op.kind = o.kind == QCW_OP_GATE ? 0 : 1;
        op.k = o.k;
        for (int j = 0; j < o.k; j++) op.qubits[j] = o.qubits[j];
        op.ncontrols = 0;
        if (o.kind == QCW_OP_GATE) {
            op.m = to_c128(matrices + o.offset, (size_t)1 << (2 * o.k));
        } else {
            op.m = kraus_superop(to_c128(matrices + o.offset, (size_t)o.nkraus << (2 * o.k)), o.nkraus, o.k);
        }
        out.push_back(std::move(op));
    }
    return QCW_OK;
}

extern "C" qcw_status qcw_apply_ops(qcw_ctx *ctx, const qcw_op *ops, int nops, const double *matrices)
{
    CHECK_CTX(ctx);
    std::vector<QOp> conv;
    qcw_status st = convert_ops(ctx->n, ops, nops, matrices, conv, ctx->validate);
    if (st) return st;
    for (QOp &op : conv) {
        st = submit(ctx, std::move(op));
        if (st) return st;
    }
    return QCW_OK;
}

extern "C" qcw_status qcw_flush(qcw_ctx *ctx)
{
    CHECK_CTX(ctx);
    return fused_flush(ctx);
}

extern "C" qcw_status qcw_sync(qcw_ctx *ctx)
{
    CHECK_CTX(ctx);
    qcw_status st = fused_flush(ctx);
    if (!st) st = ensure_full(ctx);
    if (st) return st;
    CK(cudaMemcpyAsync(ctx->h_result + kErrSlot, device_error_word(ctx), sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned long long w;
    memcpy(&w, ctx->h_result + kErrSlot, sizeof w);
    return check_error_word(ctx, w);
}

// ------------------------------------------------------------------ readouts
// Copy the result block (with the error word) to the pinned mirror and wait for it.
static qcw_status fetch_results(qcw_ctx *c)
{
    CK(cudaMemcpyAsync(c->h_result, c->d_result, 64 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    unsigned long long w;
    memcpy(&w, c->h_result + kErrSlot, sizeof w);
    return check_error_word(c, w);
}
static qcw_status diag_readout(qcw_ctx *c)
{
    qcw_status st = fused_flush(c);
    if (st) return st;
    launch_diag_reduce(c->rho, c->n, c->d_partials, c->d_result, c->red_blocks, c->stream);
    CKLAUNCH(c, launches_per_reduce());
    return fetch_results(c);
}

extern "C" qcw_status qcw_trace(qcw_ctx *ctx, double *re, double *im)
{
    CHECK_CTX(ctx);
    qcw_status st = diag_readout(ctx);
    if (st) return st;
    if (re) *re = ctx->h_result[0];
    if (im) *im = ctx->h_result[1];
    return QCW_OK;
}

extern "C" qcw_status qcw_probabilities(qcw_ctx *ctx, double *p1_out)
{
    CHECK_CTX(ctx);
    if (!p1_out) return set_error(QCW_EINVAL, "null output");
    qcw_status st = diag_readout(ctx);
    if (st) return st;
    for (int q = 0; q < ctx->n; q++) p1_out[q] = ctx->h_result[2 + q];
    return QCW_OK;
}

extern "C" qcw_status qcw_purity(qcw_ctx *ctx, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    const double *part = nullptr;
    int nb = 0;
    if (fused_purity_partials(ctx, &part, &nb)) {
        launch_fold(part, nb, ctx->d_result, ctx->stream);  // summed by the last pass as it wrote rho
        CKLAUNCH(ctx, 1);
    } else {
        if (ctx->half) launch_purity_lower(ctx->rho, ctx->n, ctx->d_partials, ctx->d_result, ctx->red_blocks, ctx->stream);
        else launch_purity(ctx->rho, ctx->n, ctx->d_partials, ctx->d_result, ctx->red_blocks, ctx->stream);
        CKLAUNCH(ctx, launches_per_reduce());
    }
    st = fetch_results(ctx);
    if (st) return st;
    *out = ctx->h_result[0];
    return QCW_OK;
}

// ------------------------------------------------------------------ Pauli expectations
// Term (qubit q, Pauli p = 1, 2, 3) added to a string's masks.
static void pauli_add(PauliTerms &T, int s, int n, int q, int p)
{
    const unsigned b = 1u << (n - 1 - q);
    if (p == 1) T.flip[s] |= b;
    if (p == 2) T.flip[s] |= b, T.ym[s] |= b, T.ny[s]++;
    if (p == 3) T.zm[s] |= b;
}

static qcw_status pauli_readout(qcw_ctx *c, const PauliTerms &T)
{
    qcw_status st = fused_flush(c);
    if (st) return st;
    launch_pauli_expect(c->rho, c->n, T, c->d_partials, c->red_blocks * (QCW_MAX_QUBITS + 2), c->d_result, c->stream);
    CKLAUNCH(c, 2);
    return fetch_results(c);
}

extern "C" qcw_status qcw_polarization(qcw_ctx *ctx, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    PauliTerms T{};
    T.count = 3 * ctx->n;
    for (int q = 0; q < ctx->n; q++)
        for (int i = 0; i < 3; i++) pauli_add(T, 3 * q + i, ctx->n, q, i + 1);
    qcw_status st = pauli_readout(ctx, T);
    if (st) return st;
    memcpy(out, ctx->h_result, sizeof(double) * (size_t)T.count);
    return QCW_OK;
}

extern "C" qcw_status qcw_correlation(qcw_ctx *ctx, int q1, int q2, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    if (q1 < 0 || q1 >= ctx->n || q2 < 0 || q2 >= ctx->n || q1 == q2) return set_error(QCW_EINVAL, "bad qubits");
    PauliTerms T{};
    T.count = 9;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            pauli_add(T, 3 * i + j, ctx->n, q1, i + 1);
            pauli_add(T, 3 * i + j, ctx->n, q2, j + 1);
        }
    qcw_status st = pauli_readout(ctx, T);
    if (st) return st;
    memcpy(out, ctx->h_result, sizeof(double) * 9);
    return QCW_OK;
}

// ------------------------------------------------------------------ entropy and fidelity
static const int kSpectralMaxQubits = 6;

// Reduced state of `keep` on the host, made exactly Hermitian ((A + A^dagger) / 2).
static qcw_status reduced_state(qcw_ctx *c, const int *keep, int nkeep, std::vector<c128> &ra)
{
    if (!keep || nkeep < 1 || nkeep > kSpectralMaxQubits) return set_error(QCW_EINVAL, "1 to 6 kept qubits");
    const int N = 1 << nkeep;
    ra.assign((size_t)N * N, c128(0, 0));
    qcw_status st = qcw_partial_trace(c, keep, nkeep, reinterpret_cast<double *>(ra.data()));
    if (st) return st;
    for (int a = 0; a < N; a++)
        for (int b = a; b < N; b++) {
            const c128 h = 0.5 * (ra[(size_t)a * N + b] + std::conj(ra[(size_t)b * N + a]));
            ra[(size_t)a * N + b] = h;
            ra[(size_t)b * N + a] = std::conj(h);
        }
    return QCW_OK;
}

extern "C" qcw_status qcw_entropy(qcw_ctx *ctx, const int *keep, int nkeep, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    std::vector<c128> ra;
    qcw_status st = reduced_state(ctx, keep, nkeep, ra);
    if (st) return st;
    const int N = 1 << nkeep;
    std::vector<double> w(N);
    herm_eig(ra.data(), N, w.data(), nullptr);
    *out = entropy_bits(w.data(), N);
    return QCW_OK;
}

extern "C" qcw_status qcw_eigenvalues(qcw_ctx *ctx, const int *keep, int nkeep, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    std::vector<c128> ra;
    qcw_status st = reduced_state(ctx, keep, nkeep, ra);
    if (st) return st;
    herm_eig(ra.data(), 1 << nkeep, out, nullptr);
    return QCW_OK;
}

extern "C" qcw_status qcw_fidelity(qcw_ctx *ctx, const int *keep, int nkeep, const double *sigma_c128, double *out)
{
    CHECK_CTX(ctx);
    if (!out || !sigma_c128) return set_error(QCW_EINVAL, "null argument");
    std::vector<c128> ra;
    qcw_status st = reduced_state(ctx, keep, nkeep, ra);
    if (st) return st;
    const int N = 1 << nkeep;
    std::vector<c128> sigma(reinterpret_cast<const c128 *>(sigma_c128), reinterpret_cast<const c128 *>(sigma_c128) + (size_t)N * N);
    *out = fidelity_root(ra.data(), sigma.data(), N);
    return QCW_OK;
}

// ------------------------------------------------------------------ asynchronous readouts
// Slot layout: Re tr, Im tr, P(q = 1) for q < QCW_MAX_QUBITS (n used), purity at 2 + n, and the
// context's error word in the last entry.
static const int kCkptVals = QCW_MAX_QUBITS + 4;

extern "C" qcw_status qcw_checkpoint(qcw_ctx *ctx, long long *ticket)
{
    CHECK_CTX(ctx);
    if (!ticket) return set_error(QCW_EINVAL, "null ticket");
    if (!ctx->d_ckpt) {
        // All or nothing: the ring is published into the context only once every piece exists,
        // so a failure here leaves the context as it was (the next call tries again).
        const size_t bytes = sizeof(double) * QCW_CHECKPOINT_SLOTS * kCkptVals;
        double *dbuf = nullptr, *hbuf = nullptr;
        cudaEvent_t ev[QCW_CHECKPOINT_SLOTS] = {};
        bool ok = cudaMalloc(&dbuf, bytes) == cudaSuccess && cudaMallocHost(&hbuf, bytes) == cudaSuccess;
        for (int i = 0; ok && i < QCW_CHECKPOINT_SLOTS; i++)
            ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
            if (hbuf) cudaFreeHost(hbuf);
            if (dbuf) cudaFree(dbuf);
            return set_error(QCW_ENOMEM, "checkpoint slots");
        }
        for (int i = 0; i < QCW_CHECKPOINT_SLOTS; i++) {
            ctx->ckpt_ticket[i] = -1;
            ctx->ckpt_ev[i] = ev[i];
        }
        ctx->h_ckpt = hbuf;
        ctx->d_ckpt = dbuf;
    }
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    const long long t = ctx->ckpt_next;
    const int slot = (int)(t % QCW_CHECKPOINT_SLOTS);
    double *d = ctx->d_ckpt + (size_t)slot * kCkptVals;
    double *h = ctx->h_ckpt + (size_t)slot * kCkptVals;
    const int n = ctx->n;
    launch_diag_reduce(ctx->rho, n, ctx->d_partials, d, ctx->red_blocks, ctx->stream);
    CKLAUNCH(ctx, launches_per_reduce());
    const double *part = nullptr;
    int nb = 0;
    if (fused_purity_partials(ctx, &part, &nb)) {
        launch_fold(part, nb, d + 2 + n, ctx->stream);
        CKLAUNCH(ctx, 1);
    } else {
        if (ctx->half) launch_purity_lower(ctx->rho, n, ctx->d_partials, d + 2 + n, ctx->red_blocks, ctx->stream);
        else launch_purity(ctx->rho, n, ctx->d_partials, d + 2 + n, ctx->red_blocks, ctx->stream);
        CKLAUNCH(ctx, launches_per_reduce());
    }
    CK(cudaMemcpyAsync(h, d, sizeof(double) * (size_t)(n + 3), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h + kCkptVals - 1, device_error_word(ctx), sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaEventRecord(ctx->ckpt_ev[slot], ctx->stream));
    ctx->ckpt_ticket[slot] = t;
    ctx->ckpt_next = t + 1;
    *ticket = t;
    return QCW_OK;
}

extern "C" qcw_status qcw_checkpoint_read(qcw_ctx *ctx, long long ticket, double *out)
{
    CHECK_CTX(ctx);
    if (!out) return set_error(QCW_EINVAL, "null output");
    if (ticket < 0 || ticket >= ctx->ckpt_next || !ctx->d_ckpt) return set_error(QCW_EINVAL, "unknown checkpoint");
    const int slot = (int)(ticket % QCW_CHECKPOINT_SLOTS);
    if (ctx->ckpt_ticket[slot] != ticket) return set_error(QCW_EINVAL, "checkpoint overwritten");
    CK(cudaEventSynchronize(ctx->ckpt_ev[slot]));
    const double *h = ctx->h_ckpt + (size_t)slot * kCkptVals;
    unsigned long long w;
    memcpy(&w, h + kCkptVals - 1, sizeof w);
    qcw_status st = check_error_word(ctx, w);
    if (st) return st;
    memcpy(out, h, sizeof(double) * (size_t)(ctx->n + 3));
    return QCW_OK;
}

extern "C" qcw_status qcw_measure(qcw_ctx *ctx, int qubit, int forced, double u, int *outcome, double *prob)
{
    CHECK_CTX(ctx);
    if (qubit < 0 || qubit >= ctx->n || forced < -1 || forced > 1) return set_error(QCW_EINVAL, "bad measurement");
    if (!std::isfinite(u)) return set_error(QCW_EINVAL, "non-finite draw");
    qcw_status st = diag_readout(ctx);
    if (st) return st;
    double p1 = ctx->h_result[2 + qubit];
    double p0 = ctx->h_result[0] - p1;
    int m = forced >= 0 ? forced : (u < p0 ? 0 : 1);
    double pm = m ? p1 : p0;
    if (outcome) *outcome = m;
    if (prob) *prob = pm;
    if (!(pm >= 1e-12)) return set_error(QCW_EZEROPROB, "outcome probability below 1e-12");
    ctx->state_ver++;
    launch_project(ctx->rho, ctx->n, qubit, m, (float)(1.0 / pm), ctx->half, ctx->nsm, ctx->stream);
    CKLAUNCH(ctx, 1);
    return QCW_OK;
}

extern "C" qcw_status qcw_partial_trace(qcw_ctx *ctx, const int *keep, int nkeep, double *out_c128)
{
    CHECK_CTX(ctx);
    const int n = ctx->n;
    if (!out_c128 || nkeep < 0 || nkeep > n || (nkeep > 0 && !keep)) return set_error(QCW_EINVAL, "bad partial trace");
    for (int j = 0; j < nkeep; j++) {
        if (keep[j] < 0 || keep[j] >= n) return set_error(QCW_EINVAL, "qubit index out of range");
        if (j && keep[j] <= keep[j - 1]) return set_error(QCW_EINVAL, "kept qubits must ascend");
    }
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    PTParams p{};
    p.n = n;
    p.nkeep = nkeep;
    p.lower = ctx->half ? 1 : 0;  // half storage is read as it is: no completion pass
    unsigned kept = 0;
    for (int j = 0; j < nkeep; j++) {
        p.kpos[j] = (int8_t)(n - 1 - keep[j]);
        kept |= 1u << keep[j];
    }
    for (int q = 0; q < n; q++)
        if (!(kept & (1u << q))) p.tpos[p.ntr++] = (int8_t)(n - 1 - q);
    size_t nout = (size_t)1 << (2 * nkeep);
    double2 *d_out = nullptr;
    if (nout * sizeof(double2) <= 64 * sizeof(double)) {
        d_out = reinterpret_cast<double2 *>(ctx->d_result);
    } else {
        if (cudaMallocAsync(&d_out, nout * sizeof(double2), ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QCW_ENOMEM, "partial trace output");
        }
    }
    launch_partial_trace(ctx->rho, p, d_out, ctx->nsm, ctx->stream);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_c128, d_out, nout * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
    if (d_out != reinterpret_cast<double2 *>(ctx->d_result)) cudaFreeAsync(d_out, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(e, "partial trace");
    return QCW_OK;
}

// ------------------------------------------------------------------ diagnostics
extern "C" const char *qcw_last_error(void) { return g_err.c_str(); }

extern "C" const char *qcw_strerror(qcw_status st)
{
    switch (st) {
    case QCW_OK: return "ok";
    case QCW_EINVAL: return "invalid argument";
    case QCW_ENOMEM: return "out of memory";
    case QCW_ECUDA: return "CUDA error";
    case QCW_EZEROPROB: return "zero-probability outcome";
    case QCW_ETIMEOUT: return "timeout";
    case QCW_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

extern "C" qcw_status qcw_stats(qcw_ctx *ctx, long long *launches, long long *fused_passes, double *fused_pass_ms,
                                long long *timed_passes)
{
    CHECK_CTX(ctx);
    qcw_status st = fused_flush(ctx);
    if (st) return st;
    CK(cudaStreamSynchronize(ctx->stream));
    fused_collect_timing(ctx);
    if (launches) *launches = ctx->launches;
    if (fused_passes) *fused_passes = ctx->passes;
    if (fused_pass_ms) *fused_pass_ms = ctx->pass_ms;
    if (timed_passes) *timed_passes = ctx->timed_passes;
    return QCW_OK;
}

extern "C" qcw_status qcw_stats_reset(qcw_ctx *ctx)
{
    CHECK_CTX(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    fused_collect_timing(ctx);
    ctx->launches = ctx->passes = ctx->timed_passes = 0;
    ctx->pass_ms = 0;
    return QCW_OK;
}

extern "C" qcw_status qcw_enable_pass_timing(qcw_ctx *ctx, int on)
{
    CHECK_CTX(ctx);
    ctx->timing = on != 0;
    return QCW_OK;
}
