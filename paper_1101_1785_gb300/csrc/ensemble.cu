// Multiverse ensemble (Sec. 5.2.1, Eq. rhoE1): nvec state vectors evolved by the one- and
// two-qubit operators of Sec. 3, per-vector noise operators chosen by the caller, and the
// density matrix rho = sum_v w_v |psi_v><psi_v| formed on the GPU.
#include "qcw_device.cuh"
#include "qcw_internal.h"

#include <cmath>
#include <utility>
#include <vector>

struct qcw_ensemble {
    int n = 0, nvec = 0, dev = 0, nsm = 0;
    float2 *psi = nullptr;  // nvec x 2^n
    int *d_choice = nullptr;
    float *d_w = nullptr;
    unsigned *d_err = nullptr;  // error word of the tensor-core density (a bounded wait ran out)
    void *d_stage = nullptr;  // complex128 staging, one vector
    cudaStream_t stream = nullptr;
};

namespace qcw {

constexpr int kEnsThreads = 256;
constexpr int kEnsMaxOmega = 16;

struct EnsGate {
    float2 u[16];    // 2^k x 2^k, k <= 2
    int k;
    int pos[2];      // ascending label bits of the struck qubits
    uint64_t off[4]; // offset of local index a (first qubit = most significant bit of a)
};

struct EnsNoise {
    float2 om[kEnsMaxOmega][4];
    int pos;
};

static unsigned ens_grid(uint64_t items, int nsm)
{
    uint64_t g = (items + kEnsThreads - 1) / kEnsThreads;
    const uint64_t cap = (uint64_t)nsm * 16;
    return (unsigned)(g < 1 ? 1 : g > cap ? cap : g);
}

// One thread per (vector, group of 2^k amplitudes differing in the struck bits): the pair /
// quartet update of Eqs. resmat1 / resmat2.
template <int K>
__global__ void k_ens_gate(float2 *__restrict__ psi, int n, uint64_t items, const __grid_constant__ EnsGate p)
{
    constexpr int M = 1 << K;
    const int sh = n - K;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < items;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = t >> sh;
        uint64_t g = t & ((1ull << sh) - 1);
#pragma unroll
        for (int j = 0; j < K; j++) g = insert0(g, p.pos[j]);
        float2 *b = psi + (v << n) + g;
        float2 x[M];
#pragma unroll
        for (int a = 0; a < M; a++) x[a] = b[p.off[a]];
#pragma unroll
        for (int a = 0; a < M; a++) {
            float2 y = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < M; c++) cfma(y, p.u[M * a + c], x[c]);
            b[p.off[a]] = y;
        }
    }
}

__global__ void k_ens_noise(float2 *__restrict__ psi, int n, uint64_t items, const int *__restrict__ choice,
                            const __grid_constant__ EnsNoise p)
{
    const int sh = n - 1;
    const uint64_t bit = 1ull << p.pos;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < items;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = t >> sh;
        const uint64_t g = insert0(t & ((1ull << sh) - 1), p.pos);
        const float2 *u = p.om[choice[v]];
        float2 *b = psi + (v << n) + g;
        const float2 x0 = b[0], x1 = b[bit];
        float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
        cfma(y0, u[0], x0), cfma(y0, u[1], x1);
        cfma(y1, u[2], x0), cfma(y1, u[3], x1);
        b[0] = y0, b[bit] = y1;
    }
}

// rho[r][c] = sum_v w_v psi_v[r] conj(psi_v[c]); consecutive threads take consecutive c.
__global__ void k_ens_density(const float2 *__restrict__ psi, int nvec, int n, const float *__restrict__ w,
                              float2 *__restrict__ rho)
{
    const uint64_t dim = 1ull << n, items = dim * dim;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < items;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = t >> n, c = t & (dim - 1);
        float2 acc = make_float2(0.f, 0.f);
        for (int v = 0; v < nvec; v++) {
            const float2 a = psi[((uint64_t)v << n) + r], b = psi[((uint64_t)v << n) + c];
            float2 ab = make_float2(0.f, 0.f);
            cfmac(ab, b, a);  // a conj(b)
            acc.x = fmaf(w[v], ab.x, acc.x);
            acc.y = fmaf(w[v], ab.y, acc.y);
        }
        rho[t] = acc;
    }
}

// Tiled form of the same rank-nvec update for n >= 6: rho = Psi^T diag(w) conj(Psi) is an outer
// product summed over the vectors, so a CTA owns a 64 x 64 tile of rho, stages 16 vectors' 64
// row amplitudes (times w_v) and 64 column amplitudes in shared memory at a time, and each thread
// accumulates a 4 x 4 block of the tile in registers: 64 FMAs per 8 shared-memory loads instead of
// two global loads per 4 FMAs.  rho is Hermitian, so only tiles on or below the diagonal are
// computed; the one above is written as the conjugate transpose through shared memory.  Tile
// pairs in the order of pair_blocked's triangle, one per CTA in a grid-stride loop.
constexpr int kDenT = 64;   // tile edge
constexpr int kDenV = 16;   // vectors staged per round
constexpr int kDenThreads = 256;

// diag_blocks: only the 64 x 64 tiles inside the 128 x 128 blocks on the diagonal (three lower
// tiles per block; the tensor-core kernel does the rest).
__global__ void __launch_bounds__(kDenThreads) k_ens_density_tiled(const float2 *__restrict__ psi, int nvec, int n,
                                                                   const float *__restrict__ w,
                                                                   float2 *__restrict__ rho, int diag_blocks)
{
    // one buffer: the staged vectors (As, Bs) while a tile accumulates, then the finished tile
    // (Tt, padded rows) for its mirrored write
    __shared__ __align__(16) float2 sbuf[kDenT * (kDenT + 1)];
    float2(*As)[kDenT] = reinterpret_cast<float2(*)[kDenT]>(sbuf);
    float2(*Bs)[kDenT] = reinterpret_cast<float2(*)[kDenT]>(sbuf + kDenV * kDenT);
    float2(*Tt)[kDenT + 1] = reinterpret_cast<float2(*)[kDenT + 1]>(sbuf);
    const uint64_t dim = 1ull << n;
    const unsigned M = (unsigned)(dim / kDenT);
    const unsigned npairs = diag_blocks ? 3 * (M / 2) : M * (M + 1) / 2;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (unsigned pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        unsigned R, C;  // row-tile R >= column-tile C
        if (diag_blocks) {  // block b: (2b, 2b), (2b + 1, 2b), (2b + 1, 2b + 1)
            const unsigned b = pr / 3, j = pr % 3;
            R = 2 * b + (j > 0 ? 1u : 0u);
            C = 2 * b + (j == 2 ? 1u : 0u);
        } else {  // pr = R (R + 1) / 2 + C
            R = (unsigned)((sqrt(8.0 * pr + 1.0) - 1.0) / 2.0);
            while (R * (R + 1) / 2 > pr) R--;
            while ((R + 1) * (R + 2) / 2 <= pr) R++;
            C = pr - R * (R + 1) / 2;
        }
        const uint64_t r0 = (uint64_t)R * kDenT, c0 = (uint64_t)C * kDenT;
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
        for (int v0 = 0; v0 < nvec; v0 += kDenV) {
            __syncthreads();  // the previous round's (or tile's) reads of As / Bs are done
            for (int e = tid; e < kDenV * kDenT; e += kDenThreads) {
                const int v = e / kDenT, i = e % kDenT;
                float2 a = make_float2(0.f, 0.f), b = a;
                if (v0 + v < nvec) {
                    const float2 *pv = psi + ((uint64_t)(v0 + v) << n);
                    const float wv = w[v0 + v];
                    a = pv[r0 + i];
                    a = make_float2(wv * a.x, wv * a.y);
                    b = pv[c0 + i];
                }
                As[v][i] = a;
                Bs[v][i] = b;
            }
            __syncthreads();
#pragma unroll 4
            for (int v = 0; v < kDenV; v++) {
                const float4 a01 = *reinterpret_cast<const float4 *>(&As[v][4 * ty]);
                const float4 a23 = *reinterpret_cast<const float4 *>(&As[v][4 * ty + 2]);
                const float4 b01 = *reinterpret_cast<const float4 *>(&Bs[v][4 * tx]);
                const float4 b23 = *reinterpret_cast<const float4 *>(&Bs[v][4 * tx + 2]);
                const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                                     make_float2(a23.z, a23.w)};
                const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                                     make_float2(b23.z, b23.w)};
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {  // acc += a_i conj(b_j)
                        acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(a[i].y, b[j].y, acc[i][j].x));
                        acc[i][j].y = fmaf(a[i].y, b[j].x, fmaf(-a[i].x, b[j].y, acc[i][j].y));
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float2 *row = rho + (r0 + 4 * ty + i) * dim + c0 + 4 * tx;
            *reinterpret_cast<float4 *>(row) = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
            *reinterpret_cast<float4 *>(row + 2) = make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y);
        }
        if (R == C) continue;
        __syncthreads();  // every thread is done reading As / Bs
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) Tt[4 * ty + i][4 * tx + j] = acc[i][j];
        __syncthreads();
        // mirror tile (C, R): element (jj, ii) = conj(tile (ii, jj)); consecutive threads take
        // consecutive columns ii of a mirror row jj
        for (int e = tid; e < kDenT * kDenT; e += kDenThreads) {
            const int jj = e / kDenT, ii = e % kDenT;
            const float2 t = Tt[ii][jj];
            rho[(c0 + jj) * dim + r0 + ii] = make_float2(t.x, -t.y);
        }
    }
}

__global__ void k_ens_zero(float2 *__restrict__ psi, int n, uint64_t items)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < items;
         t += (uint64_t)gridDim.x * blockDim.x)
        psi[t] = make_float2((t & ((1ull << n) - 1)) == 0 ? 1.f : 0.f, 0.f);
}

__global__ void k_ens_c128_to_c64(const double2 *__restrict__ src, float2 *__restrict__ dst, uint64_t cnt)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cnt; t += (uint64_t)gridDim.x * blockDim.x)
        dst[t] = make_float2((float)src[t].x, (float)src[t].y);
}

__global__ void k_ens_c64_to_c128(const float2 *__restrict__ src, double2 *__restrict__ dst, uint64_t cnt)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cnt; t += (uint64_t)gridDim.x * blockDim.x)
        dst[t] = make_double2(src[t].x, src[t].y);
}

static float2 to_f2(const double *z) { return make_float2((float)z[0], (float)z[1]); }

static bool finite_all(const double *a, size_t cnt)
{
    for (size_t i = 0; i < cnt; i++)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace qcw

using namespace qcw;

#define ENS_CK(call)                                               \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);       \
    } while (0)

static void ens_free(qcw_ensemble *e)
{
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->psi) cudaFree(e->psi);
    if (e->d_choice) cudaFree(e->d_choice);
    if (e->d_w) cudaFree(e->d_w);
    if (e->d_err) cudaFree(e->d_err);
    if (e->d_stage) cudaFree(e->d_stage);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

extern "C" qcw_status qcw_ensemble_create(int nqubits, int nvec, qcw_ensemble **out)
{
    if (!out) return set_error(QCW_EINVAL, "null output");
    *out = nullptr;
    if (nqubits < 1 || nqubits > QCW_MAX_QUBITS || nvec < 1 || nvec > 65536)
        return set_error(QCW_EINVAL, "ensemble size out of range");
    qcw_ensemble *e = new qcw_ensemble();
    e->n = nqubits;
    e->nvec = nvec;
    cudaError_t er = cudaGetDevice(&e->dev);
    if (er == cudaSuccess) er = cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, e->dev);
    if (er == cudaSuccess) er = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    const uint64_t items = (uint64_t)nvec << nqubits;
    if (er == cudaSuccess) er = cudaMalloc(&e->psi, sizeof(float2) * items);
    if (er == cudaSuccess) er = cudaMalloc(&e->d_choice, sizeof(int) * (size_t)nvec);
    if (er == cudaSuccess) er = cudaMalloc(&e->d_w, sizeof(float) * (size_t)nvec);
    if (er == cudaSuccess) er = cudaMalloc(&e->d_err, sizeof(unsigned));
    if (er == cudaSuccess) er = cudaMalloc(&e->d_stage, sizeof(double2) << nqubits);
    if (er != cudaSuccess) {
        cudaGetLastError();
        ens_free(e);
        return set_error(QCW_ENOMEM, "ensemble buffers");
    }
    k_ens_zero<<<ens_grid(items, e->nsm), kEnsThreads, 0, e->stream>>>(e->psi, nqubits, items);
    er = cudaGetLastError();
    if (er != cudaSuccess) {
        ens_free(e);
        return cuda_error(er, "ensemble init");
    }
    *out = e;
    return QCW_OK;
}

extern "C" qcw_status qcw_ensemble_destroy(qcw_ensemble *e)
{
    if (!e) return set_error(QCW_EINVAL, "null ensemble");
    ens_free(e);
    return QCW_OK;
}

extern "C" qcw_status qcw_ensemble_set(qcw_ensemble *e, const double *psi_c128)
{
    if (!e || !psi_c128) return set_error(QCW_EINVAL, "null argument");
    const uint64_t dim = 1ull << e->n;
    for (int v = 0; v < e->nvec; v++) {  // one vector at a time through the staging buffer
        ENS_CK(cudaMemcpyAsync(e->d_stage, psi_c128 + 2 * dim * v, sizeof(double2) * dim, cudaMemcpyHostToDevice,
                               e->stream));
        k_ens_c128_to_c64<<<ens_grid(dim, e->nsm), kEnsThreads, 0, e->stream>>>(
            static_cast<const double2 *>(e->d_stage), e->psi + dim * v, dim);
        ENS_CK(cudaGetLastError());
    }
    ENS_CK(cudaStreamSynchronize(e->stream));
    return QCW_OK;
}

extern "C" qcw_status qcw_ensemble_get(qcw_ensemble *e, double *psi_c128)
{
    if (!e || !psi_c128) return set_error(QCW_EINVAL, "null argument");
    const uint64_t dim = 1ull << e->n;
    for (int v = 0; v < e->nvec; v++) {
        k_ens_c64_to_c128<<<ens_grid(dim, e->nsm), kEnsThreads, 0, e->stream>>>(
            e->psi + dim * v, static_cast<double2 *>(e->d_stage), dim);
        ENS_CK(cudaGetLastError());
        ENS_CK(cudaMemcpyAsync(psi_c128 + 2 * dim * v, e->d_stage, sizeof(double2) * dim, cudaMemcpyDeviceToHost,
                               e->stream));
        ENS_CK(cudaStreamSynchronize(e->stream));
    }
    return QCW_OK;
}

static qcw_status ens_gate(qcw_ensemble *e, const double *u, const int *qs, int k)
{
    if (!e || !u) return set_error(QCW_EINVAL, "null argument");
    for (int j = 0; j < k; j++) {
        if (qs[j] < 0 || qs[j] >= e->n) return set_error(QCW_EINVAL, "qubit index out of range");
        for (int i = 0; i < j; i++)
            if (qs[i] == qs[j]) return set_error(QCW_EINVAL, "repeated qubit");
    }
    const int m = 1 << k;
    if (!finite_all(u, 2 * (size_t)m * m)) return set_error(QCW_EINVAL, "non-finite matrix entry");
    EnsGate p{};
    p.k = k;
    for (int i = 0; i < m * m; i++) p.u[i] = to_f2(u + 2 * i);
    int v[2];
    for (int j = 0; j < k; j++) v[j] = e->n - 1 - qs[j];
    for (int a = 0; a < m; a++) {
        uint64_t o = 0;
        for (int j = 0; j < k; j++)
            if ((a >> (k - 1 - j)) & 1) o |= 1ull << v[j];
        p.off[a] = o;
    }
    if (k == 2 && v[1] < v[0]) std::swap(v[0], v[1]);
    for (int j = 0; j < k; j++) p.pos[j] = v[j];
    const uint64_t items = (uint64_t)e->nvec << (e->n - k);
    if (k == 1) k_ens_gate<1><<<ens_grid(items, e->nsm), kEnsThreads, 0, e->stream>>>(e->psi, e->n, items, p);
    else k_ens_gate<2><<<ens_grid(items, e->nsm), kEnsThreads, 0, e->stream>>>(e->psi, e->n, items, p);
    ENS_CK(cudaGetLastError());
    return QCW_OK;
}

extern "C" qcw_status qcw_ensemble_apply_gate1(qcw_ensemble *e, const double u[8], int target)
{
    return ens_gate(e, u, &target, 1);
}

extern "C" qcw_status qcw_ensemble_apply_gate2(qcw_ensemble *e, const double u[32], int q1, int q2)
{
    if (e && e->n < 2) return set_error(QCW_EINVAL, "two-qubit gate on one qubit");
    const int qs[2] = {q1, q2};
    return ens_gate(e, u, qs, 2);
}

extern "C" qcw_status qcw_ensemble_apply_noise1(qcw_ensemble *e, const double *omegas, int nomega, int target,
                                              const int *choice)
{
    if (!e || !omegas || !choice) return set_error(QCW_EINVAL, "null argument");
    if (nomega < 1 || nomega > kEnsMaxOmega) return set_error(QCW_EINVAL, "1 to 16 noise operators");
    if (target < 0 || target >= e->n) return set_error(QCW_EINVAL, "qubit index out of range");
    if (!finite_all(omegas, 8 * (size_t)nomega)) return set_error(QCW_EINVAL, "non-finite matrix entry");
    for (int v = 0; v < e->nvec; v++)
        if (choice[v] < 0 || choice[v] >= nomega) return set_error(QCW_EINVAL, "noise choice out of range");
    EnsNoise p{};
    for (int k = 0; k < nomega; k++)
        for (int i = 0; i < 4; i++) p.om[k][i] = to_f2(omegas + 8 * k + 2 * i);
    p.pos = e->n - 1 - target;
    // the copy is stream-ordered before the kernel; synchronising keeps the caller's array free
    ENS_CK(cudaMemcpyAsync(e->d_choice, choice, sizeof(int) * (size_t)e->nvec, cudaMemcpyHostToDevice, e->stream));
    const uint64_t items = (uint64_t)e->nvec << (e->n - 1);
    k_ens_noise<<<ens_grid(items, e->nsm), kEnsThreads, 0, e->stream>>>(e->psi, e->n, items, e->d_choice, p);
    ENS_CK(cudaGetLastError());
    ENS_CK(cudaStreamSynchronize(e->stream));
    return QCW_OK;
}

extern "C" qcw_status qcw_ensemble_density(qcw_ensemble *e, const double *weights, qcw_ctx *ctx)
{
    if (!e || !weights || !ctx) return set_error(QCW_EINVAL, "null argument");
    if (qcw_nqubits(ctx) != e->n) return set_error(QCW_EINVAL, "qubit counts differ");
    if (!finite_all(weights, (size_t)e->nvec)) return set_error(QCW_EINVAL, "non-finite weight");
    std::vector<float> w(e->nvec);
    for (int v = 0; v < e->nvec; v++) w[v] = (float)weights[v];
    ENS_CK(cudaMemcpyAsync(e->d_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, e->stream));
    ENS_CK(cudaStreamSynchronize(e->stream));  // vectors and weights ready; w may go
    qcw_status st = begin_state_replace(ctx);
    if (st) return st;
    const uint64_t dim = 1ull << e->n;
    ENS_CK(cudaMemsetAsync(e->d_err, 0, sizeof(unsigned), ctx->stream));
    if (dim >= 2 * (uint64_t)kDenT && e->n >= 8) {
        // tiles strictly below the 128 x 128 diagonal blocks on the tensor cores, the diagonal
        // blocks (trace, probabilities) in FP32
        const uint64_t blocks = dim / (2 * kDenT), pairs = 3 * blocks;
        const uint64_t cap = (uint64_t)e->nsm * 8;
        k_ens_density_tiled<<<(unsigned)(pairs < cap ? pairs : cap), kDenThreads, 0, ctx->stream>>>(
            e->psi, e->nvec, e->n, e->d_w, ctx->rho, 1);
        ENS_CK(cudaGetLastError());
        ctx->launches++;
        if (!launch_ens_density_tc(e->psi, e->nvec, e->n, e->d_w, ctx->rho, e->d_err, e->nsm, ctx->stream))
            return set_error(QCW_ECUDA, "tensor-core density kernel could not be configured");
    } else if (dim >= (uint64_t)kDenT) {
        const uint64_t m = dim / kDenT, pairs = m * (m + 1) / 2;
        const uint64_t cap = (uint64_t)e->nsm * 8;  // 8 CTAs of 256 threads resident per SM
        k_ens_density_tiled<<<(unsigned)(pairs < cap ? pairs : cap), kDenThreads, 0, ctx->stream>>>(
            e->psi, e->nvec, e->n, e->d_w, ctx->rho, 0);
    } else {
        k_ens_density<<<ens_grid(dim * dim, e->nsm), kEnsThreads, 0, ctx->stream>>>(e->psi, e->nvec, e->n, e->d_w,
                                                                                   ctx->rho);
    }
    ENS_CK(cudaGetLastError());
    ctx->launches++;
    unsigned herr = 0;
    ENS_CK(cudaMemcpyAsync(&herr, e->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CK(cudaStreamSynchronize(ctx->stream));  // the ensemble may change right after
    if (herr) return set_error(QCW_ETIMEOUT, "ensemble density: a bounded wait ran out");
    return QCW_OK;
}
