// Fused passes: one HBM round trip of rho applies every operation the planner packed into
// the pass.
//
// A pass touches a qubit set Q (|Q| <= k).  Its tile is the set of 2^TB elements whose labels
// differ only in the "tile bits": the row and column bits of Q plus the lowest column bits
// (so that every tile is made of contiguous runs of at least 2^L elements).  One CTA owns
// one tile: it copies the tile into shared memory with cp.async (16-byte pieces), applies
// the pass's phases in place, and writes the tile back.  A phase is a composed
// superoperator on one or two qubits of Q: each thread gathers 16-element groups (the row
// quartet x column quartet of Sec. 3.2 for the two phase qubits) or 4-element groups (the
// pair x pair of Sec. 3.1) from shared memory, multiplies them by the phase superoperator
// and scatters them back.  Groups of one phase are disjoint, so phases need no atomics.
#include <cstring>

#include "planner.h"
#include "qcw_device.cuh"
#include "qcw_internal.h"

namespace qcw {

// ------------------------------------------------------------------ device descriptors
struct FPass {
    int TB;         // tile bits
    int L;          // tile bits 0..L-1 are virtual bits 0..L-1 (contiguous run)
    int nother;     // 2n - TB
    int nphase;
    int phase0;     // first phase in the phase array
    int pad;
    int8_t tbits[16];  // virtual bit of tile bit j (ascending)
    int8_t obits[40];  // virtual bits outside the tile (ascending)
};

struct FPhase {
    int nq;         // 1 or 2
    int coef;       // offset of the superoperator in the coefficient array (float2 units)
    int8_t pos[4];  // tile positions of (r_a, r_b, c_a, c_b); (r_a, c_a) when nq == 1
    int pad;
};

constexpr int FT = 256;      // threads per CTA
constexpr int TB_MAX = 14;   // largest tile: 2^14 complex64 = 128 KiB

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ unsigned ins0(unsigned x, int p)
{
    unsigned lo = x & ((1u << p) - 1u);
    return ((x ^ lo) << 1) | lo;
}

// Two-qubit phase: 16x16 superoperator S (smem, row-major) on every 16-member group.
// G groups per thread share each coefficient load.
template <int G>
__device__ __forceinline__ void phase2(float2 *__restrict__ tile, int TB, const FPhase &F, const float2 *__restrict__ S)
{
    const unsigned d0 = 1u << F.pos[0], d1 = 1u << F.pos[1], d2 = 1u << F.pos[2], d3 = 1u << F.pos[3];
    int p[4] = {F.pos[0], F.pos[1], F.pos[2], F.pos[3]};
    // ascending positions for insertion
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = a + 1; b < 4; b++)
            if (p[b] < p[a]) { int t = p[a]; p[a] = p[b]; p[b] = t; }
    const unsigned ng = 1u << (TB - 4);
    const float4 *S4 = reinterpret_cast<const float4 *>(S);
    for (unsigned g0 = threadIdx.x; g0 < ng; g0 += G * FT) {
        unsigned base[G];
        float2 x[G][16];
#pragma unroll
        for (int j = 0; j < G; j++) {
            unsigned g = g0 + j * FT;
            base[j] = ins0(ins0(ins0(ins0(g, p[0]), p[1]), p[2]), p[3]);
#pragma unroll
            for (int e = 0; e < 16; e++)
                x[j][e] = tile[base[j] + ((e & 8) ? d0 : 0u) + ((e & 4) ? d1 : 0u) + ((e & 2) ? d2 : 0u) + ((e & 1) ? d3 : 0u)];
        }
        // The member loop stays rolled so that the 256 coefficients are re-read from shared
        // memory (broadcast) instead of being hoisted into registers.
#pragma unroll 1
        for (int e = 0; e < 16; e++) {
            const unsigned oe = ((e & 8) ? d0 : 0u) + ((e & 4) ? d1 : 0u) + ((e & 2) ? d2 : 0u) + ((e & 1) ? d3 : 0u);
            float2 y[G];
#pragma unroll
            for (int j = 0; j < G; j++) y[j] = make_float2(0.f, 0.f);
#pragma unroll
            for (int f = 0; f < 16; f += 2) {
                float4 c = S4[8 * e + (f >> 1)];
                float2 c0 = make_float2(c.x, c.y), c1 = make_float2(c.z, c.w);
#pragma unroll
                for (int j = 0; j < G; j++) {
                    cfma(y[j], c0, x[j][f]);
                    cfma(y[j], c1, x[j][f + 1]);
                }
            }
#pragma unroll
            for (int j = 0; j < G; j++) tile[base[j] + oe] = y[j];
        }
    }
}

// One-qubit phase: 4x4 superoperator on every (row pair x column pair) group.
__device__ __forceinline__ void phase1(float2 *__restrict__ tile, int TB, const FPhase &F, const float2 *__restrict__ S)
{
    const int pr = F.pos[0], pc = F.pos[1];
    const int lo = pr < pc ? pr : pc, hi = pr < pc ? pc : pr;
    const unsigned dr = 1u << pr, dc = 1u << pc;
    float2 s[16];
#pragma unroll
    for (int i = 0; i < 16; i++) s[i] = S[i];
    const unsigned ng = 1u << (TB - 2);
    for (unsigned g = threadIdx.x; g < ng; g += FT) {
        unsigned b = ins0(ins0(g, lo), hi);
        float2 x[4] = {tile[b], tile[b + dc], tile[b + dr], tile[b + dr + dc]};
        float2 y[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            y[e] = make_float2(0.f, 0.f);
#pragma unroll
            for (int f = 0; f < 4; f++) cfma(y[e], s[4 * e + f], x[f]);
        }
        tile[b] = y[0];
        tile[b + dc] = y[1];
        tile[b + dr] = y[2];
        tile[b + dr + dc] = y[3];
    }
}

__global__ void __launch_bounds__(FT) k_fused_pass(float2 *__restrict__ rho, const FPass *__restrict__ passes,
                                                   const FPhase *__restrict__ phases, const float2 *__restrict__ coefs,
                                                   int pass_idx)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const FPass &P = passes[pass_idx];
    const int TB = P.TB, L = P.L;
    float2 *tile = reinterpret_cast<float2 *>(smem);
    uint64_t *hoff = reinterpret_cast<uint64_t *>(tile + (1u << TB));
    float2 *S = reinterpret_cast<float2 *>(hoff + ((1u << (TB - L)) | 1u) + 1u);  // 16-byte aligned

    uint64_t base = 0;
    {
        const uint64_t b = blockIdx.x;
        for (int j = 0; j < P.nother; j++) base |= ((b >> j) & 1ull) << P.obits[j];
    }
    for (unsigned i = threadIdx.x; i < (1u << (TB - L)); i += FT) {
        uint64_t o = 0;
        for (int j = 0; j < TB - L; j++) o |= (uint64_t)((i >> j) & 1u) << P.tbits[L + j];
        hoff[i] = o;
    }
    __syncthreads();

    const unsigned nvec = 1u << (TB - 1);
    const unsigned lmask = (1u << L) - 1u;
    for (unsigned v = threadIdx.x; v < nvec; v += FT) {
        unsigned t = 2 * v;
        cp_async16(&tile[t], rho + base + hoff[t >> L] + (t & lmask));
    }
    cp_async_wait_all();
    __syncthreads();

    for (int ph = 0; ph < P.nphase; ph++) {
        const FPhase F = phases[P.phase0 + ph];
        const int ncoef = F.nq == 2 ? 256 : 16;
        for (int i = threadIdx.x; i < ncoef; i += FT) S[i] = coefs[F.coef + i];
        __syncthreads();
        if (F.nq == 2) {
            if (TB >= 13) phase2<2>(tile, TB, F, S);
            else phase2<1>(tile, TB, F, S);
        } else {
            phase1(tile, TB, F, S);
        }
        __syncthreads();
    }

    const float4 *t4 = reinterpret_cast<const float4 *>(tile);
    for (unsigned v = threadIdx.x; v < nvec; v += FT) {
        unsigned t = 2 * v;
        *reinterpret_cast<float4 *>(rho + base + hoff[t >> L] + (t & lmask)) = t4[v];
    }
}

static size_t fused_smem_bytes(int TB, int L)
{
    return ((size_t)8 << TB) + 8 * ((((size_t)1 << (TB - L)) | 1) + 1) + 256 * sizeof(float2);
}

// ------------------------------------------------------------------ host runtime
struct CachedPlan {
    uint64_t hash = 0;
    int n = 0, k = 0, tb = 0;
    std::vector<QOp> ops;  // exact copy for verification
    std::vector<FPass> hpass;
    std::vector<int> grid;  // tiles per pass
    std::vector<size_t> smem;
    char *dbuf = nullptr;  // device copy of passes | phases | coefs
    size_t phase_off = 0, coef_off = 0;
    long long last_use = 0;
};

struct FusedRuntime {
    std::vector<CachedPlan> cache;
    long long tick = 0;
    std::vector<cudaEvent_t> ev_free, ev_pending;  // pairs: start, stop
    int smem_set_dev = -1;
    size_t smem_set_bytes = 0;
};

static uint64_t fnv(uint64_t h, const void *p, size_t n)
{
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; i++) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

static uint64_t hash_ops(const std::vector<QOp> &ops, size_t b, size_t e, int n, int k, int tb)
{
    uint64_t h = 1469598103934665603ull;
    int hdr[3] = {n, k, tb};
    h = fnv(h, hdr, sizeof(hdr));
    for (size_t i = b; i < e; i++) {
        const QOp &o = ops[i];
        int meta[3] = {o.kind, o.k, o.ncontrols};
        h = fnv(h, meta, sizeof(meta));
        h = fnv(h, o.qubits, sizeof(int) * o.k);
        h = fnv(h, o.m.data(), sizeof(c128) * o.m.size());
    }
    return h;
}

static bool same_ops(const std::vector<QOp> &a, const std::vector<QOp> &ops, size_t b, size_t e)
{
    if (a.size() != e - b) return false;
    for (size_t i = 0; i < a.size(); i++) {
        const QOp &x = a[i], &y = ops[b + i];
        if (x.kind != y.kind || x.k != y.k || x.m.size() != y.m.size()) return false;
        if (memcmp(x.qubits, y.qubits, sizeof(int) * x.k)) return false;
        if (memcmp(x.m.data(), y.m.data(), sizeof(c128) * x.m.size())) return false;
    }
    return true;
}

// Tile bits of a pass: rows and columns of Q, then the lowest column bits until TB bits.
static void tile_layout(const std::vector<int> &Q, int n, int tbmax, FPass &fp)
{
    uint64_t in = 0;
    for (int q : Q) {
        in |= 1ull << (n - 1 - q);
        in |= 1ull << (2 * n - 1 - q);
    }
    int want = tbmax < 2 * n ? tbmax : 2 * n;
    for (int v = 0; v < n && __builtin_popcountll(in) < want; v++) in |= 1ull << v;
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

static qcw_status build_plan(qcw_ctx *c, const std::vector<QOp> &ops, size_t b, size_t e, int k, int tbmax,
                             CachedPlan &cp)
{
    const int n = c->n;
    std::vector<PassPlan> plan = plan_passes(ops, b, e, n, k);
    std::vector<FPhase> hph;
    std::vector<float2> hco;
    for (const PassPlan &pp : plan) {
        FPass fp{};
        tile_layout(pp.Q, n, tbmax, fp);
        fp.nphase = (int)pp.phases.size();
        fp.phase0 = (int)hph.size();
        for (const PhasePlan &ph : pp.phases) {
            FPhase f{};
            f.nq = ph.nq;
            f.coef = (int)hco.size();
            if (ph.nq == 2) {
                f.pos[0] = (int8_t)tile_pos(fp, 2 * n - 1 - ph.qa);
                f.pos[1] = (int8_t)tile_pos(fp, 2 * n - 1 - ph.qb);
                f.pos[2] = (int8_t)tile_pos(fp, n - 1 - ph.qa);
                f.pos[3] = (int8_t)tile_pos(fp, n - 1 - ph.qb);
            } else {
                f.pos[0] = (int8_t)tile_pos(fp, 2 * n - 1 - ph.qa);
                f.pos[1] = (int8_t)tile_pos(fp, n - 1 - ph.qa);
            }
            for (const c128 &z : ph.S) hco.push_back(make_float2((float)z.real(), (float)z.imag()));
            hph.push_back(f);
        }
        cp.hpass.push_back(fp);
        cp.grid.push_back(1 << fp.nother);
        cp.smem.push_back(fused_smem_bytes(fp.TB, fp.L));
    }
    size_t sz_pass = sizeof(FPass) * cp.hpass.size();
    cp.phase_off = (sz_pass + 255) & ~(size_t)255;
    size_t sz_ph = sizeof(FPhase) * hph.size();
    cp.coef_off = (cp.phase_off + sz_ph + 255) & ~(size_t)255;
    size_t total = cp.coef_off + sizeof(float2) * hco.size();
    std::vector<char> host(total, 0);
    memcpy(host.data(), cp.hpass.data(), sz_pass);
    if (sz_ph) memcpy(host.data() + cp.phase_off, hph.data(), sz_ph);
    if (!hco.empty()) memcpy(host.data() + cp.coef_off, hco.data(), sizeof(float2) * hco.size());
    if (cudaMalloc(&cp.dbuf, total) != cudaSuccess) {
        cudaGetLastError();
        cp.dbuf = nullptr;
        return set_error(QCW_ENOMEM, "fused plan buffer");
    }
    // synchronous copy: the host vector dies at return
    cudaError_t er = cudaMemcpy(cp.dbuf, host.data(), total, cudaMemcpyHostToDevice);
    if (er != cudaSuccess) return cuda_error(er, "fused plan upload");
    return QCW_OK;
}

static void release_plan(CachedPlan &cp)
{
    if (cp.dbuf) cudaFree(cp.dbuf);
    cp.dbuf = nullptr;
}

static int auto_k(int n) { return n < 5 ? n : 5; }

static const size_t kMaxCached = 64;

static qcw_status run_segment(qcw_ctx *c, size_t b, size_t e)
{
    FusedRuntime *rt = c->fused;
    const int n = c->n;
    int k = c->fuse_k ? c->fuse_k : auto_k(n);
    if (k > n) k = n;
    const int tbmax = 13;
    uint64_t h = hash_ops(c->queue, b, e, n, k, tbmax);
    CachedPlan *hit = nullptr;
    for (CachedPlan &cp : rt->cache)
        if (cp.hash == h && cp.n == n && cp.k == k && cp.tb == tbmax && same_ops(cp.ops, c->queue, b, e)) {
            hit = &cp;
            break;
        }
    if (!hit) {
        if (rt->cache.size() >= kMaxCached) {  // evict least recently used
            size_t victim = 0;
            for (size_t i = 1; i < rt->cache.size(); i++)
                if (rt->cache[i].last_use < rt->cache[victim].last_use) victim = i;
            cudaError_t se = cudaStreamSynchronize(c->stream);
            if (se != cudaSuccess) return cuda_error(se, "stream");
            release_plan(rt->cache[victim]);
            rt->cache.erase(rt->cache.begin() + victim);
        }
        CachedPlan cp;
        cp.hash = h;
        cp.n = n;
        cp.k = k;
        cp.tb = tbmax;
        cp.ops.assign(c->queue.begin() + b, c->queue.begin() + e);
        qcw_status st = build_plan(c, c->queue, b, e, k, tbmax, cp);
        if (st) {
            release_plan(cp);
            return st;
        }
        rt->cache.push_back(std::move(cp));
        hit = &rt->cache.back();
    }
    hit->last_use = ++rt->tick;

    size_t maxsm = 0;
    for (size_t s : hit->smem) maxsm = s > maxsm ? s : maxsm;
    if (rt->smem_set_dev != c->dev || rt->smem_set_bytes < maxsm) {
        cudaError_t er = cudaFuncSetAttribute(k_fused_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxsm);
        if (er != cudaSuccess) return cuda_error(er, "fused smem attribute");
        rt->smem_set_dev = c->dev;
        rt->smem_set_bytes = maxsm;
    }
    const FPass *dp = reinterpret_cast<const FPass *>(hit->dbuf);
    const FPhase *dph = reinterpret_cast<const FPhase *>(hit->dbuf + hit->phase_off);
    const float2 *dco = reinterpret_cast<const float2 *>(hit->dbuf + hit->coef_off);
    for (size_t p = 0; p < hit->hpass.size(); p++) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->timing) {
            if (rt->ev_free.size() >= 2) {
                e1 = rt->ev_free.back(); rt->ev_free.pop_back();
                e0 = rt->ev_free.back(); rt->ev_free.pop_back();
            } else {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
            }
            cudaEventRecord(e0, c->stream);
        }
        k_fused_pass<<<hit->grid[p], FT, hit->smem[p], c->stream>>>(c->rho, dp, dph, dco, (int)p);
        c->launches++;
        c->passes++;
        if (c->timing) {
            cudaEventRecord(e1, c->stream);
            rt->ev_pending.push_back(e0);
            rt->ev_pending.push_back(e1);
        }
        cudaError_t er = cudaGetLastError();
        if (er != cudaSuccess) return cuda_error(er, "fused pass launch");
    }
    return QCW_OK;
}

// A controlled gate whose total support is at most two qubits becomes a plain 2-qubit
// unitary with the control first: diag(1, 1, U) in the (control, target) quartet order.
static bool lower_controlled(QOp &op)
{
    if (op.kind != 0 || op.ncontrols == 0) return true;
    if (op.k + op.ncontrols > 2) return false;
    std::vector<c128> m(16, c128(0, 0));
    m[0] = m[5] = 1.0;
    m[10] = op.m[0];
    m[11] = op.m[1];
    m[14] = op.m[2];
    m[15] = op.m[3];
    op.qubits[1] = op.qubits[0];
    op.qubits[0] = op.controls[0];
    op.k = 2;
    op.ncontrols = 0;
    op.m.swap(m);
    return true;
}

qcw_status fused_flush(qcw_ctx *c)
{
    if (c->queue.empty()) return QCW_OK;
    if (!c->fused) c->fused = new FusedRuntime();
    qcw_status st = QCW_OK;
    size_t b = 0;
    const size_t nq = c->queue.size();
    for (size_t i = 0; i <= nq && !st; i++) {
        bool barrier = i == nq;
        if (!barrier) {
            QOp &op = c->queue[i];
            if (!lower_controlled(op) || op.k > 2) barrier = true;
        }
        if (!barrier) continue;
        if (i > b) st = run_segment(c, b, i);
        if (!st && i < nq) st = plain_apply(c, c->queue[i]);
        b = i + 1;
    }
    c->queue.clear();
    return st;
}

void fused_collect_timing(qcw_ctx *c)
{
    FusedRuntime *rt = c->fused;
    if (!rt) return;
    for (size_t i = 0; i + 1 < rt->ev_pending.size(); i += 2) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, rt->ev_pending[i], rt->ev_pending[i + 1]) == cudaSuccess) {
            c->pass_ms += ms;
            c->timed_passes++;
        }
        rt->ev_free.push_back(rt->ev_pending[i]);
        rt->ev_free.push_back(rt->ev_pending[i + 1]);
    }
    rt->ev_pending.clear();
    cudaGetLastError();
}

void fused_destroy(qcw_ctx *c)
{
    FusedRuntime *rt = c->fused;
    if (!rt) return;
    for (CachedPlan &cp : rt->cache) release_plan(cp);
    for (cudaEvent_t e : rt->ev_free) cudaEventDestroy(e);
    for (cudaEvent_t e : rt->ev_pending) cudaEventDestroy(e);
    delete rt;
    c->fused = nullptr;
}

}  // namespace qcw
