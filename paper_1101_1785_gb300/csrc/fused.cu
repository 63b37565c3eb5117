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
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "planner.h"
#include "qcw_internal.h"
#include "tc.cuh"
#include "tile.cuh"

namespace qcw {

constexpr int FT = kTileThreads;

// One CTA per tile of one pass.
__global__ void __launch_bounds__(FT, 2) k_fused_pass(float2 *__restrict__ rho, const FPass *__restrict__ passes,
                                                   const FPhase *__restrict__ phases, const float2 *__restrict__ coefs,
                                                   int pass_idx)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const FPass &P = passes[pass_idx];
    const TileSmem sm = tile_smem(smem, P.TB, P.L);
    tile_hoff(P, sm.hoff);
    __syncthreads();
    tile_process(rho, P, blockIdx.x, phases, coefs, sm);
}

// ------------------------------------------------------------------ host runtime
// The pass's phase headers and coefficients as a kernel parameter (read through the constant
// cache, which keeps the coefficient broadcasts off the shared-memory pipe), for passes that
// fit; nph < 0 marks a pass that does not (its phases then come from shared memory).
// Every phase has a fixed slot of the largest coefficient size, so that a coefficient's address
// is the block's base plus (uniform phase counter) x slot plus a constant.
constexpr int kWsParamPhases = 24;
constexpr int kWsParamSlot = 128;  // float2: phase_coefs(PH_TWO)
struct WsParams {
    FPhase ph[kWsParamPhases];
    int nph;
    int pad[3];
    float2 coef[kWsParamPhases][kWsParamSlot];
};
static_assert(sizeof(WsParams) <= 32000, "kernel parameter block limit");

struct CachedPlan {
    uint64_t hash = 0;
    int n = 0, k = 0, tb = 0;
    bool beam = false;  // passes from the beam search (else the greedy best-absorption choice)
    std::vector<QOp> ops;  // exact copy for verification
    std::vector<FPass> hpass;
    std::vector<int> grid;  // tiles per pass
    std::vector<size_t> smem;
    char *dbuf = nullptr;  // device copy of passes | phases | coefs
    char *hbuf = nullptr;  // its pinned host source (the upload is stream-ordered)
    std::vector<WsParams> prm;  // parameter blocks of the warp-specialised kernel's passes
    std::vector<int> prm_idx;   // per pass: index into prm, -1 if the pass has none
    size_t phase_off = 0, coef_off = 0;
    long long last_use = 0;
};

// Measured choice of the fusion width (fuse_k = 0).  Segments of at least kTuneMinOps
// operations are timed with events at a candidate width until a choice is made, then the
// choice holds for the context's lifetime and for later contexts of the same device, register
// size and kernel choice (g_tuned).  Segments differ too much in content for one trial
// per width to decide, so a segment that comes back (same operations, recognised by hash, as
// in a circuit replayed step after step) is run at the other width: after kTunePairs such
// pairs the width with the smaller summed time wins.  Without repeats the widths alternate
// and, after kTuneMaxTrials trials, the smaller total time per operation wins.
constexpr int kTuneCand[2] = {4, 5};
constexpr size_t kTuneMinOps = 64;
constexpr int kTunePairs = 4;
constexpr int kTuneMaxTrials = 24;
constexpr size_t kTuneMaxSegs = 64;

struct KTuneSeg {
    uint64_t key;       // hash of the segment's operations (width-independent)
    float ms[2];
    bool have[2];
};

struct KTune {
    int chosen = 0;          // 0 until decided
    bool recorded = false;   // the choice is in the process-wide table
    int trials = 0;          // trials finished
    double ms[2] = {0, 0};   // per candidate: summed trial time
    double ops[2] = {0, 0};  // and summed operations
    int paired = 0;          // segments timed at both widths
    double pms[2] = {0, 0};  // their summed times per width
    std::vector<KTuneSeg> segs;
    bool pending = false;    // a timed trial is in flight
    int cand = 0;            // its candidate index
    uint64_t key = 0;        // and segment
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    size_t nops = 0;
};

struct FusedRuntime {
    std::vector<CachedPlan> cache;
    long long tick = 0;
    unsigned ws_grid = 0;  // CTAs of the warp-specialised kernel (resident per SM x SMs)
    unsigned tc_grid = 0;  // the same for its tensor-core variant
    double *d_ppart = nullptr;  // per-CTA purity partials of the last pass of a flush
    int ppart_nb = 0;           // CTAs that wrote them
    int ppart_cap = 0;
    std::vector<cudaEvent_t> ev_free, ev_pending;  // pairs: start, stop
    KTune tune;
};

// A width once chosen by measurement holds for every context of the same device, register size
// and kernel choice in the process: later contexts start with it and run no trials (a second
// context's trials, timed while other work shares the GPU, could otherwise pick differently).
static std::mutex g_tuned_mu;
static std::map<std::tuple<int, int, int>, int> g_tuned;

static int tuned_width(const qcw_ctx *c)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find(std::make_tuple(c->dev, c->n, c->fused_kernel));
    return it == g_tuned.end() ? 0 : it->second;
}

static void record_width(const qcw_ctx *c, int k)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned.emplace(std::make_tuple(c->dev, c->n, c->fused_kernel), k);
}

// Collect the pending trial, waiting for it: until the choice is made the host keeps pace with
// the timed segments (otherwise, with readouts that do not synchronise, the host would run
// whole steps ahead and the undecided widths would keep building plans).  Returns false.
static bool tune_poll(KTune &t)
{
    if (!t.pending) return false;
    if (cudaEventSynchronize(t.e1) != cudaSuccess) {
        cudaGetLastError();
        t.pending = false;
        return false;
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess && t.nops) {
        t.ms[t.cand] += ms;
        t.ops[t.cand] += (double)t.nops;
        for (KTuneSeg &sg : t.segs)
            if (sg.key == t.key && !sg.have[t.cand]) {
                sg.ms[t.cand] = ms;
                sg.have[t.cand] = true;
                if (sg.have[0] && sg.have[1]) {
                    t.paired++;
                    t.pms[0] += sg.ms[0];
                    t.pms[1] += sg.ms[1];
                }
                break;
            }
    }
    cudaGetLastError();
    t.pending = false;
    t.trials++;
    if (t.paired >= kTunePairs)
        t.chosen = t.pms[0] <= t.pms[1] ? kTuneCand[0] : kTuneCand[1];
    else if (t.trials >= kTuneMaxTrials && t.ops[0] > 0 && t.ops[1] > 0)
        t.chosen = t.ms[0] / t.ops[0] <= t.ms[1] / t.ops[1] ? kTuneCand[0] : kTuneCand[1];
    return false;
}

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

// Hermitian form (rho = rho^dagger, Sec. 5.2): tiles are symmetric (row and column bits of
// the same qubits), so the conjugate transpose of the tile with outside bits (o_r, o_c) is
// the tile (o_c, o_r) and the pass maps it to the conjugate transpose of its own image.  One
// CTA per unordered pair o_r <= o_c loads, evolves and stores its tile and writes the mirror
// tile as the conjugate transpose: half the phase arithmetic, 3/4 of the HBM traffic.
// Pair p -> (o_r, o_c) with o_r <= o_c, p = o_c (o_c + 1) / 2 + o_r.  FP32 estimate of the
// triangular root, corrected in integers (FP64 is far slower on this GPU).
__device__ __forceinline__ void pair_of(unsigned p, unsigned &o_r, unsigned &o_c)
{
    const unsigned long long pp = p;
    unsigned long long c = (unsigned long long)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((c + 1) * (c + 2) / 2 <= pp) c++;
    while (c * (c + 1) / 2 > pp) c--;
    o_c = (unsigned)c;
    o_r = (unsigned)(pp - c * (c + 1) / 2);
}

// Pair p -> (lo, hi), lo <= hi < M, in 4 x 4 blocks of the triangle: block rows R (pairs before
// row R: 8 R^2 + 2 R), in each the off-diagonal blocks (16 pairs, lo fastest) and then the
// diagonal block (10 pairs, triangle order).  Pairs that run side by side then cover four
// consecutive lo and four consecutive hi values, so both the evolved tiles (outside column
// bits lo) and their mirrors (outside column bits hi) fill whole cache lines together.
__device__ __forceinline__ void pair_blocked(unsigned p, unsigned M, unsigned &lo, unsigned &hi)
{
    if (M < 4) {
        pair_of(p, lo, hi);
        return;
    }
    const unsigned long long pp = p;
    unsigned long long R = (unsigned long long)((sqrtf(4.0f + 32.0f * (float)p) - 2.0f) * 0.0625f);
    while (8 * (R + 1) * (R + 1) + 2 * (R + 1) <= pp) R++;
    while (8 * R * R + 2 * R > pp) R--;
    const unsigned q = (unsigned)(pp - (8 * R * R + 2 * R)), r4 = 4 * (unsigned)R;
    if (q < 16 * (unsigned)R) {
        hi = r4 + ((q & 15u) >> 2);
        lo = 4 * (q >> 4) + (q & 3u);
    } else {
        unsigned c, r;
        pair_of(q - 16 * (unsigned)R, c, r);
        hi = r4 + r;
        lo = r4 + c;
    }
}

constexpr int HT = 128;  // threads of the Hermitian kernel: 2^12-element tiles give 2 groups each

// Mirror tile: element t' holds conj(tile[swap(t')]), swap exchanging the column half and the
// row half of the tile index.  Adjacent lanes take adjacent elements of one contiguous run
// (up to 32-byte segments) and walk the tile's rows in the other lane bits, so that the
// shared-memory reads spread over the banks.
template <int NT>
__device__ __forceinline__ void herm_mirror(float2 *__restrict__ rho, const FPass &P, uint64_t mbase,
                                            const float2 *__restrict__ tile, const uint64_t *__restrict__ hoff)
{
    const int TB = P.TB, L = P.L, h = P.TB / 2;
    const int J = L < 2 ? L : 2;
    const unsigned hmask = (1u << h) - 1u, lmask = (1u << L) - 1u, jmask = (1u << J) - 1u;
    for (unsigned idx = threadIdx.x; idx < (1u << TB); idx += NT) {
        const unsigned j = idx & jmask, u = idx >> J;
        const unsigned Rp = u & hmask, Chi = u >> h;
        const unsigned tp = (Rp << h) | (Chi << J) | j;
        const unsigned ts = (((Chi << J) | j) << h) | Rp;
        const float2 v = tile[herm_phys(ts)];
        rho[mbase + hoff[tp >> L] + (tp & lmask)] = make_float2(v.x, -v.y);
    }
}

__global__ void __launch_bounds__(HT, 4) k_fused_herm(float2 *__restrict__ rho, const FPass *__restrict__ passes,
                                                      const FPhase *__restrict__ phases,
                                                      const float2 *__restrict__ coefs, int pass_idx)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const FPass &P = passes[pass_idx];
    const int TB = P.TB, L = P.L, m = P.nother / 2;
    const TileSmem sm = tile_smem(smem, TB, L);
    tile_hoff_nt<HT>(P, sm.hoff);
    // The evolved tile is the one with o_c <= o_r (on or below the diagonal), pairs in the
    // blocked order of pair_blocked.  Outside bits ascend: m column bits (o_c) below m row
    // bits (o_r).
    unsigned o_r, o_c;
    pair_blocked(blockIdx.x, 1u << m, o_c, o_r);
    __syncthreads();
    const uint64_t t_self = ((uint64_t)o_r << m) | o_c;
    {
        const uint64_t base = tile_base(P, t_self);
        const unsigned nvec = 1u << (TB - 1), lmask = (1u << L) - 1u;
        for (unsigned v = threadIdx.x; v < nvec; v += HT) {
            unsigned e = 2 * v;
            cp_async16(&sm.tile[herm_phys(e)], rho + base + sm.hoff[e >> L] + (e & lmask));
        }
        cp_async_wait_all();
        __syncthreads();
    }
    for (int ph = 0; ph < P.nphase; ph++) {
        const FPhase F = phases[P.phase0 + ph];
        const int ncoef = phase_coefs(F.nq);
        for (int i = threadIdx.x; i < ncoef; i += HT) sm.S[i] = coefs[F.coef + i];
        __syncthreads();
        tile_apply_phase<HT, false, true>(sm.tile, TB, F, sm.S);
        __syncthreads();
    }
    tile_store_nt<HT, true>(rho, P, t_self, sm.tile, sm.hoff);
    if (o_r == o_c) return;
    herm_mirror<HT>(rho, P, tile_base(P, ((uint64_t)o_c << m) | o_r), sm.tile, sm.hoff);
}

// ------------------------------------------------------------------ warp-specialised Hermitian pass
// Persistent CTAs of kWsConsumerWarps consumer warps and kWsProducerWarps producer warps sharing
// kWsBuf tile buffers.  CTA c takes the pairs c, c + grid, c + 2 grid, ...  The producers load
// the canonical elements of a pair (see WsPair) with cp.async up to kWsBuf - 1 tiles ahead of
// the consumers and write the evolved canonical elements back while the consumers work on
// later tiles, so the pass's HBM traffic overlaps its arithmetic instead of adding to it.
// Hand-over is by mbarriers: full[b] (every producer thread, once its copies of the tile have
// landed and been completed) and empty[b] (every consumer thread); the producer warps split
// each tile's rows k and meet at a named barrier between writing a buffer back and refilling
// it.  Every wait is bounded: on running out, the side that gave up sets the pass's error word
// and returns, and the other side then runs out too.
//
// Tiles are 2^12 elements (six qubits); a producer lane covers tile bits 0..5 (an element
// pair) and the loop index k the bits 6..11, so global offsets and swizzled shared-memory
// positions split into a per-lane part and a per-k part read from a 64-entry table.  The
// pass's phase headers and coefficients are copied to shared memory once per CTA when they
// fit (else each phase's coefficients are staged before it runs).
constexpr int kWsBuf = 3;
constexpr int kWsConsumerWarps = 4;
constexpr int kWsProducerWarps = 2;  // the purity epilogue sums exactly two warps' totals
constexpr int kWsCtasPerSm = 2;
constexpr int WC = 32 * kWsConsumerWarps;  // consumer threads
constexpr int WP = 32 * kWsProducerWarps;  // producer threads
constexpr int WTH = WC + WP;
constexpr int kWsMaxPhases = 24;
constexpr int kWsCoefMax = 512;  // float2 (shared-memory fallback when the parameter block does not fit)
constexpr unsigned kWsWaitLimit = 1u << 21;  // polls (>= 0.5 s with the 256 ns back-off)

struct WsEntry {
    unsigned long long ghi;  // global offset of tile bits 6..11 = k
    unsigned phi;            // herm_phys(k << 6)
    unsigned pm;             // herm_phys(k)
};

struct WsSmem {
    float2 *buf;      // kWsBuf tiles of 2^12 elements
    float *tcB;       // kTcBFloats: B operand of the tensor-core phases (k_fused_herm_tc)
    WsEntry *tab;     // 64 entries
    unsigned long long *bt;  // 4 x 64: tile base = bt[0][o_c & 63] + bt[1][o_c >> 6] + bt[2][o_r & 63] + bt[3][o_r >> 6]
    int *stab;        // 32: shift s of a pair whose highest differing outside bit is hb
    float2 *coef;     // kWsCoefMax
    FPhase *ph;       // kWsMaxPhases headers
    int *coff;        // kWsMaxPhases offsets into coef
    uint64_t *bars;   // full[kWsBuf], empty[kWsBuf], the tensor-core phases' two MMA barriers
    double *psum;     // 2: the producer warps' purity sums
    unsigned *tslot;  // tensor-memory base address (k_fused_herm_tc)
};

__host__ __device__ constexpr size_t ws_smem_bytes()
{
    return (size_t)kWsBuf * (sizeof(float2) << 12) + kTcBFloats * sizeof(float) + 64 * sizeof(WsEntry) +
           256 * sizeof(unsigned long long) + 32 * sizeof(int) + kWsCoefMax * sizeof(float2) +
           kWsMaxPhases * sizeof(FPhase) + kWsMaxPhases * sizeof(int) + (2 * kWsBuf + 2) * sizeof(uint64_t) +
           2 * sizeof(double) + sizeof(unsigned);
}

// Canonical copy (half storage).  Element (r, c) of rho is canonical when r >= c; a pass reads
// and writes only canonical elements, so the other triangle goes stale (the host completes it
// before anything else reads rho).  For the pair (T_s, T_m) = ((o_r, o_c), (o_c, o_r)),
// o_c <= o_r: if o_r == o_c the tile is on the diagonal and (er, ec) is canonical iff er >= ec;
// else let qo be the most significant outside qubit where o_r and o_c differ (there o_r has 1)
// and t the number of tile qubits more significant than qo: T_s's element (er, ec) is canonical
// iff (er >> (6 - t)) >= (ec >> (6 - t)) (the top t tile qubits decide first, ties go to T_s),
// and otherwise its transpose in T_m is.  For t = 0 all of T_s is canonical (no mirror traffic).
struct WsPair {
    unsigned o_r, o_c;
    int s;      // 6 - t (0 on the diagonal)
    bool diag;
};

__device__ __forceinline__ WsPair ws_pair(const int *stab, unsigned p, int m)
{
    WsPair w;
    pair_blocked(p, 1u << m, w.o_c, w.o_r);
    w.diag = w.o_r == w.o_c;
    w.s = w.diag ? 0 : stab[31 - __clz(w.o_r ^ w.o_c)];
    return w;
}

__device__ __forceinline__ WsSmem ws_smem(unsigned char *smem)
{
    WsSmem w;
    w.buf = reinterpret_cast<float2 *>(smem);
    w.tcB = reinterpret_cast<float *>(w.buf + kWsBuf * 4096);
    w.tab = reinterpret_cast<WsEntry *>(w.tcB + kTcBFloats);
    w.bt = reinterpret_cast<unsigned long long *>(w.tab + 64);
    w.stab = reinterpret_cast<int *>(w.bt + 256);
    w.coef = reinterpret_cast<float2 *>(w.stab + 32);
    w.ph = reinterpret_cast<FPhase *>(w.coef + kWsCoefMax);
    w.coff = reinterpret_cast<int *>(w.ph + kWsMaxPhases);
    w.bars = reinterpret_cast<uint64_t *>(w.coff + kWsMaxPhases);
    w.psum = reinterpret_cast<double *>(w.bars + 2 * kWsBuf + 2);
    w.tslot = reinterpret_cast<unsigned *>(w.psum + 2);
    return w;
}

// TC: two-qubit phases on the tensor cores (tile_phase2_tc) when the pass's coefficients are in
// the parameter block; consumer warp 0 holds kTcCols tensor-memory columns for the kernel's life.
// PUR: also sum w |x|^2 over the write-back (purity_part, one partial per CTA).
template <bool TC, bool PUR>
__device__ __forceinline__ void ws_pass_body(float2 *__restrict__ rho, const FPass *__restrict__ passes,
                                             const FPhase *__restrict__ phases, const float2 *__restrict__ coefs,
                                             int pass_idx, unsigned npairs, unsigned long long *__restrict__ err,
                                             unsigned wait_limit, int stall_tile, double *__restrict__ purity_part,
                                             const WsParams &prm)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const WsSmem sm = ws_smem(smem);
    const FPass &P = passes[pass_idx];
    const int m = P.nother / 2, nph = P.nphase;
    const unsigned tid = threadIdx.x;
    if (tid < 64) {
        unsigned long long g = 0;
        for (int j = 0; j < 6; j++)
            if ((tid >> j) & 1u) g += 1ull << P.tbits[6 + j];
        sm.tab[tid].ghi = g;
        sm.tab[tid].phi = herm_phys(tid << 6);
        sm.tab[tid].pm = herm_phys(tid);
        // outside index bit j of the column half is obits[j], of the row half obits[m + j]
        unsigned long long b[4] = {0, 0, 0, 0};
        for (int j = 0; j < 6; j++) {
            if (!((tid >> j) & 1u)) continue;
            if (j < m) b[0] += 1ull << P.obits[j], b[2] += 1ull << P.obits[m + j];
            if (6 + j < m) b[1] += 1ull << P.obits[6 + j], b[3] += 1ull << P.obits[m + 6 + j];
        }
        for (int h = 0; h < 4; h++) sm.bt[64 * h + tid] = b[h];
    } else if (tid < 96) {
        const int hb = tid - 64;  // pair whose highest differing outside column bit is hb
        int below = 0;
        if (hb < m)
            for (int j = 0; j < 6; j++) below += P.tbits[j] < P.obits[hb];
        sm.stab[hb] = below;
    }
    if (tid == 0) {
        for (int b = 0; b < kWsBuf; b++) {
            mbar_init(&sm.bars[b], WP);  // full: every producer thread, by its copies or after finish
            mbar_init(&sm.bars[kWsBuf + b], WC);
        }
        if (TC) {
            mbar_init(&sm.bars[2 * kWsBuf], 1);  // one tcgen05.commit per MMA batch
            mbar_init(&sm.bars[2 * kWsBuf + 1], 1);
            fence_mbar_init();
        }
    }
    if (TC && tid < 32) {
        tmem_alloc(sm.tslot, kTcCols);
        tmem_relinquish();
    }
    // phase headers and coefficients: from the parameter block, else once per CTA into shared
    // memory when they fit
    const bool prmok = prm.nph >= 0;
    int total = 0;
    if (!prmok)
        for (int ph = 0; ph < nph; ph++) total += phase_coefs(phases[P.phase0 + ph].nq);
    const bool pre = !prmok && nph <= kWsMaxPhases && total <= kWsCoefMax;
    if (pre) {
        int off = 0;
        for (int ph = 0; ph < nph; ph++) {
            const FPhase F = phases[P.phase0 + ph];
            const int nc = phase_coefs(F.nq);
            if (tid == 0) {
                sm.ph[ph] = F;
                sm.coff[ph] = off;
            }
            for (int j = tid; j < nc; j += WTH) sm.coef[off + j] = coefs[F.coef + j];
            off += nc;
        }
    }
    if (TC) tc_fence_before();
    __syncthreads();
    if (TC) tc_fence_after();
    const unsigned ntile = blockIdx.x < npairs ? (npairs - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid >= WC) {  // ---- producer warps
        const unsigned lane = tid & 31u, pw = (tid - WC) >> 5;
        unsigned long long glo = 0;  // global offset of element 2 lane of a tile row (bits 0..5)
        for (int j = 0; j < 6; j++)
            if (((2 * lane) >> j) & 1u) glo += 1ull << P.tbits[j];
        const unsigned plo = herm_phys(2 * lane);
        const unsigned pm0 = herm_phys((2 * lane) << 6), pm1 = herm_phys((2 * lane + 1) << 6);
        const unsigned lc = (2 * lane);  // this lane's column pair (lc, lc + 1) of a tile row
        auto base_of = [&](unsigned o_r, unsigned o_c) {
            return sm.bt[o_c & 63u] + sm.bt[64 + (o_c >> 6)] + sm.bt[128 + (o_r & 63u)] + sm.bt[192 + (o_r >> 6)];
        };
        // Loads, row k at a time: the canonical part of T_s row k (16-byte pairs; lc and lc + 1
        // share the top bits) and, for split pairs, the canonical part of T_m row k into the
        // transposed slots of T_s (8-byte copies; the first phase conjugates them as it reads).  A
        // diagonal tile is loaded whole and completed by finish.  One cp.async group per tile;
        // tiles are released by the copies' own arrival on full, diagonal ones by finish.
        auto needs_finish = [&](unsigned i) {
            return ws_pair(sm.stab, blockIdx.x + i * gridDim.x, m).diag;
        };
        auto load = [&](unsigned i) {
            float2 *bf = sm.buf + ((i % kWsBuf) << 12);
            const WsPair w = ws_pair(sm.stab, blockIdx.x + i * gridDim.x, m);
            const uint64_t sb = base_of(w.o_r, w.o_c) + glo;
            const bool split = !w.diag && w.s < 6;
            const uint64_t mb = split ? base_of(w.o_c, w.o_r) + glo : 0;
            const unsigned ltop = lc >> w.s;
#pragma unroll 4
            for (unsigned k = pw; k < 64; k += kWsProducerWarps) {
                const WsEntry t = sm.tab[k];
                const unsigned ktop = k >> w.s;
                if (w.diag || ktop >= ltop) cp_async16(bf + (plo ^ t.phi), rho + sb + t.ghi);
                if (split && ltop < ktop) {  // T_m row k = T_s column k
                    const float2 *src = rho + mb + t.ghi;
                    cp_async8(bf + (pm0 ^ t.pm), src);
                    cp_async8(bf + (pm1 ^ t.pm), src + 1);
                }
            }
            if (!w.diag) cp_async_mbar_arrive(&sm.bars[i % kWsBuf]);
            cp_async_commit();
        };
        // A diagonal tile's copies have landed (all lanes' after the barrier): fill its upper
        // triangle from its lower one, then release it to the consumers.
        auto finish = [&](unsigned i) {
            float2 *bf = sm.buf + ((i % kWsBuf) << 12);
            bar_sync(2, WP);
            for (unsigned e = tid - WC; e < 4096; e += WP) {
                const unsigned er = e >> 6, ec = e & 63u;
                if (er < ec) {
                    const float2 v = bf[herm_phys((ec << 6) | er)];
                    bf[herm_phys(e)] = make_float2(v.x, -v.y);
                }
            }
            if (!(blockIdx.x == 0 && (int)i == stall_tile)) mbar_arrive(&sm.bars[i % kWsBuf]);
        };
        // Write-back of the canonical elements, row k at a time: T_s row k and, for split pairs,
        // T_m row k (the conjugated column k of the evolved T_s).  Row-local writes keep HBM
        // efficient.  With purity_part it also returns the sum of w |x|^2 over what it writes:
        // w = 2 below the diagonal of rho (the mirror element is not stored), 1 on it; a
        // diagonal tile (written whole) counts its upper triangle 0.
        constexpr bool pur = PUR;
        auto store = [&](unsigned i) -> float {
            float ps = 0.f;
            const float2 *bf = sm.buf + ((i % kWsBuf) << 12);
            const WsPair w = ws_pair(sm.stab, blockIdx.x + i * gridDim.x, m);
            const uint64_t sb = base_of(w.o_r, w.o_c) + glo;
            const bool split = !w.diag && w.s < 6;
            const uint64_t mb = split ? base_of(w.o_c, w.o_r) + glo : 0;
            const unsigned ltop = lc >> w.s;
#pragma unroll 4
            for (unsigned k = pw; k < 64; k += kWsProducerWarps) {
                const WsEntry t = sm.tab[k];
                const unsigned ktop = k >> w.s;
                if (w.diag || ktop >= ltop) {
                    const float4 v = *reinterpret_cast<const float4 *>(bf + (plo ^ t.phi));
                    *reinterpret_cast<float4 *>(rho + sb + t.ghi) = v;
                    if (pur) {
                        const float e0 = fmaf(v.x, v.x, v.y * v.y), e1 = fmaf(v.z, v.z, v.w * v.w);
                        const float w0 = !w.diag || k > lc ? 2.f : k == lc ? 1.f : 0.f;
                        const float w1 = !w.diag || k > lc + 1 ? 2.f : k == lc + 1 ? 1.f : 0.f;
                        ps = fmaf(w0, e0, fmaf(w1, e1, ps));
                    }
                }
                if (split && ltop < ktop) {
                    const float2 a = bf[pm0 ^ t.pm], b = bf[pm1 ^ t.pm];
                    *reinterpret_cast<float4 *>(rho + mb + t.ghi) = make_float4(a.x, -a.y, b.x, -b.y);
                    if (pur) ps = fmaf(2.f, fmaf(a.x, a.x, a.y * a.y) + fmaf(b.x, b.x, b.y * b.y), ps);
                }
            }
            return ps;
        };
        // empty[b] completes once per use of buffer b: tile i is its (i / kWsBuf)-th use.  All
        // producer threads agree on the outcome (named barrier 2).
        auto wait_empty = [&](unsigned i) {
            return bar_and(2, WP, mbar_wait(&sm.bars[kWsBuf + i % kWsBuf], (i / kWsBuf) & 1u, wait_limit));
        };
        bool ok = true;
        double pacc = 0.0;  // this thread's purity sum, tile by tile (FP32 within a tile)
        for (unsigned i = 0; i < ntile; i++) {
            if (i >= kWsBuf) {
                ok = wait_empty(i - kWsBuf);
                if (!ok) break;
                pacc += (double)store(i - kWsBuf);
                bar_sync(2, WP);  // every producer's reads of the buffer precede the new copies into it
            }
            if (!(blockIdx.x == 0 && (int)i == stall_tile)) load(i);
            else cp_async_commit();
            if (i >= 1 && needs_finish(i - 1)) {
                cp_async_wait_group1();  // tile i - 1's group
                finish(i - 1);
            }
        }
        if (ok && ntile >= 1 && needs_finish(ntile - 1)) {
            cp_async_wait_all();
            finish(ntile - 1);
        }
        for (unsigned i = ntile >= kWsBuf ? ntile - kWsBuf : 0; ok && i < ntile; i++) {
            ok = wait_empty(i);
            if (ok) pacc += (double)store(i);
        }
        cp_async_wait_all();
        if (!ok && tid == WC) atomicOr(err, 1ull);
        if (pur) {  // fixed order: shuffle tree per warp, then warp 0 + warp 1
            pacc = warp_sum(pacc);
            if (lane == 0) sm.psum[pw] = pacc;
            bar_sync(2, WP);
            if (tid == WC) purity_part[blockIdx.x] = sm.psum[0] + sm.psum[1];
        }
        return;
    }

    // ---- consumer warps: the pass's phases on each tile in turn
    TcState tc{};
    if (TC) {
        tc.tmem = *sm.tslot;
        tc.B = sm.tcB;
        tc.bar = sm.bars + 2 * kWsBuf;
    }
    bool ok = true;
    for (unsigned i = 0; i < ntile; i++) {
        const unsigned b = i % kWsBuf;
        ok = bar_and(1, WC, mbar_wait(&sm.bars[b], (i / kWsBuf) & 1u, wait_limit));
        if (!ok) break;
        float2 *tile = sm.buf + (b << 12);
        const WsPair w = ws_pair(sm.stab, blockIdx.x + i * gridDim.x, m);
        const int cs = w.diag ? 6 : w.s;  // members copied from T_m: conjugated by the first phase
        for (int ph = 0; ph < nph; ph++) {
            if (prmok) {
                const FPhase F = prm.ph[ph];  // header in registers: its positions are read per group
                if (TC && F.nq == PH_TWO) {
                    const bool good = tile_phase2_tc(tile, F, prm.coef[ph], tc, ph == 0 ? cs : 6, wait_limit);
                    ok = bar_and(1, WC, good);  // also the end-of-phase barrier
                    if (!ok) break;
                    continue;
                }
                tile_apply_phase<WC, false, true, true>(tile, 12, F, prm.coef[ph], ph == 0 ? cs : 6);
            } else if (pre) {
                tile_apply_phase<WC, false, true>(tile, 12, sm.ph[ph], sm.coef + sm.coff[ph], ph == 0 ? cs : 6);
            } else {
                const FPhase F = phases[P.phase0 + ph];
                const int nc = phase_coefs(F.nq);
                for (int j = tid; j < nc; j += WC) sm.coef[j] = coefs[F.coef + j];
                bar_sync(1, WC);
                tile_apply_phase<WC, false, true>(tile, 12, F, sm.coef, ph == 0 ? cs : 6);
            }
            bar_sync(1, WC);
        }
        if (!ok) break;
        mbar_arrive(&sm.bars[kWsBuf + b]);
    }
    if (!ok && tid == 0) atomicOr(err, 2ull);
    if (TC) {
        if (!ok && tc.batches)  // a batch that ran out may still be in flight: give it a second wait
            for (int j = 0; j < 2; j++) mbar_wait(&tc.bar[j], (tc.batches - 1) & 1u, wait_limit);
        tc_fence_before();
        bar_sync(1, WC);
        if (tid < 32) {
            tc_fence_after();
            tmem_dealloc(tc.tmem, kTcCols);
        }
    }
}

template <bool PUR>
__global__ void __launch_bounds__(WTH, kWsCtasPerSm)
    k_fused_herm_ws(float2 *__restrict__ rho, const FPass *__restrict__ passes, const FPhase *__restrict__ phases,
                    const float2 *__restrict__ coefs, int pass_idx, unsigned npairs,
                    unsigned long long *__restrict__ err, unsigned wait_limit, int stall_tile,
                    double *__restrict__ purity_part, const __grid_constant__ WsParams prm)
{
    ws_pass_body<false, PUR>(rho, passes, phases, coefs, pass_idx, npairs, err, wait_limit, stall_tile, purity_part,
                                    prm);
}

template <bool PUR>
__global__ void __launch_bounds__(WTH, kWsCtasPerSm)
    k_fused_herm_tc(float2 *__restrict__ rho, const FPass *__restrict__ passes, const FPhase *__restrict__ phases,
                    const float2 *__restrict__ coefs, int pass_idx, unsigned npairs,
                    unsigned long long *__restrict__ err, unsigned wait_limit, int stall_tile,
                    double *__restrict__ purity_part, const __grid_constant__ WsParams prm)
{
    ws_pass_body<true, PUR>(rho, passes, phases, coefs, pass_idx, npairs, err, wait_limit, stall_tile, purity_part,
                                    prm);
}

static bool herm_kernel(const qcw_ctx *c)
{
    return c->fused_kernel == QCW_FUSED_KERNEL_AUTO || c->fused_kernel == QCW_FUSED_KERNEL_HERM ||
           c->fused_kernel == QCW_FUSED_KERNEL_HERM_WS || c->fused_kernel == QCW_FUSED_KERNEL_HERM_TC;
}

// The warp-specialised pass with its two-qubit phases on the tensor cores.  Not the default:
// on GB300 it runs the 14-qubit benchmark's passes about 4 % slower than the CUDA-core kernel
// (1.049 against 1.006 ms: each phase's MMA round trip is a latency chain that two CTAs per SM
// cannot hide).
static bool tc_kernel(const qcw_ctx *c) { return c->fused_kernel == QCW_FUSED_KERNEL_HERM_TC; }

// Passes the warp-specialised kernel takes: Hermitian, 2^12-element tiles with column bit 0 of
// rho inside (element pairs contiguous in global memory).
static bool ws_pass(const qcw_ctx *c, const FPass &fp)
{
    return (c->fused_kernel == QCW_FUSED_KERNEL_AUTO || c->fused_kernel == QCW_FUSED_KERNEL_HERM_WS ||
            c->fused_kernel == QCW_FUSED_KERNEL_HERM_TC) &&
           fp.herm && fp.TB == 12 && fp.L >= 1;
}

static qcw_status build_plan(qcw_ctx *c, const std::vector<QOp> &ops, size_t b, size_t e, int k, int tbmax,
                             CachedPlan &cp, bool beam)
{
    const int n = c->n;
    TilePlan tp;
    cp.beam = beam;
    append_tile_plan(plan_passes(ops, b, e, n, k, false, beam ? PassSearch::BEAM : PassSearch::BEST), n, tbmax, tp,
                     herm_kernel(c));
    cp.hpass = tp.passes;
    cp.smem = tp.smem;
    for (const FPass &fp : tp.passes) {
        if (!fp.herm || fp.TB != 12) {
            cp.prm_idx.push_back(-1);
            continue;
        }
        cp.prm_idx.push_back((int)cp.prm.size());
        cp.prm.emplace_back();
        WsParams &w = cp.prm.back();
        memset(&w, 0, sizeof w);
        const bool fits = fp.nphase <= kWsParamPhases;
        for (int ph = 0; fits && ph < fp.nphase; ph++) {
            const FPhase &f = tp.phases[fp.phase0 + ph];
            w.ph[ph] = f;
            memcpy(&w.coef[ph][0], &tp.coefs[f.coef], sizeof(float2) * phase_coefs(f.nq));
        }
        w.nph = fits ? fp.nphase : -1;
    }
    for (const FPass &fp : tp.passes) {
        if (fp.herm) {
            const unsigned long long M = 1ull << (fp.nother / 2);
            cp.grid.push_back((int)(M * (M + 1) / 2));
        } else {
            cp.grid.push_back(1 << fp.nother);
        }
    }
    size_t sz_pass = sizeof(FPass) * tp.passes.size();
    cp.phase_off = (sz_pass + 255) & ~(size_t)255;
    size_t sz_ph = sizeof(FPhase) * tp.phases.size();
    cp.coef_off = (cp.phase_off + sz_ph + 255) & ~(size_t)255;
    size_t total = cp.coef_off + sizeof(float2) * tp.coefs.size();
    if (cudaMallocHost(&cp.hbuf, total) != cudaSuccess) {
        cudaGetLastError();
        cp.hbuf = nullptr;
        return set_error(QCW_ENOMEM, "fused plan staging");
    }
    memset(cp.hbuf, 0, total);
    memcpy(cp.hbuf, tp.passes.data(), sz_pass);
    if (sz_ph) memcpy(cp.hbuf + cp.phase_off, tp.phases.data(), sz_ph);
    if (!tp.coefs.empty()) memcpy(cp.hbuf + cp.coef_off, tp.coefs.data(), sizeof(float2) * tp.coefs.size());
    if (cudaMalloc(&cp.dbuf, total) != cudaSuccess) {
        cudaGetLastError();
        cp.dbuf = nullptr;
        return set_error(QCW_ENOMEM, "fused plan buffer");
    }
    // ordered before the passes that read it on the same stream, and not with other streams'
    // work (a plain cudaMemcpy would wait for the whole device)
    cudaError_t er = cudaMemcpyAsync(cp.dbuf, cp.hbuf, total, cudaMemcpyHostToDevice, c->stream);
    if (er != cudaSuccess) return cuda_error(er, "fused plan upload");
    return QCW_OK;
}

// Callers make sure no work on the context's stream still uses the plan (eviction synchronises
// the stream first; contexts synchronise before destruction).
static void release_plan(CachedPlan &cp)
{
    if (cp.dbuf) cudaFree(cp.dbuf);
    if (cp.hbuf) cudaFreeHost(cp.hbuf);
    cp.dbuf = nullptr;
    cp.hbuf = nullptr;
}

// Fusion width for the fused path: the candidate with the lowest modeled time.  The model
// is fitted to GB300 measurements of the Hermitian pass kernel on the 14-qubit benchmark
// circuit: a pass costs its HBM round trip, whose speed depends on the length of the tiles'
// contiguous runs (16-byte runs reach ~3.6 TB/s, 32-byte runs ~5 TB/s, longer ~5.7 TB/s),
// plus ~1.05 ps per element for each two-qubit phase (a quarter of that for one-qubit and
// half for product phases).  Both fits reproduce the measured steps within 3 %.
static double fused_cost(const TilePlan &tp, int n)
{
    const double el = (double)(1ull << (2 * n));
    double c = 0;
    for (const FPass &p : tp.passes) c += el * (p.L <= 1 ? 3.35e-12 : p.L == 2 ? 2.4e-12 : 2.2e-12);
    for (const FPhase &f : tp.phases) c += el * (f.nq == PH_TWO ? 1.05e-12 : f.nq == PH_PRODUCT ? 0.55e-12 : 0.3e-12);
    return c;
}

static int auto_k(const std::vector<QOp> &ops, size_t b, size_t e, int n, bool herm, int tbmax)
{
    if (n <= 3) return n;
    int best = 4;
    double bc = -1;
    for (int k = 3; k <= 5 && k <= n; k++) {
        TilePlan tp;
        append_tile_plan(plan_passes(ops, b, e, n, k, true, PassSearch::BEST), n, tbmax, tp, herm);
        const double c = fused_cost(tp, n);
        if (bc < 0 || c < bc) {
            bc = c;
            best = k;
        }
    }
    return best;
}

static const size_t kMaxCached = 64;
// Registers from this size up get beam-searched plans for segments that are replayed (a pass
// there costs at least ~10 us, so the planning time pays back over a few replays).
constexpr int kBeamMinQubits = 10;

// last: nothing follows this segment in the flush, so its last pass (if warp-specialised) also
// leaves the purity partials of the resulting rho.
static qcw_status run_segment(qcw_ctx *c, size_t b, size_t e, bool last)
{
    FusedRuntime *rt = c->fused;
    const int n = c->n;
    const bool herm0 = herm_kernel(c);
    KTune &tn = rt->tune;
    bool trial = false;
    int k;
    if (!c->fuse_k && !tn.chosen) tn.chosen = tuned_width(c);
    if (c->fuse_k) {
        k = c->fuse_k;
    } else if (tn.chosen) {
        k = tn.chosen;
    } else if (n >= 12 && herm0 && e - b >= kTuneMinOps && !tune_poll(tn) && !tn.chosen) {
        // a known segment runs at the width it has not been timed at; a new one alternates
        const uint64_t key = hash_ops(c->queue, b, e, n, 0, 0);
        int cand = tn.trials & 1;
        bool found = false;
        for (const KTuneSeg &sg : tn.segs)
            if (sg.key == key) {
                found = true;
                if (sg.have[0] != sg.have[1]) cand = sg.have[0] ? 1 : 0;
                break;
            }
        if (!found && tn.segs.size() < kTuneMaxSegs) tn.segs.push_back(KTuneSeg{key, {0.f, 0.f}, {false, false}});
        tn.cand = cand;
        tn.key = key;
        k = kTuneCand[cand];
        trial = true;
    } else {
        k = tn.chosen ? tn.chosen : auto_k(c->queue, b, e, n, herm0, herm0 ? 12 : 13);
    }
    if (tn.chosen && !tn.recorded) {
        record_width(c, tn.chosen);
        tn.recorded = true;
    }
    if (k > n) k = n;
    const bool herm = herm0;
    const int tbmax = herm ? 12 : 13;
    uint64_t h = hash_ops(c->queue, b, e, n, k, tbmax) ^ (0x9e3779b97f4a7c15ull * (uint64_t)(c->fused_kernel + 1));
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
        qcw_status st = build_plan(c, c->queue, b, e, k, tbmax, cp, false);
        if (st) {
            release_plan(cp);
            return st;
        }
        rt->cache.push_back(std::move(cp));
        hit = &rt->cache.back();
    } else if (!hit->beam && n >= kBeamMinQubits && !trial) {
        // The segment came back, so its plan is replayed: its planning time is paid once and the
        // passes it saves on every replay, so it is re-planned now with the beam search.  Work
        // still in flight may read the old plan's buffers.
        cudaError_t se = cudaStreamSynchronize(c->stream);
        if (se != cudaSuccess) return cuda_error(se, "stream");
        CachedPlan np;
        np.hash = hit->hash;
        np.n = hit->n;
        np.k = hit->k;
        np.tb = hit->tb;
        np.ops = std::move(hit->ops);
        qcw_status st = build_plan(c, c->queue, b, e, k, tbmax, np, true);
        if (st) {
            release_plan(np);
            hit->ops.assign(c->queue.begin() + b, c->queue.begin() + e);
            return st;
        }
        release_plan(*hit);
        *hit = std::move(np);
    }
    hit->last_use = ++rt->tick;

    size_t maxsm = 0;
    for (size_t p = 0; p < hit->smem.size(); p++) maxsm = std::max(maxsm, hit->smem[p]);
    qcw_status sst = ensure_smem_attr(reinterpret_cast<const void *>(k_fused_pass), maxsm);
    if (!sst) sst = ensure_smem_attr(reinterpret_cast<const void *>(k_fused_herm), maxsm);
    const bool tc = tc_kernel(c);
    const void *wsk[2][2] = {{reinterpret_cast<const void *>(k_fused_herm_ws<false>),
                              reinterpret_cast<const void *>(k_fused_herm_ws<true>)},
                             {reinterpret_cast<const void *>(k_fused_herm_tc<false>),
                              reinterpret_cast<const void *>(k_fused_herm_tc<true>)}};
    for (int a = 0; a < 2; a++)
        for (int pu = 0; pu < 2; pu++)
            if (!sst && (a == 0 || tc)) sst = ensure_smem_attr(wsk[a][pu], ws_smem_bytes());
    if (sst) return sst;
    unsigned &wgrid = tc ? rt->tc_grid : rt->ws_grid;
    if (!wgrid) {
        // Both kernels have the same registers, threads and shared memory; the occupancy query
        // on the tensor-core one reports a single CTA per SM, so it takes the other's answer,
        // capped by its kTcCols of the SM's 512 tensor-memory columns per CTA.
        int per_sm = 0;
        cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, reinterpret_cast<const void *>(k_fused_herm_ws<false>), WTH, ws_smem_bytes());
        if (oe != cudaSuccess) return cuda_error(oe, "occupancy");
        if (tc) per_sm = std::min(per_sm, 512 / kTcCols);
        wgrid = (unsigned)std::max(1, per_sm) * (unsigned)c->nsm;
    }
    if (trial) {
        if (!tn.e0) {
            cudaEventCreate(&tn.e0);
            cudaEventCreate(&tn.e1);
        }
        cudaEventRecord(tn.e0, c->stream);
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
        if (!ws_pass(c, hit->hpass[p])) {
            qcw_status fs = ensure_full(c);  // the other kernels read both triangles
            if (fs) return fs;
        }
        c->state_ver++;
        if (ws_pass(c, hit->hpass[p])) {
            c->half = true;
            const unsigned npairs = (unsigned)hit->grid[p];
            double *ppart = nullptr;
            if (last && p + 1 == hit->hpass.size()) {
                const int need = (int)std::min(npairs, wgrid);
                if (rt->ppart_cap < need) {
                    if (rt->d_ppart) cudaFree(rt->d_ppart);
                    rt->d_ppart = nullptr;
                    rt->ppart_cap = 0;
                    if (cudaMalloc(&rt->d_ppart, sizeof(double) * (size_t)need) != cudaSuccess) {
                        cudaGetLastError();
                        return set_error(QCW_ENOMEM, "purity partials");
                    }
                    rt->ppart_cap = need;
                }
                ppart = rt->d_ppart;
                rt->ppart_nb = need;
            }
            const unsigned wl = c->wait_limit ? c->wait_limit : kWsWaitLimit;
            auto kern = tc ? (ppart ? k_fused_herm_tc<true> : k_fused_herm_tc<false>)
                           : (ppart ? k_fused_herm_ws<true> : k_fused_herm_ws<false>);
            kern<<<std::min(npairs, wgrid), WTH, ws_smem_bytes(), c->stream>>>(
                c->rho, dp, dph, dco, (int)p, npairs, device_error_word(c), wl, c->stall_tile, ppart,
                hit->prm[hit->prm_idx[p]]);
        } else if (hit->hpass[p].herm) {
            k_fused_herm<<<hit->grid[p], HT, hit->smem[p], c->stream>>>(c->rho, dp, dph, dco, (int)p);
        } else {
            k_fused_pass<<<hit->grid[p], FT, hit->smem[p], c->stream>>>(c->rho, dp, dph, dco, (int)p);
        }
        c->launches++;
        c->passes++;
        if (c->timing) {
            cudaEventRecord(e1, c->stream);
            rt->ev_pending.push_back(e0);
            rt->ev_pending.push_back(e1);
        }
        cudaError_t er = cudaGetLastError();
        if (er != cudaSuccess) return cuda_error(er, "fused pass launch");
        if (last && p + 1 == hit->hpass.size() && ws_pass(c, hit->hpass[p])) c->purity_ver = c->state_ver;
    }
    if (trial) {
        cudaEventRecord(tn.e1, c->stream);
        tn.nops = e - b;
        tn.pending = true;
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
        if (i > b) st = run_segment(c, b, i, i == nq);
        if (!st && i < nq) st = plain_apply(c, c->queue[i]);
        b = i + 1;
    }
    c->queue.clear();
    return st;
}

bool fused_purity_partials(qcw_ctx *c, const double **partials, int *nblocks)
{
    FusedRuntime *rt = c->fused;
    if (!rt || !rt->d_ppart || c->purity_ver != c->state_ver) return false;
    *partials = rt->d_ppart;
    *nblocks = rt->ppart_nb;
    return true;
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
    if (rt->d_ppart) cudaFree(rt->d_ppart);
    for (cudaEvent_t e : rt->ev_free) cudaEventDestroy(e);
    for (cudaEvent_t e : rt->ev_pending) cudaEventDestroy(e);
    if (rt->tune.e0) cudaEventDestroy(rt->tune.e0);
    if (rt->tune.e1) cudaEventDestroy(rt->tune.e1);
    delete rt;
    c->fused = nullptr;
}

}  // namespace qcw
