// Persistent work-item kernel shared by the batched runner and the serving loop, and the
// host code that turns circuits into programs and programs into work items.
//
// Every CTA repeatedly takes the next item from a global counter.  Items are listed in an
// order where an item's dependency (the previous pass of the same circuit) always comes
// earlier in the list, so a CTA only ever waits for items that running CTAs already hold;
// every wait is bounded (spin_limit polls) and a wait that runs out sets *err instead of
// hanging.  A circuit whose rho fits one tile (2n <= tile bits) is one item: its state is
// built in shared memory, evolved through every phase and read out there, then written once.
// Larger circuits are split into one item per tile and pass, chained by per-pass counters,
// followed by readout chunks.  Each circuit is processed by a fixed item decomposition with
// a fixed thread-to-data mapping, so its result does not depend on what else is in the batch.
#include <algorithm>
#include <cstring>

#include "engine.h"
#include "qcw_internal.h"
#include "tile.cuh"

namespace qcw {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

using RedShared = double[kTileThreads / 32][kRedVals];

// Fold per-thread accumulators (first nv used) into out[0..nv) with a fixed tree.
__device__ __forceinline__ void red_store(double (&acc)[kRedVals], int nv, double *out, RedShared &sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kRedVals; v++) {
        if (v < nv) {
            double s = warp_sum(acc[v]);
            if (lane == 0) sh[w][v] = s;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        double t = 0;
        for (int j = 0; j < kTileThreads / 32; j++) t += sh[j][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// Readouts of rows [row0, row0 + rows) of an n-qubit rho stored at `src` with row stride 2^n:
// trace (re, im) and p1[q] from the diagonal, purity from every element of those rows.
__device__ __forceinline__ void readout_rows(const float2 *__restrict__ src, int n, unsigned long long row0,
                                             unsigned long long rows, double *out, RedShared &sh)
{
    double acc[kRedVals];
#pragma unroll
    for (int v = 0; v < kRedVals; v++) acc[v] = 0;
    const unsigned long long dim = 1ull << n;
    for (unsigned long long r = row0 + threadIdx.x; r < row0 + rows; r += kTileThreads) {
        float2 d = src[r * dim + r];
        acc[0] += d.x;
        acc[1] += d.y;
#pragma unroll
        for (int q = 0; q < QCW_MAX_QUBITS; q++)
            if (q < n && ((r >> (n - 1 - q)) & 1)) acc[3 + q] += d.x;
    }
    const float4 *s4 = reinterpret_cast<const float4 *>(src + row0 * dim);
    const unsigned long long n4 = rows * dim / 2;
    for (unsigned long long i = threadIdx.x; i < n4; i += 4 * kTileThreads) {
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            unsigned long long j = i + (unsigned long long)u * kTileThreads;
            if (j < n4) {
                float4 a = s4[j];
                s = fmaf(a.x, a.x, s); s = fmaf(a.y, a.y, s); s = fmaf(a.z, a.z, s); s = fmaf(a.w, a.w, s);
            }
        }
        acc[2] += (double)s;
    }
    red_store(acc, n + 3, out, sh);
}

__device__ void run_tiles(const WItem &W, unsigned char *smem)
{
    const FPass &P = *W.pass;
    const TileSmem sm = tile_smem(smem, P.TB, P.L);
    tile_hoff(P, sm.hoff);
    __syncthreads();
    for (unsigned t = W.tile0; t < W.tile0 + W.ntile; t++) {
        tile_process(W.rho, P, t, W.phases, W.coefs, sm, (W.flags & WF_INIT) != 0);
        __syncthreads();
    }
}

__device__ void run_whole(const WItem &W, unsigned char *smem, RedShared &sh)
{
    const FPass &P0 = W.pass[0];
    const TileSmem sm = tile_smem(smem, P0.TB, P0.L);
    tile_hoff(P0, sm.hoff);
    __syncthreads();
    tile_load(W.rho, P0, 0, sm, (W.flags & WF_INIT) != 0);
    for (int p = 0; p < W.npass; p++) tile_phases(W.pass[p], W.phases, W.coefs, sm);
    // the tile is the whole matrix in flat order (tile bits 0..2n-1)
    if (W.red) readout_rows(sm.tile, W.n, 0, 1ull << W.n, W.red, sh);
    tile_store(W.rho, P0, 0, sm);
}

__global__ void __launch_bounds__(kTileThreads, 2) k_engine(EngineLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ RedShared s_red;
    const int nitems = *L.nitems;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(L.next, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) return;
        const WItem W = L.items[it];
        if (W.dep) {
            if (threadIdx.x == 0) {
                long long spins = 0;
                while (ld_acquire(W.dep) < W.dep_target) {
                    if (++spins > L.spin_limit) {
                        atomicOr(L.err, 1);
                        break;
                    }
                    __nanosleep(128);
                }
            }
            __syncthreads();
        }
        if (W.kind == WI_TILES) run_tiles(W, smem);
        else if (W.kind == WI_WHOLE) run_whole(W, smem, s_red);
        else readout_rows(W.rho, W.n, W.red_row0, W.red_rows, W.red, s_red);
        __syncthreads();
        if (W.done && threadIdx.x == 0) {
            __threadfence();
            atomicAdd(W.done, 1u);
        }
    }
}

void engine_launch(const EngineLaunch &L, int grid, size_t smem, cudaStream_t s)
{
    k_engine<<<grid, kTileThreads, smem, s>>>(L);
}

qcw_status engine_prepare(int dev, size_t smem, int *grid)
{
    qcw_status st = ensure_smem_attr(reinterpret_cast<const void *>(k_engine), smem);
    if (st) return st;
    int occ = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_engine, kTileThreads, smem);
    if (e != cudaSuccess) return cuda_error(e, "engine occupancy");
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "SM count");
    if (occ < 1) return set_error(QCW_ENOTSUP, "engine kernel does not fit on an SM");
    *grid = occ * nsm;
    return QCW_OK;
}

// ------------------------------------------------------------------ host: programs
// Cost model (SM-seconds per element of rho), from GB300 measurements of k_fused_pass: one
// pass moves 16 bytes per element at ~44 GB/s per SM (6.67 TB/s / 152); a two-qubit phase
// costs ~0.54 ns per element per SM (64 FP32 FMA at the measured issue efficiency), a
// one-qubit phase about a quarter of that.
static const double kCostPass = 16.0 / 44e9;
static const double kCostPhase2 = 0.54e-9;
static const double kCostPhase1 = 0.15e-9;

double model_cost(const TilePlan &tp, int n)
{
    double el = (double)(1ull << (2 * n));
    double c = 0;
    for (const FPass &p : tp.passes) c += kCostPass * el;
    for (const FPhase &f : tp.phases)
        c += (f.nq == PH_TWO ? kCostPhase2 : f.nq == PH_PRODUCT ? 2 * kCostPhase1 : kCostPhase1) * el;
    return c;
}

int choose_fuse_k(const std::vector<QOp> &ops, size_t b, size_t e, int n, int tbmax)
{
    int best = n < 5 ? n : 5;
    double bc = -1;
    for (int k = 2; k <= 5 && k <= n; k++) {
        TilePlan tp;
        append_tile_plan(plan_passes(ops, b, e, n, k, true), n, tbmax, tp);
        double c = model_cost(tp, n);
        if (bc < 0 || c < bc) {
            bc = c;
            best = k;
        }
    }
    return best;
}

Program make_program(const std::vector<QOp> &ops, int n, int fuse_k, int tbmax)
{
    Program p;
    p.n = n;
    p.tbmax = tbmax;
    p.whole = 2 * n <= tbmax;
    std::vector<PassPlan> plan;
    if (p.whole) {
        p.k = n;
        plan = plan_passes(ops, 0, ops.size(), n, n);
        if (plan.empty()) plan.emplace_back();
        plan.resize(1);  // with k = n every op joins the first pass
        plan[0].Q.clear();
        for (int q = 0; q < n; q++) plan[0].Q.push_back(q);
    } else {
        p.k = fuse_k ? std::min(fuse_k, n) : choose_fuse_k(ops, 0, ops.size(), n, tbmax);
        plan = plan_passes(ops, 0, ops.size(), n, p.k);
        if (plan.empty()) plan.emplace_back();  // an empty pass still writes the initial state
    }
    append_tile_plan(plan, n, tbmax, p.tp);
    p.cost = model_cost(p.tp, n);
    return p;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t program_desc_bytes(const Program &p)
{
    return al256(sizeof(FPass) * p.tp.passes.size()) + al256(sizeof(FPhase) * p.tp.phases.size()) +
           al256(sizeof(float2) * p.tp.coefs.size());
}

void program_write_desc(Program &p, char *host, size_t off)
{
    p.off_pass = off;
    memcpy(host + off, p.tp.passes.data(), sizeof(FPass) * p.tp.passes.size());
    off += al256(sizeof(FPass) * p.tp.passes.size());
    p.off_phase = off;
    if (!p.tp.phases.empty()) memcpy(host + off, p.tp.phases.data(), sizeof(FPhase) * p.tp.phases.size());
    off += al256(sizeof(FPhase) * p.tp.phases.size());
    p.off_coef = off;
    if (!p.tp.coefs.empty()) memcpy(host + off, p.tp.coefs.data(), sizeof(float2) * p.tp.coefs.size());
}

void program_items(const Program &p, float2 *rho, const char *desc, unsigned *counters, double *red, int pass_begin,
                   int pass_end, bool init, bool readout, std::vector<std::vector<WItem>> &levels, int *nchunks)
{
    const FPass *dpass = reinterpret_cast<const FPass *>(desc + p.off_pass);
    const FPhase *dph = reinterpret_cast<const FPhase *>(desc + p.off_phase);
    const float2 *dco = reinterpret_cast<const float2 *>(desc + p.off_coef);
    *nchunks = 0;
    auto level = [&](size_t l) -> std::vector<WItem> & {
        if (levels.size() <= l) levels.resize(l + 1);
        return levels[l];
    };
    if (p.whole) {
        WItem w{};
        w.rho = rho;
        w.pass = dpass;
        w.phases = dph;
        w.coefs = dco;
        w.npass = (int)p.tp.passes.size();
        w.kind = WI_WHOLE;
        w.flags = init ? WF_INIT : 0;
        w.n = p.n;
        w.red = readout ? red : nullptr;
        level(0).push_back(w);
        *nchunks = readout ? 1 : 0;
        return;
    }
    for (int ps = pass_begin; ps < pass_end; ps++) {
        unsigned nt = program_tiles(p, ps);
        for (unsigned t = 0; t < nt; t++) {
            WItem w{};
            w.rho = rho;
            w.pass = dpass + ps;
            w.phases = dph;
            w.coefs = dco;
            w.tile0 = t;
            w.ntile = 1;
            w.kind = WI_TILES;
            w.flags = (init && ps == 0) ? WF_INIT : 0;
            w.n = p.n;
            if (ps > pass_begin) {
                w.dep = counters + (ps - 1 - pass_begin);
                w.dep_target = program_tiles(p, ps - 1);
            }
            w.done = counters + (ps - pass_begin);
            level(ps - pass_begin).push_back(w);
        }
    }
    if (readout && pass_end == (int)p.tp.passes.size()) {
        unsigned long long rows = reduce_rows(p.n), dim = 1ull << p.n;
        int c = 0;
        for (unsigned long long r0 = 0; r0 < dim; r0 += rows, c++) {
            WItem w{};
            w.rho = rho;
            w.kind = WI_REDUCE;
            w.n = p.n;
            w.red = red + (size_t)c * kRedVals;
            w.red_row0 = r0;
            w.red_rows = rows;
            if (pass_end > pass_begin) {
                w.dep = counters + (pass_end - 1 - pass_begin);
                w.dep_target = program_tiles(p, pass_end - 1);
            }
            level(pass_end - pass_begin).push_back(w);
        }
        *nchunks = c;
    }
}

}  // namespace qcw
