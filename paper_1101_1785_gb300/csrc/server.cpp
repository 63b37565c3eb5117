// qcw_server_*: continuous batching of circuit-simulation requests on one GPU.
//
// Requests are planned when submitted (host), wait in a FIFO, and are admitted while the
// summed footprint 16 * 4^n bytes of live requests stays within the budget (their rho lives
// in a device arena managed by a buddy allocator, next to their plan descriptors and readout
// blocks).  Each engine step launches the persistent engine kernel once over every live
// request: a request whose rho fits one tile runs to completion inside the step; a larger one
// advances by up to `passes_per_step` passes (chained by counters inside the launch) and gets
// its readout chunks in the step that finishes it.  A step waits (boundedly) for the previous
// one, harvests finished requests, admits new ones and launches; requests that arrive while
// a step runs join the next one.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>

#include "engine.h"
#include "qcw_internal.h"

using namespace qcw;

namespace {

// Power-of-two buddy allocator over [0, 2^max_order) bytes with blocks of at least 2^min_order.
class Buddy {
  public:
    void init(int min_order, int max_order)
    {
        lo_ = min_order;
        hi_ = max_order;
        free_.assign(hi_ + 1, {});
        free_[hi_].insert(0);
    }
    bool alloc(size_t bytes, size_t *off, int *order_out)
    {
        int o = lo_;
        while (o < hi_ && ((size_t)1 << o) < bytes) o++;
        if (((size_t)1 << o) < bytes) return false;
        int k = o;
        while (k <= hi_ && free_[k].empty()) k++;
        if (k > hi_) return false;
        size_t b = *free_[k].begin();
        free_[k].erase(free_[k].begin());
        while (k > o) {
            k--;
            free_[k].insert(b + ((size_t)1 << k));
        }
        *off = b;
        *order_out = o;
        return true;
    }
    void release(size_t off, int o)
    {
        while (o < hi_) {
            size_t buddy = off ^ ((size_t)1 << o);
            auto it = free_[o].find(buddy);
            if (it == free_[o].end()) break;
            free_[o].erase(it);
            off = std::min(off, buddy);
            o++;
        }
        free_[o].insert(off);
    }

  private:
    int lo_ = 0, hi_ = 0;
    std::vector<std::set<size_t>> free_;
};

int floor_log2(size_t x)
{
    int o = 0;
    while (((size_t)2 << o) <= x) o++;
    return o;
}

struct Request {
    long long id = 0;
    int n = 0;
    Program prog;
    std::vector<char> hdesc;  // host copy of the descriptors (kept until the upload completes)
    size_t rho_off = 0, desc_off = 0, red_off = 0;
    int rho_order = 0, desc_order = 0, red_order = 0;
    int next_pass = 0;
    int nchunks = 0;
    bool finishing = false;  // readout chunks are part of the step in flight
    double t_submit = 0, t_admit = 0;
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct qcw_server {
    int dev = 0, grid = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    size_t budget = 0, used = 0;
    int max_live = 0, passes_per_step = 4;
    long long spin_limit = 20000000;
    double wait_limit_s = 30.0;
    // device pools
    float2 *arena = nullptr;
    char *desc = nullptr;
    double *red = nullptr, *hred = nullptr;
    Buddy arena_alloc, desc_alloc, red_alloc;
    size_t red_bytes = 0;
    WItem *ditems = nullptr, *hitems = nullptr;
    size_t max_items = 0;
    unsigned *counters = nullptr;
    size_t max_counters = 0;
    int *dint = nullptr, *hint = nullptr;  // [0] nitems, [1] next, [2] err
    cudaEvent_t done = nullptr;
    bool in_flight = false;
    int stall_next = 0;  // diagnostics: stall one item of the next step
    // requests
    std::mutex mu;
    std::deque<Request *> waiting;
    std::vector<Request *> live;
    std::deque<qcw_result> results;
    long long next_id = 1, completed = 0;
};

static void server_free(qcw_server *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Request *r : s->waiting) delete r;
    for (Request *r : s->live) delete r;
    if (s->done) cudaEventDestroy(s->done);
    cudaFree(s->arena);
    cudaFree(s->desc);
    cudaFree(s->red);
    cudaFree(s->ditems);
    cudaFree(s->counters);
    cudaFree(s->dint);
    if (s->hred) cudaFreeHost(s->hred);
    if (s->hitems) cudaFreeHost(s->hitems);
    if (s->hint) cudaFreeHost(s->hint);
    if (s->owns_stream) cudaStreamDestroy(s->stream);
    delete s;
}

extern "C" qcw_status qcw_server_create(size_t budget_bytes, int max_live, int passes_per_step, void *cuda_stream,
                                        qcw_server **out)
{
    if (!out) return set_error(QCW_EINVAL, "null out");
    *out = nullptr;
    if (budget_bytes < 4096 || max_live < 1 || passes_per_step < 1) return set_error(QCW_EINVAL, "bad server limits");
    qcw_server *s = new qcw_server();
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!s->stream) {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return set_error(QCW_ECUDA, "server stream");
        }
        s->owns_stream = true;
    }
    s->budget = budget_bytes;
    s->max_live = max_live;
    s->passes_per_step = passes_per_step;
    // rho storage is 8 * 4^n bytes against a 16 * 4^n footprint: the arena is half the budget
    int arena_order = floor_log2(budget_bytes / 2);
    s->arena_alloc.init(8, arena_order);
    int desc_order = 26;  // 64 MiB of plan descriptors
    s->desc_alloc.init(8, desc_order);
    int red_order = 24;  // 16 MiB of readout blocks
    s->red_bytes = (size_t)1 << red_order;
    s->red_alloc.init(8, red_order);
    s->max_items = 1 << 20;
    s->max_counters = 1 << 20;
    s->smem = tile_smem_bytes(13, 3);
    qcw_status st = QCW_OK;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e != cudaSuccess) st = cuda_error(e, "cudaGetDevice");
    if (!st && (cudaMalloc(&s->arena, (size_t)1 << arena_order) != cudaSuccess ||
                cudaMalloc(&s->desc, (size_t)1 << desc_order) != cudaSuccess ||
                cudaMalloc(&s->red, s->red_bytes) != cudaSuccess ||
                cudaMallocHost(&s->hred, s->red_bytes) != cudaSuccess ||
                cudaMalloc(&s->ditems, sizeof(WItem) * s->max_items) != cudaSuccess ||
                cudaMallocHost(&s->hitems, sizeof(WItem) * s->max_items) != cudaSuccess ||
                cudaMalloc(&s->counters, sizeof(unsigned) * (s->max_counters + 1)) != cudaSuccess ||
                cudaMalloc(&s->dint, 4 * sizeof(int)) != cudaSuccess ||
                cudaMallocHost(&s->hint, 4 * sizeof(int)) != cudaSuccess)) {
        cudaGetLastError();
        st = set_error(QCW_ENOMEM, "server buffers");
    }
    if (!st) st = engine_prepare(s->dev, s->smem, &s->grid);
    if (!st) {
        e = cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMemset(s->counters + s->max_counters, 0, sizeof(unsigned));
        if (e != cudaSuccess) st = cuda_error(e, "server setup");
    }
    if (st) {
        server_free(s);
        return st;
    }
    *out = s;
    return QCW_OK;
}

extern "C" qcw_status qcw_server_submit(qcw_server *s, int nqubits, const qcw_op *ops, int nops, const double *matrices,
                                        long long *id)
{
    if (!s) return set_error(QCW_EINVAL, "null server");
    if (nqubits < 1 || nqubits > 13) return set_error(QCW_EINVAL, "served requests take 1..13 qubits");
    if (((size_t)16 << (2 * nqubits)) > s->budget) return set_error(QCW_EINVAL, "request larger than the budget");
    std::vector<QOp> q;
    qcw_status st = convert_ops(nqubits, ops, nops, matrices, q);
    if (st) return st;
    for (QOp &o : q)
        if (o.k > 2) return set_error(QCW_ENOTSUP, "served circuits take 1- and 2-qubit operations");
    Request *r = new Request();
    r->n = nqubits;
    r->prog = make_program(q, nqubits, 0, 13);
    r->hdesc.assign(program_desc_bytes(r->prog), 0);
    program_write_desc(r->prog, r->hdesc.data(), 0);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    if (id) *id = r->id;
    s->waiting.push_back(r);
    return QCW_OK;
}

static void release_request(qcw_server *s, Request *r)
{
    s->arena_alloc.release(r->rho_off, r->rho_order);
    s->desc_alloc.release(r->desc_off, r->desc_order);
    if (r->nchunks) s->red_alloc.release(r->red_off, r->red_order);
    s->used -= (size_t)16 << (2 * r->n);
}

// Wait for the step in flight and harvest the requests it finished.
static qcw_status finish_step(qcw_server *s, double limit_s)
{
    if (!s->in_flight) return QCW_OK;
    double t0 = now_s();
    for (;;) {
        cudaError_t e = cudaEventQuery(s->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_error(e, "server step");
        if (now_s() - t0 > limit_s) return set_error(QCW_ETIMEOUT, "engine step still running after the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    s->in_flight = false;
    const bool err = s->hint[2] != 0;
    const double t = now_s();
    std::vector<Request *> keep;
    for (Request *r : s->live) {
        if (r->finishing) {
            qcw_result res{};
            res.id = r->id;
            res.nqubits = r->n;
            res.status = err ? QCW_ETIMEOUT : QCW_OK;
            double acc[kRedVals] = {0};
            const double *src = s->hred + r->red_off / sizeof(double);
            for (int c = 0; c < r->nchunks; c++)
                for (int v = 0; v < r->n + 3; v++) acc[v] += src[(size_t)c * kRedVals + v];
            res.trace = acc[0];
            res.purity = acc[2];
            for (int q = 0; q < r->n; q++) res.p1[q] = acc[3 + q];
            res.t_submit = r->t_submit;
            res.t_done = t;
            release_request(s, r);
            s->results.push_back(res);
            s->completed++;
            delete r;
        } else {
            keep.push_back(r);
        }
    }
    s->live.swap(keep);
    if (err) return set_error(QCW_ETIMEOUT, "a work item's dependency wait ran out in the engine step");
    return QCW_OK;
}

extern "C" qcw_status qcw_server_step(qcw_server *s, int *launched_items)
{
    if (!s) return set_error(QCW_EINVAL, "null server");
    if (launched_items) *launched_items = 0;
    qcw_status st = finish_step(s, s->wait_limit_s);
    if (st) return st;
    // admission (FIFO) by footprint
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->waiting.empty() && (int)s->live.size() < s->max_live) {
            Request *r = s->waiting.front();
            size_t fp = (size_t)16 << (2 * r->n);
            if (s->used + fp > s->budget) break;
            size_t rho_bytes = std::max<size_t>((size_t)8 << (2 * r->n), 256);
            if (!s->arena_alloc.alloc(rho_bytes, &r->rho_off, &r->rho_order)) break;
            if (!s->desc_alloc.alloc(r->hdesc.size(), &r->desc_off, &r->desc_order)) {
                s->arena_alloc.release(r->rho_off, r->rho_order);
                break;
            }
            int chunks = r->prog.whole ? 1 : (int)(((1ull << r->n) + reduce_rows(r->n) - 1) / reduce_rows(r->n));
            if (!s->red_alloc.alloc(sizeof(double) * kRedVals * chunks, &r->red_off, &r->red_order)) {
                s->arena_alloc.release(r->rho_off, r->rho_order);
                s->desc_alloc.release(r->desc_off, r->desc_order);
                break;
            }
            r->nchunks = chunks;
            s->used += fp;
            s->waiting.pop_front();
            r->t_admit = now_s();
            cudaError_t e = cudaMemcpyAsync(s->desc + r->desc_off, r->hdesc.data(), r->hdesc.size(),
                                            cudaMemcpyHostToDevice, s->stream);
            s->live.push_back(r);
            if (e != cudaSuccess) return cuda_error(e, "descriptor upload");
        }
    }
    if (s->live.empty()) return QCW_OK;
    // work items, level by level
    std::vector<std::vector<WItem>> levels;
    size_t ncount = 0;
    for (Request *r : s->live) {
        const Program &p = r->prog;
        const int np = (int)p.tp.passes.size();
        const int p0 = r->next_pass, p1 = p.whole ? np : std::min(np, p0 + s->passes_per_step);
        const bool readout = p.whole || p1 == np;
        if (!p.whole && ncount + np > s->max_counters) continue;  // waits for the next step
        int nch = 0;
        program_items(p, s->arena + r->rho_off / sizeof(float2), s->desc + r->desc_off, s->counters + ncount,
                      s->red + r->red_off / sizeof(double), p0, p1, p0 == 0, readout, levels, &nch);
        if (!p.whole) ncount += (size_t)(p1 - p0);
        r->finishing = readout;
        r->next_pass = p1;
    }
    size_t nitems = 0;
    for (auto &lv : levels) nitems += lv.size();
    if (nitems > s->max_items) return set_error(QCW_ENOTSUP, "step exceeds the work-item buffer");
    size_t k = 0;
    for (auto &lv : levels)
        for (const WItem &w : lv) s->hitems[k++] = w;
    if (s->stall_next > 0 && nitems > 0) {  // diagnostics: one item waits on a counter nothing sets
        s->hitems[nitems - 1].dep = s->counters + s->max_counters;
        s->hitems[nitems - 1].dep_target = 1;
        s->stall_next = 0;
    }
    s->hint[0] = (int)nitems;
    EngineLaunch L;
    L.items = s->ditems;
    L.nitems = s->dint;
    L.next = s->dint + 1;
    L.err = s->dint + 2;
    L.spin_limit = s->spin_limit;
    cudaError_t e = cudaMemcpyAsync(s->ditems, s->hitems, sizeof(WItem) * nitems, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->dint, s->hint, sizeof(int), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dint + 1, 0, 2 * sizeof(int), s->stream);
    if (e == cudaSuccess && ncount) e = cudaMemsetAsync(s->counters, 0, sizeof(unsigned) * ncount, s->stream);
    if (e != cudaSuccess) return cuda_error(e, "step upload");
    engine_launch(L, s->grid, s->smem, s->stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "engine launch");
    for (Request *r : s->live)
        if (r->finishing) {
            e = cudaMemcpyAsync(s->hred + r->red_off / sizeof(double), s->red + r->red_off / sizeof(double),
                                sizeof(double) * kRedVals * r->nchunks, cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return cuda_error(e, "readout copy");
        }
    e = cudaMemcpyAsync(s->hint + 2, s->dint + 2, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->done, s->stream);
    if (e != cudaSuccess) return cuda_error(e, "step record");
    s->in_flight = true;
    if (launched_items) *launched_items = (int)nitems;
    return QCW_OK;
}

extern "C" qcw_status qcw_server_drain(qcw_server *s, double timeout_s)
{
    if (!s) return set_error(QCW_EINVAL, "null server");
    double t0 = now_s();
    for (;;) {
        qcw_status st = finish_step(s, timeout_s < 0 ? s->wait_limit_s : timeout_s);
        if (st) return st;
        bool idle;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            idle = s->waiting.empty() && s->live.empty();
        }
        if (idle) return QCW_OK;
        if (timeout_s >= 0 && now_s() - t0 > timeout_s) return set_error(QCW_ETIMEOUT, "server not drained in time");
        st = qcw_server_step(s, nullptr);
        if (st) return st;
    }
}

extern "C" qcw_status qcw_server_poll(qcw_server *s, qcw_result *out, int max, int *count)
{
    if (!s || (max > 0 && !out) || !count) return set_error(QCW_EINVAL, "bad poll arguments");
    int c = 0;
    while (c < max && !s->results.empty()) {
        out[c++] = s->results.front();
        s->results.pop_front();
    }
    *count = c;
    return QCW_OK;
}

extern "C" qcw_status qcw_server_stats(qcw_server *s, long long *waiting, long long *live, long long *completed,
                                       long long *bytes_in_use)
{
    if (!s) return set_error(QCW_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (waiting) *waiting = (long long)s->waiting.size();
    if (live) *live = (long long)s->live.size();
    if (completed) *completed = s->completed;
    if (bytes_in_use) *bytes_in_use = (long long)s->used;
    return QCW_OK;
}

extern "C" qcw_status qcw_server_set_limits(qcw_server *s, double wait_limit_s, long long polls, int stall_next_step)
{
    if (!s || polls < 1) return set_error(QCW_EINVAL, "bad limits");
    s->wait_limit_s = wait_limit_s;
    s->spin_limit = polls;
    s->stall_next = stall_next_step ? 1 : 0;
    return QCW_OK;
}

extern "C" qcw_status qcw_server_destroy(qcw_server *s)
{
    server_free(s);
    return QCW_OK;
}
