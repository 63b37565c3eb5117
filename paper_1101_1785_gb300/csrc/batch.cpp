// qcw_batch_*: many independent circuits in one persistent, graph-captured launch.
//
// The paper's multiverse evaluates independent evolution paths on separate processors
// (Sec. 5.1, Sec. 5.2.1); here independent circuits share one GPU: every circuit is planned
// into a tile program (fusion width chosen per circuit by the cost model), the programs'
// work items are listed level by level (pass order inside each circuit, circuits in
// decreasing modeled cost), and one launch of the engine kernel drains the list.  The launch
// (counter resets, kernel, readout copies) is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <thread>

#include "engine.h"
#include "qcw_internal.h"

using namespace qcw;

struct qcw_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    std::vector<Program> progs;
    std::vector<size_t> rho_off;
    std::vector<int> red_first, red_n;
    char *ddesc = nullptr;
    float2 *arena = nullptr;
    size_t arena_elems = 0;
    unsigned *counters = nullptr;
    size_t ncounters = 0;
    WItem *ditems = nullptr;
    int *dint = nullptr;  // [0] nitems, [1] next item, [2] error flag
    double *dred = nullptr, *hred = nullptr;
    int *herr = nullptr;
    size_t nred = 0;
    std::vector<WItem> items;
    int grid = 0;
    size_t smem = 0;
    long long spin_limit = 20000000;  // ~2.5 s of 128 ns polls
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool launched = false;
    long long npass = 0, nphase = 0;
    double modeled = 0;
};

#define BCK(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);        \
    } while (0)

static void batch_free(qcw_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->done) cudaEventDestroy(b->done);
    cudaFree(b->ddesc);
    cudaFree(b->arena);
    cudaFree(b->counters);
    cudaFree(b->ditems);
    cudaFree(b->dint);
    cudaFree(b->dred);
    if (b->hred) cudaFreeHost(b->hred);
    if (b->herr) cudaFreeHost(b->herr);
    if (b->owns_stream) cudaStreamDestroy(b->stream);
    delete b;
}

static qcw_status batch_capture(qcw_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    EngineLaunch L;
    L.items = b->ditems;
    L.nitems = b->dint;
    L.next = b->dint + 1;
    L.err = b->dint + 2;
    L.spin_limit = b->spin_limit;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(b->counters, 0, sizeof(unsigned) * b->ncounters, b->stream);
    cudaMemsetAsync(b->dint + 1, 0, 2 * sizeof(int), b->stream);
    engine_launch(L, b->grid, b->smem, b->stream);
    cudaMemcpyAsync(b->hred, b->dred, sizeof(double) * b->nred, cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(b->herr, b->dint + 2, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    cudaError_t e = cudaStreamEndCapture(b->stream, &b->graph);
    if (e != cudaSuccess) return cuda_error(e, "batch graph capture");
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_create(int ncirc, const int *nqubits, const long long *op_begin, const qcw_op *ops,
                                       const double *matrices, int fuse_k, void *cuda_stream, qcw_batch **out)
{
    if (!out) return set_error(QCW_EINVAL, "null out");
    *out = nullptr;
    if (ncirc < 1 || !nqubits || !op_begin) return set_error(QCW_EINVAL, "bad batch description");
    if (fuse_k != 0 && (fuse_k < 2 || fuse_k > QCW_MAX_GATE_QUBITS)) return set_error(QCW_EINVAL, "bad fuse_k");
    for (int j = 0; j < ncirc; j++) {
        if (nqubits[j] < 1 || nqubits[j] > QCW_MAX_QUBITS) return set_error(QCW_EINVAL, "nqubits out of range");
        if (op_begin[j + 1] < op_begin[j] || op_begin[j] < 0) return set_error(QCW_EINVAL, "bad op ranges");
    }
    qcw_batch *b = new qcw_batch();
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!b->stream) {  // the legacy default stream cannot be captured: use a stream of our own
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return set_error(QCW_ECUDA, "batch stream");
        }
        b->owns_stream = true;
    }
    qcw_status st = QCW_OK;
    const int tbmax = 13;
    // plan every circuit (ops are validated against its own register size)
    for (int j = 0; j < ncirc && !st; j++) {
        std::vector<QOp> q;
        st = convert_ops(nqubits[j], ops + op_begin[j], (int)(op_begin[j + 1] - op_begin[j]), matrices, q);
        for (QOp &o : q)
            if (!st && o.k > 2) st = set_error(QCW_ENOTSUP, "batched circuits take 1- and 2-qubit operations");
        if (!st) b->progs.push_back(make_program(q, nqubits[j], fuse_k, tbmax));
    }
    if (st) {
        batch_free(b);
        return st;
    }
    cudaError_t ce = cudaGetDevice(&b->dev);
    if (ce != cudaSuccess) {
        batch_free(b);
        return cuda_error(ce, "cudaGetDevice");
    }
    // descriptors, arena, counters, readout blocks
    size_t dbytes = 0, aelems = 0;
    std::vector<size_t> doff(ncirc);
    b->rho_off.resize(ncirc);
    b->red_first.resize(ncirc);
    b->red_n.resize(ncirc);
    std::vector<size_t> coff(ncirc);
    for (int j = 0; j < ncirc; j++) {
        Program &p = b->progs[j];
        doff[j] = dbytes;
        dbytes += program_desc_bytes(p);
        b->rho_off[j] = aelems;
        aelems += std::max<size_t>((size_t)1 << (2 * p.n), 32);  // 256-byte granularity
        coff[j] = b->ncounters;
        b->ncounters += p.tp.passes.size();
        unsigned long long rows = reduce_rows(p.n);
        int chunks = p.whole ? 1 : (int)(((1ull << p.n) + rows - 1) / rows);
        b->red_first[j] = (int)b->nred / kRedVals;
        b->red_n[j] = chunks;
        b->nred += (size_t)chunks * kRedVals;
        b->npass += (long long)p.tp.passes.size();
        b->nphase += (long long)p.tp.phases.size();
        b->modeled += p.cost;
    }
    std::vector<char> hdesc(dbytes);
    for (int j = 0; j < ncirc; j++) program_write_desc(b->progs[j], hdesc.data(), doff[j]);
    b->arena_elems = aelems;
    if (cudaMalloc(&b->ddesc, dbytes) != cudaSuccess || cudaMalloc(&b->arena, aelems * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&b->counters, sizeof(unsigned) * (b->ncounters + 1)) != cudaSuccess ||
        cudaMalloc(&b->dint, 4 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->dred, sizeof(double) * b->nred) != cudaSuccess ||
        cudaMallocHost(&b->hred, sizeof(double) * b->nred) != cudaSuccess ||
        cudaMallocHost(&b->herr, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return set_error(QCW_ENOMEM, "batch buffers");
    }
    // items: circuits in decreasing modeled cost, level by level
    std::vector<int> order(ncirc);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->progs[x].cost > b->progs[y].cost; });
    std::vector<std::vector<WItem>> levels;
    for (int j : order) {
        const Program &p = b->progs[j];
        int nch = 0;
        program_items(p, b->arena + b->rho_off[j], b->ddesc, b->counters + coff[j],
                      b->dred + (size_t)b->red_first[j] * kRedVals, 0, (int)p.tp.passes.size(), true, true, levels,
                      &nch);
    }
    for (auto &lv : levels) b->items.insert(b->items.end(), lv.begin(), lv.end());
    int nitems = (int)b->items.size();
    size_t smem = 0;
    for (const Program &p : b->progs)
        for (size_t s : p.tp.smem) smem = std::max(smem, s);
    b->smem = smem;
    st = engine_prepare(b->dev, smem, &b->grid);
    if (!st && cudaMalloc(&b->ditems, sizeof(WItem) * std::max(nitems, 1)) != cudaSuccess) {
        cudaGetLastError();
        st = set_error(QCW_ENOMEM, "batch items");
    }
    if (!st) {
        cudaError_t e = cudaMemcpy(b->ddesc, hdesc.data(), dbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->ditems, b->items.data(), sizeof(WItem) * nitems, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->dint, &nitems, sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
        if (e != cudaSuccess) st = cuda_error(e, "batch upload");
    }
    if (!st) st = batch_capture(b);
    if (st) {
        batch_free(b);
        return st;
    }
    *out = b;
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_run(qcw_batch *b)
{
    if (!b) return set_error(QCW_EINVAL, "null batch");
    BCK(cudaGraphLaunch(b->exec, b->stream));
    BCK(cudaEventRecord(b->done, b->stream));
    b->launched = true;
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_wait(qcw_batch *b, double timeout_s)
{
    if (!b) return set_error(QCW_EINVAL, "null batch");
    if (!b->launched) return QCW_OK;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(b->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_error(e, "batch wait");
        double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s >= 0 && dt > timeout_s) return set_error(QCW_ETIMEOUT, "batch still running after the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (*b->herr) return set_error(QCW_ETIMEOUT, "a work item's dependency wait ran out in the batch kernel");
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_results(qcw_batch *b, double *p1, double *purity, double *trace)
{
    if (!b) return set_error(QCW_EINVAL, "null batch");
    qcw_status st = qcw_batch_wait(b, -1);
    if (st) return st;
    size_t pofs = 0;
    for (size_t j = 0; j < b->progs.size(); j++) {
        const int n = b->progs[j].n;
        double acc[kRedVals] = {0};
        for (int c = 0; c < b->red_n[j]; c++)  // fixed order: chunk 0, 1, ...
            for (int v = 0; v < n + 3; v++) acc[v] += b->hred[(size_t)(b->red_first[j] + c) * kRedVals + v];
        if (trace) trace[j] = acc[0];
        if (purity) purity[j] = acc[2];
        if (p1)
            for (int q = 0; q < n; q++) p1[pofs + q] = acc[3 + q];
        pofs += n;
    }
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_get_state(qcw_batch *b, int circuit, double *rho_c128)
{
    if (!b || !rho_c128 || circuit < 0 || circuit >= (int)b->progs.size()) return set_error(QCW_EINVAL, "bad argument");
    qcw_status st = qcw_batch_wait(b, -1);
    if (st) return st;
    size_t cnt = (size_t)1 << (2 * b->progs[circuit].n);
    std::vector<float2> tmp(cnt);
    BCK(cudaMemcpy(tmp.data(), b->arena + b->rho_off[circuit], cnt * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < cnt; i++) {
        rho_c128[2 * i] = tmp[i].x;
        rho_c128[2 * i + 1] = tmp[i].y;
    }
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_info(qcw_batch *b, long long *items, long long *passes, long long *phases,
                                     double *modeled_sm_s)
{
    if (!b) return set_error(QCW_EINVAL, "null batch");
    if (items) *items = (long long)b->items.size();
    if (passes) *passes = b->npass;
    if (phases) *phases = b->nphase;
    if (modeled_sm_s) *modeled_sm_s = b->modeled;
    return QCW_OK;
}

extern "C" qcw_status qcw_batch_set_wait_limit(qcw_batch *b, long long polls, int stall_item)
{
    if (!b || polls < 1 || stall_item >= (int)b->items.size()) return set_error(QCW_EINVAL, "bad argument");
    qcw_status st = qcw_batch_wait(b, -1);
    if (st && st != QCW_ETIMEOUT) return st;
    b->spin_limit = polls;
    std::vector<WItem> items = b->items;
    if (stall_item >= 0) {  // make one item wait on a counter nothing increments
        items[stall_item].dep = b->counters + b->ncounters;
        items[stall_item].dep_target = 1;
    }
    BCK(cudaMemcpy(b->ditems, items.data(), sizeof(WItem) * items.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemset(b->counters + b->ncounters, 0, sizeof(unsigned)));
    return batch_capture(b);
}

extern "C" qcw_status qcw_batch_destroy(qcw_batch *b)
{
    batch_free(b);
    return QCW_OK;
}
