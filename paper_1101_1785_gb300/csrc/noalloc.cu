// Partial trace that allocates no device memory.
//
// qcw_partial_trace needs a device buffer for its FP64 result and gets one from
// cudaMallocAsync.  Some callers must not allocate: a process in which another thread is
// capturing a CUDA graph in global mode (cudaMalloc/cudaFree are then forbidden process-wide),
// an application whose memory allocator already owns the whole device budget, or a
// latency-critical loop that cannot afford the device-wide synchronisation cudaFree implies.
// This variant keeps its result buffer in a fixed array in device memory that is part of
// the library image, so it never calls cudaMalloc, cudaFree or an allocating library routine.
#include <mutex>

#include "qcw_internal.h"

namespace qcw {

// Result buffer of qcw_partial_trace_static: room for a 6-qubit reduced state (4^6 complex128,
// 64 KiB).  Every device that loads the library holds one copy until the process exits.
static __device__ __align__(256) double2 g_pt_static[QCW_PT_STATIC_MAX_ENTRIES];

namespace {
struct StaticSlot {
    double2 *ptr = nullptr;  // device address of g_pt_static on this device
    int nsm = 0;
    bool ready = false;
};
std::mutex g_static_mu;
StaticSlot g_static_slots[64];
}  // namespace

// Device address of g_pt_static for the current device.  In host code the symbol names a
// host-side shadow, not device memory, so the address must come from cudaGetSymbolAddress.
static qcw_status static_slot(StaticSlot **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(QCW_ENOTSUP, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticSlot &s = g_static_slots[dev];
    if (!s.ready) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pt_static);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_pt_static)");
        e = cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
        s.ptr = static_cast<double2 *>(p);
        s.ready = true;
    }
    *out = &s;
    return QCW_OK;
}

}  // namespace qcw

using namespace qcw;

extern "C" qcw_status qcw_partial_trace_static(const void *dev_rho, int nqubits, const int *keep, int nkeep,
                                               void *cuda_stream, double *out_c128)
{
    const int n = nqubits;
    if (!dev_rho || !out_c128) return set_error(QCW_EINVAL, "null rho or output");
    if (n < 1 || n > QCW_MAX_QUBITS) return set_error(QCW_EINVAL, "nqubits out of range");
    if (nkeep < 0 || nkeep > n || (nkeep > 0 && !keep)) return set_error(QCW_EINVAL, "bad kept-qubit list");
    if (((size_t)1 << (2 * nkeep)) > (size_t)QCW_PT_STATIC_MAX_ENTRIES)
        return set_error(QCW_EINVAL, "qcw_partial_trace_static keeps at most 6 qubits (4^6 result entries)");
    for (int j = 0; j < nkeep; j++) {
        if (keep[j] < 0 || keep[j] >= n) return set_error(QCW_EINVAL, "qubit index out of range");
        if (j && keep[j] <= keep[j - 1]) return set_error(QCW_EINVAL, "kept qubits must ascend");
    }
    StaticSlot *slot = nullptr;
    qcw_status st = static_slot(&slot);
    if (st) return st;
    PTParams p{};
    p.n = n;
    p.nkeep = nkeep;
    unsigned kept = 0;
    for (int j = 0; j < nkeep; j++) {
        p.kpos[j] = (int8_t)(n - 1 - keep[j]);
        kept |= 1u << keep[j];
    }
    for (int q = 0; q < n; q++)
        if (!(kept & (1u << q))) p.tpos[p.ntr++] = (int8_t)(n - 1 - q);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    launch_partial_trace(static_cast<const float2 *>(dev_rho), p, slot->ptr, slot->nsm, s);
    cudaError_t e = cudaGetLastError();
    size_t bytes = sizeof(double2) << (2 * nkeep);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_c128, slot->ptr, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "qcw_partial_trace_static");
    return QCW_OK;
}
