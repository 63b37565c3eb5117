// Fused-mode execution of queued operations.
#include "qcw_internal.h"

namespace qcw {

qcw_status fused_flush(qcw_ctx *c)
{
    for (const QOp &op : c->queue) {
        qcw_status st = plain_apply(c, op);
        if (st) {
            c->queue.clear();
            return st;
        }
    }
    c->queue.clear();
    return QCW_OK;
}

void fused_destroy(qcw_ctx *) {}
void fused_collect_timing(qcw_ctx *) {}

}  // namespace qcw
