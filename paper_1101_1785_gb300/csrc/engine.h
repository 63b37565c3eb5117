// Work-item engine shared by the batched runner (qcw_batch_*) and the serving loop
// (qcw_server_*): circuits are planned into tile programs, programs into work items, and one
// persistent kernel drains the item list.
#pragma once
#include <stdint.h>

#include <vector>

#include "tile.h"

namespace qcw {

// Kinds of work item.
enum : int {
    WI_TILES = 0,   // tiles [tile0, tile0 + ntile) of one pass of a multi-tile program
    WI_REDUCE = 1,  // FP64 readouts over rows [red_row0, red_row0 + red_rows) of rho
    WI_WHOLE = 2,   // a whole program whose rho fits one tile: load once, all passes, readouts, store
};
enum : int { WF_INIT = 1 };  // the item's tiles start as |0..0><0..0| instead of being loaded

struct WItem {
    float2 *rho;
    const FPass *pass;       // first pass of the item
    const FPhase *phases;    // phase array of the program
    const float2 *coefs;     // coefficient array of the program
    unsigned *dep;           // wait until *dep >= dep_target (nullptr: no dependency)
    unsigned *done;          // incremented once the item's stores are complete (nullptr: none)
    double *red;             // readout output (kinds 1, 2): trace re, trace im, purity, p1[n]
    unsigned long long red_row0, red_rows;
    unsigned dep_target;
    unsigned tile0, ntile;
    int npass;
    int kind;
    int flags;
    int n;
    int pad;
};

constexpr int kRedVals = 3 + QCW_MAX_QUBITS;  // values per readout block

// Launch state of the persistent kernel.
struct EngineLaunch {
    const WItem *items;
    const int *nitems;
    int *next;
    int *err;
    long long spin_limit;
};

void engine_launch(const EngineLaunch &L, int grid, size_t smem, cudaStream_t s);
qcw_status engine_prepare(int dev, size_t smem, int *grid);

// A circuit turned into device-ready descriptors.
struct Program {
    int n = 0, k = 0, tbmax = 13;
    bool whole = false;      // rho fits one tile: one WI_WHOLE item
    TilePlan tp;
    double cost = 0;         // modeled SM-seconds
    size_t off_pass = 0, off_phase = 0, off_coef = 0;  // offsets inside a descriptor buffer
};

// Plan ops for an n-qubit register; fuse_k = 0 lets the cost model choose the width.
Program make_program(const std::vector<QOp> &ops, int n, int fuse_k, int tbmax);

// Modeled cost (SM-seconds) of running a plan; used to choose the fusion width.
double model_cost(const TilePlan &tp, int n);
int choose_fuse_k(const std::vector<QOp> &ops, size_t b, size_t e, int n, int tbmax);

// Bytes a program's descriptors occupy in a descriptor buffer (256-byte aligned sections).
size_t program_desc_bytes(const Program &p);
// Copy a program's descriptors to host staging at `base + off` and record the offsets.
void program_write_desc(Program &p, char *host, size_t off);

// Number of tiles of pass p of a program.
inline unsigned program_tiles(const Program &p, size_t pass) { return 1u << p.tp.passes[pass].nother; }

// Readout chunks of a multi-tile program (rows per chunk chosen for ~2^17 elements).
inline unsigned long long reduce_rows(int n)
{
    unsigned long long rows = (1ull << 17) >> n;
    if (rows < 1) rows = 1;
    if (rows > (1ull << n)) rows = 1ull << n;
    return rows;
}

// Items of passes [pass_begin, pass_end) of one program.  Appends to `levels[l]` (level = pass
// index - pass_begin; readouts on the level after the last pass).  desc: device base of the
// descriptor buffer holding the program; counters: (pass_end - pass_begin) zeroed device
// counters, one per pass of the range; red: its readout blocks (chunk count in *nchunks).
void program_items(const Program &p, float2 *rho, const char *desc, unsigned *counters, double *red,
                   int pass_begin, int pass_end, bool init, bool readout, std::vector<std::vector<WItem>> &levels,
                   int *nchunks);

}  // namespace qcw
