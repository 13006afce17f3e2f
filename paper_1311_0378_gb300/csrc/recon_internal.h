// Internal layout shared by the host API and the kernels (not part of the ABI).
#pragma once
#include <stdint.h>

namespace rk {

constexpr int BW = 128;       // block width in pixels: one warp row, 32 lanes x 4 pixels
constexpr int WPR = BW / 4;   // interior 32-bit words per block row
// Shared-memory row = the TMA box row: pixels x0-16 .. x0+143 (160 bytes), so
// the box starts on a 16-byte boundary. Pixel x sits at byte XOFF + x; the
// interior is words W0 .. W0+31, the left halo pixel (x = -1) is the top byte
// of word WL, the right halo pixel (x = BW) the low byte of word WR.
constexpr int XOFF = 16;
constexpr int PW = (BW + 2 * XOFF) / 4;   // 40 words per shared-memory row
constexpr int W0 = XOFF / 4, WL = W0 - 1, WR = W0 + WPR;
constexpr int BOXW = BW + 2 * XOFF;       // TMA box width in bytes
constexpr int NT = 128;       // threads per CTA (4 warps)
constexpr int QCAP = 2048;    // shared-memory queue entries per BFS level
constexpr int GCAP = 16384;   // global spill entries per BFS level per CTA
constexpr unsigned EMPTY = 0xFFFFFFFFu;

// Block state word: flag bits (no flag = queued in the cold list, never
// visited) and, above them, the index of the block's tile, written once per
// launch so that a fetched block's tile comes with the fetch's atomic.
constexpr unsigned S_RUN = 1u, S_DIRTY = 2u, S_IDLE = 4u, S_VIS = 8u;
constexpr unsigned S_TILE_SHIFT = 4;   // tile index << S_TILE_SHIFT; at most 2^28 tiles per call
constexpr int MAX_TILES = 1 << 28;

struct alignas(16) TileDesc {
    const uint8_t *I;
    uint8_t *J;
    int H, W, pitch, conn;
    int nbx, nby;         // blocks across / down
    int k;                // first-visit scan pairs before the queue; < 0: scans to stability
    int fast;             // 1: rows start on 4-byte boundaries (word loads and stores)
                          // 2: also 16-byte rows: TMA loads through tmaps[2t], tmaps[2t+1]
    unsigned block_base;  // first global block index of this tile
    int gain;             // adaptive scan-to-queue switch: keep scanning while a pair raises >= gain px
    int dual;             // 1: erosion -- pixels are complemented (255 - v) as they are loaded and stored
    int fill;             // 1: FillHoles -- J is first set to I on the image border, 255 inside
};

struct Ctl {
    unsigned long long head, tail;   // ring of re-queued blocks
    unsigned outstanding;            // blocks queued or running
    unsigned cold;                   // cursor into the packing order
    int abort;                       // nonzero: a bound ran out (RECON_ETIMEOUT); the value says which
    unsigned abort_block;            // block being processed when it ran out
    int err_tile;                    // lowest failing tile index (INT_MAX if none)
};

// phase timers (ns, thread 0 of the CTA): load, scans, seeding, queue,
// write-back + notification + release, work fetch
enum { PH_LOAD = 0, PH_SCAN, PH_SEED, PH_QUEUE, PH_WRITE, PH_FETCH, NPH };

struct Work {
    unsigned long long visits, scan_rows, pops, seeds, levels, busy_ns;
    unsigned long long phase_ns[NPH];
};

struct Params {
    const TileDesc *tiles;
    int ntiles;
    const void *tmaps;             // 2 CUtensorMap (128 B each) per tile: I, J
    const int *order;              // packing order of tiles
    const unsigned *order_base;    // ntiles + 1 cumulative block counts in packing order
    unsigned nblocks;
    unsigned *state;               // per block: S_* flags | tile index << S_TILE_SHIFT
    unsigned long long *ring;      // ring_cap slots: state << 32 | block (see next_item)
    unsigned ring_cap;             // ring slots
    Ctl *ctl;
    int *tile_err;                 // per tile status
    Work *work;                    // per tile counters
    uint16_t *spill;               // per CTA: 2 * GCAP entries
    long long wait_ns;             // limit of one idle wait
    int bands;                     // warps scanning a block concurrently
    int revisit_scans;             // scan pairs a revisit runs before its queue phase
    int phantom;                   // test: extra outstanding unit that never ends
    int check;                     // check J <= I on first visits
    volatile unsigned *trace;      // optional: per-warp progress words in mapped host memory
};

// where-codes recorded in Ctl::abort when a bound runs out
enum {
    AB_RERUN = 1, AB_OVERFLOW = 2, AB_LEVELS = 3, AB_SCANS = 4, /* 5: unused */ AB_NOTIFY = 6,
    /* 7: unused */ AB_IDLE = 8, AB_PUSH = 9, AB_TMA = 10
};

}  // namespace rk
