// Grayscale morphological reconstruction by irregular wavefront propagation
// (Table II "Morphological Reconstruction"; Sec. II-B Algorithm 1; the hybrid
// scan-then-queue schedule of Sec. V-C) for sm_103a.
//
// Design. The image is cut into blocks of BH x 128 pixels. One persistent
// launch pulls blocks from a work list: first every block once, in packing
// order (the "cold" list), then blocks re-queued because a neighbour raised a
// pixel on their border (a ring in global memory). A CTA reconstructs its block
// locally in shared memory against the block's 1-pixel halo:
//   1. k raster + anti-raster scan pairs, then (adaptive variants) more pairs
//      while a pair still raises enough pixels, or scans until a pair changes
//      nothing (variant k < 0). Up to four warps scan row bands at once; a
//      scan row is one warp: a vertical max from the previous row, then a warp
//      prefix scan of clamp maps along the row, in two-plane u16x2 arithmetic;
//   2. a seeding pass: one in-place geodesic dilation whose changed pixels form
//      the frontier (Algorithm 1's initialization phase) -- after scans only
//      next to the rows the last pair changed, on revisits only on the frame;
//   3. the wavefront phase in shared memory: wide levels level-synchronously
//      (warp-ballot compaction, spill to global memory), thin ones in per-warp
//      rings; each update an atomic byte max under the mask,
//      J(q) <- max(J(q), min(J(p), I(q))).
// Erosion tiles run the same steps on complemented values (complemented as
// they are loaded and stored).
// The block then writes its changed rows and notifies each neighbour block
// whose halo can now receive a propagation. Every update is a monotone step
// towards the unique fixed point R, so any order of blocks and updates yields
// the same bytes. Each block has one writer at a time (the RUN state bit);
// a notification for a running block sets DIRTY and the runner re-reads its
// halo before it lets go. Every device-side wait is bounded.
#include <climits>
#include <cuda_runtime.h>
#include "recon_internal.h"

namespace rk {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Bounds-checked build (-DRECON_CHECKS, librecon_checks.so): the stand-in for
// a memory checker. Every queue slot and every wavefront pixel offset is
// checked before it is used; a failed check is counted, its where-code kept
// (1: queue slot, 2: wavefront pixel offset, 3: pushed pixel offset), and the
// access is skipped instead of made. Read back with recon_checks().
#ifdef RECON_CHECKS
__device__ unsigned g_check_violations;
__device__ unsigned g_check_first;
__device__ __noinline__ bool check_fail(unsigned where)
{
    atomicAdd(&g_check_violations, 1u);
    atomicCAS(&g_check_first, 0u, where);
    return false;
}
#define RK_CHECK(cond, where) ((cond) ? true : check_fail(where))
#else
#define RK_CHECK(cond, where) true
#endif

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


// Rows of a block held in shared memory: BH + 2 (with the halo), loaded by
// one TMA box -- or, above 256 rows (the largest box), by two boxes of TBOX
// rows, TBOX a multiple of 4 so that the second box starts 128-byte aligned;
// the rows past the halo row are loaded but never used.
template <int BH>
struct Boxes {
    static constexpr int N = BH + 2 > 256 ? 2 : 1;
    static constexpr int TBOX = N == 1 ? BH + 2 : ((BH + 2) / 2 + 3) / 4 * 4;
    static constexpr int ROWS = N * TBOX;
    static_assert(TBOX <= 256 && ROWS >= BH + 2 && (TBOX * BOXW) % 128 == 0 || N == 1, "TMA boxes");
};

template <int BH>
struct Smem {
    alignas(128) uint32_t J[Boxes<BH>::ROWS * PW];   // TMA destinations: 128-byte aligned
    alignas(128) uint32_t I[Boxes<BH>::ROWS * PW];   // 0 on the halo: nothing ever propagates into it
    unsigned long long mbar;                  // TMA completion barrier
    uint16_t q[2][QCAP];          // BFS levels (byte offsets into J)
    uint8_t hIt[BW + 2], hIb[BW + 2];  // halo mask, top / bottom rows, x = -1 .. BW
    uint8_t hIl[BH], hIr[BH];          // halo mask, left / right columns
    uint8_t eT[BW], eB[BW], eL[BH], eR[BH];  // edge values when neighbours last saw them
    unsigned rowmask[BH / 32];    // rows changed since the block was loaded
    unsigned pairmask[BH / 32];   // rows changed by the latest scan pair
    unsigned claim[2][BH * BW / 32];  // wavefront ownership bits, one per interior pixel, by level parity
    unsigned cq[3];               // level sizes, rotating by level (see run_queue)
    unsigned solo_src, solo_L;    // queue buffer and level count after a warp-solo run
    unsigned item, tile, flag, overflow, notify, visited;
    unsigned phase;               // parity of the TMA barrier's next completion
    unsigned abrt;                // block-uniform copy of the abort word
    Work acc;                     // thread 0: counters of consecutive visits to tile acc_tile
    int acc_tile;
};

__device__ __forceinline__ int find_tile(const Params &P, unsigned b)
{
    int lo = 0, hi = P.ntiles - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.tiles[mid].block_base <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned cold_block(const Params &P, unsigned c)
{
    int lo = 0, hi = P.ntiles - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.order_base[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return P.tiles[P.order[lo]].block_base + (c - P.order_base[lo]);
}

// Records the first bound that ran out (see AB_*); every CTA then winds down.
__device__ void set_abort(const Params &P, int where)
{
    atomicCAS(&P.ctl->abort, 0, where);
}

__device__ __forceinline__ bool aborted(const Params &P) { return *(volatile int *)&P.ctl->abort != 0; }

// progress trace (debug): lane 0 of each warp writes (code << 24 | block & 0xFFFFFF)
__device__ __forceinline__ void trace(const Params &P, unsigned code, unsigned b)
{
    if (P.trace && (threadIdx.x & 31) == 0)
        P.trace[blockIdx.x * (NT / 32) + (threadIdx.x >> 5)] = (code << 24) | (b & 0xFFFFFFu);
}

// The ring of re-queued blocks. Position t (from the tail for producers,
// from the head for consumers, one atomicAdd each) uses slot t % ring_cap in
// lap L = t / ring_cap. A slot word holds state << 32 | block, with state
// 4L + 0 (free for lap L), 4L + 1 (holds lap L's block) or 4L + 2 (lap L's
// ticket was given up). Producer and consumer of a position each wait for
// their own lap's state, so laps never mix, whatever the ring size.
__device__ __forceinline__ unsigned long long slot_word(unsigned state, unsigned b)
{
    return ((unsigned long long)state << 32) | b;
}

// Appends block b to the ring (the caller already moved its state from IDLE
// to queued and counted it as outstanding). If the position's ticket was
// given up, the slot is freed for the next lap and b goes to a new position.
__device__ void push_hot(const Params &P, unsigned b)
{
    for (int attempt = 0;; ++attempt) {
        if (attempt > (1 << 20)) { set_abort(P, AB_PUSH); return; }
        const unsigned long long t = atomicAdd(&P.ctl->tail, 1ull);
        unsigned long long *slot = &P.ring[t % P.ring_cap];
        const unsigned lap4 = (unsigned)(t / P.ring_cap) * 4u;
        // a slot free for this lap holds exactly slot_word(lap4, 0): publish
        // on that guess first, and otherwise go on from the word the CAS saw
        unsigned long long w = atomicCAS(slot, slot_word(lap4, 0), slot_word(lap4 + 1, b));
        if (w == slot_word(lap4, 0)) return;
        bool moved = false;
        for (int it = 0; !moved; ++it) {
            const unsigned st = (unsigned)(w >> 32);
            if (st == lap4) {                 // free for this lap: publish b
                const unsigned long long prev = atomicCAS(slot, w, slot_word(lap4 + 1, b));
                if (prev == w) return;
                w = prev;                     // the ticket holder gave it up meanwhile
                continue;
            }
            if (st == lap4 + 2) {             // given up: free it for the next lap, move on
                atomicExch(slot, slot_word(lap4 + 4, 0));
                moved = true;
                continue;
            }
            // an earlier lap's block not yet taken: wait for its consumer
            if (it > (1 << 22)) { set_abort(P, AB_PUSH); return; }
            __nanosleep(64);
            w = *(volatile unsigned long long *)slot;
        }
    }
}

// Marks block a (of the tile whose index is tb >> S_TILE_SHIFT) as needing
// (re)processing because a neighbour changed. A notified block is idle most of
// the time, so the first compare-and-swap assumes that state, and later ones
// start from the word the previous one returned.
__device__ void notify_block(const Params &P, unsigned a, unsigned tb)
{
    unsigned old = tb | S_IDLE | S_VIS;
    unsigned nw;
    for (int it = 0;; ++it) {
        if (it > (1 << 20)) { set_abort(P, AB_NOTIFY); return; }
        if (old & S_RUN) {
            if (old & S_DIRTY) return;
            nw = old | S_DIRTY;
        } else if (old & S_IDLE) {
            nw = old & ~S_IDLE;
        } else {
            return;  // already queued
        }
        unsigned prev = atomicCAS(&P.state[a], old, nw);
        if (prev == old) break;
        old = prev;
    }
    if (!(old & S_RUN)) {
        atomicAdd(&P.ctl->outstanding, 1u);
        push_hot(P, a);
    }
}

#ifndef IDLE_SLEEP_MAX_NS
#define IDLE_SLEEP_MAX_NS 4096   // longest back-off of an idle CTA between polls
#endif

// Thread 0: next block to process, or EMPTY when all work is done / aborted.
// Re-queued blocks are handed out by tickets (one atomicAdd on the ring head,
// never retried, so hundreds of CTAs asking at once do not contend in a
// compare-and-swap loop), taken only while the ring looks non-empty -- and,
// while first-visit (cold) blocks remain, only while it holds more than a few
// items. A ticket below the tail waits for its producer to publish the block.
// A ticket at or past the tail (other CTAs took the last items first) waits
// for a later push, unless cold blocks remain: then its holder gives it up
// (the slot's state for this lap goes from free to given-up, so the producer
// pushes that block again elsewhere) and takes a cold block. So a CTA never
// runs a block while it holds a ticket, and no CTA waits while cold blocks
// are left. When no block is queued or running, none can be pushed any more:
// the CTA leaves, dropping an unserved ticket.
__device__ unsigned next_item(const Params &P)
{
    constexpr unsigned long long RING_MIN = 4;   // below this, prefer cold blocks over a ticket
    Ctl *c = P.ctl;
    unsigned long long idle0 = 0;
    unsigned sleep = 32;
    for (;;) {
        if (*(volatile int *)&c->abort) return EMPTY;
        const unsigned long long h = *(volatile unsigned long long *)&c->head;
        const unsigned long long t = *(volatile unsigned long long *)&c->tail;
        const bool cold_left = *(volatile unsigned *)&c->cold < P.nblocks;
        if (h < t && (!cold_left || t - h > RING_MIN)) {
            const unsigned long long tk = atomicAdd(&c->head, 1ull);
            unsigned long long *slot = &P.ring[tk % P.ring_cap];
            const unsigned lap4 = (unsigned)(tk / P.ring_cap) * 4u;
            unsigned wait = 32;
            for (;;) {
                const unsigned long long w = *(volatile unsigned long long *)slot;
                if ((unsigned)(w >> 32) == lap4 + 1) {   // this lap's block: take it, free the slot
                    atomicExch(slot, slot_word(lap4 + 4, 0));
                    return (unsigned)w;
                }
                if (*(volatile int *)&c->abort) return EMPTY;
                if (tk < *(volatile unsigned long long *)&c->tail) {
                    __nanosleep(32);   // its producer is publishing the block
                    continue;
                }
                if ((unsigned)(w >> 32) == lap4 && *(volatile unsigned *)&c->cold < P.nblocks) {
                    // other work exists: give the ticket up (unless its block just arrived)
                    if (atomicCAS(slot, w, slot_word(lap4 + 2, 0)) == w) break;
                    continue;
                }
                if (*(volatile unsigned *)&c->outstanding == 0) return EMPTY;
                const unsigned long long now = gtimer();
                if (idle0 == 0) idle0 = now;
                else if ((long long)(now - idle0) > P.wait_ns) { set_abort(P, AB_IDLE); return EMPTY; }
                __nanosleep(wait);
                if (wait < IDLE_SLEEP_MAX_NS) wait <<= 1;
            }
        }
        if (*(volatile unsigned *)&c->cold < P.nblocks) {
            unsigned k = atomicAdd(&c->cold, 1u);
            if (k < P.nblocks) return cold_block(P, k);
        }
        if (*(volatile unsigned long long *)&c->head < *(volatile unsigned long long *)&c->tail) continue;
        if (*(volatile unsigned *)&c->outstanding == 0) return EMPTY;
        unsigned long long now = gtimer();
        if (idle0 == 0) idle0 = now;
        else if ((long long)(now - idle0) > P.wait_ns) { set_abort(P, AB_IDLE); return EMPTY; }
        __nanosleep(sleep);
        if (sleep < IDLE_SLEEP_MAX_NS) sleep <<= 1;
    }
}

// ---------------------------------------------------------------------------
// loads

__device__ __forceinline__ uint32_t ld_j_word(const uint8_t *p) { return __ldcg((const unsigned int *)p); }
__device__ __forceinline__ uint32_t ld_j_byte(const uint8_t *p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ld_i_word(const uint8_t *p) { return __ldg((const unsigned int *)p); }
__device__ __forceinline__ uint32_t ld_i_byte(const uint8_t *p) { return __ldg(p); }

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// TMA: the (BH+2) x 160-byte box of I and of J at (x0 - XOFF, y0 - 1) into
// shared memory; out-of-image pixels arrive as 0 (the border rule: absent
// neighbours act as J = 0, the identity of max). One thread issues; every
// thread waits on the CTA's mbarrier (bounded).
// Bytes of the shared-memory word holding pixels x .. x+3 that lie inside
// 0 <= x < W (the pixels of an erosion tile that get complemented).
__device__ __forceinline__ uint32_t inimage_mask(int x, int W)
{
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (x + b >= 0 && x + b < W) m |= 0xFFu << (8 * b);
    return m;
}

// Erosion tiles (the dual operation) run as dilation on complemented values:
// every loaded in-image pixel v becomes 255 - v (= ~v for a byte). Pixels
// outside the image stay 0, i.e. absent, as for dilation.
template <int BH>
__device__ void complement_box(Smem<BH> &S, const TileDesc &D, int y0, int x0)
{
    constexpr int NW = WR - WL + 1;
    for (int idx = threadIdx.x; idx < (BH + 2) * NW; idx += NT) {
        const int r = idx / NW, w = WL + (idx - r * NW);
        const int yy = y0 - 1 + r;
        if (yy < 0 || yy >= D.H) continue;
        const uint32_t m = inimage_mask(x0 + 4 * (w - W0), D.W);
        S.J[r * PW + w] ^= m;
        S.I[r * PW + w] ^= m;
    }
}

template <int BH>
__device__ void tma_load_block(Smem<BH> &S, const Params &P, const TileDesc &D, int t, int y0, int x0)
{
    const unsigned bar = smem_addr(&S.mbar);
    if (threadIdx.x == 0) {
        const char *tm = (const char *)P.tmaps + (size_t)t * 256;
        const unsigned long long mI = (unsigned long long)tm, mJ = (unsigned long long)(tm + 128);
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" :: "l"(mI) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" :: "l"(mJ) : "memory");
        // Neighbour blocks wrote J (halo rows) with generic stores and published
        // them through the block-state atomics this thread acquired; the TMA
        // reads through the async proxy, so order generic before async accesses
        // of global memory as well as of this CTA's shared memory.
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const unsigned bytes = 2u * (unsigned)(Boxes<BH>::ROWS * BOXW);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
        const int cx = x0 - XOFF, cy = y0 - 1;
        constexpr int NBOX = Boxes<BH>::N, TBOX = Boxes<BH>::TBOX;
#pragma unroll
        for (int bx = 0; bx < NBOX; ++bx) {
            const unsigned so = (unsigned)(bx * TBOX * BOXW);
            asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                         :: "r"(smem_addr(S.J) + so), "l"(mJ), "r"(cx), "r"(cy + bx * TBOX), "r"(bar) : "memory");
            asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                         :: "r"(smem_addr(S.I) + so), "l"(mI), "r"(cx), "r"(cy + bx * TBOX), "r"(bar) : "memory");
        }
    }
    const unsigned ph = S.phase;
    unsigned done = 0;
    for (long it = 0; !done; ++it) {
        asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
                     : "=r"(done) : "r"(bar), "r"(ph) : "memory");
        if (!done && it > (1l << 26)) { set_abort(P, AB_TMA); break; }
    }
    __syncthreads();
    if (threadIdx.x == 0) S.phase = ph ^ 1u;
    if (D.dual) {
        complement_box(S, D, y0, x0);
        __syncthreads();
    }
    // halo mask out of the box, then zero it in S.I
    const uint8_t *Ib = (const uint8_t *)S.I;
    constexpr int RB = PW * 4;
    for (int x = threadIdx.x - 1; x <= BW; x += NT) {
        S.hIt[x + 1] = Ib[XOFF + x];
        S.hIb[x + 1] = Ib[(BH + 1) * RB + XOFF + x];
    }
    for (int r = threadIdx.x; r < BH; r += NT) {
        S.hIl[r] = Ib[(r + 1) * RB + XOFF - 1];
        S.hIr[r] = Ib[(r + 1) * RB + XOFF + BW];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * (BH + 2) + 2 * PW; i += NT) {
        if (i < BH + 2) S.I[i * PW + WL] = 0u;
        else if (i < 2 * (BH + 2)) S.I[(i - (BH + 2)) * PW + WR] = 0u;
        else if (i < 2 * (BH + 2) + PW) S.I[i - 2 * (BH + 2)] = 0u;
        else S.I[(BH + 1) * PW + (i - 2 * (BH + 2) - PW)] = 0u;
    }
}

// Loads the block (rows y0-1 .. y0+BH, columns x0-1 .. x0+BW) into shared
// memory with plain loads (any pitch / alignment).
// halo_only: reload just the J halo ring (the interior is ours and unchanged).
template <int BH>
__device__ void load_block(Smem<BH> &S, const TileDesc &D, int y0, int x0, bool halo_only)
{
    const int H = D.H, W = D.W;
    const size_t pitch = (size_t)D.pitch;
    constexpr int NW = WR - WL + 1;   // 34 words per row: halo, 32 interior, halo
    // halo_only: the two halo rows, then the left and right halo words of rows 1..BH
    const int nitems = halo_only ? 2 * NW + 2 * BH : (BH + 2) * NW;
    for (int idx = threadIdx.x; idx < nitems; idx += NT) {
        int r, w;
        if (!halo_only) { r = idx / NW; w = WL + (idx - r * NW); }
        else if (idx < NW) { r = 0; w = WL + idx; }
        else if (idx < 2 * NW) { r = BH + 1; w = WL + (idx - NW); }
        else if (idx < 2 * NW + BH) { r = 1 + (idx - 2 * NW); w = WL; }
        else { r = 1 + (idx - 2 * NW - BH); w = WR; }
        const bool hrow = (r == 0 || r == BH + 1), hword = (w == WL || w == WR);
        const int yy = y0 - 1 + r;
        uint32_t jv = 0, iv = 0, loaded = 0;   // loaded: the bytes read from the image
        const bool rowin = (yy >= 0 && yy < H);
        if (w == WL) {
            const int x = x0 - 1;
            if (rowin && x >= 0) {
                jv = ld_j_byte(D.J + yy * pitch + x) << 24;
                if (!halo_only) iv = ld_i_byte(D.I + yy * pitch + x) << 24;
                loaded = 0xFF000000u;
            }
        } else if (w == WR) {
            const int x = x0 + BW;
            if (rowin && x < W) {
                jv = ld_j_byte(D.J + yy * pitch + x);
                if (!halo_only) iv = ld_i_byte(D.I + yy * pitch + x);
                loaded = 0xFFu;
            }
        } else if (rowin) {
            const int x = x0 + 4 * (w - W0);
            loaded = inimage_mask(x, W);
            if (D.fast && x + 3 < W) {
                jv = ld_j_word(D.J + yy * pitch + x);
                if (!halo_only) iv = ld_i_word(D.I + yy * pitch + x);
            } else {
                for (int b = 0; b < 4; ++b)
                    if (x + b < W) {
                        jv |= ld_j_byte(D.J + yy * pitch + x + b) << (8 * b);
                        if (!halo_only) iv |= ld_i_byte(D.I + yy * pitch + x + b) << (8 * b);
                    }
            }
        }
        if (D.dual) { jv ^= loaded; iv ^= loaded; }   // erosion: complemented values
        S.J[r * PW + w] = jv;
        if (halo_only) continue;
        S.I[r * PW + w] = (hrow || hword) ? 0u : iv;
        if (hrow) {
            uint8_t *h = (r == 0) ? S.hIt : S.hIb;
            if (w == WL) h[0] = (uint8_t)(iv >> 24);
            else if (w == WR) h[BW + 1] = (uint8_t)iv;
            else for (int b = 0; b < 4; ++b) h[4 * (w - W0) + b + 1] = (uint8_t)(iv >> (8 * b));
        } else if (w == WL) {
            S.hIl[r - 1] = (uint8_t)(iv >> 24);
        } else if (w == WR) {
            S.hIr[r - 1] = (uint8_t)iv;
        }
    }
}

template <int BH>
__device__ __forceinline__ uint8_t jbyte(const Smem<BH> &S, int r, int x)  // x in -1 .. BW
{
    return ((const volatile uint8_t *)S.J)[r * PW * 4 + XOFF + x];
}

template <int BH>
__device__ void save_edges(Smem<BH> &S)
{
    for (int i = threadIdx.x; i < BW; i += NT) {
        S.eT[i] = jbyte(S, 1, i);
        S.eB[i] = jbyte(S, BH, i);
    }
    for (int i = threadIdx.x; i < BH; i += NT) {
        S.eL[i] = jbyte(S, i + 1, 0);
        S.eR[i] = jbyte(S, i + 1, BW - 1);
    }
}

// ---------------------------------------------------------------------------
// scans: one warp over rows [r0, r1) of the block (shared-memory row indices)


// Two-plane byte arithmetic. A shared-memory word holds pixels x..x+3 in
// bytes 0..3; the scans work on its even plane E (pixels x, x+2 as two u16
// lanes) and odd plane O (pixels x+1, x+3), where max / min are native u16x2
// instructions (the byte-wise __vmaxu4 / __vminu4 are emulated).
__device__ __forceinline__ uint32_t pmax(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t pmin(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t even_plane(uint32_t w) { return __byte_perm(w, 0u, 0x4240); }
__device__ __forceinline__ uint32_t odd_plane(uint32_t w) { return __byte_perm(w, 0u, 0x4341); }
__device__ __forceinline__ uint32_t merge_planes(uint32_t e, uint32_t o) { return __byte_perm(e, o, 0x6240); }
// clamp-map composition f o g on both u16 lanes, f = (fA, fC), g = (gA, gC)
__device__ __forceinline__ void pcompose(uint32_t fA, uint32_t fC, uint32_t gA, uint32_t gC, uint32_t &A, uint32_t &C)
{
    A = pmin(fC, pmax(fA, gA));
    C = pmin(fC, pmax(fA, gC));
}

// A clamp map v -> min(C, max(A, v)) packed as A | C << 16 (one per lane of a
// row); g o f on such packed maps is two byte broadcasts and two u16x2 ops.
__device__ __forceinline__ uint32_t map_pack(uint32_t A, uint32_t C) { return A | (C << 16); }
__device__ __forceinline__ uint32_t compose(uint32_t g, uint32_t f)
{
    const uint32_t A2 = __byte_perm(g, 0u, 0x4040), C2 = __byte_perm(g, 0u, 0x4242);
    return pmin(C2, pmax(A2, f));
}

// Row recurrence of the scans. The previous row's result stays in registers
// (the neighbouring lanes' planes arrive by shuffle, the halo words by a
// broadcast load), and the next row's mask and marker words are loaded while
// the current row is computed. Changed rows and pixels are counted per lane and
// reduced over the warp once per group of 32 rows, so no row waits on a warp
// reduction before the next one starts.
template <int CONN, bool DOWN>
__device__ __forceinline__ unsigned scan_rows(uint32_t *SJ, const uint32_t *SI, unsigned *rowmask,
                                              unsigned *pairmask, int r0, int r1)
{
    const int lane = threadIdx.x & 31, w = lane + W0;
    const int step = DOWN ? 1 : -1;
    const int yb = DOWN ? r0 : r1 - 1, ye = DOWN ? r1 : r0 - 1;
    constexpr uint32_t ID_C = 0x00FF00FFu;    // identity map: A = 0, C = 255 (both lanes)
    unsigned any = 0, rbits = 0;   // this lane's changed pixels; rows it changed in the current group
    __syncwarp();
    const uint32_t pw0 = SJ[(yb - step) * PW + w];
    uint32_t pE = even_plane(pw0), pO = odd_plane(pw0);
    uint32_t j = SJ[yb * PW + w], i = SI[yb * PW + w];
    for (int y = yb; y != ye; y += step) {
        const int yn = y + step;
        uint32_t jn = 0, in = 0;
        if (yn != ye) {
            jn = SJ[yn * PW + w];
            in = SI[yn * PW + w];
        }
        uint32_t vE = pE, vO = pO;
        if (CONN == 8) {
            const int yp = y - step;
            uint32_t oW = __shfl_up_sync(FULL, pO, 1);     // odd plane of the word to the left
            uint32_t eE = __shfl_down_sync(FULL, pE, 1);   // even plane of the word to the right
            if (lane == 0) oW = odd_plane(SJ[yp * PW + WL]);
            if (lane == 31) eE = even_plane(SJ[yp * PW + WR]);
            const uint32_t westE = __funnelshift_l(oW, pO, 16);   // pixels x-1, x+1 of the even pixels
            const uint32_t eastO = __funnelshift_r(pE, eE, 16);   // pixels x+2, x+4 of the odd pixels
            vE = __vimax3_u16x2(pE, westE, pO);
            vO = __vimax3_u16x2(pO, pE, eastO);
        }
        const uint32_t jE = even_plane(j), jO = odd_plane(j), iE = even_plane(i), iO = odd_plane(i);
        const uint32_t aE = pmin(iE, pmax(jE, vE)), aO = pmin(iO, pmax(jO, vO));
        uint32_t AE, CE, AO, CO;   // prefix clamp maps of every pixel inside the word
        uint32_t m;
        if (DOWN) {   // left to right: pixel order E.l0, O.l0, E.l1, O.l1
            uint32_t A1O, C1O, A1E, C1E;
            pcompose(aO, iO, aE, iE, A1O, C1O);                          // x+1 o x, x+3 o x+2
            pcompose(aE, iE, aO << 16, (iO << 16) | 0x00FFu, A1E, C1E);   // x o id, x+2 o x+1
            pcompose(A1E, C1E, A1E << 16, (C1E << 16) | 0x00FFu, AE, CE);
            pcompose(A1O, C1O, A1O << 16, (C1O << 16) | 0x00FFu, AO, CO);
            m = (AO >> 16) | (CO & 0xFFFF0000u);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(FULL, m, d);
                if (lane >= d) m = compose(m, o);
            }
        } else {      // right to left: pixel order O.l1, E.l1, O.l0, E.l0
            uint32_t A1E, C1E, A1O, C1O;
            pcompose(aE, iE, aO, iO, A1E, C1E);                               // x o x+1, x+2 o x+3
            pcompose(aO, iO, aE >> 16, (iE >> 16) | 0x00FF0000u, A1O, C1O);    // x+1 o x+2, x+3 o id
            pcompose(A1E, C1E, A1E >> 16, (C1E >> 16) | 0x00FF0000u, AE, CE);
            pcompose(A1O, C1O, A1O >> 16, (C1O >> 16) | 0x00FF0000u, AO, CO);
            m = (AE & 0xFFFFu) | (CE << 16);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_down_sync(FULL, m, d);
                if (lane + d < 32) m = compose(m, o);
            }
        }
        (void)ID_C;
        uint32_t ex = DOWN ? __shfl_up_sync(FULL, m, 1) : __shfl_down_sync(FULL, m, 1);
        if (lane == (DOWN ? 0 : 31)) ex = map_pack(0, 255);
        // the row's halo pixel on the side the scan starts from (x = -1 or x = BW)
        const uint32_t h = DOWN ? (SJ[y * PW + WL] >> 24) : (SJ[y * PW + WR] & 0xFF);
        const uint32_t vin = min(ex >> 16, max(ex & 0xFFFFu, h)) * 0x00010001u;
        const uint32_t rE = pmin(CE, pmax(AE, vin)), rO = pmin(CO, pmax(AO, vin));
        const uint32_t dE = rE ^ jE, dO = rO ^ jO;
        const unsigned nd = ((dE & 0xFFFFu) != 0) + ((dE >> 16) != 0) + ((dO & 0xFFFFu) != 0) + ((dO >> 16) != 0);
        if (nd) SJ[y * PW + w] = merge_planes(rE, rO);
        any += nd;
        rbits |= (nd ? 1u : 0u) << ((y - 1) & 31);
        if (((DOWN ? y : y - 1) & 31) == 0 || yn == ye) {   // leaving a group of 32 rows (0-based y - 1)
            const unsigned g = __reduce_or_sync(FULL, rbits);
            if (lane == 0 && g) {
                atomicOr(&rowmask[(y - 1) >> 5], g);
                atomicOr(&pairmask[(y - 1) >> 5], g);
            }
            rbits = 0;
        }
        pE = rE;
        pO = rO;
        j = jn;
        i = in;
    }
    return __reduce_add_sync(FULL, any);   // pixels changed (warp-uniform)
}

template <int BH, int CONN>
__device__ unsigned raster_rows(Smem<BH> &S, int r0, int r1)
{
    return scan_rows<CONN, true>(S.J, S.I, S.rowmask, S.pairmask, r0, r1);
}

template <int BH, int CONN>
__device__ unsigned antiraster_rows(Smem<BH> &S, int r0, int r1)
{
    return scan_rows<CONN, false>(S.J, S.I, S.rowmask, S.pairmask, r0, r1);
}

// One raster + anti-raster pair over the whole block; `bands` warps each take a
// horizontal band of rows. Returns (block-uniformly) whether any pixel changed.
template <int BH, int CONN>
__device__ unsigned scan_pair(Smem<BH> &S, int bands, unsigned long long &rows)
{
    // returns the number of pixels the pair changed (block-uniform)
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) S.flag = 0;
    for (int i = threadIdx.x; i < BH / 32; i += NT) S.pairmask[i] = 0;
    __syncthreads();
    unsigned ch = 0;
    if (warp < bands) {
        const int r0 = 1 + warp * BH / bands, r1 = 1 + (warp + 1) * BH / bands;
        ch = raster_rows<BH, CONN>(S, r0, r1);
        ch += antiraster_rows<BH, CONN>(S, r0, r1);
    }
    if (ch && (threadIdx.x & 31) == 0) atomicAdd(&S.flag, ch);
    rows += 2 * BH;
    __syncthreads();
    const unsigned n = S.flag;
    __syncthreads();  // everyone has read the count before it is reset again
    return n;
}

// ---------------------------------------------------------------------------
// queue phase

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int BH>
__device__ __forceinline__ void put_entry(Smem<BH> &S, uint16_t *gsp, int lvl, unsigned slot, uint16_t v)
{
    if (!RK_CHECK(v >= (unsigned)(PW * 4) && v < (unsigned)((BH + 1) * PW * 4) &&
                  (unsigned)(v % (PW * 4) - XOFF) < (unsigned)BW, 3))
        return;
    if (slot < (unsigned)QCAP) S.q[lvl][slot] = v;
    else if (slot - QCAP < (unsigned)GCAP) gsp[lvl * GCAP + (slot - QCAP)] = v;
    else S.overflow = 1;
}

template <int BH>
__device__ __forceinline__ uint16_t get_entry(const Smem<BH> &S, const uint16_t *gsp, int lvl, unsigned i)
{
    if (!RK_CHECK(i < (unsigned)(QCAP + GCAP), 1)) return (uint16_t)(PW * 4 + XOFF);
    return i < (unsigned)QCAP ? S.q[lvl][i] : gsp[lvl * GCAP + (i - QCAP)];
}

// warp-aggregated append of pixel offset v (when pred) to level lvl
template <int BH>
__device__ __forceinline__ void warp_push(Smem<BH> &S, uint16_t *gsp, int lvl, bool pred, uint16_t v)
{
    const unsigned bal = __ballot_sync(FULL, pred);
    if (!bal) return;
    const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&S.cq[lvl], (unsigned)__popc(bal));
    base = __shfl_sync(FULL, base, leader);
    if (pred) put_entry(S, gsp, lvl, base + __popc(bal & lanemask_lt()), v);
}

// Seeding pass: J(p) <- max(J(p), min(I(p), max over N(p) of J)) in place;
// every raised pixel joins level 0. Returns the level's size.
template <int BH, int CONN>
__device__ unsigned seed_pass(Smem<BH> &S, uint16_t *gsp, const unsigned *filter = nullptr)
{
    // filter (optional): visit only rows within one row of a row set in it.
    // After a scan pair every pixel has taken all eight directions into
    // account, so only pixels next to a pixel that pair changed can still be
    // raised: filter = the pair's changed rows.
    unsigned rm[BH / 32];
#pragma unroll
    for (int i = 0; i < BH / 32; ++i) rm[i] = filter ? filter[i] : 0u;
    __syncthreads();
    if (threadIdx.x == 0) { S.cq[0] = 0; S.cq[1] = 0; S.cq[2] = 0; S.overflow = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = lane + W0;
    for (int y = 1 + (threadIdx.x >> 5); y <= BH; y += NT / 32) {
        if (filter) {
            bool act = false;
#pragma unroll
            for (int d = -1; d <= 1; ++d) {
                const int r = y - 1 + d;   // 0-based block row
                if (r >= 0 && r < BH && ((rm[r >> 5] >> (r & 31)) & 1u)) act = true;
            }
            if (!act) continue;
        }
        // one geodesic dilation step in the two-plane form (see scan_rows)
        const uint32_t *rw = &S.J[y * PW];
        const uint32_t c = rw[w];
        const uint32_t cE = even_plane(c), cO = odd_plane(c);
        // maxima over pixels x-1, x, x+1 of one row, for the even and the odd pixels
        auto hmax = [](const uint32_t *row, int ww, uint32_t &hE, uint32_t &hO) {
            const uint32_t v = row[ww], vE = even_plane(v), vO = odd_plane(v);
            hE = __vimax3_u16x2(vE, __funnelshift_l(odd_plane(row[ww - 1]), vO, 16), vO);
            hO = __vimax3_u16x2(vO, vE, __funnelshift_r(vE, even_plane(row[ww + 1]), 16));
        };
        uint32_t mE, mO;
        hmax(rw, w, mE, mO);
        const uint32_t *up = rw - PW, *dn = rw + PW;
        if (CONN == 8) {
            uint32_t uE, uO, dE, dO;
            hmax(up, w, uE, uO);
            hmax(dn, w, dE, dO);
            mE = __vimax3_u16x2(mE, uE, dE);
            mO = __vimax3_u16x2(mO, uO, dO);
        } else {
            const uint32_t u = up[w], d = dn[w];
            mE = __vimax3_u16x2(mE, even_plane(u), even_plane(d));
            mO = __vimax3_u16x2(mO, odd_plane(u), odd_plane(d));
        }
        const uint32_t iw = S.I[y * PW + w];
        const uint32_t nv = merge_planes(pmin(even_plane(iw), mE), pmin(odd_plane(iw), mO));
        const uint32_t diff = nv ^ c;
        if (diff) S.J[y * PW + w] = nv;
        if (__any_sync(FULL, diff != 0) && lane == 0)
            atomicOr(&S.rowmask[(y - 1) >> 5], 1u << ((y - 1) & 31));
        {   // the row's raised pixels join level 0: one slot reservation per warp and row
            const unsigned lt = lanemask_lt();
            unsigned off[4], tot = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const unsigned bk = __ballot_sync(FULL, ((diff >> (8 * b)) & 0xFFu) != 0);
                off[b] = tot + __popc(bk & lt);
                tot += __popc(bk);
            }
            if (tot) {
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(&S.cq[0], tot);
                base = __shfl_sync(FULL, base, 0);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if ((diff >> (8 * b)) & 0xFFu) put_entry(S, gsp, 0, base + off[b], (uint16_t)((y * PW + w) * 4 + b));
            }
        }
    }
    __syncthreads();
    return S.cq[0];
}


// Seeding of a block that was already at its fixed point for its previous
// halo (a revisit): its interior is unchanged since, so only the pixels next to
// the halo (the block's 1-pixel frame) can be raised. Each frame pixel takes
// one geodesic dilation step; the raised ones form level 0.
template <int BH, int CONN>
__device__ unsigned seed_frame(Smem<BH> &S, uint16_t *gsp)
{
    constexpr int RB = PW * 4;
    constexpr int NFR = 2 * BW + 2 * (BH - 2);
    if (threadIdx.x == 0) { S.cq[0] = 0; S.cq[1] = 0; S.cq[2] = 0; S.overflow = 0; }
    __syncthreads();
    const volatile uint8_t *Jb = (const volatile uint8_t *)S.J;
    const uint8_t *Ib = (const uint8_t *)S.I;
    for (int base = 0; base < NFR; base += NT) {
        const int i = base + threadIdx.x;
        const bool act = i < NFR;
        int r = 1, x = 0;
        if (i < BW) { r = 1; x = i; }
        else if (i < 2 * BW) { r = BH; x = i - BW; }
        else if (i < 2 * BW + (BH - 2)) { r = 2 + (i - 2 * BW); x = 0; }
        else { r = 2 + (i - 2 * BW - (BH - 2)); x = BW - 1; }
        const unsigned p = (unsigned)(r * RB + XOFF + x);
        bool raised = false;
        if (act) {
            uint32_t m = Jb[p - RB];
            m = max(m, (uint32_t)Jb[p + RB]);
            m = max(m, (uint32_t)Jb[p - 1]);
            m = max(m, (uint32_t)Jb[p + 1]);
            if (CONN == 8) {
                m = max(m, (uint32_t)Jb[p - RB - 1]);
                m = max(m, (uint32_t)Jb[p - RB + 1]);
                m = max(m, (uint32_t)Jb[p + RB - 1]);
                m = max(m, (uint32_t)Jb[p + RB + 1]);
            }
            const uint32_t nv = min(m, (uint32_t)Ib[p]);
            if (nv > Jb[p]) {   // one writer per frame pixel
                ((volatile uint8_t *)S.J)[p] = (uint8_t)nv;
                raised = true;
                atomicOr(&S.rowmask[(r - 1) >> 5], 1u << ((r - 1) & 31));
            }
        }
        warp_push(S, gsp, 0, raised, (uint16_t)p);
    }
    __syncthreads();
    return S.cq[0];
}



// Neighbour k of a pixel, as (row, column) steps: 8-connectivity NW, N, NE,
// W, E, SW, S, SE; 4-connectivity N, W, E, S.
template <int CONN>
__device__ __forceinline__ constexpr int nb_dy(int k)
{
    return CONN == 8 ? (k < 3 ? -1 : (k < 5 ? 0 : 1)) : (k == 0 ? -1 : (k == 3 ? 1 : 0));
}
template <int CONN>
__device__ __forceinline__ constexpr int nb_dx(int k)
{
    return CONN == 8 ? (k == 0 || k == 3 || k == 5 ? -1 : (k == 2 || k == 4 || k == 7 ? 1 : 0))
                     : (k == 1 ? -1 : (k == 2 ? 1 : 0));
}
// byte offset of neighbour k in the shared-memory J / I rows
template <int CONN>
__device__ __forceinline__ constexpr int nb_off(int k)
{
    return nb_dy<CONN>(k) * (PW * 4) + nb_dx<CONN>(k);
}

__device__ __forceinline__ uint32_t max3u(uint32_t a, uint32_t b, uint32_t c) { return __vimax3_u32(a, b, c); }

// One pop of Algorithm 1's propagation phase, for frontier pixel p (a
// shared-memory byte offset; act = false for an idle thread). Its neighbours q
// that satisfy the propagation condition J(q) < min(J(p), I(q)) are
// candidates. A candidate is updated by the one thread that claims it in this
// level's ownership bitmap `claim` (an atomic OR, never retried); the owner
// sets J(q) <- min(I(q), max over N(q) of J) -- one geodesic dilation step at
// q (Table II) -- with a plain byte store. With one writer per pixel and level
// and J only ever raised, no atomics touch J. An offer whose claim fails is
// not lost: the owner's maximum includes J(p), written before the barrier
// that opened this level, and a neighbour raised during the level is itself in
// the next frontier and offers its value again.
// The maxima of all directions come from a 5 x 5 window of J around p held in
// registers: the 3 x 3 centre is read for the propagation test, the outer
// ring when p has a candidate. Returns the raised neighbours
// (bit k) with their new values in nv[k]; `own` gets the candidates this
// thread claimed, and `gm` the groups of BH / 32 block rows it changed.
template <int BH, int CONN>
__device__ __forceinline__ unsigned expand(Smem<BH> &S, unsigned *claim, unsigned p, bool act,
                                           uint32_t (&nv)[CONN], unsigned &own, unsigned &gm)
{
    constexpr int RB = PW * 4;
    const volatile uint8_t *Jb = (const volatile uint8_t *)S.J;
    volatile uint8_t *Jm = (volatile uint8_t *)S.J;
    const uint8_t *Ib = (const uint8_t *)S.I;
    own = 0;
#ifdef RECON_CHECKS
    // an interior pixel of the block: rows 1 .. BH of J, columns XOFF .. XOFF + BW - 1
    if (act && !RK_CHECK(p >= (unsigned)RB && p < (unsigned)((BH + 1) * RB) && (unsigned)(p % RB - XOFF) < (unsigned)BW,
                         2)) {
        act = false;
        p = RB + XOFF;
    }
#endif
    if (!act) return 0;
    const uint32_t v = Jb[p];
    uint32_t iq[CONN], jq[CONN];
    unsigned cand = 0;
#pragma unroll
    for (int k = 0; k < CONN; ++k) {
        iq[k] = Ib[p + nb_off<CONN>(k)];
        jq[k] = Jb[p + nb_off<CONN>(k)];
        cand |= (jq[k] < min(v, iq[k]) ? 1u : 0u) << k;
    }
    if (!cand) return 0;
    // claims: every candidate is interior (a halo pixel's mask is 0 in S.I)
    const int r = (int)(p / (unsigned)RB), x = (int)p - r * RB - XOFF;   // row 1..BH, column 0..BW-1
    const int pb = (r - 1) * BW + x;
    unsigned old[CONN];
#pragma unroll
    for (int k = 0; k < CONN; ++k) {
        const int qb = pb + nb_dy<CONN>(k) * BW + nb_dx<CONN>(k);
        old[k] = ((cand >> k) & 1u) ? atomicOr(&claim[qb >> 5], 1u << (qb & 31)) : ~0u;
    }
    // outer ring of the 5 x 5 window, read while the claims are in flight;
    // rows p - 2 and p + 2 exist only for rows 2 .. BH - 1 (elsewhere they are
    // needed only for halo pixels, which are never owned, so a valid row is
    // read in their place)
    const unsigned um = r >= 2 ? p - 2 * RB : p - RB, dm = r <= BH - 1 ? p + 2 * RB : p + RB;
    uint32_t M[CONN];
    if (CONN == 8) {
        // w[a][b] = J(p + (a - 2) rows + (b - 2) columns)
        uint32_t w[5][5];
        w[0][0] = Jb[um - 2]; w[0][1] = Jb[um - 1]; w[0][2] = Jb[um]; w[0][3] = Jb[um + 1]; w[0][4] = Jb[um + 2];
        w[4][0] = Jb[dm - 2]; w[4][1] = Jb[dm - 1]; w[4][2] = Jb[dm]; w[4][3] = Jb[dm + 1]; w[4][4] = Jb[dm + 2];
        w[1][0] = Jb[p - RB - 2]; w[2][0] = Jb[p - 2]; w[3][0] = Jb[p + RB - 2];
        w[1][4] = Jb[p - RB + 2]; w[2][4] = Jb[p + 2]; w[3][4] = Jb[p + RB + 2];
        w[1][1] = jq[0]; w[1][2] = jq[1]; w[1][3] = jq[2];
        w[2][1] = jq[3]; w[2][2] = v;     w[2][3] = jq[4];
        w[3][1] = jq[5]; w[3][2] = jq[6]; w[3][3] = jq[7];
        uint32_t h[5][3];   // h[a][c] = max over columns c .. c + 2 of row a
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[a][c] = max3u(w[a][c], w[a][c + 1], w[a][c + 2]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int a = nb_dy<8>(k) + 1, c = nb_dx<8>(k) + 1;   // top-left of q's 3 x 3 in the window
            M[k] = max3u(h[a][c], h[a + 1][c], h[a + 2][c]);
        }
    } else {
        const uint32_t nw = Jb[p - RB - 1], ne = Jb[p - RB + 1], sw = Jb[p + RB - 1], se = Jb[p + RB + 1];
        const uint32_t n2 = Jb[um], s2 = Jb[dm], w2 = Jb[p - 2], e2 = Jb[p + 2];
        M[0] = max(max3u(n2, nw, ne), v);   // N(q) of q = N: its N, W, E and p
        M[1] = max(max3u(w2, nw, sw), v);   // q = W
        M[2] = max(max3u(e2, ne, se), v);   // q = E
        M[3] = max(max3u(s2, sw, se), v);   // q = S
    }
#pragma unroll
    for (int k = 0; k < CONN; ++k) {
        const int qb = pb + nb_dy<CONN>(k) * BW + nb_dx<CONN>(k);
        own |= ((old[k] >> (qb & 31)) & 1u) ? 0u : (1u << k);
    }
    unsigned raised = 0;
#pragma unroll
    for (int k = 0; k < CONN; ++k) {
        nv[k] = min(iq[k], M[k]);
        // jq[k] is current: q has one writer per level, and it is this thread
        if (((own >> k) & 1u) && nv[k] > jq[k]) {
            Jm[p + nb_off<CONN>(k)] = (uint8_t)nv[k];
            raised |= 1u << k;
        }
    }
    if (raised) {   // groups of BH / 32 rows changed (0-based rows r - 2, r - 1, r), kept in a register
        const unsigned up = CONN == 8 ? (raised & 0x07u) : (raised & 0x1u);
        const unsigned mid = CONN == 8 ? (raised & 0x18u) : (raised & 0x6u);
        const unsigned dn = CONN == 8 ? (raised & 0xE0u) : (raised & 0x8u);
        constexpr int GSH = BH == 32 ? 0 : (BH == 64 ? 1 : (BH == 128 ? 2 : 3));   // log2 rows per group
        if (up) gm |= 1u << (max(r - 2, 0) >> GSH);
        if (mid) gm |= 1u << ((r - 1) >> GSH);
        if (dn) gm |= 1u << (min(r, BH - 1) >> GSH);
    }
    return raised;
}


// Processes the wavefront level by level until it is empty (Algorithm 1's
// propagation phase). Level L reads queue L % 2 and appends to (L + 1) % 2;
// its size is counted in cq[(L + 1) % 3], and cq[(L + 2) % 3] is reset during
// level L, so one barrier per level suffices. Level L claims pixels in bitmap
// claim[L % 2]; the other bitmap, last used by level L - 1, is cleared during
// level L for level L + 1. n0 = size of level 0 (counted in cq[0]; the seeding
// pass zeroed cq[1], cq[2]). Returns entries processed; the row groups the
// levels changed are added to rowmask (whole groups: a write-back of a
// group's unchanged rows stores the values they already hold).
constexpr unsigned SOLO_MAX = 32;   // levels this small run in warp 0 alone

template <int BH, int CONN>
__device__ unsigned long long run_queue(Smem<BH> &S, const Params &P, uint16_t *gsp, unsigned n0,
                                        unsigned long long &nlevels)
{
    constexpr unsigned MAX_LEVELS = 1u << 21;
    constexpr int NCW = BH * BW / 32;   // claim words per bitmap
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long pops = 0;
    unsigned gm = 0;   // groups of BH / 32 rows this thread changed
    for (int i = threadIdx.x; i < 2 * NCW; i += NT) (&S.claim[0][0])[i] = 0u;
    __syncthreads();
    unsigned n = n0;
    int src = 0, ccur = 0;   // queue buffer and level-size counter of the current level
    for (unsigned L = 0; n > 0; ++L) {
        if (L > MAX_LEVELS) {
            if (threadIdx.x == 0) set_abort(P, AB_LEVELS);
            break;
        }
        if (n <= SOLO_MAX) {
            // Thin wavefront: warp 0 runs the levels alone, one pixel per
            // lane, with __syncwarp as the level barrier, while the other
            // warps wait at one CTA barrier. The levels alternate between the
            // two claim bitmaps as between the queue buffers; during a level
            // each lane zeroes the bitmap words that its claims of the level
            // before set (every set bit has an owner, so whole words can go),
            // so one __syncwarp per level suffices. Slots of the next level
            // come from ballots. When a level outgrows the warp, the CTA
            // takes it over.
            if (warp == 0) {
                for (int i = lane; i < NCW; i += 32) S.claim[src ^ 1][i] = 0u;
                __syncwarp();
                unsigned m = n;
                int s = src;
                unsigned pprev = 0, oprev = 0;   // this lane's pixel and owned candidates in the level before
                while (m > 0 && m <= SOLO_MAX) {
                    if (++L > MAX_LEVELS) {
                        if (lane == 0) set_abort(P, AB_LEVELS);
                        m = 0;
                        break;
                    }
                    pops += m;
                    ++nlevels;
                    if (oprev) {   // zero the bitmap words its claims of the level before set
                        constexpr int RB = PW * 4;
                        unsigned *cprev = S.claim[s ^ 1];
                        const int r = (int)(pprev / (unsigned)RB), x = (int)pprev - r * RB - XOFF;
                        const int pb = (r - 1) * BW + x;
#pragma unroll
                        for (int k = 0; k < CONN; ++k)
                            if ((oprev >> k) & 1u) cprev[(pb + nb_dy<CONN>(k) * BW + nb_dx<CONN>(k)) >> 5] = 0u;
                    }
                    const bool act = (unsigned)lane < m;
                    const unsigned p = act ? get_entry(S, gsp, s, lane) : 0u;
                    uint32_t nv[CONN];
                    unsigned own;
                    const unsigned raised = expand<BH, CONN>(S, S.claim[s], p, act, nv, own, gm);
                    const unsigned lt = lanemask_lt();
                    unsigned tot = 0;
#pragma unroll
                    for (int k = 0; k < CONN; ++k) {
                        const unsigned bk = __ballot_sync(FULL, (raised >> k) & 1u);
                        if ((raised >> k) & 1u) put_entry(S, gsp, s ^ 1, tot + __popc(bk & lt), (uint16_t)(p + nb_off<CONN>(k)));
                        tot += __popc(bk);
                    }
                    __syncwarp();
                    pprev = p;
                    oprev = own;
                    m = tot;
                    s ^= 1;
                }
                if (lane == 0) {
                    S.cq[0] = m;
                    S.cq[1] = 0;
                    S.cq[2] = 0;
                    S.solo_src = (unsigned)s;
                    S.solo_L = L;
                }
            }
            __syncthreads();
            n = S.cq[0];
            src = (int)S.solo_src;
            ccur = 0;
            L = S.solo_L;   // the same in every thread
            continue;
        }
        const unsigned navail = min(n, (unsigned)(QCAP + GCAP));
        pops += navail;
        ++nlevels;
        const int dst = src ^ 1;
        const int cnext = ccur == 2 ? 0 : ccur + 1, cfree = cnext == 2 ? 0 : cnext + 1;
        if (threadIdx.x == 0) S.cq[cfree] = 0;   // last read two barriers ago
        for (int i = threadIdx.x; i < NCW; i += NT) S.claim[dst][i] = 0u;   // for level L + 1
        unsigned *claim = S.claim[src];
        for (unsigned base = 0; base < navail; base += NT) {
            const unsigned i = base + threadIdx.x;
            const bool act = i < navail;
            const unsigned p = act ? get_entry(S, gsp, src, i) : 0u;
            uint32_t nv[CONN];
            unsigned own;
            const unsigned raised = expand<BH, CONN>(S, claim, p, act, nv, own, gm);
            if (raised) {
                unsigned slot = atomicAdd(&S.cq[cnext], (unsigned)__popc(raised));
#pragma unroll
                for (int k = 0; k < CONN; ++k)
                    if ((raised >> k) & 1u) put_entry(S, gsp, dst, slot++, (uint16_t)(p + nb_off<CONN>(k)));
            }
        }
        __syncthreads();
        n = S.cq[cnext];
        src = dst;
        ccur = cnext;
    }
    {   // rows of the changed groups, for the write-back
        constexpr int GS = BH / 32;
        const unsigned g = __reduce_or_sync(FULL, gm);
        if ((g >> lane) & 1u) atomicOr(&S.rowmask[(lane * GS) >> 5], ((1u << GS) - 1u) << ((lane * GS) & 31));
    }
    return pops;
}

// ---------------------------------------------------------------------------

template <int BH>
__device__ void write_back(Smem<BH> &S, const TileDesc &D, int y0, int x0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t pitch = (size_t)D.pitch;
    for (int r = warp; r < BH; r += NT / 32) {
        if (!((S.rowmask[r >> 5] >> (r & 31)) & 1u)) continue;
        const int yy = y0 + r;
        if (yy >= D.H) break;
        const int x = x0 + 4 * lane;
        const uint32_t v = S.J[(r + 1) * PW + lane + W0] ^ (D.dual ? 0xFFFFFFFFu : 0u);
        uint8_t *dst = D.J + yy * pitch + x;
        if (D.fast && x + 3 < D.W) {
            *(uint32_t *)dst = v;
        } else {
            for (int b = 0; b < 4; ++b)
                if (x + b < D.W) dst[b] = (uint8_t)(v >> (8 * b));
        }
    }
}

// direction bits for neighbour notification
enum { DN = 1, DS = 2, DW = 4, DE = 8, DNW = 16, DNE = 32, DSW = 64, DSE = 128 };

template <int BH, int CONN>
__device__ void edge_notify_bits(Smem<BH> &S)
{
    unsigned bits = 0;
    for (int x = threadIdx.x; x < BW; x += NT) {
        const uint32_t vt = jbyte(S, 1, x), vb = jbyte(S, BH, x);
        for (int dx = (CONN == 8 ? -1 : 0); dx <= (CONN == 8 ? 1 : 0); ++dx) {
            const int qx = x + dx;
            const unsigned dirN = qx < 0 ? DNW : (qx >= BW ? DNE : DN);
            const unsigned dirS = qx < 0 ? DSW : (qx >= BW ? DSE : DS);
            if (vt != S.eT[x] && jbyte(S, 0, qx) < min(vt, (uint32_t)S.hIt[qx + 1])) bits |= dirN;
            if (vb != S.eB[x] && jbyte(S, BH + 1, qx) < min(vb, (uint32_t)S.hIb[qx + 1])) bits |= dirS;
        }
    }
    for (int r = 1 + threadIdx.x; r <= BH; r += NT) {
        const uint32_t vl = jbyte(S, r, 0), vr = jbyte(S, r, BW - 1);
        for (int dy = (CONN == 8 ? -1 : 0); dy <= (CONN == 8 ? 1 : 0); ++dy) {
            const int qr = r + dy;
            const uint32_t il = qr == 0 ? S.hIt[0] : (qr == BH + 1 ? S.hIb[0] : S.hIl[qr - 1]);
            const uint32_t ir = qr == 0 ? S.hIt[BW + 1] : (qr == BH + 1 ? S.hIb[BW + 1] : S.hIr[qr - 1]);
            const unsigned dirW = qr == 0 ? DNW : (qr == BH + 1 ? DSW : DW);
            const unsigned dirE = qr == 0 ? DNE : (qr == BH + 1 ? DSE : DE);
            if (vl != S.eL[r - 1] && jbyte(S, qr, -1) < min(vl, il)) bits |= dirW;
            if (vr != S.eR[r - 1] && jbyte(S, qr, BW) < min(vr, ir)) bits |= dirE;
        }
    }
    if (bits) atomicOr(&S.notify, bits);
}

// Phase clock of thread 0: adds the time since the last tick to wk.phase_ns[ph].
struct PhaseClock {
    unsigned long long last;
    __device__ __forceinline__ void tick(Work &wk, int ph)
    {
        if (threadIdx.x == 0) {
            const unsigned long long now = gtimer();
            wk.phase_ns[ph] += now - last;
            last = now;
        }
    }
};

// Block-uniform read of the abort word.
template <int BH>
__device__ bool block_aborted(Smem<BH> &S, const Params &P)
{
    if (threadIdx.x == 0) S.abrt = (unsigned)*(volatile int *)&P.ctl->abort;
    __syncthreads();
    const bool a = S.abrt != 0;
    __syncthreads();
    return a;
}

// Returns true when the block's state was released here (normal path), false
// when the caller must release it (tile failed the marker check).
template <int BH, int CONN>
__device__ bool process_block(Smem<BH> &S, const Params &P, const TileDesc &D, unsigned b,
                              int t, uint16_t *gsp, Work &wk)
{
    const unsigned local = b - D.block_base;
    const int by = (int)(local / (unsigned)D.nbx), bx = (int)(local % (unsigned)D.nbx);
    const int y0 = by * BH, x0 = bx * BW;
    const bool visited = S.visited != 0;
    PhaseClock clk{threadIdx.x == 0 ? gtimer() : 0ull};

    for (int i = threadIdx.x; i < BH / 32; i += NT) S.rowmask[i] = 0;
    if (threadIdx.x == 0) { S.notify = 0; S.flag = 0; }
    if (D.fast == 2) tma_load_block(S, P, D, t, y0, x0);
    else load_block(S, D, y0, x0, false);
    __syncthreads();
    trace(P, 2, b);

    if (!visited && P.check) {
        bool bad = false;
        for (int idx = threadIdx.x; idx < BH * WPR; idx += NT) {
            const int o = (1 + idx / WPR) * PW + W0 + idx % WPR;
            if (__vcmpgtu4(S.J[o], S.I[o])) bad = true;
        }
        if (bad) S.flag = 1;
        __syncthreads();
        if (S.flag) {
            if (threadIdx.x == 0) {
                atomicExch(&P.tile_err[t], 2);
                atomicMin(&P.ctl->err_tile, t);
            }
            return false;
        }
    }
    save_edges(S);
    __syncthreads();
    clk.tick(wk, PH_LOAD);

    const int k = D.k;
    bool need_seed = true;
    // a visited block sits at its fixed point for the halo it last saw
    bool frame_only = visited;
    constexpr int MAX_SCAN_PAIRS = 1 << 16, MAX_RERUNS = 1 << 14, MAX_OVERFLOWS = 1 << 12, MAX_ADAPTIVE = 64;
    constexpr int REVISIT_SCAN_MIN = 64;   // frame pixels raised before a revisit turns to scans
    // A revisit seeds from its frame first; only when that raised many frame
    // pixels (a wide change arrived through the halo) does it switch to scan
    // pairs -- fixed ones, then more while a pair still raises at least gain
    // pixels (the tuned scan-to-queue switch, Sec. V-C) -- and seed the whole block.
    const bool scan_on_revisit = k >= 0 && (P.revisit_scans > 0 || D.gain > 0);
    auto revisit_scans = [&]() {
        for (int s = 0; s < MAX_ADAPTIVE; ++s) {
            const unsigned g = scan_pair<BH, CONN>(S, P.bands, wk.scan_rows);
            if (g == 0 || (s + 1 >= P.revisit_scans && (D.gain == 0 || g < (unsigned)D.gain))) break;
        }
    };
    bool scanned = false;   // a scan pair ran this visit (its changed rows bound the seeding)
    if (!visited || k < 0) {
        const int pairs = k < 0 ? MAX_SCAN_PAIRS : k;
        int s = 0;
        scanned = pairs > 0;
        for (; s < pairs; ++s) {
            if (!scan_pair<BH, CONN>(S, P.bands, wk.scan_rows)) { if (k < 0) need_seed = false; break; }
        }
        if (k < 0 && s == pairs && threadIdx.x == 0) set_abort(P, AB_SCANS);
        if (k >= 0 && s == pairs && D.gain > 0) {
            for (int a = 0; a < MAX_ADAPTIVE; ++a)
                if (scan_pair<BH, CONN>(S, P.bands, wk.scan_rows) < (unsigned)D.gain) break;
        }
    }
    trace(P, 3, b);
    clk.tick(wk, PH_SCAN);
    for (int rerun = 0;; ++rerun) {
        if (rerun > MAX_RERUNS) {
            if (threadIdx.x == 0) set_abort(P, AB_RERUN);
            return true;
        }
        if (need_seed) {
            unsigned n;
            if (frame_only) {
                n = seed_frame<BH, CONN>(S, gsp);
                if (scan_on_revisit && n >= (unsigned)REVISIT_SCAN_MIN) {
                    revisit_scans();
                    n = seed_pass<BH, CONN>(S, gsp, S.pairmask);
                }
            } else {
                n = seed_pass<BH, CONN>(S, gsp, scanned ? S.pairmask : nullptr);
            }
            wk.seeds += 1;
            trace(P, 4, b);
            clk.tick(wk, PH_SEED);
            wk.pops += run_queue<BH, CONN>(S, P, gsp, n, wk.levels);
            for (int ov = 0; S.overflow; ++ov) {  // a level overflowed: rediscover the frontier
                __syncthreads();
                if (ov > MAX_OVERFLOWS) {
                    if (threadIdx.x == 0) set_abort(P, AB_OVERFLOW);
                    break;
                }
                n = seed_pass<BH, CONN>(S, gsp);
                wk.seeds += 1;
                wk.pops += run_queue<BH, CONN>(S, P, gsp, n, wk.levels);
            }
            trace(P, 5, b);
            clk.tick(wk, PH_QUEUE);
        }
        __syncthreads();
        write_back(S, D, y0, x0);
        __threadfence();
        edge_notify_bits<BH, CONN>(S);
        __syncthreads();
        if (threadIdx.x < 8) {   // one lane of warp 0 per direction, concurrently
            const unsigned bits = S.notify;
            const int d = threadIdx.x;
            const int dy = (d == 0 || d == 4 || d == 5) ? -1 : ((d == 1 || d == 6 || d == 7) ? 1 : 0);
            const int dx = (d == 2 || d == 4 || d == 6) ? -1 : ((d == 3 || d == 5 || d == 7) ? 1 : 0);
            if (bits & (1u << d)) {
                const int ny = by + dy, nx = bx + dx;
                if (ny >= 0 && ny < D.nby && nx >= 0 && nx < D.nbx)
                    notify_block(P, D.block_base + (unsigned)(ny * D.nbx + nx), (unsigned)t << S_TILE_SHIFT);
            }
        } else if (threadIdx.x == 32) {
            // meanwhile (another warp): let go of the block unless a neighbour
            // changed our halo while it ran
            const unsigned tb = (unsigned)t << S_TILE_SHIFT;
            const unsigned prev = atomicCAS(&P.state[b], tb | S_RUN | S_VIS, tb | S_IDLE | S_VIS);
            S.flag = (prev == (tb | S_RUN | S_VIS)) ? 0u : 1u;
            if (S.flag) atomicAnd(&P.state[b], ~S_DIRTY);
        }
        __syncwarp();
        if (threadIdx.x == 0) S.notify = 0;
        save_edges(S);
        for (int i = threadIdx.x; i < BH / 32; i += NT) S.rowmask[i] = 0;
        __syncthreads();
        trace(P, 6, b);
        clk.tick(wk, PH_WRITE);
        if (!S.flag) return true;
        if (block_aborted(S, P)) return true;
        __threadfence();
        load_block(S, D, y0, x0, true);  // fresh halo, then converge again
        wk.visits += 1;
        __syncthreads();
        trace(P, 7, b);
        clk.tick(wk, PH_LOAD);
        if (k < 0) {
            need_seed = false;
            int sp = 0;
            while (scan_pair<BH, CONN>(S, P.bands, wk.scan_rows)) {
                if (++sp > MAX_SCAN_PAIRS) {
                    if (threadIdx.x == 0) set_abort(P, AB_SCANS);
                    break;
                }
            }
        } else {
            need_seed = true;
            frame_only = true;
        }
        clk.tick(wk, PH_SCAN);
    }
}

template <int BH>
__global__ void __launch_bounds__(NT, BH == 256 ? 2 : (BH == 128 ? 4 : 6)) recon_persistent(Params P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<BH> &S = *reinterpret_cast<Smem<BH> *>(smem_raw);
    uint16_t *gsp = P.spill + (size_t)blockIdx.x * 2 * GCAP;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.phase = 0;
    }
    __syncthreads();
    // thread 0 accumulates the work counters of consecutive visits to one tile
    // and publishes them when the CTA moves to another tile or leaves
    Work &acc = S.acc;
    int &acc_tile = S.acc_tile;
    if (threadIdx.x == 0) {
        acc = Work{0, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}};
        acc_tile = -1;
    }
    auto flush = [&]() {
        if (threadIdx.x != 0 || acc_tile < 0) return;
        Work &g = P.work[acc_tile];
        atomicAdd(&g.visits, acc.visits);
        if (acc.scan_rows) atomicAdd(&g.scan_rows, acc.scan_rows);
        if (acc.pops) atomicAdd(&g.pops, acc.pops);
        if (acc.seeds) atomicAdd(&g.seeds, acc.seeds);
        if (acc.levels) atomicAdd(&g.levels, acc.levels);
        atomicAdd(&g.busy_ns, acc.busy_ns);
        for (int ph = 0; ph < NPH; ++ph)
            if (acc.phase_ns[ph]) atomicAdd(&g.phase_ns[ph], acc.phase_ns[ph]);
        acc = Work{0, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}};
    };
    for (;;) {
        const unsigned long long t_fetch = threadIdx.x == 0 ? gtimer() : 0ull;
        if (threadIdx.x == 0) {
            const unsigned b = next_item(P);
            S.item = b;
            if (b != EMPTY) {
                const unsigned old = atomicOr(&P.state[b], S_RUN | S_VIS);
                const int t = (int)(old >> S_TILE_SHIFT);   // written by the init kernel
                S.tile = (unsigned)t;
                S.visited = (old & S_VIS) ? 1u : 0u;
                S.flag = (*(volatile int *)&P.tile_err[t] == 0) ? 1u : 0u;  // one read, shared
            }
        }
        __syncthreads();
        const unsigned b = S.item;
        if (b == EMPTY) {
            flush();
            trace(P, 15, 0);
            return;
        }
        trace(P, 1, b);
        const int t = (int)S.tile;
        const TileDesc D = P.tiles[t];
        Work wk = {1, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}};
        const unsigned long long t_start = gtimer();
        wk.phase_ns[PH_FETCH] = t_start - t_fetch;
        bool released = false;
        const bool live = S.flag != 0;
        __syncthreads();  // S.flag is reused inside process_block
        if (live) {
            if (D.conn == 8) released = process_block<BH, 8>(S, P, D, b, t, gsp, wk);
            else released = process_block<BH, 4>(S, P, D, b, t, gsp, wk);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // failed tile: drop the block without touching its pixels
            if (!released) atomicExch(&P.state[b], ((unsigned)t << S_TILE_SHIFT) | S_IDLE | S_VIS);
            if (t != acc_tile) {
                flush();
                acc_tile = t;
            }
            acc.visits += wk.visits;
            acc.scan_rows += wk.scan_rows;
            acc.pops += wk.pops;
            acc.seeds += wk.seeds;
            acc.levels += wk.levels;
            acc.busy_ns += gtimer() - t_start;
            for (int ph = 0; ph < NPH; ++ph) acc.phase_ns[ph] += wk.phase_ns[ph];
            __threadfence();
            atomicSub(&P.ctl->outstanding, 1u);
        }
        trace(P, 9, b);
    }
}

__global__ void recon_init_kernel(Params P)
{
    const size_t n = P.nblocks;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        P.state[i] = (unsigned)find_tile(P, (unsigned)i) << S_TILE_SHIFT;   // not queued, not visited
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)P.ring_cap;
         i += (size_t)gridDim.x * blockDim.x)
        P.ring[i] = 0ull;   // state 0: free for lap 0
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)P.ntiles;
         i += (size_t)gridDim.x * blockDim.x) {
        P.tile_err[i] = 0;
        P.work[i] = Work{0, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.ctl->head = 0;
        P.ctl->tail = 0;
        P.ctl->outstanding = P.nblocks + (P.phantom ? 1u : 0u);
        P.ctl->cold = 0;
        P.ctl->abort = 0;
        P.ctl->abort_block = 0;
        P.ctl->err_tile = INT_MAX;
    }
}

// FillHoles tiles: J <- I on the one-pixel image border, 255 inside -- the
// marker whose reconstruction by erosion under I fills the holes of I (the
// flood of the background starts at the border). CTA (x, k) writes rows
// x, x + gridDim.x, ... of tile list[k]; 16-byte stores where rows allow.
__global__ void __launch_bounds__(256) fill_marker_kernel(const TileDesc *tiles, const int *list)
{
    const TileDesc D = tiles[list[blockIdx.y]];
    const bool vec = (D.pitch % 16) == 0 && ((uintptr_t)D.I % 16) == 0 && ((uintptr_t)D.J % 16) == 0;
    const int nv = vec ? D.W >> 4 : 0;
    for (int y = blockIdx.x; y < D.H; y += gridDim.x) {
        const uint8_t *irow = D.I + (size_t)y * D.pitch;
        uint8_t *jrow = D.J + (size_t)y * D.pitch;
        const bool edge_row = (y == 0 || y == D.H - 1);
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            uint4 o;
            if (edge_row) {
                o = __ldg((const uint4 *)irow + v);
            } else {
                o = make_uint4(~0u, ~0u, ~0u, ~0u);
                uint32_t *ow = (uint32_t *)&o;
                const int x = 16 * v;
                if (x == 0) ow[0] = (ow[0] & ~0xFFu) | irow[0];
                if (x + 15 >= D.W - 1) {
                    const int b = D.W - 1 - x;
                    ow[b >> 2] = (ow[b >> 2] & ~(0xFFu << (8 * (b & 3)))) | ((uint32_t)irow[D.W - 1] << (8 * (b & 3)));
                }
            }
            ((uint4 *)jrow)[v] = o;
        }
        for (int x = 16 * nv + threadIdx.x; x < D.W; x += blockDim.x)
            jrow[x] = (edge_row || x == 0 || x == D.W - 1) ? irow[x] : (uint8_t)255;
    }
}

}  // namespace rk

// ---------------------------------------------------------------------------
// launch helpers used by the host API

extern "C" size_t rk_smem_bytes(int bh)
{
    switch (bh) {
    case 32: return sizeof(rk::Smem<32>);
    case 64: return sizeof(rk::Smem<64>);
    case 128: return sizeof(rk::Smem<128>);
    case 256: return sizeof(rk::Smem<256>);
    }
    return 0;
}

extern "C" cudaError_t rk_configure(int bh, int *ctas_per_sm)
{
    const void *fn = nullptr;
    switch (bh) {
    case 32: fn = (const void *)rk::recon_persistent<32>; break;
    case 64: fn = (const void *)rk::recon_persistent<64>; break;
    case 128: fn = (const void *)rk::recon_persistent<128>; break;
    case 256: fn = (const void *)rk::recon_persistent<256>; break;
    default: return cudaErrorInvalidValue;
    }
    const size_t sm = rk_smem_bytes(bh);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, rk::NT, sm);
}

extern "C" cudaError_t rk_launch_init(int grid, const rk::Params *P, cudaStream_t st)
{
    rk::recon_init_kernel<<<grid, 256, 0, st>>>(*P);
    return cudaGetLastError();
}

// Bounds-checked build only: *enabled = 1, the number of failed checks since
// the last reset and the where-code of the first. Other builds: *enabled = 0.
extern "C" int recon_checks(int *enabled, unsigned *violations, unsigned *first, int reset)
{
    if (!enabled || !violations || !first) return 1;
#ifdef RECON_CHECKS
    *enabled = 1;
    if (cudaMemcpyFromSymbol(violations, rk::g_check_violations, sizeof(unsigned)) != cudaSuccess ||
        cudaMemcpyFromSymbol(first, rk::g_check_first, sizeof(unsigned)) != cudaSuccess)
        return 4;
    if (reset) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(rk::g_check_violations, &z, sizeof(z)) != cudaSuccess ||
            cudaMemcpyToSymbol(rk::g_check_first, &z, sizeof(z)) != cudaSuccess)
            return 4;
    }
#else
    *enabled = 0;
    *violations = 0;
    *first = 0;
    (void)reset;
#endif
    return 0;
}

extern "C" cudaError_t rk_launch_fill(const rk::TileDesc *tiles, const int *list, int nlist, cudaStream_t st)
{
    if (nlist <= 0) return cudaSuccess;
    if (nlist > 65535) return cudaErrorInvalidValue;
    rk::fill_marker_kernel<<<dim3(64, (unsigned)nlist), 256, 0, st>>>(tiles, list);
    return cudaGetLastError();
}

extern "C" cudaError_t rk_launch_main(int bh, int grid, const rk::Params *P, cudaStream_t st)
{
    const size_t sm = rk_smem_bytes(bh);
    switch (bh) {
    case 32: rk::recon_persistent<32><<<grid, rk::NT, sm, st>>>(*P); break;
    case 64: rk::recon_persistent<64><<<grid, rk::NT, sm, st>>>(*P); break;
    case 128: rk::recon_persistent<128><<<grid, rk::NT, sm, st>>>(*P); break;
    case 256: rk::recon_persistent<256><<<grid, rk::NT, sm, st>>>(*P); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
