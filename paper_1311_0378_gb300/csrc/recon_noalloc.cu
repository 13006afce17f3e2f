// recon_run_noalloc: the one entry point that allocates no memory at all.
//
// Who needs it: callers that must not call cudaMalloc (or anything that
// allocates device or pinned memory) once they are running -- for example a
// plugin inside a host framework that has already handed all device memory to
// its own pool allocator, or a latency-critical pipeline that forbids the
// implicit device synchronisation an allocation can bring. Such callers can
// still pass their own input and output buffers, but the library must find its
// scratch space elsewhere.
//
// How: the persistent reconstruction kernel's scratch (control word, one tile
// descriptor, per-block state and ring, the per-CTA overflow areas of the
// wavefront queues) lives in one file-scope device array, g_noalloc_scratch,
// of NOALLOC_BYTES (11 MiB). It is part of the module image, so every GPU that
// loads this library holds those 11 MiB until the process exits. In host code
// the array's name is only a host-side stand-in, not a device address, so the
// first call on each device looks up the real address with
// cudaGetSymbolAddress (with that device current) and caches it; kernels get
// that address. Make that first call outside any CUDA stream capture.
//
// Limits: one tile, row stride = W, blocks of 64 x 128 pixels, at most
// NOALLOC_MAX_BLOCKS = 4096 blocks (e.g. 4096 x 8192 or 8192 x 4096 pixels),
// and at most NOALLOC_MAX_CTAS = 160 CTAs. Larger inputs are rejected with
// RECON_EINVAL before anything runs.
//
// Sharing: every call uses the same array, which keeps the last call's
// contents; the init kernel clears what must start at zero (control word,
// block states, ring, status, counters) at the start of every call. Calls
// whose work overlaps on the GPU (from two host threads or on two streams)
// race on the array and must not be issued.
#include <climits>
#include <cstring>
#include <mutex>
#include <cuda_runtime.h>

#include "recon.h"
#include "recon_internal.h"

extern "C" cudaError_t rk_configure(int bh, int *ctas_per_sm);
extern "C" cudaError_t rk_launch_init(int grid, const rk::Params *P, cudaStream_t st);
extern "C" cudaError_t rk_launch_main(int bh, int grid, const rk::Params *P, cudaStream_t st);

namespace {

constexpr int NOALLOC_BH = 64;
constexpr unsigned NOALLOC_MAX_BLOCKS = 4096;
constexpr int NOALLOC_MAX_CTAS = 160;

// byte offsets inside the scratch array
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_DESC = 256;            // TileDesc (64 B) + order (4 B) + order_base (8 B)
constexpr size_t OFF_ORDER = OFF_DESC + 64;
constexpr size_t OFF_BASE = OFF_DESC + 80;
constexpr size_t OFF_ERR = 512;
constexpr size_t OFF_WORK = 576;
constexpr size_t OFF_STATE = 1024;
constexpr size_t OFF_RING = OFF_STATE + 4 * NOALLOC_MAX_BLOCKS;
constexpr size_t RING_SLOTS = 2 * NOALLOC_MAX_BLOCKS + 2 * NOALLOC_MAX_CTAS;   // 8-byte slots
constexpr size_t OFF_SPILL = 131072;
constexpr size_t SPILL_BYTES = (size_t)NOALLOC_MAX_CTAS * 2 * rk::GCAP * sizeof(uint16_t);
constexpr size_t NOALLOC_BYTES = 11u << 20;

static_assert(sizeof(rk::Ctl) <= OFF_DESC - OFF_CTL, "control word");
static_assert(sizeof(rk::TileDesc) <= 64, "descriptor");
static_assert(OFF_BASE + 8 <= OFF_ERR && OFF_WORK + sizeof(rk::Work) <= OFF_STATE, "layout");
static_assert(OFF_RING % 8 == 0 && OFF_RING + 8 * RING_SLOTS <= OFF_SPILL, "state and ring");
static_assert(OFF_SPILL + SPILL_BYTES <= NOALLOC_BYTES, "spill areas");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[256];   // device address of g_noalloc_scratch, per device
int g_max_ctas[256];

// Once per device, with that device current: the array's device address and
// the kernel's shared-memory setting. Returns RECON_OK or an error code.
int setup_device(int dev, unsigned char **base, int *max_ctas)
{
    if (dev < 0 || dev >= 256) return RECON_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RECON_ECUDA;
        int occ = 0, sms = 0;
        if (rk_configure(NOALLOC_BH, &occ) != cudaSuccess) return RECON_ECUDA;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RECON_ECUDA;
        long ctas = (long)(occ > 0 ? occ : 1) * (long)sms;
        g_max_ctas[dev] = (int)(ctas < NOALLOC_MAX_CTAS ? ctas : NOALLOC_MAX_CTAS);
        g_scratch_dev[dev] = (unsigned char *)p;
    }
    *base = g_scratch_dev[dev];
    *max_ctas = g_max_ctas[dev];
    return RECON_OK;
}

}  // namespace

extern "C" int recon_run_noalloc(const uint8_t *I, uint8_t *J, int H, int W, int conn, void *cuda_stream)
{
    if (!I || !J || H < 1 || W < 1 || (conn != 4 && conn != 8)) return RECON_EINVAL;
    // block counts in 64-bit arithmetic: no overflow for any int H, W
    const long long nbx_ll = ((long long)W + rk::BW - 1) / rk::BW, nby_ll = ((long long)H + NOALLOC_BH - 1) / NOALLOC_BH;
    if (nbx_ll * nby_ll > (long long)NOALLOC_MAX_BLOCKS) return RECON_EINVAL;  // beyond the fixed scratch
    const unsigned nbx = (unsigned)nbx_ll, nby = (unsigned)nby_ll;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RECON_ECUDA;
    unsigned char *base = nullptr;
    int grid = 0;
    int rc = setup_device(dev, &base, &grid);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // the one tile's descriptor and packing tables, staged from the host stack
    unsigned char stage[OFF_BASE + 8 - OFF_DESC];
    memset(stage, 0, sizeof(stage));
    rk::TileDesc d;
    memset(&d, 0, sizeof(d));
    d.I = I; d.J = J; d.H = H; d.W = W; d.pitch = W; d.conn = conn;
    d.nbx = (int)nbx; d.nby = (int)nby;
    d.k = 1;
    d.fast = ((W % 4) == 0 && ((uintptr_t)I % 4) == 0 && ((uintptr_t)J % 4) == 0) ? 1 : 0;  // plain loads
    d.block_base = 0;
    memcpy(stage, &d, sizeof(d));
    const int order0 = 0;
    const unsigned ob[2] = {0u, nbx * nby};
    memcpy(stage + (OFF_ORDER - OFF_DESC), &order0, sizeof(order0));
    memcpy(stage + (OFF_BASE - OFF_DESC), ob, sizeof(ob));
    if (cudaMemcpyAsync(base + OFF_DESC, stage, sizeof(stage), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RECON_ECUDA;

    rk::Params P;
    memset(&P, 0, sizeof(P));
    P.tiles = (const rk::TileDesc *)(base + OFF_DESC);
    P.ntiles = 1;
    P.tmaps = base + OFF_DESC;   // never read: the tile uses plain loads
    P.order = (const int *)(base + OFF_ORDER);
    P.order_base = (const unsigned *)(base + OFF_BASE);
    P.nblocks = nbx * nby;
    P.state = (unsigned *)(base + OFF_STATE);
    P.ring = (unsigned long long *)(base + OFF_RING);
    P.ring_cap = 2 * (nbx * nby) + 2 * (unsigned)grid;
    P.ctl = (rk::Ctl *)(base + OFF_CTL);
    P.tile_err = (int *)(base + OFF_ERR);
    P.work = (rk::Work *)(base + OFF_WORK);
    P.spill = (uint16_t *)(base + OFF_SPILL);
    P.wait_ns = 2000000000ll;
    P.bands = 4;
    P.revisit_scans = 0;
    P.phantom = 0;
    P.check = 1;
    P.trace = nullptr;
    // the init kernel zeroes control word, states, ring, status and counters
    if (rk_launch_init(grid, &P, st) != cudaSuccess) return RECON_ECUDA;
    if (rk_launch_main(NOALLOC_BH, grid, &P, st) != cudaSuccess) return RECON_ECUDA;
    // the status word comes back on the caller's stream, and only that stream
    // is waited on (a plain cudaMemcpy would also wait for other work on the device)
    rk::Ctl h;
    if (cudaMemcpyAsync(&h, base + OFF_CTL, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RECON_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RECON_ECUDA;
    if (h.abort) return RECON_ETIMEOUT;
    if (h.err_tile != INT_MAX) return RECON_EMARKER;
    return RECON_OK;
}
