// Host side of the C ABI declared in include/recon.h: argument checks, scratch
// management, the launch of the persistent reconstruction kernel, CUDA-graph
// replay of repeated batches, and the end-to-end (host buffer) entry points.
#include <climits>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#include <map>
#include <tuple>
#include <algorithm>
#include <time.h>
#include <cmath>
#include <cuda.h>
#include <cuda_runtime.h>

#include "recon.h"
#include "recon_internal.h"
#include "recon_sched.h"
#include "recon_learn.h"
#include "recon_dt.h"

extern "C" size_t rk_smem_bytes(int bh);
extern "C" cudaError_t rk_configure(int bh, int *ctas_per_sm);
extern "C" cudaError_t rk_launch_init(int grid, const rk::Params *P, cudaStream_t st);
extern "C" cudaError_t rk_launch_main(int bh, int grid, const rk::Params *P, cudaStream_t st);
extern "C" cudaError_t rk_launch_fill(const rk::TileDesc *tiles, const int *list, int nlist, cudaStream_t st);

constexpr int HOST_SEGMENTS = 4;   // pipeline segments of the end-to-end (host buffer) calls

struct recon_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    unsigned flags = 0;
    int sms = 0;
    // tunables
    // defaults: 128-row blocks, one scan pair on a first visit, then more pairs
    // while a pair still raises >= 2048 pixels (first visits and revisits)
    int bh = 128, k = 1, grid = 0, bands = 4, order_policy = 1, phantom = 0, use_tma = 1, revisit_scans = 0, scan_gain = 2048;
    long long wait_ns = 2000000000ll;
    // device scratch
    unsigned char *d_meta = nullptr; size_t cap_meta = 0;      // descriptors + order tables
    unsigned *d_state = nullptr; size_t cap_blocks = 0, cap_ring = 0;
    unsigned long long *d_ring = nullptr;
    rk::Ctl *d_ctl = nullptr;
    int *d_tile_err = nullptr; rk::Work *d_work = nullptr; size_t cap_tiles = 0;
    uint16_t *d_spill = nullptr; size_t cap_spill_ctas = 0;
    // host staging (pinned)
    unsigned char *h_meta = nullptr; size_t cap_hmeta = 0;
    cudaEvent_t meta_free = nullptr, ev0 = nullptr, ev1 = nullptr;
    // end-to-end buffers and the copy streams of its pipeline
    uint8_t *d_img = nullptr; size_t cap_img = 0;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr, s_plan = nullptr;
    cudaEvent_t ev_in[HOST_SEGMENTS] = {}, ev_out[HOST_SEGMENTS] = {};
    rk::Ctl *h_seg_ctl = nullptr;   // pinned: each segment's control word, copied right after its kernel
    // last call
    int last_n = 0;
    int launched = 0;
    int last_err_tile = -1;
    int last_abort = 0;
    int host_status = 0;     // 1: last_err_tile / last_abort hold the last recon_batch_host call's status
    // diagnostics: per-warp progress words in mapped host memory
    unsigned *h_trace = nullptr; unsigned *d_trace = nullptr; size_t cap_trace = 0; int trace_on = 0;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gsig;
    // learned scheduler
    recon_sched *sched = nullptr;
    // distance transform scratch
    unsigned char *d_dt = nullptr; size_t cap_dt = 0;
    int *d_dt_site = nullptr; size_t cap_dt_site = 0;
    unsigned *h_dt_cnt = nullptr;
    int dt_levels = 0;
    // autotuner results: (size bucket, connectivities, marker class) -> {bh, bands, k, gain}
    std::map<std::tuple<int, int, int>, std::vector<int>> tune_cache;
    int tune_from_cache = 0;
};

static int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return RECON_OK;
    if (e == cudaErrorMemoryAllocation) return RECON_ENOMEM;
    return RECON_ECUDA;
}

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_status(e_); } while (0)

template <typename T>
static int grow(T **p, size_t *cap, size_t need)
{
    if (*cap >= need && *p) return RECON_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = std::max(need, (size_t)1);
    const cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();   // an allocation failure leaves the context usable: clear it
        *p = nullptr;
        return cuda_status(e);
    }
    *cap = n;
    return RECON_OK;
}

static void drop_graph(recon_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gsig.clear();
}

extern "C" int recon_init(recon_ctx **out, int device, void *cuda_stream, unsigned flags)
{
    if (!out) return RECON_EINVAL;
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return RECON_EINVAL;
    CK(cudaSetDevice(device));
    recon_ctx *c = new (std::nothrow) recon_ctx();
    if (!c) return RECON_ENOMEM;
    c->device = device;
    c->flags = flags;
    cudaError_t e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->meta_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_ctl, sizeof(rk::Ctl));
    if (e == cudaSuccess) {
        int occ = 0;
        for (int bh : {32, 64, 128, 256})
            if (e == cudaSuccess) e = rk_configure(bh, &occ);
    }
    if (e != cudaSuccess) {
        recon_free(c);
        return cuda_status(e);
    }
    c->sched = recon_sched_create();
    // environment overrides of the context defaults (RECON_BLOCK_H=64 ...);
    // a malformed or out-of-range value fails the call rather than being ignored
    static const struct { const char *name; int key; } env[] = {
        {"RECON_BLOCK_H", RECON_P_BLOCK_H}, {"RECON_SWEEPS", RECON_P_SWEEPS}, {"RECON_BANDS", RECON_P_BANDS},
        {"RECON_GRID", RECON_P_GRID}, {"RECON_WAIT_NS", RECON_P_WAIT_NS}, {"RECON_ORDER", RECON_P_ORDER},
        {"RECON_TMA", RECON_P_TMA}, {"RECON_REVISIT_SCANS", RECON_P_REVISIT_SCANS},
        {"RECON_SCAN_GAIN", RECON_P_SCAN_GAIN}};
    for (const auto &ev : env) {
        const char *v = getenv(ev.name);
        if (!v || !*v) continue;
        char *end = nullptr;
        const long long x = strtoll(v, &end, 10);
        if (*end != '\0' || recon_set_param(c, ev.key, (int64_t)x) != RECON_OK) {
            recon_free(c);
            return RECON_EINVAL;
        }
    }
    *out = c;
    return RECON_OK;
}

extern "C" int recon_free(recon_ctx *c)
{
    if (!c) return RECON_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    cudaFree(c->d_meta);
    cudaFree(c->d_state);
    cudaFree(c->d_ring);
    cudaFree(c->d_ctl);
    cudaFree(c->d_tile_err);
    cudaFree(c->d_work);
    cudaFree(c->d_spill);
    cudaFree(c->d_img);
    cudaFree(c->d_dt);
    cudaFree(c->d_dt_site);
    if (c->h_dt_cnt) cudaFreeHost(c->h_dt_cnt);
    if (c->h_meta) cudaFreeHost(c->h_meta);
    if (c->h_trace) cudaFreeHost(c->h_trace);
    if (c->meta_free) cudaEventDestroy(c->meta_free);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (int s = 0; s < HOST_SEGMENTS; ++s)
        if (c->ev_in[s]) cudaEventDestroy(c->ev_in[s]);
    for (int s = 0; s < HOST_SEGMENTS; ++s)
        if (c->ev_out[s]) cudaEventDestroy(c->ev_out[s]);
    if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
    if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
    if (c->s_plan) cudaStreamDestroy(c->s_plan);
    if (c->h_seg_ctl) cudaFreeHost(c->h_seg_ctl);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    recon_sched_destroy(c->sched);
    delete c;
    return RECON_OK;
}

extern "C" const char *recon_strerror(int s)
{
    switch (s) {
    case RECON_OK: return "ok";
    case RECON_EINVAL: return "invalid argument";
    case RECON_EMARKER: return "marker exceeds mask (J > I) at some pixel";
    case RECON_ENOMEM: return "out of memory";
    case RECON_ECUDA: return "CUDA runtime error";
    case RECON_ETIMEOUT: return "bounded device wait ran out";
    }
    return "unknown status";
}

static int tile_ok(const recon_tile &t)
{
    if (!t.I || !t.J || t.H < 1 || t.W < 1 || t.pitch < t.W) return 0;
    if (t.conn != 4 && t.conn != 8) return 0;
    if (t.op != RECON_OP_DILATE && t.op != RECON_OP_ERODE && t.op != RECON_OP_FILL_HOLES) return 0;
    if ((double)t.H * (double)t.pitch > 9.0e18) return 0;
    return 1;
}

extern "C" int recon_set_param(recon_ctx *c, int key, int64_t v)
{
    if (!c) return RECON_EINVAL;
    switch (key) {
    case RECON_P_BLOCK_H:
        if (v != 32 && v != 64 && v != 128 && v != 256) return RECON_EINVAL;
        c->bh = (int)v; break;
    case RECON_P_SWEEPS:
        if (v < -1 || v > 64) return RECON_EINVAL;
        c->k = (int)v; break;
    case RECON_P_GRID:
        if (v < 0 || v > (1 << 20)) return RECON_EINVAL;
        c->grid = (int)v; break;
    case RECON_P_BANDS:
        if (v != 1 && v != 2 && v != 4) return RECON_EINVAL;
        c->bands = (int)v; break;
    case RECON_P_WAIT_NS:
        if (v < 1000 || v > 600000000000ll) return RECON_EINVAL;
        c->wait_ns = v; break;
    case RECON_P_ORDER:
        if (v != 0 && v != 1) return RECON_EINVAL;
        c->order_policy = (int)v; break;
    case RECON_P_TEST_STALL:
        if (v != 0 && v != 1) return RECON_EINVAL;
        c->phantom = (int)v; break;
    case RECON_P_TMA:
        if (v != 0 && v != 1) return RECON_EINVAL;
        c->use_tma = (int)v; break;
    case RECON_P_TRACE:
        if (v != 0 && v != 1) return RECON_EINVAL;
        c->trace_on = (int)v; break;
    case RECON_P_REVISIT_SCANS:
        if (v < 0 || v > 16) return RECON_EINVAL;
        c->revisit_scans = (int)v; break;
    case RECON_P_SCAN_GAIN:
        if (v < 0 || v > (1 << 20)) return RECON_EINVAL;
        c->scan_gain = (int)v; break;
    default: return RECON_EINVAL;
    }
    drop_graph(c);
    return RECON_OK;
}

extern "C" int64_t recon_get_param(recon_ctx *c, int key)
{
    if (!c) return -1;
    switch (key) {
    case RECON_P_BLOCK_H: return c->bh;
    case RECON_P_SWEEPS: return c->k;
    case RECON_P_GRID: {
        if (c->grid) return c->grid;
        int occ = 0;
        if (rk_configure(c->bh, &occ) != cudaSuccess) return -1;
        return (int64_t)occ * c->sms;
    }
    case RECON_P_BANDS: return c->bands;
    case RECON_P_WAIT_NS: return c->wait_ns;
    case RECON_P_ORDER: return c->order_policy;
    case RECON_P_TEST_STALL: return c->phantom;
    case RECON_P_TMA: return c->use_tma;
    case RECON_P_TRACE: return c->trace_on;
    case RECON_P_REVISIT_SCANS: return c->revisit_scans;
    case RECON_P_SCAN_GAIN: return c->scan_gain;
    case RECON_P_LAST_ABORT: return c->last_abort;
    case RECON_P_TUNE_FROM_CACHE: return c->tune_from_cache;
    }
    return -1;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda needed).
typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static encode_fn get_encode()
{
    static encode_fn fn = nullptr;
    static int tried = 0;
    if (!tried) {
        tried = 1;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (encode_fn)p;
    }
    return fn;
}

// Tensor map of one uint8 image: dims (W, H), row stride pitch, box of
// BOXW x (bh + 2) bytes; out-of-bounds elements read as zero.
static int encode_map(CUtensorMap *m, const void *base, int H, int W, int pitch, int bh)
{
    encode_fn fn = get_encode();
    if (!fn) return 0;
    cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    // at most 256 rows per box: taller blocks are loaded as two boxes whose
    // height is a multiple of 4 rows (the kernel's Boxes<BH>)
    const int rows = bh + 2 > 256 ? ((bh + 2) / 2 + 3) / 4 * 4 : bh + 2;
    cuuint32_t box[2] = {(cuuint32_t)rk::BOXW, (cuuint32_t)rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct MetaLayout {
    size_t off_order, off_base, off_fill, off_maps, total;
};

// descriptors | packing order | block bases | FillHoles tile list | tensor maps
static MetaLayout meta_layout(int n)
{
    MetaLayout L;
    L.off_order = align_up(sizeof(rk::TileDesc) * n, 16);
    L.off_base = align_up(L.off_order + sizeof(int) * n, 16);
    L.off_fill = align_up(L.off_base + sizeof(unsigned) * (n + 1), 16);
    L.off_maps = align_up(L.off_fill + sizeof(int) * n, 128);
    L.total = L.off_maps + 256 * (size_t)n;
    return L;
}

// Builds the descriptor table + packing tables in the pinned staging buffer.
// Returns bytes used, or 0 on failure.
static int stage_meta(recon_ctx *c, const recon_tile *tiles, int n, const int *variant,
                      const int *order, size_t *bytes, unsigned *nblocks, int *nfill)
{
    const MetaLayout L = meta_layout(n);
    const size_t off_order = L.off_order, off_base = L.off_base, total = L.total;
    // the previous call's copy out of the staging buffer must be done (its
    // event is recorded right after that copy, not after the kernels)
    CK(cudaEventSynchronize(c->meta_free));
    if (c->cap_hmeta < total) {
        if (c->h_meta) cudaFreeHost(c->h_meta);
        c->h_meta = nullptr;
        c->cap_hmeta = 0;
        CK(cudaMallocHost((void **)&c->h_meta, total));
        c->cap_hmeta = total;
    }
    rk::TileDesc *D = (rk::TileDesc *)c->h_meta;
    int *ord = (int *)(c->h_meta + off_order);
    unsigned *base = (unsigned *)(c->h_meta + off_base);
    int *fill = (int *)(c->h_meta + L.off_fill);
    int nf = 0;
    unsigned long long nb = 0;
    for (int t = 0; t < n; ++t) {
        const recon_tile &T = tiles[t];
        rk::TileDesc d;
        memset(&d, 0, sizeof(d));
        d.I = T.I; d.J = T.J; d.H = T.H; d.W = T.W; d.pitch = T.pitch; d.conn = T.conn;
        d.dual = T.op != RECON_OP_DILATE ? 1 : 0;
        d.fill = T.op == RECON_OP_FILL_HOLES ? 1 : 0;
        if (d.fill) fill[nf++] = t;
        d.nbx = (T.W + rk::BW - 1) / rk::BW;
        d.nby = (T.H + c->bh - 1) / c->bh;
        // variant: -1 = scans to stability; else k + 256 * (gain / 64)
        if (variant) {
            d.k = variant[t] == -1 ? -1 : (variant[t] & 0xFF);
            d.gain = variant[t] == -1 ? 0 : (variant[t] >> 8) * 64;
        } else {
            d.k = c->k;
            d.gain = c->scan_gain;
        }
        d.fast = ((T.pitch % 4) == 0 && ((uintptr_t)T.I % 4) == 0 && ((uintptr_t)T.J % 4) == 0) ? 1 : 0;
        CUtensorMap *maps = (CUtensorMap *)(c->h_meta + L.off_maps + 256 * (size_t)t);
        memset(maps, 0, 256);
        if (c->use_tma && (T.pitch % 16) == 0 && ((uintptr_t)T.I % 16) == 0 && ((uintptr_t)T.J % 16) == 0 &&
            encode_map(&maps[0], T.I, T.H, T.W, T.pitch, c->bh) && encode_map(&maps[1], T.J, T.H, T.W, T.pitch, c->bh))
            d.fast = 2;
        d.block_base = (unsigned)nb;
        nb += (unsigned long long)d.nbx * (unsigned long long)d.nby;
        if (nb >= 0xFFFFFFF0ull) return RECON_EINVAL;
        D[t] = d;
    }
    if (order) {
        std::vector<char> seen(n, 0);
        for (int i = 0; i < n; ++i) {
            if (order[i] < 0 || order[i] >= n || seen[order[i]]) return RECON_EINVAL;
            seen[order[i]] = 1;
            ord[i] = order[i];
        }
    } else {
        for (int i = 0; i < n; ++i) ord[i] = i;
        if (c->order_policy == 1)
            std::stable_sort(ord, ord + n, [&](int a, int b) {
                return (long long)tiles[a].H * tiles[a].W > (long long)tiles[b].H * tiles[b].W;
            });
    }
    unsigned acc = 0;
    for (int i = 0; i < n; ++i) {
        base[i] = acc;
        acc += (unsigned)(D[ord[i]].nbx * D[ord[i]].nby);
    }
    base[n] = acc;
    memset(fill + nf, 0, sizeof(int) * (size_t)(n - nf));
    *bytes = total;
    *nblocks = (unsigned)nb;
    *nfill = nf;
    return RECON_OK;
}

static int batch_impl(recon_ctx *c, const recon_tile *tiles, int n, const int *variant, const int *order)
{
    if (!c || !tiles || n < 1 || n > rk::MAX_TILES) return RECON_EINVAL;
    for (int t = 0; t < n; ++t)
        if (!tile_ok(tiles[t])) return RECON_EINVAL;
    if (variant)
        for (int t = 0; t < n; ++t)
            if (variant[t] < -1 || (variant[t] >= 0 && ((variant[t] & 0xFF) > 64 || (variant[t] >> 8) > 4096)))
                return RECON_EINVAL;
    CK(cudaSetDevice(c->device));

    std::vector<int> lv, lo;
    if ((c->flags & RECON_FLAG_LEARNED) && !variant && !order && c->sched) {
        int rc = recon_sched_plan(c->sched, tiles, n, c->sms, c->stream, &lv, &lo);
        if (rc == RECON_OK) { variant = lv.data(); order = lo.data(); }
    }

    size_t bytes = 0;
    unsigned nblocks = 0;
    int nfill = 0;
    int rc = stage_meta(c, tiles, n, variant, order, &bytes, &nblocks, &nfill);
    if (rc) return rc;
    if (nfill > 65535) return RECON_EINVAL;

    int grid = c->grid;
    if (!grid) {
        int occ = 0;
        CK(rk_configure(c->bh, &occ));
        grid = std::max(1, occ) * c->sms;
    }
    // scratch: grow only between launches (nothing in flight uses the old buffers)
    // ring slots: any number is correct (laps are tagged); this many keeps
    // producers from waiting for an earlier lap's block to be taken
    const size_t ring_cap = std::min<size_t>(2 * (size_t)nblocks + 2 * (size_t)grid, (size_t)1 << 31);
    const bool need = c->cap_meta < bytes || c->cap_blocks < nblocks || c->cap_ring < ring_cap ||
                      c->cap_tiles < (size_t)n || c->cap_spill_ctas < (size_t)grid || !c->d_state || !c->d_ring;
    if (need) {
        CK(cudaStreamSynchronize(c->stream));
        drop_graph(c);
        if ((rc = grow(&c->d_meta, &c->cap_meta, bytes))) return rc;
        if (c->cap_blocks < nblocks || c->cap_ring < ring_cap || !c->d_state || !c->d_ring) {
            size_t a = 0, b = 0;
            if (c->d_state) cudaFree(c->d_state);
            if (c->d_ring) cudaFree(c->d_ring);
            c->d_state = nullptr; c->d_ring = nullptr; c->cap_blocks = 0; c->cap_ring = 0;
            if ((rc = grow(&c->d_state, &a, nblocks))) return rc;
            if ((rc = grow(&c->d_ring, &b, ring_cap))) return rc;
            c->cap_blocks = a;
            c->cap_ring = b;
        }
        if (c->cap_tiles < (size_t)n || !c->d_tile_err || !c->d_work) {
            size_t a = 0, b = 0;
            if (c->d_tile_err) cudaFree(c->d_tile_err);
            if (c->d_work) cudaFree(c->d_work);
            c->d_tile_err = nullptr; c->d_work = nullptr; c->cap_tiles = 0;
            if ((rc = grow(&c->d_tile_err, &a, (size_t)n))) return rc;
            if ((rc = grow(&c->d_work, &b, (size_t)n))) return rc;
            c->cap_tiles = std::min(a, b);
        }
        if (c->cap_spill_ctas < (size_t)grid) {
            size_t a = 0;
            if (c->d_spill) cudaFree(c->d_spill);
            c->d_spill = nullptr; c->cap_spill_ctas = 0;
            if ((rc = grow(&c->d_spill, &a, (size_t)grid * 2 * rk::GCAP))) return rc;
            c->cap_spill_ctas = (size_t)grid;
        }
    }

    rk::Params P;
    memset(&P, 0, sizeof(P));
    const MetaLayout ML = meta_layout(n);
    P.tiles = (const rk::TileDesc *)c->d_meta;
    P.ntiles = n;
    P.tmaps = (const void *)(c->d_meta + ML.off_maps);
    P.order = (const int *)(c->d_meta + ML.off_order);
    P.order_base = (const unsigned *)(c->d_meta + ML.off_base);
    P.nblocks = nblocks;
    P.state = c->d_state;
    P.ring = c->d_ring;
    P.ring_cap = (unsigned)ring_cap;
    P.ctl = c->d_ctl;
    P.tile_err = c->d_tile_err;
    P.work = c->d_work;
    P.spill = c->d_spill;
    P.wait_ns = c->wait_ns;
    P.bands = c->bands;
    P.revisit_scans = c->revisit_scans;
    P.phantom = c->phantom;
    P.check = (c->flags & RECON_FLAG_NO_CHECK) ? 0 : 1;
    P.trace = nullptr;
    if (c->trace_on) {
        const size_t words = (size_t)grid * (rk::NT / 32);
        if (c->cap_trace < words) {
            CK(cudaStreamSynchronize(c->stream));
            drop_graph(c);
            if (c->h_trace) cudaFreeHost(c->h_trace);
            c->h_trace = nullptr;
            c->cap_trace = 0;
            CK(cudaHostAlloc((void **)&c->h_trace, words * sizeof(unsigned), cudaHostAllocMapped));
            CK(cudaHostGetDevicePointer((void **)&c->d_trace, c->h_trace, 0));
            c->cap_trace = words;
        }
        memset(c->h_trace, 0, c->cap_trace * sizeof(unsigned));
        P.trace = c->d_trace;
    }

    // signature of this launch: replay the captured graph when it repeats
    std::vector<unsigned char> sig(bytes + sizeof(P) + 2 * sizeof(int));
    memcpy(sig.data(), c->h_meta, bytes);
    memcpy(sig.data() + bytes, &P, sizeof(P));
    memcpy(sig.data() + bytes + sizeof(P), &grid, sizeof(int));
    memcpy(sig.data() + bytes + sizeof(P) + sizeof(int), &c->bh, sizeof(int));

    c->last_n = n;
    c->last_err_tile = -1;
    c->host_status = 0;
    const bool use_graph = !(c->flags & RECON_FLAG_NO_GRAPH);
    if (use_graph && c->gexec && sig == c->gsig) {
        // the graph records meta_free itself, right after its descriptor copy
        CK(cudaGraphLaunch(c->gexec, c->stream));
    } else {
        drop_graph(c);
        cudaGraph_t g = nullptr;
        if (use_graph) CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        // inside a capture, only an external record becomes an event node
        const unsigned evf = use_graph ? cudaEventRecordExternal : cudaEventRecordDefault;
        cudaError_t e = cudaMemcpyAsync(c->d_meta, c->h_meta, bytes, cudaMemcpyHostToDevice, c->stream);
        // the staging buffer is free once this copy is done: the next call may
        // refill it while this call's kernels still run
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->meta_free, c->stream, evf);
        // FillHoles tiles: write their border markers first
        if (e == cudaSuccess && nfill)
            e = rk_launch_fill(P.tiles, (const int *)(c->d_meta + ML.off_fill), nfill, c->stream);
        if (e == cudaSuccess) e = rk_launch_init(std::min(grid, 4 * c->sms), &P, c->stream);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->ev0, c->stream, evf);
        if (e == cudaSuccess) e = rk_launch_main(c->bh, grid, &P, c->stream);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->ev1, c->stream, evf);
        if (use_graph) {
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) e = cudaGraphLaunch(c->gexec, c->stream);
            if (e == cudaSuccess) c->gsig.swap(sig);
            else drop_graph(c);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    c->launched = 1;
    if (c->flags & RECON_FLAG_SYNC) return recon_sync(c);
    return RECON_OK;
}

extern "C" int recon_batch_ex(recon_ctx *c, const recon_tile *tiles, int n, const int *variant,
                              const int *order)
{
    return batch_impl(c, tiles, n, variant, order);
}

extern "C" int recon_batch(recon_ctx *c, const recon_tile *tiles, int n)
{
    return batch_impl(c, tiles, n, nullptr, nullptr);
}

extern "C" int recon_run(recon_ctx *c, const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    return recon_run_op(c, I, J, H, W, conn, RECON_OP_DILATE);
}

extern "C" int recon_run_op(recon_ctx *c, const uint8_t *I, uint8_t *J, int H, int W, int conn, int op)
{
    recon_tile t;
    t.I = I; t.J = J; t.H = H; t.W = W; t.pitch = W; t.conn = conn; t.op = op;
    return batch_impl(c, &t, 1, nullptr, nullptr);
}

extern "C" int recon_sync(recon_ctx *c)
{
    if (!c) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    if (!c->launched) return RECON_OK;
    if (!c->host_status) {   // a host batch records its own status (its segments share the control word)
        rk::Ctl h;
        CK(cudaMemcpy(&h, c->d_ctl, sizeof(h), cudaMemcpyDeviceToHost));
        c->last_err_tile = (h.err_tile == INT_MAX) ? -1 : h.err_tile;
        c->last_abort = h.abort;
    }
    if (c->last_abort) return RECON_ETIMEOUT;
    if (c->last_err_tile >= 0) return RECON_EMARKER;
    return RECON_OK;
}

extern "C" int recon_last_error_tile(recon_ctx *c)
{
    if (!c) return -1;
    recon_sync(c);
    return c->last_err_tile;
}

extern "C" int recon_get_work(recon_ctx *c, recon_work *out, int n)
{
    if (!c || !out || n < 0 || n > c->last_n) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    if (n == 0) return RECON_OK;
    std::vector<rk::Work> w(n);
    CK(cudaMemcpy(w.data(), c->d_work, sizeof(rk::Work) * n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) {
        out[i].visits = w[i].visits;
        out[i].scan_rows = w[i].scan_rows;
        out[i].pops = w[i].pops;
        out[i].seeds = w[i].seeds;
        out[i].levels = w[i].levels;
        out[i].busy_ns = w[i].busy_ns;
        for (int k = 0; k < 6; ++k) out[i].phase_ns[k] = w[i].phase_ns[k];
    }
    return RECON_OK;
}

extern "C" int recon_last_kernel_ms(recon_ctx *c, float *ms)
{
    if (!c || !ms || !c->launched) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaEventElapsedTime(ms, c->ev0, c->ev1));
    return RECON_OK;
}

// ---------------------------------------------------------------------------
// end-to-end entry points (host buffers)

// Rows of `width` bytes between host and device: one linear copy when both
// sides are contiguous, a 2-D copy otherwise.
static cudaError_t copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t height,
                             cudaMemcpyKind kind, cudaStream_t st)
{
    if (dpitch == width && spitch == width)
        return cudaMemcpyAsync(dst, src, width * height, kind, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, st);
}

// Streams and events of the end-to-end pipeline (created on first use).
static int ensure_pipeline(recon_ctx *c)
{
    if (!c->s_h2d) CK(cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking));
    if (!c->s_d2h) CK(cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking));
    if (!c->s_plan) CK(cudaStreamCreateWithFlags(&c->s_plan, cudaStreamNonBlocking));
    for (int s = 0; s < HOST_SEGMENTS; ++s) {
        if (!c->ev_in[s]) CK(cudaEventCreateWithFlags(&c->ev_in[s], cudaEventDisableTiming));
        if (!c->ev_out[s]) CK(cudaEventCreateWithFlags(&c->ev_out[s], cudaEventDisableTiming));
    }
    if (!c->h_seg_ctl) CK(cudaMallocHost((void **)&c->h_seg_ctl, sizeof(rk::Ctl) * HOST_SEGMENTS));
    return RECON_OK;
}

// End to end: the batch is cut into up to HOST_SEGMENTS runs of consecutive
// tiles with about equal pixel counts. A segment's host-to-device copies are
// queued on one stream a segment ahead of its use; the segment is planned (the
// learned schedule's feature pass, on a side stream, once its inputs are in)
// and launched on the context stream behind the segment before it, so the
// device runs the segments back to back while the host plans the next one.
// Each segment's control word is copied to pinned memory right after its
// kernel; the host checks it when the segment is done and only then queues
// that segment's results back to the caller on a third stream.
extern "C" int recon_batch_host(recon_ctx *c, const recon_tile *tiles, int n)
{
    if (!c || !tiles || n < 1) return RECON_EINVAL;
    for (int t = 0; t < n; ++t)
        if (!tile_ok(tiles[t])) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    size_t total = 0;
    std::vector<size_t> off(n);
    for (int t = 0; t < n; ++t) {
        off[t] = total;
        total += align_up((size_t)tiles[t].H * (size_t)tiles[t].W, 256);
    }
    if (c->cap_img < 2 * total) {
        CK(cudaStreamSynchronize(c->stream));
        drop_graph(c);
    }
    int rc = grow(&c->d_img, &c->cap_img, 2 * total);
    if (rc) return rc;
    if ((rc = ensure_pipeline(c))) return rc;
    // the previous call's copies out of d_img are finished (that call waited)
    std::vector<recon_tile> dt(n);
    for (int t = 0; t < n; ++t) {
        dt[t] = tiles[t];
        dt[t].I = c->d_img + off[t];
        dt[t].J = c->d_img + total + off[t];
        dt[t].pitch = tiles[t].W;
    }
    // segment boundaries: cut when a segment reaches total / HOST_SEGMENTS pixels
    const int nseg_max = total >= ((size_t)256 << 20) ? HOST_SEGMENTS : 1;
    std::vector<int> seg_end;
    {
        size_t acc = 0;
        for (int t = 0; t < n; ++t) {
            acc += (size_t)tiles[t].H * tiles[t].W;
            const size_t goal = total / (size_t)nseg_max * (seg_end.size() + 1);
            if (t == n - 1 || ((int)seg_end.size() + 1 < nseg_max && acc >= goal)) seg_end.push_back(t + 1);
        }
    }
    const int nseg = (int)seg_end.size();
    auto first = [&](int s) { return s ? seg_end[s - 1] : 0; };
    auto queue_inputs = [&](int s) -> int {
        for (int t = first(s); t < seg_end[s]; ++t) {
            const recon_tile &T = tiles[t];
            CK(copy_rows(c->d_img + off[t], T.W, T.I, T.pitch, T.W, T.H, cudaMemcpyHostToDevice, c->s_h2d));
            if (T.op != RECON_OP_FILL_HOLES)   // a FillHoles tile's J is output only
                CK(copy_rows(dt[t].J, T.W, T.J, T.pitch, T.W, T.H, cudaMemcpyHostToDevice, c->s_h2d));
        }
        CK(cudaEventRecord(c->ev_in[s], c->s_h2d));
        return RECON_OK;
    };
    const unsigned fl = c->flags;
    auto launch = [&](int s) -> int {
        const int t0 = first(s), ns = seg_end[s] - t0;
        std::vector<int> lv, lo;
        const int *var = nullptr, *ord = nullptr;
        if ((fl & RECON_FLAG_LEARNED) && c->sched && recon_sched_has_model(c->sched)) {
            CK(cudaStreamWaitEvent(c->s_plan, c->ev_in[s], 0));
            const int prc = recon_sched_plan(c->sched, dt.data() + t0, ns, c->sms, c->s_plan, &lv, &lo);
            if (prc != RECON_OK) return prc;
            var = lv.data();
            ord = lo.data();
        }
        CK(cudaStreamWaitEvent(c->stream, c->ev_in[s], 0));
        const int brc = batch_impl(c, dt.data() + t0, ns, var, ord);
        if (brc != RECON_OK) return brc;
        CK(cudaMemcpyAsync(&c->h_seg_ctl[s], c->d_ctl, sizeof(rk::Ctl), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaEventRecord(c->ev_out[s], c->stream));
        return RECON_OK;
    };
    c->flags = (fl & ~RECON_FLAG_SYNC) | (nseg > 1 ? RECON_FLAG_NO_GRAPH : 0u);
    int err_tile = -1, abort_code = 0;
    rc = queue_inputs(0);
    if (rc == RECON_OK && nseg > 1) rc = queue_inputs(1);
    if (rc == RECON_OK) rc = launch(0);
    for (int s = 0; s < nseg && rc == RECON_OK; ++s) {
        if (s + 2 < nseg) rc = queue_inputs(s + 2);
        if (rc == RECON_OK && s + 1 < nseg) rc = launch(s + 1);   // queued behind segment s
        if (rc != RECON_OK) break;
        cudaError_t e = cudaEventSynchronize(c->ev_out[s]);
        if (e != cudaSuccess) { rc = cuda_status(e); break; }
        const rk::Ctl &h = c->h_seg_ctl[s];
        if (h.abort || h.err_tile != INT_MAX) {   // this segment failed: its results stay on the device
            abort_code = h.abort;
            err_tile = h.err_tile == INT_MAX ? -1 : first(s) + h.err_tile;   // in the caller's indexing
            rc = h.abort ? RECON_ETIMEOUT : RECON_EMARKER;
            break;
        }
        for (int t = first(s); t < seg_end[s] && rc == RECON_OK; ++t) {
            const recon_tile &T = tiles[t];
            rc = cuda_status(copy_rows(T.J, T.pitch, dt[t].J, T.W, T.W, T.H, cudaMemcpyDeviceToHost, c->s_d2h));
        }
    }
    c->flags = fl;
    const cudaError_t e0 = cudaStreamSynchronize(c->stream);
    const cudaError_t e1 = cudaStreamSynchronize(c->s_h2d), e2 = cudaStreamSynchronize(c->s_d2h);
    c->last_err_tile = err_tile;
    c->last_abort = abort_code;
    c->host_status = 1;
    if (rc != RECON_OK) return rc;
    if (e0 != cudaSuccess) return cuda_status(e0);
    if (e1 != cudaSuccess) return cuda_status(e1);
    return cuda_status(e2);
}

extern "C" int recon_run_host(recon_ctx *c, const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    recon_tile t;
    t.I = I; t.J = J; t.H = H; t.W = W; t.pitch = W; t.conn = conn; t.op = RECON_OP_DILATE;
    return recon_batch_host(c, &t, 1);
}

// ---------------------------------------------------------------------------
// learned cost model entry points

extern "C" int recon_features(recon_ctx *c, const recon_tile *tiles, int n, float *feat)
{
    if (!c || !tiles || n < 1 || !feat) return RECON_EINVAL;
    for (int t = 0; t < n; ++t)
        if (!tile_ok(tiles[t])) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<rl_tile> rt(n);
    for (int t = 0; t < n; ++t)
        rt[t] = rl_tile{tiles[t].I, tiles[t].J, tiles[t].H, tiles[t].W, tiles[t].pitch, tiles[t].op};
    const size_t sb = rl_features_scratch(n), hb = rl_features_stage(n);
    void *d = nullptr, *h = nullptr;
    CK(cudaMalloc(&d, sb));
    cudaError_t e = cudaMallocHost(&h, hb);
    if (e == cudaSuccess) e = rl_features(rt.data(), n, d, sb, feat, nullptr, c->sms, c->stream, h, hb);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (h) cudaFreeHost(h);
    return cuda_status(e);
}

extern "C" int recon_mlp_forward(recon_ctx *c, const float *theta, const float *X, int n, float *Y)
{
    if (!c || !theta || !X || !Y || n < 1) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(rl_forward(theta, X, n, Y, c->stream));
    if (c->flags & RECON_FLAG_SYNC) CK(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

extern "C" int recon_mlp_grad(recon_ctx *c, const float *theta, const float *X, const float *T, const int *idx,
                              int n, float *grad, float *loss)
{
    if (!c || !theta || !X || !T || !grad || n < 1) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(rl_grad(theta, X, T, idx, n, grad, loss, c->stream));
    if (c->flags & RECON_FLAG_SYNC) CK(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

extern "C" int recon_mlp_adam(recon_ctx *c, float *theta, float *grad, float *m, float *v, int t, float lr)
{
    if (!c || !theta || !grad || !m || !v || t < 1 || !(lr > 0.0f)) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(rl_adam(theta, grad, m, v, t, lr, c->stream));
    if (c->flags & RECON_FLAG_SYNC) CK(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

static uint64_t sm64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

extern "C" int recon_mlp_train_resume(recon_ctx *c, float *theta, float *adam_mv, int *step, int epoch0,
                                      const float *X, const float *T, int n, int epochs, int batch, float lr,
                                      uint64_t seed, float *epoch_loss)
{
    if (!c || !theta || !adam_mv || !step || *step < 0 || epoch0 < 0 || !X || !T || n < 1 || epochs < 1 ||
        batch < 1 || !(lr > 0.0f))
        return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    float *m = adam_mv, *v = adam_mv + MLP_NPARAMS, *g = nullptr, *dl = nullptr;
    int *didx = nullptr;
    cudaError_t e = cudaMalloc((void **)&g, sizeof(float) * MLP_NPARAMS);
    if (e == cudaSuccess) e = cudaMemsetAsync(g, 0, sizeof(float) * MLP_NPARAMS, c->stream);
    if (e == cudaSuccess) e = cudaMalloc((void **)&didx, sizeof(int) * (size_t)n * 2);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dl, sizeof(float) * epochs);
    if (e == cudaSuccess) e = cudaMemsetAsync(dl, 0, sizeof(float) * epochs, c->stream);
    std::vector<int> perm(n);
    int t = *step;
    const int nbatches = (n + batch - 1) / batch;
    for (int k = 0; k < epochs && e == cudaSuccess; ++k) {
        const int ep = epoch0 + k;   // the shuffle depends on the absolute epoch, so a resumed run repeats it
        // Fisher-Yates shuffle driven by SplitMix64 outputs of (seed, epoch)
        for (int i = 0; i < n; ++i) perm[i] = i;
        uint64_t st = sm64(seed ^ sm64((uint64_t)ep + 1));
        for (int i = n - 1; i > 0; --i) {
            st = sm64(st);
            const int j = (int)(st % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        int *buf = didx + (size_t)(k & 1) * n;  // double-buffered: the copy of epoch e+1 cannot race epoch e
        e = cudaMemcpyAsync(buf, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // perm is pageable and reused
        for (int s = 0; s < n && e == cudaSuccess; s += batch) {
            const int nb = std::min(batch, n - s);
            e = rl_grad(theta, X, T, buf + s, nb, g, dl + k, c->stream);
            if (e == cudaSuccess) e = rl_adam(theta, g, m, v, ++t, lr, c->stream);
        }
    }
    if (e == cudaSuccess && epoch_loss) {
        e = cudaMemcpyAsync(epoch_loss, dl, sizeof(float) * epochs, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        for (int i = 0; i < epochs; ++i) epoch_loss[i] /= (float)nbatches;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) *step = t;
    cudaFree(g);
    cudaFree(didx);
    cudaFree(dl);
    return cuda_status(e);
}

extern "C" int recon_mlp_train(recon_ctx *c, float *theta, const float *X, const float *T, int n, int epochs,
                               int batch, float lr, uint64_t seed, float *epoch_loss)
{
    if (!c) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    float *mv = nullptr;
    CK(cudaMalloc((void **)&mv, sizeof(float) * MLP_NPARAMS * 2));
    int step = 0;
    cudaError_t e = cudaMemsetAsync(mv, 0, sizeof(float) * MLP_NPARAMS * 2, c->stream);
    int rc = e == cudaSuccess ? recon_mlp_train_resume(c, theta, mv, &step, 0, X, T, n, epochs, batch, lr, seed,
                                                       epoch_loss)
                              : cuda_status(e);
    cudaFree(mv);
    return rc;
}

extern "C" int recon_sched_set_model(recon_ctx *c, const float *theta, const float *norm, int variant_a,
                                     int variant_b)
{
    if (!c) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    const int rc = recon_sched_set(c->sched, theta, norm, variant_a, variant_b);
    if (rc == RECON_OK) drop_graph(c);
    return rc;
}

extern "C" int recon_sched_plan_batch(recon_ctx *c, const recon_tile *tiles, int n, int *variant, int *order,
                                      float *pred)
{
    if (!c || !tiles || n < 1 || !variant || !order) return RECON_EINVAL;
    for (int t = 0; t < n; ++t)
        if (!tile_ok(tiles[t])) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    std::vector<int> lv, lo;
    const int rc = recon_sched_plan(c->sched, tiles, n, c->sms, c->stream, &lv, &lo);
    if (rc) return rc;
    std::copy(lv.begin(), lv.end(), variant);
    std::copy(lo.begin(), lo.end(), order);
    if (pred) {
        const std::vector<float> &p = recon_sched_last_pred(c->sched);
        std::copy(p.begin(), p.begin() + 2 * (size_t)n, pred);
    }
    return RECON_OK;
}

// ---------------------------------------------------------------------------
// autotuner: times candidate (block height, bands, first-visit scan pairs) on
// the caller's batch and keeps the fastest. Results never differ (R is unique),
// only the time does.

// The autotuner's cache key of a batch: size bucket = round(log2(mean tile
// area)), the set of connectivities (bit 0: 4, bit 1: 8), and the marker
// class (1 when most of the batch's marker pixels are 0, as for border-seeded
// markers such as FillHoles; 0 otherwise), from the cost model's feature pass.
static int tune_key(recon_ctx *c, const recon_tile *tiles, int n, std::tuple<int, int, int> *key)
{
    double area = 0.0;
    int conns = 0;
    for (int t = 0; t < n; ++t) {
        area += (double)tiles[t].H * tiles[t].W;
        conns |= tiles[t].conn == 4 ? 1 : 2;
    }
    float *feat = nullptr;
    CK(cudaMalloc((void **)&feat, sizeof(float) * RECON_NFEAT * (size_t)n));
    int rc = recon_features(c, tiles, n, feat);
    std::vector<float> h((size_t)RECON_NFEAT * n);
    if (rc == RECON_OK && cudaMemcpy(h.data(), feat, sizeof(float) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = RECON_ECUDA;
    cudaFree(feat);
    if (rc) return rc;
    double zero = 0.0;
    for (int t = 0; t < n; ++t) zero += (double)h[(size_t)t * RECON_NFEAT + 17] * tiles[t].H * tiles[t].W;
    const int bucket = (int)std::lround(std::log2(std::max(area / n, 1.0)));
    *key = std::make_tuple(bucket, conns, zero >= 0.5 * area ? 1 : 0);
    return RECON_OK;
}

extern "C" int recon_autotune_cache(recon_ctx *c, int *entries, int max_entries)
{
    if (!c || max_entries < 0 || (max_entries > 0 && !entries)) return -RECON_EINVAL;
    int i = 0;
    for (const auto &kv : c->tune_cache) {
        if (i >= max_entries) break;
        int *e = entries + 7 * i++;
        e[0] = std::get<0>(kv.first); e[1] = std::get<1>(kv.first); e[2] = std::get<2>(kv.first);
        for (int k = 0; k < 4; ++k) e[3 + k] = kv.second[k];
    }
    return (int)c->tune_cache.size();
}

extern "C" int recon_autotune_cache_load(recon_ctx *c, const int *entries, int count)
{
    if (!c || count < 0 || (count > 0 && !entries)) return RECON_EINVAL;
    for (int i = 0; i < count; ++i) {
        const int *e = entries + 7 * i;
        if ((e[3] != 32 && e[3] != 64 && e[3] != 128 && e[3] != 256) || (e[4] != 1 && e[4] != 2 && e[4] != 4) || e[5] < -1 ||
            e[5] > 64 || e[6] < 0 || e[6] > (1 << 20) || e[1] < 1 || e[1] > 3 || (e[2] != 0 && e[2] != 1))
            return RECON_EINVAL;
    }
    if (count == 0) c->tune_cache.clear();
    for (int i = 0; i < count; ++i) {
        const int *e = entries + 7 * i;
        c->tune_cache[std::make_tuple(e[0], e[1], e[2])] = std::vector<int>{e[3], e[4], e[5], e[6]};
    }
    return RECON_OK;
}

extern "C" int recon_autotune(recon_ctx *c, const recon_tile *tiles, int n, int reps, int *best)
{
    if (!c || !tiles || n < 1 || !best || reps < 1 || reps > 100) return RECON_EINVAL;
    for (int t = 0; t < n; ++t)
        if (!tile_ok(tiles[t])) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    std::tuple<int, int, int> key;
    int krc = tune_key(c, tiles, n, &key);
    if (krc) return krc;
    c->tune_from_cache = 0;
    const auto hit = c->tune_cache.find(key);
    if (hit != c->tune_cache.end()) {   // this kind of batch was tuned before: no trials
        c->bh = hit->second[0]; c->bands = hit->second[1]; c->k = hit->second[2]; c->scan_gain = hit->second[3];
        for (int k = 0; k < 4; ++k) best[k] = hit->second[k];
        c->tune_from_cache = 1;
        drop_graph(c);
        return RECON_OK;
    }
    // backup of every marker so each trial starts from the same J
    size_t total = 0;
    std::vector<size_t> off(n);
    for (int t = 0; t < n; ++t) {
        off[t] = total;
        total += align_up((size_t)tiles[t].H * (size_t)tiles[t].pitch, 256);
    }
    uint8_t *bk = nullptr;
    CK(cudaMalloc((void **)&bk, total));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < n && e == cudaSuccess; ++t)
        e = cudaMemcpyAsync(bk + off[t], tiles[t].J, (size_t)tiles[t].H * tiles[t].pitch, cudaMemcpyDeviceToDevice,
                            c->stream);
    const int save_bh = c->bh, save_bands = c->bands, save_k = c->k, save_gain = c->scan_gain;
    const unsigned save_flags = c->flags;
    c->flags &= ~RECON_FLAG_SYNC;
    float best_ms = 1e30f;
    int bb[4] = {save_bh, save_bands, save_k, save_gain};
    int rc = RECON_OK;
    const int BHs[3] = {32, 64, 128}, BANDS[2] = {2, 4}, KS[3] = {0, 1, 2}, GAINS[2] = {0, 2048};
    for (int a = 0; a < 3 && e == cudaSuccess && rc == RECON_OK; ++a)
        for (int b = 0; b < 2 && e == cudaSuccess && rc == RECON_OK; ++b)
            for (int k = 0; k < 3 && e == cudaSuccess && rc == RECON_OK; ++k)
            for (int gi = 0; gi < 2 && e == cudaSuccess && rc == RECON_OK; ++gi) {
                c->bh = BHs[a]; c->bands = BANDS[b]; c->k = KS[k]; c->scan_gain = GAINS[gi];
                drop_graph(c);
                float sum = 0.0f;
                for (int r = 0; r < reps + 1 && e == cudaSuccess && rc == RECON_OK; ++r) {
                    for (int t = 0; t < n && e == cudaSuccess; ++t)
                        e = cudaMemcpyAsync(tiles[t].J, bk + off[t], (size_t)tiles[t].H * tiles[t].pitch,
                                            cudaMemcpyDeviceToDevice, c->stream);
                    if (e != cudaSuccess) break;
                    rc = batch_impl(c, tiles, n, nullptr, nullptr);
                    if (rc == RECON_OK) rc = recon_sync(c);
                    float ms = 0.0f;
                    if (rc == RECON_OK) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
                    if (r > 0) sum += ms;   // the first run warms up (and builds the graph)
                }
                if (rc == RECON_OK && e == cudaSuccess && sum / reps < best_ms) {
                    best_ms = sum / reps;
                    bb[0] = BHs[a]; bb[1] = BANDS[b]; bb[2] = KS[k]; bb[3] = GAINS[gi];
                }
            }
    for (int t = 0; t < n && e == cudaSuccess; ++t)
        e = cudaMemcpyAsync(tiles[t].J, bk + off[t], (size_t)tiles[t].H * tiles[t].pitch, cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(bk);
    c->flags = save_flags;
    drop_graph(c);
    if (rc != RECON_OK || e != cudaSuccess) {
        c->bh = save_bh; c->bands = save_bands; c->k = save_k; c->scan_gain = save_gain;
        return rc != RECON_OK ? rc : cuda_status(e);
    }
    c->bh = bb[0]; c->bands = bb[1]; c->k = bb[2]; c->scan_gain = bb[3];
    best[0] = bb[0]; best[1] = bb[1]; best[2] = bb[2]; best[3] = bb[3];
    c->tune_cache[key] = std::vector<int>{bb[0], bb[1], bb[2], bb[3]};
    return RECON_OK;
}

// ---------------------------------------------------------------------------
// diagnostics

extern "C" int recon_sync_for(recon_ctx *c, int timeout_ms)
{
    if (!c || timeout_ms < 0) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    for (long waited_us = 0;; waited_us += 200) {
        const cudaError_t q = cudaStreamQuery(c->stream);
        if (q == cudaSuccess) return recon_sync(c);
        if (q != cudaErrorNotReady) return cuda_status(q);
        if (waited_us / 1000 >= timeout_ms) return RECON_ETIMEOUT;
        struct timespec ts = {0, 200000};
        nanosleep(&ts, nullptr);
    }
}

extern "C" int recon_trace(recon_ctx *c, unsigned *out, int n)
{
    if (!c || !out || n < 0) return -1;
    if (!c->h_trace) return 0;
    const int m = (int)std::min((size_t)n, c->cap_trace);
    for (int i = 0; i < m; ++i) out[i] = ((volatile unsigned *)c->h_trace)[i];
    return m;
}

// ---------------------------------------------------------------------------
// distance transform (recon_dt.cu)

extern "C" int recon_dt(recon_ctx *c, const uint8_t *B, uint32_t *d2, int32_t *site, int H, int W)
{
    if (!c || !B || !d2 || H < 1 || W < 1 || H > 32768 || W > 32768) return RECON_EINVAL;
    if ((long long)H * W > 0x7FFFFFFFll) return RECON_EINVAL;
    CK(cudaSetDevice(c->device));
    const size_t n = (size_t)H * W;
    const size_t need = dt_scratch_bytes(H, W);
    if (c->cap_dt < need || (!site && c->cap_dt_site < n) || !c->h_dt_cnt) {
        CK(cudaStreamSynchronize(c->stream));
        int rc;
        if ((rc = grow(&c->d_dt, &c->cap_dt, need))) return rc;
        if (!site && (rc = grow(&c->d_dt_site, &c->cap_dt_site, n))) return rc;
        if (!c->h_dt_cnt) CK(cudaMallocHost((void **)&c->h_dt_cnt, 4 * sizeof(unsigned)));
    }
    int *s = site ? (int *)site : c->d_dt_site;
    const int rc = dt_run(B, H, W, s, (unsigned *)d2, c->d_dt, c->h_dt_cnt, 8 * c->sms, c->stream, &c->dt_levels);
    if (rc == DT_ECUDA) return RECON_ECUDA;
    CK(cudaStreamSynchronize(c->stream));
    return rc == DT_ELIMIT ? RECON_ETIMEOUT : RECON_OK;
}

extern "C" int recon_dt_levels(recon_ctx *c)
{
    return c ? c->dt_levels : -1;
}
