/*
 * recon.h -- C ABI of the GB300 (sm_103a) grayscale morphological
 * reconstruction library.
 *
 * Operation (Table II, "Morphological Reconstruction": flood-fill of a marker
 * image J limited by a mask image I, 4- or 8-connected, after Vincent 1993):
 *     R = lim_n delta_I^n(J),   delta_I(X)(p) = min( max_{q in N(p)} X(q), I(p) ),
 * N(p) = p and its 4 or 8 neighbours inside the image. R is computed by the
 * irregular wavefront propagation pattern (Sec. II-B, Algorithm 1) in the
 * hybrid form of Sec. V-C (irregular operations): raster / anti-raster scans
 * first, then queue-driven propagation. R is unique, so every schedule returns
 * the same bytes.
 *
 * Two more operations run on the same engine (recon_tile.op):
 *   reconstruction by erosion, the dual: R = lim_n eps_I^n(J),
 *     eps_I(X)(p) = max( min_{q in N(p)} X(q), I(p) ), for J >= I;
 *   FillHoles (Table II: fill the holes of image objects by a flood of the
 *     background from selected points, here the image border): the erosion of
 *     the marker "I on the one-pixel image border, 255 inside" under I, which
 *     equals complement -> border-seeded reconstruction by dilation ->
 *     complement. A pixel the border flood cannot reach is raised to the
 *     lowest level that encloses it.
 * Both are the dilation run on complemented values (255 - v): the kernels
 * complement pixels as they load and store them, and treat pixels outside the
 * image as absent, so no complemented copy of I or J is ever written.
 *
 * Images are uint8, row-major, `pitch` bytes between rows (pitch >= W). All
 * image pointers handed to recon_run / recon_batch are DEVICE pointers owned by
 * the caller; J is read as the marker and overwritten in place with R (as D is
 * updated in place in Algorithm 1). The library owns only its scratch memory.
 *
 * Calls are asynchronous on the context's stream: the return value is the
 * argument-check status; the device status (marker check, bounded waits) is
 * returned by recon_sync, or at once when the context has RECON_FLAG_SYNC.
 * No function aborts, traps or spins without a bound; errors are status codes.
 * A context is used by one host thread at a time.
 */
#ifndef RECON_H
#define RECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct recon_ctx recon_ctx;

/* Status codes. */
enum {
    RECON_OK = 0,
    RECON_EINVAL = 1,    /* bad argument (null pointer, size, conn not 4/8, pitch < W) */
    RECON_EMARKER = 2,   /* the marker violates its operation's precondition at some
                            pixel (dilation: J > I; erosion: J < I). J of that tile
                            is then left in an unspecified state. */
    RECON_ENOMEM = 3,    /* device or host allocation failed */
    RECON_ECUDA = 4,     /* a CUDA runtime call failed */
    RECON_ETIMEOUT = 5   /* a bounded device-side wait ran out; outputs unspecified */
};

/* Flags for recon_init. */
#define RECON_FLAG_SYNC      0x1u  /* each call waits for the device and returns its status */
#define RECON_FLAG_NO_CHECK  0x2u  /* skip the J <= I check (caller guarantees it) */
#define RECON_FLAG_LEARNED   0x4u  /* recon_batch: the cost model picks variant and order */
#define RECON_FLAG_NO_GRAPH  0x8u  /* recon_batch: never capture / replay a CUDA graph */

/* Operations (recon_tile.op). */
enum {
    RECON_OP_DILATE = 0,     /* reconstruction by dilation (Table II), J <= I */
    RECON_OP_ERODE = 1,      /* reconstruction by erosion (the dual), J >= I */
    RECON_OP_FILL_HOLES = 2  /* FillHoles (Table II) of I; J's input is ignored and
                                J receives the result */
};

/* One tile of a batch: device pointers, caller-owned. */
typedef struct {
    const uint8_t *I;   /* mask, H x W, row stride `pitch` bytes */
    uint8_t *J;         /* marker in, R out (in place) */
    int H, W, pitch;    /* H, W >= 1; pitch >= W */
    int conn;           /* 4 or 8 */
    int op;             /* RECON_OP_*; 0 (dilation) when zero-initialised */
} recon_tile;

/* Creates a context on CUDA device `device`: the library's scratch for the
 * state Algorithm 1 (Sec. II-B) keeps beside the image D it updates in place --
 * the wavefront queues' overflow areas, per-block state and work list, tile
 * descriptors and status words -- plus the cost model. It owns no image data.
 * `cuda_stream` is a cudaStream_t
 * (NULL: the context creates its own non-blocking stream). flags: RECON_FLAG_*.
 * The environment variables RECON_BLOCK_H, RECON_SWEEPS, RECON_BANDS,
 * RECON_GRID, RECON_WAIT_NS, RECON_ORDER, RECON_TMA, RECON_REVISIT_SCANS and
 * RECON_SCAN_GAIN, when set, override the matching RECON_P_* defaults (decimal
 * integers; an invalid value makes the call return RECON_EINVAL).
 * Returns RECON_OK and *ctx, or an error code with *ctx = NULL. */
int recon_init(recon_ctx **ctx, int device, void *cuda_stream, unsigned flags);

/* Reconstructs one tile (Table II; Algorithm 1 with the hybrid scan + queue
 * schedule of Sec. V-C). I, J: device pointers, pitch = W. J <- R in place. */
int recon_run(recon_ctx *ctx, const uint8_t *I, uint8_t *J, int H, int W, int conn);

/* recon_run for any operation: op = RECON_OP_DILATE, RECON_OP_ERODE (J >= I,
 * J <- the reconstruction by erosion) or RECON_OP_FILL_HOLES (J <- FillHoles(I);
 * J need not be initialised). Device pointers, pitch = W. */
int recon_run_op(recon_ctx *ctx, const uint8_t *I, uint8_t *J, int H, int W, int conn, int op);

/* Reconstructs n independent tiles of any sizes in one persistent launch
 * (tiles are processed concurrently, as the 4K x 4K tiles of Sec. V are).
 * `tiles` is a HOST array of n descriptors with device image pointers.
 * Tiles must not overlap in memory. With RECON_FLAG_LEARNED the cost model
 * chooses each tile's variant and the packing order (never the pixel values).
 * 1 <= n <= 2^28 (RECON_EINVAL otherwise).
 * On a device error, recon_last_error_tile names the first failing tile. */
int recon_batch(recon_ctx *ctx, const recon_tile *tiles, int n);

/* As recon_batch with an explicit schedule. variant[t] = -1: scan pairs to
 * stability, no queue; otherwise variant[t] = k + 256 * g: a block runs k
 * raster + anti-raster pairs on its first visit, then (g > 0) keeps scanning,
 * on first visits and revisits, while a pair still raises at least 64 * g
 * pixels, then switches to its queue phase (0 <= k <= 64, 0 <= g <= 4096).
 * order[] = permutation of 0..n-1 giving the packing order. Either array may
 * be NULL (context defaults). */
int recon_batch_ex(recon_ctx *ctx, const recon_tile *tiles, int n, const int *variant,
                   const int *order);

/* End-to-end form: I, J are HOST pointers (pinned or pageable), pitch = W.
 * Copies in, reconstructs, copies R back into J, and waits. */
int recon_run_host(recon_ctx *ctx, const uint8_t *I, uint8_t *J, int H, int W, int conn);

/* End-to-end batch: tiles[].I / tiles[].J are HOST pointers; waits. The J of
 * a FillHoles tile is only written. A batch of 256 Mpx or more is cut into
 * four runs of consecutive tiles with about equal pixel counts, processed as
 * a pipeline: a run's inputs are copied in one run ahead of its use, each run
 * is planned (RECON_FLAG_LEARNED) while the run before it is reconstructed
 * and then queued behind it, and a run's results are copied back while the
 * next run is reconstructed (copies from pinned host memory overlap the
 * reconstruction). Each run's device status is checked before its results are
 * copied back; on an error no later run's results are copied back, the call
 * returns once the runs already queued have finished, and
 * recon_last_error_tile (and recon_sync) report the failing tile by its index
 * in `tiles`. recon_get_work and recon_last_kernel_ms describe the last run
 * that was launched. */
int recon_batch_host(recon_ctx *ctx, const recon_tile *tiles, int n);

/* Waits for the context's stream; returns the device status of the last call. */
int recon_sync(recon_ctx *ctx);

/* Index of the first tile of the last batch that failed, or -1. Syncs. */
int recon_last_error_tile(recon_ctx *ctx);

/* Frees the context and its scratch memory (the queue and work-list state of
 * Algorithm 1, Sec. II-B; see recon_init) after waiting for its stream. The
 * caller's images are not touched. NULL is accepted. */
int recon_free(recon_ctx *ctx);

/* Static description of a status code: the argument checks, the precondition
 * of the operation (Table II's reconstruction needs J <= I; its dual J >= I),
 * allocation and runtime failures, and the bounded waits of the wavefront
 * propagation (Algorithm 1's loop "while the queue is not empty" runs under
 * iteration and time limits). The string is static; never NULL. */
const char *recon_strerror(int status);

/* Tunables (recon_set_param / recon_get_param). */
enum {
    RECON_P_BLOCK_H = 1,     /* block height in rows: 32, 64, 128 (default) or 256 (block width is 128) */
    RECON_P_SWEEPS = 2,      /* default variant: scan pairs before the queue; -1 = scans only */
    RECON_P_GRID = 3,        /* CTAs of the persistent launch; 0 = SMs x occupancy */
    RECON_P_BANDS = 4,       /* warps that scan a block concurrently (1, 2 or 4) */
    RECON_P_WAIT_NS = 5,     /* limit of one device-side idle wait, ns (default 2e9) */
    RECON_P_ORDER = 6,       /* default packing order: 0 = as given, 1 = largest area first */
    RECON_P_TEST_STALL = 7,  /* testing: 1 = add a phantom unit of work that never ends,
                                so the bounded wait must run out (RECON_ETIMEOUT) */
    RECON_P_TMA = 8,         /* 1 (default): tiles whose rows and bases are 16-byte aligned
                                are loaded into shared memory by TMA; 0 = plain loads */
    RECON_P_TRACE = 9,       /* diagnostics: 1 = kernels record per-warp progress in mapped
                                host memory (read with recon_trace, even while running) */
    RECON_P_LAST_ABORT = 10, /* read-only: which device-side bound ran out in the last call
                                (0 = none; 1 rerun, 2 overflow, 3 levels, 4 scans, 5 unused,
                                6 notify, 7 unused, 8 idle wait, 9 ring push, 10 TMA) */
    RECON_P_REVISIT_SCANS = 11, /* scan pairs a block runs when revisited (after a neighbour
                                   raised its halo) before its queue phase; default 0 */
    RECON_P_SCAN_GAIN = 12,     /* default adaptive scan-to-queue switch: after its fixed scan
                                   pairs a block keeps scanning while a pair raises at least this
                                   many pixels (first visits and revisits); 0 = off; default 2048 */
    RECON_P_TUNE_FROM_CACHE = 13 /* read-only: 1 if the last recon_autotune call took its
                                   result from the cache instead of timing trials */
};
int recon_set_param(recon_ctx *ctx, int key, int64_t value);
int64_t recon_get_param(recon_ctx *ctx, int key);

/* Work counters of one tile in the last call (propagation work measured by
 * the method itself: what the cost model learns from). */
typedef struct {
    uint64_t visits;      /* block visits (first visits + revisits after a halo change) */
    uint64_t scan_rows;   /* rows processed by raster / anti-raster scans */
    uint64_t pops;        /* queue entries processed */
    uint64_t seeds;       /* seeding passes over a block */
    uint64_t levels;      /* wavefront levels processed (sequential steps of the queue phase) */
    uint64_t busy_ns;     /* sum over block visits of the time a CTA spent on them */
    uint64_t phase_ns[6]; /* that time by phase: load, scans, seeding, queue,
                             write-back + notification, and the work fetch before it */
} recon_work;

/* Waits at most timeout_ms for the context's stream: the device status as
 * recon_sync when it finished in time, RECON_ETIMEOUT (nothing changed) if not. */
int recon_sync_for(recon_ctx *ctx, int timeout_ms);

/* Diagnostics (RECON_P_TRACE = 1): copies up to n progress words of the last
 * launch, one per warp: (code << 24) | block index. Readable while a kernel is
 * still running. Returns the number of words copied. */
int recon_trace(recon_ctx *ctx, unsigned *out, int n);

/* Copies the counters of the last call's first n tiles into out[] (syncs). */
int recon_get_work(recon_ctx *ctx, recon_work *out, int n);

/* Device time of the last call's persistent kernel in ms (CUDA events on the
 * context's stream; syncs). */
int recon_last_kernel_ms(recon_ctx *ctx, float *ms);


/* Allocation-free reconstruction of one tile (the paper has no counterpart:
 * this serves callers that must not allocate device or pinned memory once
 * running -- e.g. a plugin whose host framework owns all device memory through
 * its own pool, or a latency-critical pipeline that cannot accept the implicit
 * synchronisation an allocation may cause). No context is needed and nothing
 * is allocated: the scratch space is one 11 MiB array compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits. I, J: device pointers, row stride = W, J <- R in place; runs on
 * `cuda_stream` (NULL = the default stream) of the current device and blocks
 * the calling host thread until that stream has finished the call (it waits on
 * that stream only; the descriptor upload from host stack memory and the status
 * read-back are ordered on it too). The first call on each device looks up the array's device address;
 * make that first call outside any stream capture. Limits: at most 4096 blocks
 * of 64 x 128 pixels (e.g. 4096 x 8192); larger inputs return RECON_EINVAL.
 * Every call reuses the same array (cleared where it must start at zero), so
 * calls that overlap on the GPU race: issue them one at a time. */
int recon_run_noalloc(const uint8_t *I, uint8_t *J, int H, int W, int conn, void *cuda_stream);

/* Autotuner: times every candidate block height {32, 64, 128} x bands
 * {2, 4} x first-visit scan pairs {0, 1, 2} x adaptive scan gain {0, 2048} on
 * this batch (each `reps` times after one warm-up run, J restored from a
 * device backup before every run), installs the fastest in the context and
 * writes it to best[4] = {block height, bands, scan pairs, scan gain}. J
 * holds its original marker on return. The paper tunes its scan-to-queue
 * switch point the same way (Sec. V-C). */
int recon_autotune(recon_ctx *ctx, const recon_tile *tiles, int n, int reps, int *best);
/* The autotuner keeps its results in the context, keyed by the batch's size
 * bucket (round(log2 of the mean tile area)), its connectivities (bit 0: 4,
 * bit 1: 8) and its marker class (1 when most marker pixels are 0, as for
 * border-seeded markers; 0 otherwise). A recon_autotune call on a batch whose
 * key is cached installs the cached result without timing anything
 * (RECON_P_TUNE_FROM_CACHE reads 1 afterwards).
 * recon_autotune_cache copies up to max_entries entries of 7 ints {bucket,
 * connectivities, marker class, block height, bands, scan pairs, scan gain}
 * into entries (HOST) and returns how many the cache holds (negative status on
 * bad arguments). recon_autotune_cache_load adds such entries (count = 0
 * clears the cache); it validates every entry first and returns RECON_EINVAL,
 * changing nothing, if one is out of range. Together they persist the cache. */
int recon_autotune_cache(recon_ctx *ctx, int *entries, int max_entries);
int recon_autotune_cache_load(recon_ctx *ctx, const int *entries, int count);

/* ---- learned cost model ------------------------------------------------
 * The scheduler's analogue of the paper's performance-aware task scheduling
 * (Sec. IV, PATS: per-task speedup estimates choose where each task runs):
 * a multilayer perceptron 20 -> 64 -> 64 -> 2 (ReLU, fp32) maps per-tile
 * features to the predicted log cost of two variants; the scheduler gives each
 * tile its cheaper variant and packs tiles by decreasing predicted cost. It
 * only reorders and re-parameterises work; pixel values are never touched.
 * All float pointers below are DEVICE pointers owned by the caller, in the
 * flat parameter layout W1 (64x20), b1 (64), W2 (64x64), b2 (64), W3 (2x64),
 * b3 (2), row-major. */
#define RECON_NFEAT 20
#define RECON_MLP_NPARAMS 5634

/* Features of n tiles into feat (n x 20 fp32): [0..15] fraction of pixels with
 * (I - J) >> 4 == k, [16] fraction with I >= 100 (blob pixels), [17] fraction
 * with J == 0, [18] log2(H) / 12, [19] log2(W) / 12. One pass over I and J.
 * Erosion and FillHoles tiles are described by their complemented values (for
 * FillHoles with J = 0 inside), the dilation problem the kernel solves. Syncs. */
int recon_features(recon_ctx *ctx, const recon_tile *tiles, int n, float *feat);

/* Y (n x 2) = MLP(theta, X (n x 20)). */
int recon_mlp_forward(recon_ctx *ctx, const float *theta, const float *X, int n, float *Y);

/* Adds to grad (5634 floats) the gradient of L = 1/(2n) sum (Y - T)^2 over the
 * samples idx[0..n) (idx NULL: 0..n-1) and, when loss is not NULL, adds L to
 * *loss. The caller zeroes grad and loss first. */
int recon_mlp_grad(recon_ctx *ctx, const float *theta, const float *X, const float *T, const int *idx,
                   int n, float *grad, float *loss);

/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8), step
 * number t >= 1; grad is zeroed afterwards. */
int recon_mlp_adam(recon_ctx *ctx, float *theta, float *grad, float *m, float *v, int t, float lr);

/* Mini-batch Adam for `epochs` epochs over X (n x 20), T (n x 2), shuffled per
 * epoch by a SplitMix64-driven Fisher-Yates permutation of (seed, epoch).
 * epoch_loss (HOST, optional, `epochs` floats) receives each epoch's mean batch
 * loss. Syncs. */
int recon_mlp_train(recon_ctx *ctx, float *theta, const float *X, const float *T, int n, int epochs,
                    int batch, float lr, uint64_t seed, float *epoch_loss);

/* Resumable form of recon_mlp_train (checkpoint / resume of the cost model's
 * training). adam_mv: DEVICE, 2 * RECON_MLP_NPARAMS floats, Adam's first then
 * second moment estimates (zeros to start). *step (HOST, in/out): Adam steps
 * taken so far (0 to start). epoch0: index of the first epoch to run; the
 * mini-batch shuffle of epoch e depends only on (seed, e), so running epochs
 * [0, a) and then, from the saved theta / adam_mv / step, [a, a + b) follows
 * the same sequence of updates as running [0, a + b) at once (up to the
 * summation order of the gradient reduction). Other arguments as in
 * recon_mlp_train; epoch_loss receives `epochs` values. Syncs. */
int recon_mlp_train_resume(recon_ctx *ctx, float *theta, float *adam_mv, int *step, int epoch0,
                           const float *X, const float *T, int n, int epochs, int batch, float lr,
                           uint64_t seed, float *epoch_loss);

/* Installs a trained model for RECON_FLAG_LEARNED batches. theta and norm are
 * HOST pointers: norm = (mean_a, std_a, mean_b, std_b) de-normalising the two
 * outputs; variant_a / variant_b are the variants (as in recon_batch_ex) that
 * outputs 0 and 1 predict. */
int recon_sched_set_model(recon_ctx *ctx, const float *theta, const float *norm, int variant_a,
                          int variant_b);

/* The plan the model makes for a batch (HOST outputs): variant[n], order[n]
 * and, optionally, pred[2n] (predicted log costs). Syncs. */
int recon_sched_plan_batch(recon_ctx *ctx, const recon_tile *tiles, int n, int *variant, int *order,
                           float *pred);

/* Bounds-checked build (librecon_checks.so, built with RECON_CHECKS): the
 * reconstruction kernel checks every wavefront queue slot and pixel offset
 * before using it, counts failed checks and skips those accesses instead of
 * making them (the stand-in for a memory checker). recon_checks reports
 * *enabled (1 in that build, 0 otherwise), the number of failed checks since
 * the last reset and the where-code of the first (1: queue slot, 2: wavefront
 * pixel, 3: pushed pixel); reset != 0 clears them. Returns 0, or nonzero on
 * bad arguments or a CUDA error. */
int recon_checks(int *enabled, unsigned *violations, unsigned *first, int reset);

/* ---- distance transform (Table II) ----
 * For each foreground pixel (B != 0) of the H x W image B (device uint8,
 * pitch = W), the squared Euclidean distance to the background pixel that the
 * 8-connected irregular wavefront propagation assigns to it: Algorithm 1 with
 * elements D(p) = the nearest background pixel ("site") found so far, seeded
 * from the background pixels that touch the foreground; a foreground neighbour
 * q takes site s when (|q - s|^2, s) < (|q - site(q)|^2, site(q)).
 * d2: device uint32 H x W out (0 on background; 0xFFFFFFFF everywhere when B
 * has no background pixel). site: device int32 H x W out, index y*W + x of the
 * assigned background pixel (-1 without background), or NULL (the context then
 * keeps it in its scratch). 1 <= H, W <= 32768, H * W < 2^31.
 * Like Danielsson's vector propagation this approximates the exact Euclidean
 * transform (a pixel passes on only the site it holds); the result depends on
 * the processing order, but every site is a background pixel and no pixel has
 * an 8-neighbour holding a closer site. Runs on the context stream and waits;
 * RECON_ETIMEOUT if an iteration bound ran out. */
int recon_dt(recon_ctx *ctx, const uint8_t *B, uint32_t *d2, int32_t *site, int H, int W);

/* Wavefront levels the last recon_dt call ran (diagnostics), or -1. */
int recon_dt_levels(recon_ctx *ctx);

/* ---- device micro-benchmarks (Sec. V-C, Tables III and IV) ----
 * GB300 versions of the paper's random-access and atomic micro-benchmarks,
 * which bound the irregular (wavefront) phase. Both run on the CURRENT CUDA
 * device and its default stream, wait for completion, and return the kernel's
 * CUDA-event time in *ms. They allocate at most 8 bytes of scratch. */

/* Number of threads the micro-benchmark kernels launch on `device`
 * (SMs x 8 CTAs x 256), or a negative status. */
int recon_mb_threads(int device);

/* Table III: `ops` random 32-bit accesses to the device matrix `matrix` of
 * 2^log2n elements (1 <= log2n <= 34; the paper's 4K x 4K matrix is log2n = 24).
 * Access k (k = 0 .. ops-1) goes to element SplitMix64(seed, k + 1) >> (64 - log2n),
 * where SplitMix64(s, n) is output n of the SplitMix64 generator seeded with s
 * (s + n * 0x9E3779B97F4A7C15, then the generator's published mixing steps).
 * write = 0: reads; *checksum receives the sum of the values read (mod 2^64).
 * write = 1: element i is set to (uint32)(i * 0x9E3779B1) ^ 0x5A5A5A5A (a value of
 * the index only, so colliding writes agree); checksum may be NULL.
 * Bandwidth = ops * 4 bytes / *ms. */
int recon_mb_random(const void *matrix, int log2n, uint64_t ops, int write, uint64_t seed,
                    uint64_t *checksum, float *ms);

/* Table IV: every thread performs `iters` atomic adds of 1.
 *   mode 0: all threads on counters[0] (one variable, global memory);
 *   mode 1: thread t on counters[t] (an array indexed by thread, global);
 *   mode 2: all threads of a CTA on one shared-memory word; the CTA then writes
 *           its total to counters[cta];
 *   mode 3: each thread on its own shared-memory word, written to counters[t].
 * counters: device array of recon_mb_threads(device) entries, zeroed by the
 * caller for modes 0 and 1. Throughput = threads * iters / *ms. */
int recon_mb_atomic(unsigned *counters, int mode, int iters, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* RECON_H */
