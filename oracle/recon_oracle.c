/*
 * CPU ORACLE for grayscale morphological reconstruction by dilation.
 * TEST INFRASTRUCTURE ONLY: it is called by the tests, by the smoke check and by
 * the benchmark's CPU-baseline leg, never by the library. It shares no code,
 * header or table with the CUDA path.
 *
 * What is computed (Table II, "Morphological Reconstruction": flood-fill a
 * marker image limited by a mask image, 4-/8-connected, citing Vincent 1993):
 *     R = lim_n delta_I^n(J),  delta_I(X)(p) = min( max_{q in N(p)} X(q), I(p) ),
 * N(p) = p plus its 4 or 8 neighbours that lie inside the image.
 * Precondition J <= I pixel-wise (otherwise status 2 and J is left untouched).
 *
 * oracle_recon        -- the method's regular phase (Sec. V-C, irregular
 *                        operations: raster / anti-raster scans) run alone until
 *                        a full raster + anti-raster pair changes no pixel.
 * oracle_recon_widest -- an independent exact route used as a cross-check and for
 *                        large inputs: R(p) = max over sources q and paths q->p of
 *                        min(J(q), min of I on the path), computed as a
 *                        maximum-bottleneck (widest-path) flood that finalises
 *                        pixels in decreasing value order with 256 buckets.
 * oracle_recon_erode -- reconstruction by erosion, the dual operation:
 *                        R = lim_n eps_I^n(J), eps_I(X)(p) = max( min_{q in N(p)} X(q), I(p) ),
 *                        precondition J >= I. Written out with min and max
 *                        exchanged (absent neighbours are skipped, as above), not
 *                        through complements, so the duality
 *                        R^eps_I(J) = 255 - R^delta_{255-I}(255-J) tests it.
 *                        It is what FillHoles (Table II) computes when the marker
 *                        is I on the image border and 255 inside.
 * Both are single-threaded per tile; oracle_recon_tiles runs tiles on threads.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_EMARKER 2
#define ORACLE_ENOMEM 3

static inline uint8_t u8max(uint8_t a, uint8_t b) { return a > b ? a : b; }
static inline uint8_t u8min(uint8_t a, uint8_t b) { return a < b ? a : b; }

static int check(const uint8_t *I, const uint8_t *J, int H, int W, int conn)
{
    if (!I || !J || H <= 0 || W <= 0 || (conn != 4 && conn != 8)) return ORACLE_EINVAL;
    size_t n = (size_t)H * (size_t)W;
    for (size_t i = 0; i < n; ++i)
        if (J[i] > I[i]) return ORACLE_EMARKER;
    return ORACLE_OK;
}

/* Raster scan, y = 0..H-1, x = 0..W-1:
 *   J(p) <- min(I(p), max(J(p), J over N+(p))),
 * N+(p) = {(y, x-1), (y-1, x)} for 4-conn, plus {(y-1, x-1), (y-1, x+1)} for 8-conn. */
static int raster(const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    int changed = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            uint8_t m = J[p];
            if (x > 0) m = u8max(m, J[p - 1]);
            if (y > 0) {
                m = u8max(m, J[p - W]);
                if (conn == 8) {
                    if (x > 0) m = u8max(m, J[p - W - 1]);
                    if (x < W - 1) m = u8max(m, J[p - W + 1]);
                }
            }
            uint8_t v = u8min(m, I[p]);
            if (v != J[p]) { J[p] = v; changed = 1; }
        }
    return changed;
}

/* Anti-raster scan, y = H-1..0, x = W-1..0, with the mirrored set N-(p). */
static int antiraster(const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    int changed = 0;
    for (int y = H - 1; y >= 0; --y)
        for (int x = W - 1; x >= 0; --x) {
            size_t p = (size_t)y * W + x;
            uint8_t m = J[p];
            if (x < W - 1) m = u8max(m, J[p + 1]);
            if (y < H - 1) {
                m = u8max(m, J[p + W]);
                if (conn == 8) {
                    if (x < W - 1) m = u8max(m, J[p + W + 1]);
                    if (x > 0) m = u8max(m, J[p + W - 1]);
                }
            }
            uint8_t v = u8min(m, I[p]);
            if (v != J[p]) { J[p] = v; changed = 1; }
        }
    return changed;
}

/* Sweeps to stability. J is overwritten with R. *pairs (optional) receives
 * the number of raster + anti-raster pairs run, the last one included. */
int oracle_recon(const uint8_t *I, uint8_t *J, int H, int W, int conn, int *pairs)
{
    int rc = check(I, J, H, W, conn);
    if (rc) return rc;
    int n = 0;
    for (;;) {
        int c1 = raster(I, J, H, W, conn);
        int c2 = antiraster(I, J, H, W, conn);
        ++n;
        if (!c1 && !c2) break;
    }
    if (pairs) *pairs = n;
    return ORACLE_OK;
}

/* One geodesic dilation X <- min(delta(X), I) over the whole image at once
 * (every pixel reads the old X). Returns 1 if any pixel changed. */
int oracle_dilate_step(const uint8_t *I, uint8_t *X, int H, int W, int conn)
{
    if (!I || !X || H <= 0 || W <= 0 || (conn != 4 && conn != 8)) return -ORACLE_EINVAL;
    size_t n = (size_t)H * (size_t)W;
    uint8_t *old = (uint8_t *)malloc(n);
    if (!old) return -ORACLE_ENOMEM;
    memcpy(old, X, n);
    int changed = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t m = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (conn == 4 && dy != 0 && dx != 0) continue;
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    m = u8max(m, old[(size_t)yy * W + xx]);
                }
            uint8_t v = u8min(m, I[(size_t)y * W + x]);
            if (v != X[(size_t)y * W + x]) { X[(size_t)y * W + x] = v; changed = 1; }
        }
    free(old);
    return changed;
}

/* ---- reconstruction by erosion ---- */

static int check_erode(const uint8_t *I, const uint8_t *J, int H, int W, int conn)
{
    if (!I || !J || H <= 0 || W <= 0 || (conn != 4 && conn != 8)) return ORACLE_EINVAL;
    size_t n = (size_t)H * (size_t)W;
    for (size_t i = 0; i < n; ++i)
        if (J[i] < I[i]) return ORACLE_EMARKER;
    return ORACLE_OK;
}

/* Raster scan of the erosion: J(p) <- max(I(p), min(J(p), J over N+(p))). */
static int raster_erode(const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    int changed = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            uint8_t m = J[p];
            if (x > 0) m = u8min(m, J[p - 1]);
            if (y > 0) {
                m = u8min(m, J[p - W]);
                if (conn == 8) {
                    if (x > 0) m = u8min(m, J[p - W - 1]);
                    if (x < W - 1) m = u8min(m, J[p - W + 1]);
                }
            }
            uint8_t v = u8max(m, I[p]);
            if (v != J[p]) { J[p] = v; changed = 1; }
        }
    return changed;
}

/* Anti-raster scan of the erosion, with the mirrored set N-(p). */
static int antiraster_erode(const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    int changed = 0;
    for (int y = H - 1; y >= 0; --y)
        for (int x = W - 1; x >= 0; --x) {
            size_t p = (size_t)y * W + x;
            uint8_t m = J[p];
            if (x < W - 1) m = u8min(m, J[p + 1]);
            if (y < H - 1) {
                m = u8min(m, J[p + W]);
                if (conn == 8) {
                    if (x < W - 1) m = u8min(m, J[p + W + 1]);
                    if (x > 0) m = u8min(m, J[p + W - 1]);
                }
            }
            uint8_t v = u8max(m, I[p]);
            if (v != J[p]) { J[p] = v; changed = 1; }
        }
    return changed;
}

/* Erosion sweeps to stability (J >= I required, else status 2). */
int oracle_recon_erode(const uint8_t *I, uint8_t *J, int H, int W, int conn, int *pairs)
{
    int rc = check_erode(I, J, H, W, conn);
    if (rc) return rc;
    int n = 0;
    for (;;) {
        int c1 = raster_erode(I, J, H, W, conn);
        int c2 = antiraster_erode(I, J, H, W, conn);
        ++n;
        if (!c1 && !c2) break;
    }
    if (pairs) *pairs = n;
    return ORACLE_OK;
}

/* One whole-image geodesic erosion X <- max(eps(X), I), every pixel reading
 * the old X. Returns 1 if any pixel changed. */
int oracle_erode_step(const uint8_t *I, uint8_t *X, int H, int W, int conn)
{
    if (!I || !X || H <= 0 || W <= 0 || (conn != 4 && conn != 8)) return -ORACLE_EINVAL;
    size_t n = (size_t)H * (size_t)W;
    uint8_t *old = (uint8_t *)malloc(n);
    if (!old) return -ORACLE_ENOMEM;
    memcpy(old, X, n);
    int changed = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t m = 255;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (conn == 4 && dy != 0 && dx != 0) continue;
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    m = u8min(m, old[(size_t)yy * W + xx]);
                }
            uint8_t v = u8max(m, I[(size_t)y * W + x]);
            if (v != X[(size_t)y * W + x]) { X[(size_t)y * W + x] = v; changed = 1; }
        }
    free(old);
    return changed;
}

/* ---- maximum-bottleneck flood (test cross-check / large inputs) ---- */
typedef struct { uint32_t *v; size_t n, cap; } bucket_t;

static int bpush(bucket_t *b, uint32_t p)
{
    if (b->n == b->cap) {
        size_t nc = b->cap ? 2 * b->cap : 1024;
        uint32_t *nv = (uint32_t *)realloc(b->v, nc * sizeof(uint32_t));
        if (!nv) return 0;
        b->v = nv; b->cap = nc;
    }
    b->v[b->n++] = p;
    return 1;
}

int oracle_recon_widest(const uint8_t *I, uint8_t *J, int H, int W, int conn)
{
    int rc = check(I, J, H, W, conn);
    if (rc) return rc;
    size_t n = (size_t)H * (size_t)W;
    if (n > 0xFFFFFFFFull) return ORACLE_EINVAL;
    bucket_t bk[256];
    memset(bk, 0, sizeof(bk));
    uint8_t *done = (uint8_t *)calloc(n, 1);
    int ok = done != NULL;
    for (size_t p = 0; ok && p < n; ++p) ok = bpush(&bk[J[p]], (uint32_t)p);
    static const int dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 1}, dx8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    static const int dy4[4] = {-1, 0, 0, 1}, dx4[4] = {0, -1, 1, 0};
    const int *dy = conn == 8 ? dy8 : dy4, *dx = conn == 8 ? dx8 : dx4;
    for (int b = 255; ok && b >= 0; --b) {
        /* pushes made while draining bucket b land in b or lower */
        while (ok && bk[b].n > 0) {
            uint32_t p = bk[b].v[--bk[b].n];
            if (done[p] || J[p] != b) continue;
            done[p] = 1;
            int y = (int)(p / (uint32_t)W), x = (int)(p % (uint32_t)W);
            for (int k = 0; k < conn; ++k) {
                int yy = y + dy[k], xx = x + dx[k];
                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                size_t q = (size_t)yy * W + xx;
                uint8_t c = u8min((uint8_t)b, I[q]);
                if (!done[q] && c > J[q]) {
                    J[q] = c;
                    ok = bpush(&bk[c], (uint32_t)q);
                }
            }
        }
    }
    for (int b = 0; b < 256; ++b) free(bk[b].v);
    free(done);
    return ok ? ORACLE_OK : ORACLE_ENOMEM;
}

/* ---- many tiles on host threads ---- */
typedef struct {
    int n, method, next;
    const uint8_t *const *I;
    uint8_t *const *J;
    const int *H, *W, *conn;
    int *status;
    pthread_mutex_t mu;
} tjob_t;

static void *tworker(void *arg)
{
    tjob_t *t = (tjob_t *)arg;
    for (;;) {
        pthread_mutex_lock(&t->mu);
        int i = t->next++;
        pthread_mutex_unlock(&t->mu);
        if (i >= t->n) break;
        int rc = t->method == 1 ? oracle_recon_widest(t->I[i], t->J[i], t->H[i], t->W[i], t->conn[i])
               : t->method == 2 ? oracle_recon_erode(t->I[i], t->J[i], t->H[i], t->W[i], t->conn[i], NULL)
                                : oracle_recon(t->I[i], t->J[i], t->H[i], t->W[i], t->conn[i], NULL);
        if (t->status) t->status[i] = rc;
    }
    return NULL;
}

/* Runs n independent tiles. method 0 = sweeps to stability, 1 = widest flood,
 * 2 = erosion sweeps to stability.
 * status[i] (optional) receives each tile's code. Returns the number of threads used. */
int oracle_recon_tiles(int n, const uint8_t *const *I, uint8_t *const *J, const int *H,
                       const int *W, const int *conn, int method, int nthreads, int *status)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    tjob_t t;
    t.n = n; t.method = method; t.next = 0; t.I = I; t.J = J; t.H = H; t.W = W;
    t.conn = conn; t.status = status;
    pthread_mutex_init(&t.mu, NULL);
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[started], NULL, tworker, &t) == 0) ++started;
    tworker(&t);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&t.mu);
    return started + 1;
}
