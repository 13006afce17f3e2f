/*
 * Seeded synthetic tissue-like tiles: the mask I and the marker J.
 *
 * This module only builds inputs. It holds none of the reconstruction's
 * arithmetic and is shared, as a plain input source, by the CUDA path's tests
 * and benchmark and by the CPU oracle's tests.
 *
 * Recipe (stands in for the paper's 4K x 4K brain-tumour slide tiles, Sec. V):
 *   - every random number is an output of a SplitMix64 stream (Steele, Lea and
 *     Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
 *     seeded per (seed, tile, purpose); pixel i of a tile takes output i of the
 *     noise stream, so any pixel can be regenerated on its own;
 *   - noise: I0 = 20 + (u mod 41), i.e. integers in [20, 60];
 *   - blobs: centre (u mod W, u mod H), radius r in [rmin, rmax], peak P in
 *     [120, 230]; Gaussian profile P * exp(-d^2 / (2 sigma^2)), sigma = r / 2,
 *     cut at d <= r, added in 1/256 gray-level fixed point from a per-radius
 *     table q[r][d^2] = round(65536 * exp(-2 d^2 / r^2));
 *   - I = min(255, (256 * I0 + sum_b (P_b * q + 128) >> 8 + 128) >> 8);
 *   - markers: h-dome J = max(I - 10, 0); fill-holes J = I on the 1-pixel
 *     image border and 0 inside.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_RMAX 64

static inline uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number n (n >= 1) of the SplitMix64 stream seeded with s. */
static inline uint64_t sm64_at(uint64_t s, uint64_t n)
{
    return sm64_mix(s + n * 0x9E3779B97F4A7C15ULL);
}

/* Stream seed for (seed, tile, purpose). */
uint64_t synth_stream(uint64_t seed, uint64_t tile, uint64_t purpose)
{
    uint64_t a = sm64_at(seed, 1);
    uint64_t b = sm64_at(a ^ tile, 1);
    return sm64_at(b ^ (purpose * 0xD1B54A32D192ED03ULL), 1);
}

uint64_t synth_u64(uint64_t stream, uint64_t n) { return sm64_at(stream, n); }

enum { PURPOSE_NOISE = 1, PURPOSE_BLOBS = 2 };

typedef struct {
    int H, W, pitch;    /* rows, columns, row stride in bytes (>= W) */
    int nblobs, rmin, rmax;
    int marker;         /* 0 = h-dome, 1 = fill-holes, -1 = leave J untouched */
    int pad;
    uint64_t tile;      /* tile index inside the seed's family */
} synth_desc;

static void profile_table(uint32_t *q, int r)
{
    /* q[d2] for d2 in [0, r*r] */
    double r2 = (double)r * (double)r;
    for (int d2 = 0; d2 <= r * r; ++d2)
        q[d2] = (uint32_t)floor(65536.0 * exp(-2.0 * (double)d2 / r2) + 0.5);
}

static void gen_one(const synth_desc *d, uint64_t seed, uint8_t *I, uint8_t *J,
                    uint32_t *acc, uint32_t *q)
{
    const int H = d->H, W = d->W, P = d->pitch;
    const uint64_t sn = synth_stream(seed, d->tile, PURPOSE_NOISE);
    const uint64_t sb = synth_stream(seed, d->tile, PURPOSE_BLOBS);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint64_t i = (uint64_t)y * (uint64_t)W + (uint64_t)x;
            acc[i] = 256u * (20u + (uint32_t)(sm64_at(sn, i + 1) % 41u));
        }
    int last_r = -1;
    for (int b = 0; b < d->nblobs; ++b) {
        uint64_t k = 4 * (uint64_t)b;
        int cx = (int)(sm64_at(sb, k + 1) % (uint64_t)W);
        int cy = (int)(sm64_at(sb, k + 2) % (uint64_t)H);
        int r = d->rmin + (int)(sm64_at(sb, k + 3) % (uint64_t)(d->rmax - d->rmin + 1));
        uint32_t peak = 120u + (uint32_t)(sm64_at(sb, k + 4) % 111u);
        if (r != last_r) { profile_table(q, r); last_r = r; }
        for (int dy = -r; dy <= r; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= H) continue;
            for (int dx = -r; dx <= r; ++dx) {
                int x = cx + dx;
                int d2 = dy * dy + dx * dx;
                if (x < 0 || x >= W || d2 > r * r) continue;
                acc[(uint64_t)y * W + x] += (peak * q[d2] + 128u) >> 8;
            }
        }
    }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint32_t v = (acc[(uint64_t)y * W + x] + 128u) >> 8;
            I[(uint64_t)y * P + x] = (uint8_t)(v > 255u ? 255u : v);
        }
    if (d->marker == 0) {
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                uint8_t v = I[(uint64_t)y * P + x];
                J[(uint64_t)y * P + x] = (uint8_t)(v > 10 ? v - 10 : 0);
            }
    } else if (d->marker == 1) {
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int border = (y == 0 || x == 0 || y == H - 1 || x == W - 1);
                J[(uint64_t)y * P + x] = border ? I[(uint64_t)y * P + x] : 0;
            }
    }
}

static int desc_ok(const synth_desc *d)
{
    return d->H > 0 && d->W > 0 && d->pitch >= d->W && d->nblobs >= 0 &&
           d->rmin >= 1 && d->rmax >= d->rmin && d->rmax <= SYNTH_RMAX;
}

typedef struct {
    const synth_desc *d;
    uint8_t *const *I;
    uint8_t *const *J;
    uint64_t seed;
    int n, next, err;
    pthread_mutex_t mu;
} job_t;

static void *worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * (SYNTH_RMAX * SYNTH_RMAX + 1));
    uint32_t *acc = NULL;
    size_t cap = 0;
    for (;;) {
        pthread_mutex_lock(&jb->mu);
        int t = jb->next++;
        pthread_mutex_unlock(&jb->mu);
        if (t >= jb->n) break;
        size_t need = (size_t)jb->d[t].H * (size_t)jb->d[t].W;
        if (need > cap) {
            free(acc);
            acc = (uint32_t *)malloc(need * sizeof(uint32_t));
            cap = acc ? need : 0;
        }
        if (!acc || !q) {
            pthread_mutex_lock(&jb->mu);
            jb->err = 3;
            pthread_mutex_unlock(&jb->mu);
            break;
        }
        gen_one(&jb->d[t], jb->seed, jb->I[t], jb->J[t], acc, q);
    }
    free(acc);
    free(q);
    return NULL;
}

/* Fills I[t] and J[t] for n tiles on nthreads host threads.
 * Returns 0, 1 for a bad descriptor, 3 when memory runs out. */
int synth_batch(int n, const synth_desc *d, uint8_t *const *I, uint8_t *const *J,
                uint64_t seed, int nthreads)
{
    for (int t = 0; t < n; ++t)
        if (!desc_ok(&d[t]) || !I[t] || (d[t].marker >= 0 && !J[t])) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    job_t jb;
    jb.d = d; jb.I = I; jb.J = J; jb.seed = seed; jb.n = n; jb.next = 0; jb.err = 0;
    pthread_mutex_init(&jb.mu, NULL);
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[started], NULL, worker, &jb) == 0) ++started;
    worker(&jb);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&jb.mu);
    return jb.err;
}
