/*
 * CPU ORACLE for the distance transform by irregular wavefront propagation.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, the benchmark's CPU legs);
 * it shares no code with the CUDA path.
 *
 * Operation (Table II, "Distance Transform": for each foreground pixel, the
 * distance to the closest background pixel; irregular, 8-connected, IWPP).
 * Method: Algorithm 1 with the data elements D(p) = the background pixel (the
 * "site") nearest to p found so far. Initialization: every background pixel is
 * its own site, foreground pixels have none; the active set S holds the
 * background pixels that touch a foreground pixel (raster order). Propagation:
 * extract e_i from S (FIFO); for each 8-neighbour e_j that is foreground, the
 * propagation condition is key(e_j, site(e_i)) < key(e_j, site(e_j)), with
 * key(q, s) = (|q - s|^2, s) (squared Euclidean distance, ties to the lower
 * site index; no site = +infinity); Update: site(e_j) <- site(e_i); e_j joins S.
 * Result: site map and squared distances |p - site(p)|^2 (0 on background).
 *
 * The propagation is an approximation of the exact Euclidean distance
 * transform (a pixel passes on only the site it holds, as in Danielsson's
 * vector propagation), and its result depends on the processing order; the
 * tests therefore pin it to the exact transform within a bound and check the
 * fixed-point property, not bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DT_OK 0
#define DT_EINVAL 1
#define DT_ENOMEM 3

static uint64_t key_of(int W, int64_t q, int64_t s)
{
    if (s < 0) return UINT64_MAX;
    int64_t qy = q / W, qx = q % W, sy = s / W, sx = s % W;
    uint64_t d2 = (uint64_t)((qy - sy) * (qy - sy) + (qx - sx) * (qx - sx));
    return (d2 << 32) | (uint64_t)s;
}

/* B: H x W bytes, nonzero = foreground. site: H*W int32 out (-1 = no
 * background in the image). d2: H*W uint32 out (UINT32_MAX where no site).
 * Returns DT_OK or an error code. */
int oracle_dt(const uint8_t *B, int H, int W, int32_t *site, uint32_t *d2)
{
    if (!B || !site || !d2 || H < 1 || W < 1 || H > 32768 || W > 32768) return DT_EINVAL;
    const int64_t n = (int64_t)H * W;
    /* FIFO: each pixel enters at most once per improvement; a ring of n+1 slots
     * suffices when a pixel already waiting is not queued twice */
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    uint8_t *inq = (uint8_t *)calloc((size_t)n, 1);
    if (!q || !inq) { free(q); free(inq); return DT_ENOMEM; }
    int64_t head = 0, tail = 0, cap = n + 1;
    for (int64_t p = 0; p < n; ++p) site[p] = B[p] ? -1 : (int32_t)p;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            if (B[p]) continue;
            int touches = 0;
            for (int dy = -1; dy <= 1 && !touches; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int yy = y + dy, xx = x + dx;
                    if ((dy || dx) && yy >= 0 && yy < H && xx >= 0 && xx < W && B[(int64_t)yy * W + xx]) {
                        touches = 1;
                        break;
                    }
                }
            if (touches) { q[tail] = (int32_t)p; tail = (tail + 1) % cap; inq[p] = 1; }
        }
    static const int DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1}, DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    while (head != tail) {
        const int64_t p = q[head];
        head = (head + 1) % cap;
        inq[p] = 0;
        const int64_t s = site[p];
        const int y = (int)(p / W), x = (int)(p % W);
        for (int k = 0; k < 8; ++k) {
            int yy = y + DY[k], xx = x + DX[k];
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            int64_t r = (int64_t)yy * W + xx;
            if (!B[r]) continue;
            if (key_of(W, r, s) < key_of(W, r, site[r])) {
                site[r] = (int32_t)s;
                if (!inq[r]) { q[tail] = (int32_t)r; tail = (tail + 1) % cap; inq[r] = 1; }
            }
        }
    }
    for (int64_t p = 0; p < n; ++p)
        d2[p] = site[p] < 0 ? UINT32_MAX : (uint32_t)(key_of(W, p, site[p]) >> 32);
    free(q);
    free(inq);
    return DT_OK;
}
