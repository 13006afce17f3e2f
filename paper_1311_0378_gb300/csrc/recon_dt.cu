// Distance transform by irregular wavefront propagation (Table II, "Distance
// Transform": for each foreground pixel the distance to the closest background
// pixel; irregular, 8-connected, IWPP).
//
// Algorithm 1 with data elements D(p) = the background pixel ("site") nearest
// to p found so far. Initialization: background pixels are their own sites,
// foreground pixels have none; the wavefront S = background pixels touching a
// foreground pixel. Propagation: for an element p of S with site s, every
// foreground 8-neighbour q with key(q, s) < key(q, site(q)) takes s and joins
// S, key(q, s) = (|q - s|^2, s) (ties to the lower site index).
//
// GB300 form: the wavefront is processed level-synchronously in global memory,
// one launch per level over a compacted frontier; a site is taken by a 32-bit
// compare-and-swap, and a per-pixel level stamp keeps each pixel at most once
// in a level's frontier. While the transform runs, sites and frontier entries
// are packed coordinates (y << 16 | x), which order like y * W + x and need no
// division; the final pass writes indices y * W + x. Three rotating level
// counters let consecutive level launches run back to back without a host
// round trip; the host reads a counter once per batch of levels to learn when
// S is empty. A CTA reserves the slots of all its new frontier entries with one
// global atomic add (a single global counter is the contended resource).
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "recon_dt.h"

namespace dt {

// packed coordinates: y << 16 | x (y, x < 32768)
__device__ __forceinline__ unsigned dist2(int q, int s)
{
    const int dy = (q >> 16) - (s >> 16), dx = (q & 0xFFFF) - (s & 0xFFFF);
    return (unsigned)(dy * dy) + (unsigned)(dx * dx);
}

// key(q, s) = (|q - s|^2, s); no site = +infinity. Packed sites order like
// their indices y * W + x, so the tie-break is the same.
__device__ __forceinline__ unsigned long long key_of(int q, int s)
{
    if (s < 0) return ~0ull;
    return ((unsigned long long)dist2(q, s) << 32) | (unsigned)s;
}

// warp-aggregated append of v to list (count *cnt) when pred
__device__ __forceinline__ void push(int *list, unsigned *cnt, bool pred, int v)
{
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred);
    if (!bal) return;
    const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(bal));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (pred) list[base + __popc(bal & ((1u << lane) - 1u))] = v;
}

__global__ void __launch_bounds__(256) init_kernel(const uint8_t *B, int H, int W, int *site, int *stamp, int *F0,
                                                   unsigned *cnt)
{
    const long long n = (long long)H * W;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // whole warps iterate together (the ballot in push needs every lane)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        const long long p = base + threadIdx.x;
        bool seed = false;
        if (p < n) {
            const bool fg = B[p] != 0;
            const int y = (int)(p / W), x = (int)(p - (long long)y * W);
            site[p] = fg ? -1 : (y << 16 | x);
            stamp[p] = 0;
            if (!fg) {
                for (int dy = -1; dy <= 1 && !seed; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int yy = y + dy, xx = x + dx;
                        if ((dy || dx) && yy >= 0 && yy < H && xx >= 0 && xx < W && B[(long long)yy * W + xx]) {
                            seed = true;
                            break;
                        }
                    }
            }
        }
        push(F0, &cnt[0], seed, p < n ? (int)((p / W) << 16 | (p % W)) : 0);
    }
}

// Level L: reads frontier Fin (count cnt[L % 3]), appends to Fout (count
// cnt[(L + 1) % 3]) and resets cnt[(L + 2) % 3], which no launch reads again
// before level L + 2 (it was level L - 1's input count).
__global__ void __launch_bounds__(256) level_kernel(const uint8_t *B, int H, int W, int *site, int *stamp,
                                                    const int *Fin, int *Fout, unsigned *cnt, int L, int *err)
{
    __shared__ unsigned s_tot, s_base;
    const unsigned n = cnt[L % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(L + 2) % 3] = 0;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const unsigned i = base + threadIdx.x;
        unsigned raised = 0;   // bit k: neighbour k took this site and is new in the next level
        int p = 0;   // packed coordinates
        if (i < n) {
            p = Fin[i];
            const int y = p >> 16, x = p & 0xFFFF;
            const int s = __ldcg(site + (y * W + x));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int dy = k < 3 ? -1 : (k < 5 ? 0 : 1);
                const int dx = (k == 0 || k == 3 || k == 5) ? -1 : ((k == 1 || k == 6) ? 0 : 1);
                const int yy = y + dy, xx = x + dx;
                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                const int qi = yy * W + xx, q = yy << 16 | xx;
                if (!B[qi]) continue;
                const unsigned long long kn = key_of(q, s);
                int cur = __ldcg(site + qi);
                for (int it = 0; kn < key_of(q, cur); ++it) {
                    if (it > (1 << 16)) { atomicExch(err, 1); break; }
                    const int prev = atomicCAS(site + qi, cur, s);
                    if (prev == cur) {
                        if (atomicExch(stamp + qi, L + 1) != L + 1) raised |= 1u << k;
                        break;
                    }
                    cur = prev;
                }
            }
        }
        unsigned bal[8], tot = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            bal[k] = __ballot_sync(0xFFFFFFFFu, (raised >> k) & 1u);
            tot += __popc(bal[k]);
        }
        // slots: warp offset inside the CTA (shared atomic), then one global
        // atomic per CTA; the loop is block-uniform, so the barriers are safe
        const int lane = threadIdx.x & 31;
        unsigned o = 0;
        if (lane == 0 && tot) o = atomicAdd(&s_tot, tot);
        __syncthreads();
        if (threadIdx.x == 0) {
            s_base = s_tot ? atomicAdd(&cnt[(L + 1) % 3], s_tot) : 0u;
            s_tot = 0;
        }
        __syncthreads();
        if (tot) {
            o = __shfl_sync(0xFFFFFFFFu, o, 0) + s_base;
            const unsigned lt = (1u << lane) - 1u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int dy = k < 3 ? -1 : (k < 5 ? 0 : 1);
                const int dx = (k == 0 || k == 3 || k == 5) ? -1 : ((k == 1 || k == 6) ? 0 : 1);
                if ((raised >> k) & 1u) Fout[o + __popc(bal[k] & lt)] = p + dy * 65536 + dx;
                o += __popc(bal[k]);
            }
        }
    }
}

// d2 from the packed sites, and the sites rewritten as indices y * W + x
__global__ void __launch_bounds__(256) final_kernel(int H, int W, int *site, unsigned *d2)
{
    const long long n = (long long)H * W;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int s = site[p];
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
        if (d2) d2[p] = s < 0 ? 0xFFFFFFFFu : dist2(y << 16 | x, s);
        site[p] = s < 0 ? -1 : (s >> 16) * W + (s & 0xFFFF);
    }
}

}  // namespace dt

size_t dt_scratch_bytes(int H, int W)
{
    const size_t n = (size_t)H * W;
    return 256 + n * sizeof(int) * 3;   // counters + error | stamp | two frontiers
}

int dt_run(const uint8_t *B, int H, int W, int *site, unsigned *d2, void *scratch, unsigned *h_cnt,
           int grid, cudaStream_t st, int *levels_out)
{
    const size_t n = (size_t)H * W;
    unsigned char *base = (unsigned char *)scratch;
    unsigned *cnt = (unsigned *)base;      // cnt[0..2]
    int *err = (int *)(base + 64);
    int *stamp = (int *)(base + 256);
    int *F[2] = {stamp + n, stamp + 2 * n};
    if (cudaMemsetAsync(base, 0, 256, st) != cudaSuccess) return DT_ECUDA;   // counters, error word
    dt::init_kernel<<<grid, 256, 0, st>>>(B, H, W, site, stamp, F[0], cnt);
    if (cudaGetLastError() != cudaSuccess) return DT_ECUDA;
    // every level improves some pixel's key; keys only decrease and each
    // pixel's key has at most H*W + 1 values, but in practice a level count
    // of a few times the largest distance suffices: bound it generously
    const long long max_levels = 8ll * (H + W) + 1024;
    constexpr int BATCH = 16;
    int L = 0;
    for (;;) {
        for (int b = 0; b < BATCH; ++b, ++L) {
            dt::level_kernel<<<grid, 256, 0, st>>>(B, H, W, site, stamp, F[L & 1], F[(L + 1) & 1], cnt, L, err);
        }
        if (cudaGetLastError() != cudaSuccess) return DT_ECUDA;
        if (cudaMemcpyAsync(h_cnt, cnt, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return DT_ECUDA;
        if (h_cnt[L % 3] == 0) break;   // level L has nothing to do: S is empty
        if (L > max_levels) return DT_ELIMIT;
    }
    int herr = 0;
    if (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DT_ECUDA;
    if (herr) return DT_ELIMIT;
    dt::final_kernel<<<grid, 256, 0, st>>>(H, W, site, d2);
    if (cudaGetLastError() != cudaSuccess) return DT_ECUDA;
    if (levels_out) *levels_out = L;
    return DT_OK;
}
