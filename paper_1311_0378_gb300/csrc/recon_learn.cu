// Learned cost model kernels (the scheduler's analogue of the paper's
// performance-aware task scheduling, Sec. IV: estimated per-task costs choose
// where and how each task runs). Never touches pixel values.
//
//   features_kernel  one pass over I and J of every tile: 16-bin histogram of
//                    I - J (bins of width 16), count of I >= 100 (blob pixels),
//                    count of J == 0 (fill-holes markers), J > I violations.
//                    Erosion tiles are counted on complemented values (the
//                    dilation problem the kernel actually solves); FillHoles
//                    tiles as complemented I with J = 0 (their interior marker)
//   finalize_kernel  counts -> 20 fp32 features per tile
//   mlp_forward      20 -> 64 -> 64 -> 2, ReLU hidden units, fp32
//   mlp_grad         forward + backward of L = 1/(2N) sum (Y - T)^2 over a
//                    mini-batch, gradients accumulated per CTA in shared memory
//   adam_kernel      Adam update (Kingma & Ba 2015, Algorithm 1); zeroes the gradient
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>
#include "recon_learn.h"

namespace rl {

struct FeatTile {
    const uint8_t *I, *J;
    int H, W, pitch, op;
    int crow;   // rows per chunk (about CHUNK_PX pixels)
};

__device__ __forceinline__ int find_chunk_tile(const unsigned *chunk_base, int n, unsigned c)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (chunk_base[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// counts: per tile NCOUNT u32: [0..15] histogram, [16] bright, [17] zero J, [18] violations
constexpr int NCOUNT = 19;
constexpr int CHUNK_PX = 1 << 16;   // pixels per chunk of a tile (a whole number of rows, at least one)

// Per-thread counts. The 16 histogram bins are one-hot counters in 8-bit
// fields of two 64-bit words (bins 0-7 and 8-15: one shift and two adds per
// pixel), moved into the 32-bit totals at least every 255 pixels; blob pixels,
// zero markers and J > I violations are plain counters.
struct Counts {
    unsigned long long lo = 0, hi = 0;   // 8-bit fields: bins 0..7, 8..15
    unsigned tot[NCOUNT] = {};
    unsigned pend = 0;                   // pixels in the 8-bit fields

    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            tot[k] += (unsigned)(lo >> (8 * k)) & 0xFFu;
            tot[8 + k] += (unsigned)(hi >> (8 * k)) & 0xFFu;
        }
        lo = hi = 0;
        pend = 0;
    }
    // one pixel; op: the tile's operation (0 dilation, 1 erosion, 2 FillHoles)
    __device__ __forceinline__ void add(uint32_t i, uint32_t j, int op)
    {
        if (op != 0) {
            i ^= 0xFFu;
            j = (op == 2) ? 0u : (j ^ 0xFFu);
        }
        const bool bad = j > i;
        const uint32_t bin = (i - j) >> 4;   // 0..15 unless bad
        const unsigned long long one = bad ? 0ull : (1ull << (8 * (bin & 7)));
        lo += bin < 8 ? one : 0ull;
        hi += bin < 8 ? 0ull : one;
        tot[18] += bad;
        tot[16] += (i >= 100);
        tot[17] += (j == 0);
    }
    // 16 pixels from one 16-byte vector of I and of J (<= 255 pixels pending)
    __device__ __forceinline__ void add16(uint4 a, uint4 b, int op)
    {
        if (pend > 255 - 16) flush();
        const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int s = 0; s < 4; ++s) add((aw[q] >> (8 * s)) & 0xFF, (bw[q] >> (8 * s)) & 0xFF, op);
        pend += 16;
    }
    __device__ __forceinline__ void add1(uint32_t i, uint32_t j, int op)
    {
        if (pend > 254) flush();
        add(i, j, op);
        pend += 1;
    }
};

__global__ void __launch_bounds__(256) features_kernel(const FeatTile *T, int n, const unsigned *chunk_base,
                                                       unsigned nchunks, unsigned *counts)
{
    __shared__ unsigned sh[NCOUNT];
    for (unsigned c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (threadIdx.x < NCOUNT) sh[threadIdx.x] = 0;
        __syncthreads();
        const int t = find_chunk_tile(chunk_base, n, c);
        const FeatTile d = T[t];
        const int y0 = (int)(c - chunk_base[t]) * d.crow;
        const int rows = min(d.H, y0 + d.crow) - y0;
        Counts loc;
        const bool vec = ((d.pitch & 15) == 0) && (((uintptr_t)d.I & 15) == 0) && (((uintptr_t)d.J & 15) == 0);
        // every thread strides over the chunk's 16-byte vectors (rows x W/16),
        // so narrow tiles keep the whole CTA busy and each thread has several
        // loads in flight; the ragged column tail and unaligned tiles go byte by byte
        const int nv = vec ? d.W >> 4 : 0;
        const int nvec = rows * nv;
#pragma unroll 4
        for (int e = threadIdx.x; e < nvec; e += blockDim.x) {
            const int r = e / nv, v = e - r * nv;
            const size_t o = (size_t)(y0 + r) * d.pitch;
            loc.add16(__ldg((const uint4 *)(d.I + o) + v), __ldg((const uint4 *)(d.J + o) + v), d.op);
        }
        const int tw = d.W - 16 * nv;   // pixels per row not covered by vectors
        for (int e = threadIdx.x; e < rows * tw; e += blockDim.x) {
            const int r = e / tw, x = 16 * nv + (e - r * tw);
            const size_t o = (size_t)(y0 + r) * d.pitch + x;
            loc.add1(d.I[o], d.J[o], d.op);
        }
        loc.flush();
#pragma unroll
        for (int k = 0; k < NCOUNT; ++k)
            if (loc.tot[k]) atomicAdd(&sh[k], loc.tot[k]);
        __syncthreads();
        if (threadIdx.x < NCOUNT && sh[threadIdx.x]) atomicAdd(&counts[t * NCOUNT + threadIdx.x], sh[threadIdx.x]);
        __syncthreads();
    }
}

__global__ void finalize_kernel(const FeatTile *T, int n, const unsigned *counts, float *feat, int *violations)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float px = (float)T[t].H * (float)T[t].W;
    const unsigned *c = counts + t * NCOUNT;
    float *f = feat + t * NFEAT;
    for (int k = 0; k < 16; ++k) f[k] = (float)c[k] / px;
    f[16] = (float)c[16] / px;
    f[17] = (float)c[17] / px;
    f[18] = log2f((float)T[t].H) / 12.0f;
    f[19] = log2f((float)T[t].W) / 12.0f;
    if (violations) violations[t] = c[18] ? 1 : 0;
}

// ---------------------------------------------------------------------------
// MLP: parameter blob layout W1 (64x20) b1 (64) W2 (64x64) b2 (64) W3 (2x64) b3 (2)

constexpr int D0 = NFEAT, D1 = 64, D2 = 64, D3 = 2;
constexpr int OW1 = 0, OB1 = OW1 + D1 * D0, OW2 = OB1 + D1, OB2 = OW2 + D2 * D1, OW3 = OB2 + D2,
              OB3 = OW3 + D3 * D2, NP = OB3 + D3;
static_assert(NP == MLP_NPARAMS, "parameter count");

__global__ void __launch_bounds__(64) mlp_forward(const float *theta, const float *X, int n, float *Y)
{
    __shared__ float P[NP];
    __shared__ float x[D0], a1[D1], a2[D2];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = theta[i];
    __syncthreads();
    const int j = threadIdx.x;
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        if (j < D0) x[j] = X[(size_t)s * D0 + j];
        __syncthreads();
        float z = P[OB1 + j];
        for (int i = 0; i < D0; ++i) z = fmaf(P[OW1 + j * D0 + i], x[i], z);
        a1[j] = fmaxf(z, 0.0f);
        __syncthreads();
        z = P[OB2 + j];
        for (int k = 0; k < D1; ++k) z = fmaf(P[OW2 + j * D1 + k], a1[k], z);
        a2[j] = fmaxf(z, 0.0f);
        __syncthreads();
        if (j < D3) {
            float y = P[OB3 + j];
            for (int k = 0; k < D2; ++k) y = fmaf(P[OW3 + j * D2 + k], a2[k], y);
            Y[(size_t)s * D3 + j] = y;
        }
        __syncthreads();
    }
}

// Gradient of L over the samples idx[0..nb) (idx NULL: 0..nb-1), added into grad.
__global__ void __launch_bounds__(64) mlp_grad(const float *theta, const float *X, const float *T,
                                               const int *idx, int nb, float *grad, float *loss)
{
    __shared__ float P[NP];
    __shared__ float G[NP];
    __shared__ float x[D0], z1[D1], a1[D1], z2[D2], a2[D2], dz2[D2], dy[D3];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) { P[i] = theta[i]; G[i] = 0.0f; }
    __syncthreads();
    const int j = threadIdx.x;
    const float invN = 1.0f / (float)nb;
    float lsum = 0.0f;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int s = idx ? idx[b] : b;
        if (j < D0) x[j] = X[(size_t)s * D0 + j];
        __syncthreads();
        float z = P[OB1 + j];
        for (int i = 0; i < D0; ++i) z = fmaf(P[OW1 + j * D0 + i], x[i], z);
        z1[j] = z;
        a1[j] = fmaxf(z, 0.0f);
        __syncthreads();
        z = P[OB2 + j];
        for (int k = 0; k < D1; ++k) z = fmaf(P[OW2 + j * D1 + k], a1[k], z);
        z2[j] = z;
        a2[j] = fmaxf(z, 0.0f);
        __syncthreads();
        if (j < D3) {
            float y = P[OB3 + j];
            for (int k = 0; k < D2; ++k) y = fmaf(P[OW3 + j * D2 + k], a2[k], y);
            const float e = y - T[(size_t)s * D3 + j];
            dy[j] = e * invN;
            lsum += 0.5f * e * e * invN;
        }
        __syncthreads();
        // output layer
        for (int o = 0; o < D3; ++o) G[OW3 + o * D2 + j] += dy[o] * a2[j];
        if (j < D3) G[OB3 + j] += dy[j];
        float g2 = 0.0f;
        for (int o = 0; o < D3; ++o) g2 = fmaf(dy[o], P[OW3 + o * D2 + j], g2);
        dz2[j] = z2[j] > 0.0f ? g2 : 0.0f;
        __syncthreads();
        // hidden layer 2: thread j owns row j of W2
        for (int k = 0; k < D1; ++k) G[OW2 + j * D1 + k] += dz2[j] * a1[k];
        G[OB2 + j] += dz2[j];
        // hidden layer 1: thread j = unit j of layer 1
        float g1 = 0.0f;
        for (int k = 0; k < D2; ++k) g1 = fmaf(dz2[k], P[OW2 + k * D1 + j], g1);
        const float dz1 = z1[j] > 0.0f ? g1 : 0.0f;
        for (int i = 0; i < D0; ++i) G[OW1 + j * D0 + i] += dz1 * x[i];
        G[OB1 + j] += dz1;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < NP; i += blockDim.x)
        if (G[i] != 0.0f) atomicAdd(&grad[i], G[i]);
    if (loss && j < D3 && lsum != 0.0f) atomicAdd(loss, lsum);
}

__global__ void adam_kernel(float *theta, float *grad, float *m, float *v, int t, float lr, float b1,
                            float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)t));
    const float vh = vi / (1.0f - powf(b2, (float)t));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
    grad[i] = 0.0f;
}

}  // namespace rl

// ---------------------------------------------------------------------------
// host-side launchers (internal)

cudaError_t rl_features(const rl_tile *tiles, int n, void *scratch, size_t scratch_bytes, float *feat_dev,
                        int *viol_dev, int grid, cudaStream_t st, void *host_stage, size_t stage_bytes)
{
    // scratch: [FeatTile n][chunk_base n+1][counts n*NCOUNT]
    const size_t o_base = ((sizeof(rl::FeatTile) * n + 15) / 16) * 16;
    const size_t o_cnt = ((o_base + sizeof(unsigned) * (n + 1) + 15) / 16) * 16;
    const size_t need = o_cnt + sizeof(unsigned) * n * rl::NCOUNT;
    if (scratch_bytes < need || stage_bytes < o_cnt) return cudaErrorInvalidValue;
    unsigned char *h = (unsigned char *)host_stage;
    rl::FeatTile *F = (rl::FeatTile *)h;
    unsigned *base = (unsigned *)(h + o_base);
    unsigned acc = 0;
    for (int t = 0; t < n; ++t) {
        F[t].I = tiles[t].I; F[t].J = tiles[t].J; F[t].H = tiles[t].H; F[t].W = tiles[t].W;
        F[t].pitch = tiles[t].pitch; F[t].op = tiles[t].op;
        F[t].crow = std::max(1, std::min(tiles[t].H, rl::CHUNK_PX / std::max(tiles[t].W, 1)));
        base[t] = acc;
        acc += (unsigned)((tiles[t].H + F[t].crow - 1) / F[t].crow);
    }
    base[n] = acc;
    unsigned char *d = (unsigned char *)scratch;
    cudaError_t e = cudaMemcpyAsync(d, h, o_cnt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d + o_cnt, 0, sizeof(unsigned) * n * rl::NCOUNT, st);
    if (e != cudaSuccess) return e;
    rl::features_kernel<<<grid, 256, 0, st>>>((const rl::FeatTile *)d, n, (const unsigned *)(d + o_base), acc,
                                             (unsigned *)(d + o_cnt));
    rl::finalize_kernel<<<(n + 127) / 128, 128, 0, st>>>((const rl::FeatTile *)d, n, (const unsigned *)(d + o_cnt),
                                                         feat_dev, viol_dev);
    return cudaGetLastError();
}

size_t rl_features_scratch(int n)
{
    const size_t o_base = ((sizeof(rl::FeatTile) * n + 15) / 16) * 16;
    const size_t o_cnt = ((o_base + sizeof(unsigned) * (n + 1) + 15) / 16) * 16;
    return o_cnt + sizeof(unsigned) * n * rl::NCOUNT;
}

size_t rl_features_stage(int n)
{
    const size_t o_base = ((sizeof(rl::FeatTile) * n + 15) / 16) * 16;
    return ((o_base + sizeof(unsigned) * (n + 1) + 15) / 16) * 16;
}

cudaError_t rl_forward(const float *theta, const float *X, int n, float *Y, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    rl::mlp_forward<<<n < 1216 ? n : 1216, 64, 0, st>>>(theta, X, n, Y);
    return cudaGetLastError();
}

cudaError_t rl_grad(const float *theta, const float *X, const float *T, const int *idx, int nb, float *grad,
                    float *loss, cudaStream_t st)
{
    if (nb <= 0) return cudaSuccess;
    int g = (nb + 15) / 16;
    if (g > 304) g = 304;
    rl::mlp_grad<<<g, 64, 0, st>>>(theta, X, T, idx, nb, grad, loss);
    return cudaGetLastError();
}

cudaError_t rl_adam(float *theta, float *grad, float *m, float *v, int t, float lr, cudaStream_t st)
{
    rl::adam_kernel<<<(MLP_NPARAMS + 255) / 256, 256, 0, st>>>(theta, grad, m, v, t, lr, 0.9f, 0.999f, 1e-8f);
    return cudaGetLastError();
}
