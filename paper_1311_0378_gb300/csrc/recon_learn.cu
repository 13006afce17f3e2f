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

constexpr int FT = 256;   // threads of features_kernel

// Four pixels at once (bytes of a 32-bit word). d gets the per-byte
// difference a - b modulo 256 and the high bit of each byte of `borrow` is set
// where b > a (the bytes subtract independently: the high bit of each byte of
// a is set first so that no borrow crosses a byte boundary, then restored).
__device__ __forceinline__ void sub_bytes(uint32_t a, uint32_t b, uint32_t &d, uint32_t &borrow)
{
    constexpr uint32_t H = 0x80808080u;
    d = ((a | H) - (b & ~H)) ^ ((a ^ ~b) & H);
    borrow = ((~a & b) | (~(a ^ b) & d)) & H;
}

// Counts of one thread: the 16 histogram bins live in the thread's own column
// of a shared array (row = bin, column = thread: the 32 lanes of a warp always
// touch 32 different banks), with row 16 taking the pixels whose I - J bin is
// undefined (J > I); the blob-pixel, zero-marker and violation counts are
// registers, counted four pixels at a time.
struct Counts {
    unsigned *col;                       // &hist[threadIdx.x], rows FT apart
    unsigned bright = 0, zero = 0, bad = 0;

    // one 32-bit word of I and of J; op: 0 dilation, 1 erosion, 2 FillHoles
    __device__ __forceinline__ void add4(uint32_t i, uint32_t j, int op, int npx = 4)
    {
        if (op != 0) {
            i = ~i;
            j = (op == 2) ? 0u : ~j;
        }
        uint32_t d, jgt, e, lt100;
        sub_bytes(i, j, d, jgt);
        sub_bytes(i, 0x64646464u, e, lt100);   // bytes of I below 100
        const uint32_t z = ~(((j & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | j | 0x7F7F7F7Fu);   // bytes of J equal to 0
        const uint32_t valid = npx == 4 ? 0x80808080u : (0x80808080u >> (8 * (4 - npx)));
        bright += __popc(~lt100 & valid);
        zero += __popc(z & valid);
        bad += __popc(jgt & valid);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (b >= npx) break;
            const unsigned bin = ((jgt >> (8 * b + 7)) & 1u) ? 16u : ((d >> (8 * b + 4)) & 15u);
            col[bin * FT] += 1u;
        }
    }
};

__global__ void __launch_bounds__(FT) features_kernel(const FeatTile *T, int n, const unsigned *chunk_base,
                                                      unsigned nchunks, unsigned *counts)
{
    __shared__ unsigned hist[17 * FT];
    __shared__ unsigned sh[NCOUNT];
    for (unsigned c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (threadIdx.x < NCOUNT) sh[threadIdx.x] = 0;
        for (int b = 0; b < 17; ++b) hist[b * FT + threadIdx.x] = 0u;   // this thread's column
        __syncthreads();
        const int t = find_chunk_tile(chunk_base, n, c);
        const FeatTile d = T[t];
        const int y0 = (int)(c - chunk_base[t]) * d.crow;
        const int rows = min(d.H, y0 + d.crow) - y0;
        Counts loc;
        loc.col = &hist[threadIdx.x];
        const bool vec = ((d.pitch & 15) == 0) && (((uintptr_t)d.I & 15) == 0) && (((uintptr_t)d.J & 15) == 0);
        // every thread strides over the chunk's 16-byte vectors (rows x W/16),
        // so narrow tiles keep the whole CTA busy and each thread has several
        // loads in flight; the ragged column tail and unaligned tiles go byte by byte
        const int nv = vec ? d.W >> 4 : 0;
        const int nvec = rows * nv;
        // (row, vector) of index e, stepped by FT = q rows + rem vectors
        const int q = nv ? FT / nv : 0, rem = FT - q * nv;
        int r = nv ? (int)threadIdx.x / nv : 0, v = (int)threadIdx.x - r * nv;
#pragma unroll 2
        for (int e = threadIdx.x; e < nvec; e += FT) {
            const size_t o = (size_t)(y0 + r) * d.pitch;
            const uint4 a = __ldg((const uint4 *)(d.I + o) + v), b = __ldg((const uint4 *)(d.J + o) + v);
            loc.add4(a.x, b.x, d.op);
            loc.add4(a.y, b.y, d.op);
            loc.add4(a.z, b.z, d.op);
            loc.add4(a.w, b.w, d.op);
            r += q;
            v += rem;
            if (v >= nv) {
                v -= nv;
                ++r;
            }
        }
        const int tw = d.W - 16 * nv;   // pixels per row not covered by vectors
        for (int e = threadIdx.x; e < rows * tw; e += FT) {
            const int r = e / tw, x = 16 * nv + (e - r * tw);
            const size_t o = (size_t)(y0 + r) * d.pitch + x;
            loc.add4(d.I[o], d.J[o], d.op, 1);
        }
        if (loc.bright) atomicAdd(&sh[16], loc.bright);
        if (loc.zero) atomicAdd(&sh[17], loc.zero);
        if (loc.bad) atomicAdd(&sh[18], loc.bad);
        __syncthreads();
        {   // bin (thread & 15) over the 16 columns of thread group (thread >> 4)
            const int bin = threadIdx.x & 15, g = threadIdx.x >> 4;
            unsigned s = 0;
#pragma unroll
            for (int q = 0; q < FT / 16; ++q) s += hist[bin * FT + g * (FT / 16) + q];
            if (s) atomicAdd(&sh[bin], s);
        }
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
                        int *viol_dev, int sms, cudaStream_t st, void *host_stage, size_t stage_bytes)
{
    static int occ = 0;   // resident CTAs of features_kernel per SM (it is latency-bound: fill the SMs)
    if (!occ && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rl::features_kernel, rl::FT, 0) != cudaSuccess)
        occ = 4;
    const int grid = std::max(1, occ) * std::max(1, sms);
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
    rl::features_kernel<<<grid, rl::FT, 0, st>>>((const rl::FeatTile *)d, n, (const unsigned *)(d + o_base), acc,
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
