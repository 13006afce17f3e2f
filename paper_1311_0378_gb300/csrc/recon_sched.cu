// Batch scheduler: the learned cost model picks each tile's variant (two scan
// / queue settings) and orders tiles of equal size by decreasing predicted
// cost; tiles of different sizes go largest first (on 1000-tile batches,
// ordering by predicted cost alone was 2-4% slower than by area). Its outputs
// only reorder and re-parameterise work; pixel values are never touched, and
// without a model the plain schedule applies.
#include <algorithm>
#include <numeric>
#include <vector>
#include <cuda_runtime.h>
#include "recon_learn.h"
#include "recon_sched.h"

struct recon_sched {
    int have_model = 0;
    float *d_theta = nullptr;
    float norm[4] = {0, 1, 0, 1};
    int variant[2] = {-1, 1};
    // scratch
    void *d_scratch = nullptr; size_t cap_scratch = 0;
    float *d_feat = nullptr, *d_pred = nullptr; size_t cap_n = 0;
    void *h_stage = nullptr; size_t cap_stage = 0;
    std::vector<float> pred;
};

recon_sched *recon_sched_create() { return new recon_sched(); }

void recon_sched_destroy(recon_sched *s)
{
    if (!s) return;
    cudaFree(s->d_theta);
    cudaFree(s->d_scratch);
    cudaFree(s->d_feat);
    cudaFree(s->d_pred);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    delete s;
}

int recon_sched_set(recon_sched *s, const float *theta, const float *norm, int va, int vb)
{
    // variants use the recon_batch_ex encoding: -1, or k + 256 * g (k <= 64, g <= 4096)
    auto ok = [](int v) { return v == -1 || (v >= 0 && (v & 0xFF) <= 64 && (v >> 8) <= 4096); };
    if (!s || !theta || !norm || !ok(va) || !ok(vb)) return RECON_EINVAL;
    if (!s->d_theta && cudaMalloc((void **)&s->d_theta, sizeof(float) * MLP_NPARAMS) != cudaSuccess)
        return RECON_ENOMEM;
    if (cudaMemcpy(s->d_theta, theta, sizeof(float) * MLP_NPARAMS, cudaMemcpyHostToDevice) != cudaSuccess)
        return RECON_ECUDA;
    for (int i = 0; i < 4; ++i) s->norm[i] = norm[i];
    s->variant[0] = va;
    s->variant[1] = vb;
    s->have_model = 1;
    return RECON_OK;
}

int recon_sched_has_model(const recon_sched *s) { return s && s->have_model; }

const std::vector<float> &recon_sched_last_pred(const recon_sched *s) { return s->pred; }

static int ensure(recon_sched *s, int n)
{
    const size_t sb = rl_features_scratch(n), hb = rl_features_stage(n);
    if (s->cap_scratch < sb) {
        cudaFree(s->d_scratch);
        s->d_scratch = nullptr;
        s->cap_scratch = 0;
        if (cudaMalloc(&s->d_scratch, sb) != cudaSuccess) return RECON_ENOMEM;
        s->cap_scratch = sb;
    }
    if (s->cap_stage < hb) {
        if (s->h_stage) cudaFreeHost(s->h_stage);
        s->h_stage = nullptr;
        s->cap_stage = 0;
        if (cudaMallocHost(&s->h_stage, hb) != cudaSuccess) return RECON_ENOMEM;
        s->cap_stage = hb;
    }
    if (s->cap_n < (size_t)n) {
        cudaFree(s->d_feat);
        cudaFree(s->d_pred);
        s->d_feat = s->d_pred = nullptr;
        s->cap_n = 0;
        if (cudaMalloc((void **)&s->d_feat, sizeof(float) * NFEAT * n) != cudaSuccess) return RECON_ENOMEM;
        if (cudaMalloc((void **)&s->d_pred, sizeof(float) * 2 * n) != cudaSuccess) return RECON_ENOMEM;
        s->cap_n = (size_t)n;
    }
    return RECON_OK;
}

int recon_sched_plan(recon_sched *s, const recon_tile *tiles, int n, int sms, cudaStream_t st,
                     std::vector<int> *variant, std::vector<int> *order)
{
    if (!s || !s->have_model) return RECON_EINVAL;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RECON_ECUDA;  // staging buffer reuse
    int rc = ensure(s, n);
    if (rc) return rc;
    std::vector<rl_tile> rt(n);
    for (int t = 0; t < n; ++t)
        rt[t] = rl_tile{tiles[t].I, tiles[t].J, tiles[t].H, tiles[t].W, tiles[t].pitch, tiles[t].op};
    cudaError_t e = rl_features(rt.data(), n, s->d_scratch, s->cap_scratch, s->d_feat, nullptr, sms, st,
                                s->h_stage, s->cap_stage);
    if (e == cudaSuccess) e = rl_forward(s->d_theta, s->d_feat, n, s->d_pred, st);
    s->pred.resize(2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->pred.data(), s->d_pred, sizeof(float) * 2 * n,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return RECON_ECUDA;
    std::vector<float> cost(n);
    variant->resize(n);
    order->resize(n);
    for (int t = 0; t < n; ++t) {
        const float a = s->pred[2 * t] * s->norm[1] + s->norm[0];
        const float b = s->pred[2 * t + 1] * s->norm[3] + s->norm[2];
        s->pred[2 * t] = a;
        s->pred[2 * t + 1] = b;
        (*variant)[t] = a < b ? s->variant[0] : s->variant[1];
        cost[t] = a < b ? a : b;
    }
    std::iota(order->begin(), order->end(), 0);
    std::stable_sort(order->begin(), order->end(), [&](int x, int y) {
        const long long ax = (long long)tiles[x].H * tiles[x].W, ay = (long long)tiles[y].H * tiles[y].W;
        return ax != ay ? ax > ay : cost[x] > cost[y];
    });
    return RECON_OK;
}
