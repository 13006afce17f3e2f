// Learned cost model: internal launchers (see recon_learn.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#define NFEAT 20
#define MLP_NPARAMS 5634

struct rl_tile {
    const uint8_t *I, *J;
    int H, W, pitch;
    int op;   // RECON_OP_*: erosion and FillHoles tiles are described by their complemented values
};

size_t rl_features_scratch(int n);
size_t rl_features_stage(int n);
cudaError_t rl_features(const rl_tile *tiles, int n, void *scratch, size_t scratch_bytes, float *feat_dev,
                        int *viol_dev, int sms, cudaStream_t st, void *host_stage, size_t stage_bytes);
cudaError_t rl_forward(const float *theta, const float *X, int n, float *Y, cudaStream_t st);
cudaError_t rl_grad(const float *theta, const float *X, const float *T, const int *idx, int nb, float *grad,
                    float *loss, cudaStream_t st);
cudaError_t rl_adam(float *theta, float *grad, float *m, float *v, int t, float lr, cudaStream_t st);
