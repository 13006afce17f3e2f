// Batch scheduler: per-tile variant and packing order (internal).
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "recon.h"

struct recon_sched;
recon_sched *recon_sched_create();
void recon_sched_destroy(recon_sched *s);
// Loads a trained model: theta (host, MLP_NPARAMS floats), target de-normalisation
// (mean0, std0, mean1, std1) and the two variants its outputs stand for.
int recon_sched_set(recon_sched *s, const float *theta, const float *norm, int variant_a, int variant_b);
int recon_sched_has_model(const recon_sched *s);
// Plans a batch: features (one pass over I, J), MLP forward, then per tile the
// variant with the lower predicted cost and the order of decreasing predicted
// cost (longest processing time first). Synchronises the stream.
int recon_sched_plan(recon_sched *s, const recon_tile *tiles, int n, int sms, cudaStream_t st,
                     std::vector<int> *variant, std::vector<int> *order);
// Last plan's predictions (de-normalised log costs, 2 per tile).
const std::vector<float> &recon_sched_last_pred(const recon_sched *s);
