// Distance transform by irregular wavefront propagation: internal launcher
// (see recon_dt.cu). Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

enum { DT_OK = 0, DT_ECUDA = 1, DT_ELIMIT = 2 };

// Device scratch bytes for an H x W image (counters, level stamps, two frontiers).
size_t dt_scratch_bytes(int H, int W);

// Runs the whole transform on stream st and waits for it. B: device H x W
// bytes (nonzero = foreground); site: device int32 H x W out; d2: device uint32
// H x W out (may be NULL); scratch: dt_scratch_bytes(H, W) device bytes; h_cnt:
// 4 pinned host words; grid: CTAs per launch. levels_out (optional): levels run.
int dt_run(const uint8_t *B, int H, int W, int *site, unsigned *d2, void *scratch, unsigned *h_cnt,
           int grid, cudaStream_t st, int *levels_out);
