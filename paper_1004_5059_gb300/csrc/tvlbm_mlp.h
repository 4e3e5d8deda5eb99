// Private: what the closure step needs from the network (tvlbm_mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include "tvlbm_closure.h"

namespace tvlbm {
// Forward pass of `rows` rows of x (device BF16 [rows][64]) into y (device FP32 [rows][16]),
// queued on the network's stream.  TVLBM_* status.
int mlp_forward_async(tvlbm_mlp* m, const void* x, int rows, float* y);
// The closure learned step's inputs, built inside the forward kernel: row c = y nx + x is the
// normalised 3 x 3 periodic neighbourhood of the six moments m6 (device [6][ny][nx]): feature
// 6 k + q = (m6[q] of neighbour k - mu[q]) isg[q] rounded to BF16, neighbour k = 3 (dy + 1) +
// (dx + 1), features 54 .. 63 zero.
struct MlpFeatures {
    const float* m6;
    int nx, ny;
    float mu[6], isg[6];
};
// Forward pass of the nx ny rows those features make (rows = nx ny, a multiple of 128).
int mlp_forward_features_async(tvlbm_mlp* m, const MlpFeatures& feat, int rows, float* y);
int mlp_max_rows(const tvlbm_mlp* m);
float* mlp_ybuf(tvlbm_mlp* m);  // the network's own [max_rows][16] output buffer
int mlp_set_stream(tvlbm_mlp* m, cudaStream_t s);
int mlp_status(tvlbm_mlp* m);  // synchronises; ETIMEOUT if a device wait gave up
unsigned long long mlp_uid(const tvlbm_mlp* m);  // unique over the process's networks
cudaStream_t mlp_stream(const tvlbm_mlp* m);
}  // namespace tvlbm
