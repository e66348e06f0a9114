// TMA form of the 3-D fused iteration (vector3d_tma.cu).
#pragma once

#include "internal.h"
#include "vector3d.cuh"

namespace vomt {

struct Tma3Plan;

// True when the TMA form applies: 40 <= n <= 1024 with n a multiple of 4
// (16-byte strides), k <= 6 channels, norms u in {L12, L2, L1} and w in
// {L1, L2} (and the nuclear norms for compact 2 x 2 and 3 x 3 matrices, k = 3
// and 6 channels), the stage ring fits the SM (two blocks for k <= 4, one for
// k = 5, 6), and the driver provides cuTensorMapEncodeTiled.
bool tma3_supported(int n, int k, int l, int un, int wn);

// Tensor maps over the two ping-pong states (volumes phi[k], u_x[k], u_y[k],
// u_z[k], w[l], each n^3) and b; nullptr if they cannot be built.
Tma3Plan *tma3_plan_create(int n, int k, int l, int un, int wn, const float *state0, const float *state1,
                           const float *b);
void tma3_plan_destroy(Tma3Plan *pl);

// One iteration from state `in_state` (0 or 1) into `out`; blocks march zc planes.
void tma3_launch_step(const Tma3Plan *pl, int in_state, v3::S3Out out, const OpDev &g, const StepDev &s,
                      DevStatus *st, int zc, cudaStream_t stream);

}  // namespace vomt
