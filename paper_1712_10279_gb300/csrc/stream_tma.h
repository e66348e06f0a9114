// TMA form of the streaming engine's fused iteration (stream_tma.cu).
#pragma once

#include "internal.h"

namespace vomt {

struct TmaPlan;

// True when the TMA step applies: n a multiple of 4 (16-byte strides), k <= 4,
// at least 16 MB of iterate and 304 tiles (below either the plain step is as
// fast), the tile's shared memory fits two blocks per SM, and the driver
// provides cuTensorMapEncodeTiled.
bool tma_step_supported(int n, int k, int l, int un, int wn);

// Tensor maps over the two ping-pong states (planes phi[k], u_x[k], u_y[k],
// w[l], each n x n) and b; nullptr if the maps cannot be built.
TmaPlan *tma_plan_create(int n, int k, int l, int un, int wn, const float *state0, const float *state1,
                         const float *b);
void tma_plan_destroy(TmaPlan *pl);

// One iteration from state `in_state` (0 or 1) into the state at out_state.
// pdl: launch as a programmatic dependent of the previous kernel on the stream (its
// blocks are scheduled while that kernel drains and wait for its writes in the kernel)
void tma_launch_step(const TmaPlan *pl, int in_state, float *out_state, const OpDev &g, const StepDev &s,
                     DevStatus *st, cudaStream_t stream, bool pdl = false);

}  // namespace vomt
