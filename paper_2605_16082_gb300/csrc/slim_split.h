// Split-IMEX internal step with the subcycled 2D external mode.
#pragma once

#include "slim_internal.h"

namespace slim {
struct SplitBufs;
size_t split_aux2d_len(const DevMesh& m);
slim_status split_alloc(slim_state* s);
void split_free(slim_state* s);
void* split_field(slim_state* s, int field);  // 2D double buffers of the last stage, or null
slim_status split_hpg(slim_state* s, cudaStream_t st);
slim_status split_rhs2d(slim_state* s, double t, double* out, cudaStream_t st);
slim_status split_rhs3d_momentum(slim_state* s, int field, void* out, cudaStream_t st);
slim_status split_step(slim_state* s, double t, double dt, cudaStream_t st);
int split_kernel_count(const slim_state* s);
// the step's time kernel (its first argument is the step's start time)
const void* split_time_kernel();
// the time kernel's argument (a struct of at most 128 bytes) for a step at t, dt
void split_time_args(const slim_state* s, double t, double dt, void* out);
}  // namespace slim
