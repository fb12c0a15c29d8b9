// Launchers of the device kernels (host-callable, one per operation and precision).
#pragma once

#include "slim_internal.h"

namespace slim {

enum : int {
  SLIM_ERRBIT_NONFINITE = 1,
  SLIM_ERRBIT_BOUNDS = 2,
  SLIM_ERRBIT_TIMEOUT = 4,
};

struct StageParams {
  double kappa;      // vertical diffusivity of the solved field
  double penalty;    // vertical SIPG penalty factor
  double flux_top;   // prescribed kappa dT/dz at the surface
  double flux_bot;   // prescribed kappa dT/dz at the bed
};

// stretch 1 + eta/h of every vertex column
template <typename R>
cudaError_t launch_stretch(const DevMesh& m, const double* eta, R* st, cudaStream_t st_);

template <typename R>
cudaError_t launch_continuity(const DevMesh& m, int TP, const R* U, const R* V, const double* eta,
                              const R* st_cur, double* eta_out, R* st_out, R* W, double dt,
                              cudaStream_t st);

template <typename R>
cudaError_t launch_tracer_stage(const DevMesh& m, int TP, const R* U, const R* V, const R* Tn,
                                const R* Tp, const R* Text, const R* W, R* Tout, const R* st_n,
                                const R* st_np1, double th_p, double th_s, double alpha,
                                double beta, double dt, const StageParams& sp, int* err,
                                cudaStream_t st);

template <typename R>
cudaError_t launch_rhs3d(const DevMesh& m, int TP, const R* U, const R* V, const R* T,
                         const R* Text, const R* st, R* out, cudaStream_t stm);

template <typename R>
cudaError_t launch_vertical_solve(const DevMesh& m, int TP, const R* W, const R* st, const R* rhs,
                                  R* out, double bdt, const StageParams& sp, int* err,
                                  cudaStream_t st_);

// rhs2d of the tracer scheme: column sums of R_h(q, 1), 3*n_tri doubles
template <typename R>
cudaError_t launch_column_divergence(const DevMesh& m, int TP, const R* U, const R* V,
                                     const R* st_cur, double* out, cudaStream_t st);

// mass: block partials (2 doubles per tile: sum, compensation) then one final block;
// consistent: the consistent mass of the coupled column system instead of the lumped one
template <typename R>
cudaError_t launch_mass(const DevMesh& m, int TP, const R* T, const double* eta, double* partials,
                        double* result, cudaStream_t st, bool consistent);

// coupled (consistent-mass, 6x6 blocks per prism) column system of the tracer scheme
size_t coupled_smem_bytes(const DevMesh& m, int TP, size_t esz);
template <typename R>
cudaError_t launch_continuity_cpl(const DevMesh& m, int TP, const R* U, const R* V, const double* eta,
                                  const R* st_cur, double* eta_out, R* st_out, R* W, double dt,
                                  cudaStream_t st);
template <typename R>
cudaError_t launch_tracer_stage_cpl(const DevMesh& m, int TP, const R* U, const R* V, const R* Tn,
                                    const R* Tp, const R* Text, const R* W, R* Tout, const R* st_n,
                                    const R* st_np1, double th_p, double th_s, double alpha,
                                    double beta, double dt, const StageParams& sp, int* err,
                                    cudaStream_t st);
template <typename R>
cudaError_t launch_vertical_solve_cpl(const DevMesh& m, int TP, const R* W, const R* st, const R* rhs,
                                      R* out, double bdt, const StageParams& sp, int* err,
                                      cudaStream_t stm);

// float <-> double conversion
cudaError_t launch_convert_d2f(const double* in, float* out, size_t n, cudaStream_t st);
cudaError_t launch_convert_f2d(const float* in, double* out, size_t n, cudaStream_t st);

}  // namespace slim
