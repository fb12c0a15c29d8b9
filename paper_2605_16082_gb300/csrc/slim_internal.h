// Internal structures shared by the translation units of libslim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/slim.h"

struct slim_state;

namespace slim {
struct SplitBufs;

// thread-local message of the last failing call
void set_error(const std::string& msg);
void clear_error();

#define SLIM_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::slim::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
      return (_e == cudaErrorMemoryAllocation) ? SLIM_ERR_OOM : SLIM_ERR_CUDA;     \
    }                                                                              \
  } while (0)

// Device-side view of the mesh.  Per-triangle arrays are structure-of-arrays:
// entry (j, t) of a [3][n_tri] array sits at j * n_tri + t.
struct DevMesh {
  int n_tri;
  int P;            // prisms
  int n_tiles;
  int max_layers;
  int max_tile_tris; // most triangles in one tile
  int n_levels;     // 0 for sigma layers
  const int* col_off;    // [n_tri + 1]
  const int* tile_t0;    // [n_tiles + 1] first triangle of each thread-block tile
  const int4* tile_info; // [n_tiles] (first triangle, triangles, first prism, prisms)
  const int4* einfo;     // [3][n_tri] per edge: (neighbour or -1 wall / -2 open, its first
                         // prism, its layer count, neighbour-local vertices l0 | l1 << 2)
  const double* jh;      // [n_tri] 2 x triangle area
  const double* gx;      // [3][n_tri] d phi_a / dx
  const double* gy;      // [3][n_tri]
  const double* enx;     // [3][n_tri] outward unit normal of edge e
  const double* eny;
  const double* elen;    // [3][n_tri] edge length
  const double* rin;     // [n_tri] inradius
  const float* rin_f;
  const double* h;       // [3][n_tri] rest depth at the vertices
  const int* nbr;        // [3][n_tri] neighbour triangle, -1 wall, -2 open boundary
  const int* nloc;       // [3][n_tri] neighbour-local vertices of own e, e+1: l0 | l1 << 2
  const double* levels;  // [n_levels] or null
  const double* hN;      // [3][n_tri] h / N (rest layer thickness of sigma columns)
  const double* ih;      // [3][n_tri] 1 / h
  const float* hN_f;
  const float* ih_f;
  const float* h_f;
  const float* levels_f;
  // float copies of the geometry for the mixed-precision kernels
  const float* jh_f;
  const float* gx_f;
  const float* gy_f;
  const float* enx_f;
  const float* eny_f;
  const float* elen_f;
  // [3][n_tri] 1 / min(r_in^-, r_in^+) of interior edges (0 elsewhere): the SIPG
  // penalty length of the horizontal diffusion
  const double* esig;
  const float* esig_f;
};

// Event pair around one kernel launch while profiling is on.
struct ProfScope {
  struct ::slim_state* s;
  int idx;
  cudaStream_t st;
  ProfScope(struct ::slim_state* s_, int phase, cudaStream_t st_);
  ~ProfScope();
};

}  // namespace slim

struct slim_mesh {
  slim::DevMesh d;
  std::vector<void*> allocs;
  int tile_prisms;
  // host copies used by host-side set-up
  std::vector<int> col_off_h;
  std::vector<int> tile_t0_h;
  std::vector<int> nbr_h;
  // first tile of each triangle class of a partition mesh (0 owned next to a ghost,
  // 1 owned interior, 2 ghost) and the tile count; 0, 0, 0, n_tiles otherwise
  int class_tile[4] = {0, 0, 0, 0};
};

struct slim_state {
  const slim_mesh* mesh;
  slim_precision prec;
  slim_params par;
  size_t esz;  // bytes per 3D value
  // 3D fields (compute type)
  void* T = nullptr; void* S = nullptr; void* U = nullptr; void* V = nullptr;
  void* W = nullptr;
  void* Text = nullptr; void* Sext = nullptr;   // open-boundary exterior profiles
  // open-boundary forcing of the split scheme: exterior velocity at the two forcing
  // times and the exterior tracers at the second (null for the tracer scheme)
  void* Uxa = nullptr; void* Vxa = nullptr; void* Uxb = nullptr; void* Vxb = nullptr;
  void* Textb = nullptr; void* Sextb = nullptr;
  void* tmp[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // stage buffers
  void* Rx = nullptr; void* Ry = nullptr;       // baroclinic pressure gradient
  // 2D fields (double)
  double* eta = nullptr; double* eta_next = nullptr;
  void* st_cur = nullptr; void* st_next = nullptr;  // stretch 1 + eta/h per vertex column (compute type)
  double* Qx = nullptr; double* Qy = nullptr;
  double* Qbx = nullptr; double* Qby = nullptr;
  double* aux2d = nullptr;  // scratch 2D storage (split scheme)
  size_t aux2d_len = 0;
  // reductions
  double* red = nullptr;    // block partials of the mass sum
  int red_blocks = 0;
  double* red_out = nullptr;
  // split scheme (2D external mode and coupling; allocated for SLIM_SCHEME_SPLIT)
  slim::SplitBufs* sp = nullptr;
  int* err = nullptr;       // device error flags
  double* stage64 = nullptr;  // 6P doubles: conversion staging of the mixed form
  int steps_since_check = 0;
  // CUDA graph of the whole step
  cudaStream_t g_stream = nullptr;
  cudaGraph_t g_graph = nullptr;      // kept alive: its node handles address the exec
  cudaGraphExec_t g_exec = nullptr;
  cudaEvent_t g_in = nullptr, g_out = nullptr;
  cudaGraphNode_t g_time_node = nullptr;
  cudaKernelNodeParams g_time_params{};
  double g_dt = 0.0;
  alignas(16) unsigned char g_time_args[128];  // the time kernel's argument for the next replay
  // phase timing (slim_profile_*)
  bool prof_on = false;
  int prof_max = 0;
  int prof_n = 0;
  std::vector<cudaEvent_t> prof_ev;  // 2 per recorded launch
  std::vector<int> prof_phase;
  std::vector<void*> allocs;
};
