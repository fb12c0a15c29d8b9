// Tracer mass into caller memory without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// tracer mass: code running under a caching or pool allocator that forbids
// direct cudaMalloc/cudaFree, code inside a region where the host must not
// block or synchronize (cudaMalloc and cudaFree can do both), or embedders
// whose memory budget is fixed in advance.  slim_tracer_mass writes its block
// partials into a buffer of the state and copies the result to the host; this
// variant keeps the block partials in a fixed device array of this file and
// writes the result to a device address the caller passes, so the call itself
// allocates nothing and does not wait for the GPU.
#include <mutex>
#include <string>

#include "slim_device.cuh"
#include "slim_kernels.h"

namespace slim {
namespace {

// 2 doubles (compensated sum) per thread-block tile: at most 65536 tiles,
// 1 MiB held on every GPU that loads the library until the process exits.
constexpr int kNoAllocMaxTiles = 65536;
__device__ __align__(256) double g_mass_partials[2 * kNoAllocMaxTiles];

// Device address of g_mass_partials per device, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_partials_ptr[kMaxDevices] = {nullptr};
std::mutex g_partials_mu;

struct CS {
  double s, c;
};
__device__ __forceinline__ CS cs_add(CS x, CS y) {
  const double s = x.s + y.s;
  const double bp = s - x.s;
  const double err = (x.s - (s - bp)) + (y.s - bp);
  return {s, x.c + y.c + err};
}
template <int TP>
__device__ __forceinline__ CS cs_block(CS v, double* s_s, double* s_c) {
  s_s[threadIdx.x] = v.s;
  s_c[threadIdx.x] = v.c;
  __syncthreads();
  for (int w = TP / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      const CS r = cs_add({s_s[threadIdx.x], s_c[threadIdx.x]}, {s_s[threadIdx.x + w], s_c[threadIdx.x + w]});
      s_s[threadIdx.x] = r.s;
      s_c[threadIdx.x] = r.c;
    }
    __syncthreads();
  }
  return {s_s[0], s_c[0]};
}

// the same per-tile sum as the tracer-mass reduction, partials into `part`
template <typename R, int TP>
__global__ void __launch_bounds__(TP) k_mass_tiles(DevMesh m, const R* __restrict__ T,
                                                   const double* __restrict__ eta,
                                                   double* __restrict__ part) {
  __shared__ int s_off[TP + 1];
  __shared__ double s_s[TP], s_c[TP];
  const Tile tl = load_tile<TP>(m, s_off);
  const int i = threadIdx.x;
  CS v = {0.0, 0.0};
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    const int p = tl.p0 + i, nt = m.n_tri;
    const double w12 = m.jh[t] * (1.0 / 12.0);
    for (int a = 0; a < 3; ++a) {
      const double dz = dz_r<double>(m, a * nt + t, eta[a * nt + t], k, N);
      const double x = w12 * dz * ((double)T[(size_t)a * m.P + p] + (double)T[(size_t)(3 + a) * m.P + p]);
      v = cs_add(v, {x, 0.0});
    }
  }
  const CS r = cs_block<TP>(v, s_s, s_c);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r.s;
    part[2 * blockIdx.x + 1] = r.c;
  }
}

template <int TP>
__global__ void __launch_bounds__(TP) k_mass_total(const double* __restrict__ part, int n,
                                                   double* __restrict__ out) {
  __shared__ double s_s[TP], s_c[TP];
  CS v = {0.0, 0.0};
  for (int j = threadIdx.x; j < n; j += TP) v = cs_add(v, {part[2 * j], part[2 * j + 1]});
  const CS r = cs_block<TP>(v, s_s, s_c);
  if (threadIdx.x == 0) out[0] = r.s + r.c;
}

template <typename R>
cudaError_t launch_tiles(const DevMesh& m, int TP, const R* T, const double* eta, double* part,
                         cudaStream_t st) {
  switch (TP) {
    case 128: k_mass_tiles<R, 128><<<m.n_tiles, 128, 0, st>>>(m, T, eta, part); break;
    case 256: k_mass_tiles<R, 256><<<m.n_tiles, 256, 0, st>>>(m, T, eta, part); break;
    case 512: k_mass_tiles<R, 512><<<m.n_tiles, 512, 0, st>>>(m, T, eta, part); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// device address of the partials array on the current device (set-up on first use)
slim_status partials_ptr(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal above the supported range"); return SLIM_ERR_ARG; }
  std::lock_guard<std::mutex> lock(g_partials_mu);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mass_partials);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return SLIM_ERR_CUDA;
    }
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return SLIM_OK;
}

}  // namespace
}  // namespace slim

using namespace slim;

extern "C" slim_status slim_tracer_mass_noalloc(slim_state* s, int field, double* mass_dev,
                                                void* stream) {
  clear_error();
  if (!s || !mass_dev) { set_error("null argument"); return SLIM_ERR_ARG; }
  if (field != SLIM_FIELD_T && field != SLIM_FIELD_S) { set_error("field must be T or S"); return SLIM_ERR_ARG; }
  const DevMesh& m = s->mesh->d;
  if (m.n_tiles > kNoAllocMaxTiles) {
    set_error("mesh has " + std::to_string(m.n_tiles) + " tiles; slim_tracer_mass_noalloc supports at most " +
              std::to_string(kNoAllocMaxTiles) + " (use slim_tracer_mass or larger tiles)");
    return SLIM_ERR_ARG;
  }
  double* part = nullptr;
  slim_status r = partials_ptr(&part);
  if (r != SLIM_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const void* T = field == SLIM_FIELD_T ? s->T : s->S;
  cudaError_t e = s->prec == SLIM_FP64
                      ? launch_tiles<double>(m, s->mesh->tile_prisms, (const double*)T, s->eta, part, st)
                      : launch_tiles<float>(m, s->mesh->tile_prisms, (const float*)T, s->eta, part, st);
  if (e != cudaSuccess) { set_error(std::string("mass tiles: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  k_mass_total<256><<<1, 256, 0, st>>>(part, m.n_tiles, mass_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("mass total: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  return SLIM_OK;
}
