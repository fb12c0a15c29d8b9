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
// allocates nothing.  It runs the same two reduction kernels as slim_tracer_mass,
// so both give the same bits.
#include <mutex>
#include <string>

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
  // the reduction kernels of slim_tracer_mass (same order, same bits), with the
  // partials in the library array and the result at the caller's address
  const cudaError_t e =
      s->prec == SLIM_FP64
          ? launch_mass<double>(m, s->mesh->tile_prisms, (const double*)T, s->eta, part, mass_dev, st,
                                s->par.vertical != 0)
          : launch_mass<float>(m, s->mesh->tile_prisms, (const float*)T, s->eta, part, mass_dev, st,
                               s->par.vertical != 0);
  if (e != cudaSuccess) { set_error(std::string("tracer mass: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  return SLIM_OK;
}
