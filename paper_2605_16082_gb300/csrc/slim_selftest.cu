// Diagnostics of device building blocks against the compiler's own operations.
#include <string>

#include "slim_barrier.cuh"
#include "slim_device.cuh"
#include "slim_kernels.h"

namespace slim {
namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// i-th test pattern: raw bits (every class) or a double near the binary32 range
__global__ void k_conv_check(long long n, unsigned long long seed, unsigned long long* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r = splitmix64(seed ^ (unsigned long long)i * 0xd1342543de82ef95ull);
    unsigned long long db = r;
    if (i & 1) {  // exponent within [866, 1156]: subnormal, normal and overflowing binary32
      const unsigned long long E = 866 + (r >> 52) % 291;
      db = (r & 0x800fffffffffffffull) | (E << 52);
    }
    if ((i & 7) == 2) db &= 0xffffffffe0000000ull | ((r >> 7) & 0x10000000ull);  // exact halves
    const double x = __longlong_as_double((long long)db);
    const float a = d2f_bits(x), b = (float)x;
    const bool ok1 = (__float_as_uint(a) == __float_as_uint(b)) || (a != a && b != b);
    const float y = __uint_as_float((unsigned)(r >> 17));
    const double c = f2d_bits(y), d = (double)y;
    const bool ok2 = (__double_as_longlong(c) == __double_as_longlong(d)) || (c != c && d != d);
    if (!ok1) atomicAdd(&bad[0], 1ull);
    if (!ok2) atomicAdd(&bad[1], 1ull);
  }
}

// rounds of the grid barrier; block skip_block (if >= 0) leaves before the first
__global__ void k_barrier_check(unsigned* bar, int* err, int skip_block, int rounds, int* arrivals) {
  __shared__ int s_fail;
  for (int r = 0; r < rounds; ++r) {
    if ((int)blockIdx.x == skip_block) return;
    if (threadIdx.x == 0) atomicAdd(arrivals, 1);
    if (!grid_barrier(bar, gridDim.x, err, &s_fail)) return;
  }
}

// rounds of the neighbour waits of the persistent 2D run on a ring of blocks (block
// b waits for b - 1 and b + 1); block skip_block (if >= 0) leaves before the first
__global__ void k_nbwait_check(unsigned* done, int* err, int skip_block, int rounds, int* arrivals) {
  __shared__ int s_fail;
  __shared__ int s_nb[2];
  const int G = gridDim.x, b = blockIdx.x;
  const int nn = G > 2 ? 2 : G - 1;
  if (threadIdx.x == 0) {
    s_fail = 0;
    s_nb[0] = (b + G - 1) % G;
    s_nb[1] = (b + 1) % G;
  }
  __syncthreads();
  for (int r = 0; r < rounds; ++r) {
    if (b == skip_block) return;
    if (threadIdx.x == 0) atomicAdd(arrivals, 1);
    if (!neighbour_wait(done, (unsigned)(r + 1), s_nb, nn, err, &s_fail)) return;
  }
}

// Arithmetic peak: every thread runs 8 independent FMA chains (enough independent
// work to keep the pipe busy at full occupancy); a result is stored only when it
// is NaN, which never happens, so that the chains are not removed.
template <typename R>
__global__ void __launch_bounds__(256) k_fma_peak(long long iters, R b, R c, R* out) {
  R a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (R)(threadIdx.x + j) * (R)1e-3;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  R s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s != s) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace slim

using namespace slim;

extern "C" slim_status slim_selftest_fma_peak(int precision, long long iters, double* flops_per_s,
                                              double* ms) {
  clear_error();
  if ((precision != SLIM_FP64 && precision != SLIM_MIXED) || iters < 1 || !flops_per_s || !ms) {
    set_error("bad argument");
    return SLIM_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = 8 * sms, threads = 256;
  void* d = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d, (size_t)blocks * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float t = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0);
    if (precision == SLIM_FP64)
      k_fma_peak<double><<<blocks, threads>>>(iters, 0.999999, 1e-7, (double*)d);
    else
      k_fma_peak<float><<<blocks, threads>>>(iters, 0.9999f, 1e-4f, (float*)d);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d) cudaFree(d);
  if (e != cudaSuccess) { set_error(std::string("selftest: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  *ms = t;
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (t * 1e-3);
  return SLIM_OK;
}

extern "C" slim_status slim_selftest_barrier(int n_blocks, int skip_block, int rounds, int* err_bits,
                                             int* arrivals) {
  clear_error();
  if (n_blocks < 1 || n_blocks > 1024 || rounds < 0 || !err_bits || !arrivals) {
    set_error("bad argument");
    return SLIM_ERR_ARG;
  }
  int* d = nullptr;  // [0] error bits, [1] arrivals, [2..3] barrier words
  cudaError_t e = cudaMalloc((void**)&d, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 4 * sizeof(int));
  if (e == cudaSuccess) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_blocks);
    cfg.blockDim = dim3(128);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_barrier_check, reinterpret_cast<unsigned*>(d + 2), d, skip_block,
                           rounds, d + 1);
  }
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) { set_error(std::string("selftest: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  *err_bits = h[0];
  *arrivals = h[1];
  return SLIM_OK;
}

extern "C" slim_status slim_selftest_neighbour_wait(int n_blocks, int skip_block, int rounds, int* err_bits,
                                                    int* arrivals) {
  clear_error();
  if (n_blocks < 2 || n_blocks > 1024 || rounds < 0 || !err_bits || !arrivals) {
    set_error("bad argument");
    return SLIM_ERR_ARG;
  }
  int* d = nullptr;  // [0] error bits, [1] arrivals, [2 ..] one stage counter per block
  const size_t words = 2 + (size_t)n_blocks;
  cudaError_t e = cudaMalloc((void**)&d, words * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, words * sizeof(int));
  if (e == cudaSuccess) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_blocks);
    cfg.blockDim = dim3(128);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_nbwait_check, reinterpret_cast<unsigned*>(d + 2), d, skip_block, rounds,
                           d + 1);
  }
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) { set_error(std::string("selftest: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  *err_bits = h[0];
  *arrivals = h[1];
  return SLIM_OK;
}

extern "C" slim_status slim_selftest_conversions(long long n, unsigned long long seed,
                                                 long long* bad_d2f, long long* bad_f2d) {
  clear_error();
  if (n < 0 || !bad_d2f || !bad_f2d) { set_error("bad argument"); return SLIM_ERR_ARG; }
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc((void**)&d, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && n > 0) {
    k_conv_check<<<4 * 152, 256>>>(n, seed, d);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) { set_error(std::string("selftest: ") + cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  *bad_d2f = (long long)h[0];
  *bad_f2d = (long long)h[1];
  return SLIM_OK;
}
