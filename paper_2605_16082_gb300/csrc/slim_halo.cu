// Partitioned tracer step on one device: the horizontal domain decomposition of
// Sec. 3 ("Multi-GPU") emulated in one process.  Every partition is a state on
// its own mesh: its owned triangles (those next to another partition first, then
// the interior ones) followed by one layer of ghost triangles (the other
// partitions' triangles across its edges).  After every phase whose kernels read
// lateral neighbours, the owners' boundary values are copied into the ghosts:
// a pack kernel gathers them into a send buffer, one device-to-device
// cudaMemcpyAsync per partition pair moves the buffer, an unpack kernel scatters
// it into the ghost columns.  The boundary tiles of a stage run first on a
// high-priority stream that then carries the exchange, while the interior tiles
// run on a second stream (the boundary/interior split of Sec. 3).
//
// Lateral reads of the tracer scheme: the horizontal residual of the continuity
// (velocity, static within a step, and the elevation's stretch at t_n) and of
// each stage (the stage input tracer).  So a step exchanges the stage outputs
// (three 3D exchanges) and, at its end, the new elevation (one 2D exchange), after
// which every column's stretch is recomputed from its elevation.
#include <algorithm>
#include <string>
#include <vector>

#include "slim_kernels.h"

struct slim_halo {
  std::vector<slim_state*> parts;
  int K = 0;
  // pair (i -> j), i != j, with at least one triangle
  struct Pair {
    int src, dst, n;           // partitions, triangles
    int n_prisms;              // prisms of those columns
    int* d_src = nullptr;      // [n] local triangle ids in src
    int* d_dst = nullptr;      // [n] local ghost ids in dst
    int* d_off = nullptr;      // [n + 1] prism offsets of the triangles in the buffers
    void* send = nullptr;      // 6 x n_prisms values (3D) or 3 n doubles (2D), whichever is larger
    void* recv = nullptr;
  };
  std::vector<Pair> pairs;
  cudaStream_t s_bnd = nullptr, s_int = nullptr;
  std::vector<cudaEvent_t> ev;  // scratch events
  std::vector<void*> allocs;
};

namespace slim {
namespace {

// pack: column values of the listed owner triangles, all layers and node planes
template <typename R>
__global__ void k_pack3(const int* __restrict__ col_off, int P, const R* __restrict__ f,
                        const int* __restrict__ tri, const int* __restrict__ off, int n, R* __restrict__ buf) {
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const int t = tri[q], p0 = col_off[t], N = col_off[t + 1] - p0, b0 = off[q];
    for (int j = threadIdx.x; j < 6 * N; j += blockDim.x) {
      const int r = j / N, k = j - r * N;
      buf[(size_t)6 * b0 + j] = f[(size_t)r * P + p0 + k];
    }
  }
}

template <typename R>
__global__ void k_unpack3(const int* __restrict__ col_off, int P, R* __restrict__ f,
                          const int* __restrict__ tri, const int* __restrict__ off, int n,
                          const R* __restrict__ buf) {
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const int t = tri[q], p0 = col_off[t], N = col_off[t + 1] - p0, b0 = off[q];
    for (int j = threadIdx.x; j < 6 * N; j += blockDim.x) {
      const int r = j / N, k = j - r * N;
      f[(size_t)r * P + p0 + k] = buf[(size_t)6 * b0 + j];
    }
  }
}

// 2D nodal field (double, [3][n_tri])
__global__ void k_pack2(int nt, const double* __restrict__ f, const int* __restrict__ tri, int n,
                        double* __restrict__ buf) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 3 * n; j += gridDim.x * blockDim.x) {
    const int a = j / n, q = j - a * n;
    buf[j] = f[(size_t)a * nt + tri[q]];
  }
}
__global__ void k_unpack2(int nt, double* __restrict__ f, const int* __restrict__ tri, int n,
                          const double* __restrict__ buf) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 3 * n; j += gridDim.x * blockDim.x) {
    const int a = j / n, q = j - a * n;
    f[(size_t)a * nt + tri[q]] = buf[j];
  }
}

#define SLIM_HT(expr)                                                          \
  do {                                                                         \
    cudaError_t _e = (expr);                                                   \
    if (_e != cudaSuccess) {                                                   \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));           \
      return _e == cudaErrorMemoryAllocation ? SLIM_ERR_OOM : SLIM_ERR_CUDA;   \
    }                                                                          \
  } while (0)

// device address of a 3D field of a state by id (the tracer scheme's fields)
void* field3(slim_state* s, int field) {
  switch (field) {
    case SLIM_FIELD_T: return s->T;
    case SLIM_FIELD_S: return s->S;
    case SLIM_FIELD_U: return s->U;
    case SLIM_FIELD_V: return s->V;
    case SLIM_FIELD_W: return s->W;
  }
  return nullptr;
}

// exchange of a 3D buffer (one per partition, e.g. the stage output) on stream st
slim_status exchange3(slim_halo* h, void* const* bufs, cudaStream_t st) {
  for (auto& pr : h->pairs) {
    slim_state* a = h->parts[pr.src];
    const DevMesh& ma = a->mesh->d;
    const int grid = std::min(pr.n, 1024);
    if (a->prec == SLIM_FP64)
      k_pack3<double><<<grid, 128, 0, st>>>(ma.col_off, ma.P, (const double*)bufs[pr.src], pr.d_src, pr.d_off,
                                            pr.n, (double*)pr.send);
    else
      k_pack3<float><<<grid, 128, 0, st>>>(ma.col_off, ma.P, (const float*)bufs[pr.src], pr.d_src, pr.d_off,
                                           pr.n, (float*)pr.send);
    SLIM_HT(cudaGetLastError());
  }
  for (auto& pr : h->pairs)
    SLIM_HT(cudaMemcpyAsync(pr.recv, pr.send, (size_t)6 * pr.n_prisms * h->parts[pr.src]->esz,
                            cudaMemcpyDeviceToDevice, st));
  for (auto& pr : h->pairs) {
    slim_state* b = h->parts[pr.dst];
    const DevMesh& mb = b->mesh->d;
    const int grid = std::min(pr.n, 1024);
    if (b->prec == SLIM_FP64)
      k_unpack3<double><<<grid, 128, 0, st>>>(mb.col_off, mb.P, (double*)bufs[pr.dst], pr.d_dst, pr.d_off, pr.n,
                                              (const double*)pr.recv);
    else
      k_unpack3<float><<<grid, 128, 0, st>>>(mb.col_off, mb.P, (float*)bufs[pr.dst], pr.d_dst, pr.d_off, pr.n,
                                             (const float*)pr.recv);
    SLIM_HT(cudaGetLastError());
  }
  return SLIM_OK;
}

slim_status exchange_eta(slim_halo* h, cudaStream_t st) {
  for (auto& pr : h->pairs) {
    const int nt = h->parts[pr.src]->mesh->d.n_tri;
    k_pack2<<<std::min((3 * pr.n + 255) / 256, 1024), 256, 0, st>>>(nt, h->parts[pr.src]->eta, pr.d_src, pr.n,
                                                                      (double*)pr.send);
    SLIM_HT(cudaGetLastError());
  }
  for (auto& pr : h->pairs)
    SLIM_HT(cudaMemcpyAsync(pr.recv, pr.send, (size_t)3 * pr.n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  for (auto& pr : h->pairs) {
    const int nt = h->parts[pr.dst]->mesh->d.n_tri;
    k_unpack2<<<std::min((3 * pr.n + 255) / 256, 1024), 256, 0, st>>>(nt, h->parts[pr.dst]->eta, pr.d_dst, pr.n,
                                                                        (const double*)pr.recv);
    SLIM_HT(cudaGetLastError());
  }
  return SLIM_OK;
}

// the mesh restricted to tiles [t0, t1)
DevMesh tile_range(const DevMesh& m, int t0, int t1) {
  DevMesh r = m;
  r.tile_info = m.tile_info + t0;
  r.n_tiles = t1 - t0;
  return r;
}

cudaEvent_t ev(slim_halo* h, size_t i) { return h->ev[i]; }

template <typename R>
slim_status halo_step_t(slim_halo* h, double dt, cudaStream_t user) {
  const int K = h->K;
  // all partitions start after the caller's stream
  SLIM_HT(cudaEventRecord(ev(h, 0), user));
  SLIM_HT(cudaStreamWaitEvent(h->s_bnd, ev(h, 0), 0));
  SLIM_HT(cudaStreamWaitEvent(h->s_int, ev(h, 0), 0));
  // continuity over the owned tiles (no lateral output is read within the step)
  for (int p = 0; p < K; ++p) {
    slim_state* s = h->parts[p];
    const slim_mesh* me = s->mesh;
    const DevMesh mo = tile_range(me->d, 0, me->class_tile[2]);
    if (mo.n_tiles == 0) continue;
    const R* U = (const R*)s->U;
    const R* V = (const R*)s->V;
    cudaError_t e = s->par.vertical
        ? launch_continuity_cpl<R>(mo, me->tile_prisms, U, V, s->eta, (const R*)s->st_cur, s->eta_next,
                                   (R*)s->st_next, (R*)s->W, dt, h->s_bnd)
        : launch_continuity<R>(mo, me->tile_prisms, U, V, s->eta, (const R*)s->st_cur, s->eta_next,
                               (R*)s->st_next, (R*)s->W, dt, h->s_bnd);
    SLIM_HT(e);
  }
  SLIM_HT(cudaEventRecord(ev(h, 1), h->s_bnd));
  SLIM_HT(cudaStreamWaitEvent(h->s_int, ev(h, 1), 0));
  // three SSP-RK3 stages (the weights and stage elevations of slim_step)
  const double th_p[3] = {0.0, 1.0, 0.5}, th_s[3] = {1.0, 0.5, 1.0};
  const double al[3] = {0.0, 0.75, 1.0 / 3.0}, be[3] = {1.0, 0.25, 2.0 / 3.0};
  std::vector<void*> outs(K);
  for (int st = 0; st < 3; ++st) {
    for (int p = 0; p < K; ++p) {
      slim_state* s = h->parts[p];
      const slim_mesh* me = s->mesh;
      const R* Tp = (const R*)(st == 0 ? s->T : s->tmp[st - 1]);
      R* To = (R*)(st == 2 ? s->T : s->tmp[st]);
      outs[p] = To;
      StageParams sp{s->par.kappa_v, s->par.penalty_v, s->par.flux_top, s->par.flux_bot};
      // boundary tiles first (their outputs are what the neighbours need), then the
      // interior tiles on the other stream
      for (int part = 0; part < 2; ++part) {
        const DevMesh mr = part == 0 ? tile_range(me->d, 0, me->class_tile[1])
                                     : tile_range(me->d, me->class_tile[1], me->class_tile[2]);
        if (mr.n_tiles == 0) continue;
        cudaStream_t sm = part == 0 ? h->s_bnd : h->s_int;
        cudaError_t e = s->par.vertical
            ? launch_tracer_stage_cpl<R>(mr, me->tile_prisms, (const R*)s->U, (const R*)s->V, (const R*)s->T, Tp,
                                         (const R*)s->Text, (const R*)s->W, To, (const R*)s->st_cur,
                                         (const R*)s->st_next, th_p[st], th_s[st], al[st], be[st], dt, sp, s->err,
                                         sm)
            : launch_tracer_stage<R>(mr, me->tile_prisms, (const R*)s->U, (const R*)s->V, (const R*)s->T, Tp,
                                     (const R*)s->Text, (const R*)s->W, To, (const R*)s->st_cur,
                                     (const R*)s->st_next, th_p[st], th_s[st], al[st], be[st], dt, sp, s->err, sm);
        SLIM_HT(e);
      }
    }
    // the exchange follows the boundary tiles on their stream and overlaps the interior
    slim_status r = exchange3(h, outs.data(), h->s_bnd);
    if (r != SLIM_OK) return r;
    // the next stage needs both
    SLIM_HT(cudaEventRecord(ev(h, 2), h->s_int));
    SLIM_HT(cudaStreamWaitEvent(h->s_bnd, ev(h, 2), 0));
    SLIM_HT(cudaEventRecord(ev(h, 3), h->s_bnd));
    SLIM_HT(cudaStreamWaitEvent(h->s_int, ev(h, 3), 0));
  }
  // eta <- eta', exchange it, and every column's stretch from its elevation
  for (int p = 0; p < K; ++p) {
    slim_state* s = h->parts[p];
    SLIM_HT(cudaMemcpyAsync(s->eta, s->eta_next, sizeof(double) * 3 * s->mesh->d.n_tri, cudaMemcpyDeviceToDevice,
                            h->s_bnd));
  }
  slim_status r = exchange_eta(h, h->s_bnd);
  if (r != SLIM_OK) return r;
  for (int p = 0; p < K; ++p) {
    slim_state* s = h->parts[p];
    SLIM_HT(launch_stretch<R>(s->mesh->d, s->eta, (R*)s->st_cur, h->s_bnd));
  }
  SLIM_HT(cudaEventRecord(ev(h, 4), h->s_bnd));
  SLIM_HT(cudaStreamWaitEvent(user, ev(h, 4), 0));
  return SLIM_OK;
}

void free_halo(slim_halo* h) {
  if (!h) return;
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->s_bnd) cudaStreamDestroy(h->s_bnd);
  if (h->s_int) cudaStreamDestroy(h->s_int);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

}  // namespace
}  // namespace slim

using namespace slim;

extern "C" slim_status slim_halo_create(slim_state* const* parts, int n_parts, const int* pair_count,
                                        const int* send_tris, const int* recv_tris, slim_halo** out) {
  clear_error();
  if (!out) { set_error("out is null"); return SLIM_ERR_ARG; }
  *out = nullptr;
  if (!parts || n_parts < 1 || n_parts > 1024 || !pair_count) { set_error("null argument or bad count"); return SLIM_ERR_ARG; }
  for (int p = 0; p < n_parts; ++p) {
    if (!parts[p]) { set_error("null state"); return SLIM_ERR_ARG; }
    if (parts[p]->par.scheme != SLIM_SCHEME_TRACER) {
      set_error("the partitioned step is built for the tracer scheme");
      return SLIM_ERR_UNSUPPORTED;
    }
    if (parts[p]->prec != parts[0]->prec || parts[p]->par.vertical != parts[0]->par.vertical) {
      set_error("partitions differ in precision or column system");
      return SLIM_ERR_ARG;
    }
  }
  slim_halo* h = new slim_halo();
  h->K = n_parts;
  h->parts.assign(parts, parts + n_parts);
  auto fail = [&](slim_status st) { free_halo(h); return st; };
  size_t pos = 0;
  for (int i = 0; i < n_parts; ++i)
    for (int j = 0; j < n_parts; ++j) {
      const int n = pair_count[i * n_parts + j];
      if (n < 0 || (i == j && n != 0)) { set_error("bad pair count"); return fail(SLIM_ERR_ARG); }
      if (n == 0) continue;
      if (!send_tris || !recv_tris) { set_error("null triangle lists"); return fail(SLIM_ERR_ARG); }
      const slim_mesh* ma = parts[i]->mesh;
      const slim_mesh* mb = parts[j]->mesh;
      slim_halo::Pair pr;
      pr.src = i; pr.dst = j; pr.n = n;
      std::vector<int> src(send_tris + pos, send_tris + pos + n), dst(recv_tris + pos, recv_tris + pos + n);
      std::vector<int> off(n + 1, 0);
      for (int q = 0; q < n; ++q) {
        const int ts = src[q], td = dst[q];
        if (ts < 0 || ts >= ma->d.n_tri || td < 0 || td >= mb->d.n_tri) {
          set_error("triangle id out of range in the pair lists");
          return fail(SLIM_ERR_ARG);
        }
        const int Ns = ma->col_off_h[ts + 1] - ma->col_off_h[ts];
        const int Nd = mb->col_off_h[td + 1] - mb->col_off_h[td];
        if (Ns != Nd) { set_error("sender and ghost columns differ in layers"); return fail(SLIM_ERR_MESH); }
        off[q + 1] = off[q] + Ns;
      }
      pr.n_prisms = off[n];
      pos += n;
      const size_t bytes = std::max((size_t)6 * pr.n_prisms * parts[i]->esz, (size_t)3 * n * sizeof(double));
      void* d[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
      const size_t sz[5] = {n * sizeof(int), n * sizeof(int), (n + 1) * sizeof(int), bytes, bytes};
      for (int k = 0; k < 5; ++k) {
        cudaError_t e = cudaMalloc(&d[k], sz[k]);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return fail(SLIM_ERR_OOM); }
        h->allocs.push_back(d[k]);
      }
      pr.d_src = (int*)d[0]; pr.d_dst = (int*)d[1]; pr.d_off = (int*)d[2]; pr.send = d[3]; pr.recv = d[4];
      cudaError_t e = cudaMemcpy(pr.d_src, src.data(), sz[0], cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(pr.d_dst, dst.data(), sz[1], cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(pr.d_off, off.data(), sz[2], cudaMemcpyHostToDevice);
      if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return fail(SLIM_ERR_CUDA); }
      h->pairs.push_back(pr);
    }
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->s_bnd, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->s_int, cudaStreamNonBlocking, lo);
  h->ev.assign(5, nullptr);
  for (size_t k = 0; k < h->ev.size() && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&h->ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return fail(SLIM_ERR_CUDA); }
  *out = h;
  return SLIM_OK;
}

extern "C" void slim_halo_destroy(slim_halo* h) { free_halo(h); }

extern "C" slim_status slim_halo_exchange(slim_halo* h, int field, void* stream) {
  clear_error();
  if (!h) { set_error("halo is null"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (field == SLIM_FIELD_ETA) return exchange_eta(h, st);
  std::vector<void*> bufs(h->K);
  for (int p = 0; p < h->K; ++p) {
    bufs[p] = field3(h->parts[p], field);
    if (!bufs[p]) { set_error("field cannot be exchanged"); return SLIM_ERR_ARG; }
  }
  return exchange3(h, bufs.data(), st);
}

extern "C" slim_status slim_halo_step(slim_halo* h, double t, double dt, void* stream) {
  clear_error();
  (void)t;
  if (!h) { set_error("halo is null"); return SLIM_ERR_ARG; }
  if (!(dt > 0)) { set_error("dt must be positive"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  return h->parts[0]->prec == SLIM_FP64 ? halo_step_t<double>(h, dt, st) : halo_step_t<float>(h, dt, st);
}
