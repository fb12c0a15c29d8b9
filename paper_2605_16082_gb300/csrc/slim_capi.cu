// C ABI: parameters, state management, field transfer and the hot-path
// operations (dispatch on the state's precision to the kernel launchers).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "slim_internal.h"
#include "slim_kernels.h"
#include "slim_split.h"

using namespace slim;

extern "C" slim_status slim_params_default(slim_params* p) {
  if (!p) { set_error("params is null"); return SLIM_ERR_ARG; }
  std::memset(p, 0, sizeof(*p));
  p->g = 9.81;
  p->rho0 = 1025.0;
  p->coriolis_f = 1e-4;
  p->eos_alpha = 2e-4;
  p->eos_beta = 7.6e-4;
  p->eos_T0 = 10.0;
  p->eos_S0 = 35.0;
  p->kappa_v = 1e-3;
  p->nu_v = 1e-3;
  p->kappa_h = 0.0;
  p->nu_h = 0.0;
  p->drag_cd = 2.5e-3;
  p->flux_top = 0.0;
  p->flux_bot = 0.0;
  p->penalty_v = 4.0;
  p->penalty_h = 6.0;
  p->tide_amp = 1.0;
  p->tide_period = 44712.0;
  p->scheme = SLIM_SCHEME_TRACER;
  p->n_sub = 20;
  p->tile_prisms = 256;
  p->check_every = 0;
  p->blocks_per_sm = 0;
  p->use_graph = 1;
  p->persistent_2d = 1;
  p->forcing_t_a = 0.0;
  p->forcing_t_b = 1.0;
  p->forcing = 0;
  p->vertical = 0;
  return SLIM_OK;
}

namespace {

slim_status check_params(const slim_params* par) {
  if (!par) { set_error("params is null"); return SLIM_ERR_ARG; }
  if (par->scheme != SLIM_SCHEME_TRACER && par->scheme != SLIM_SCHEME_SPLIT) {
    set_error("unknown scheme");
    return SLIM_ERR_ARG;
  }
  if (par->scheme == SLIM_SCHEME_SPLIT && (par->n_sub < 2 || (par->n_sub % 2) != 0)) {
    set_error("n_sub must be even and >= 2 for the split scheme");
    return SLIM_ERR_ARG;
  }
  if (!(par->kappa_v >= 0) || !(par->nu_v >= 0) || !(par->penalty_v > 0)) {
    set_error("diffusivities must be >= 0 and penalty > 0");
    return SLIM_ERR_ARG;
  }
  if (par->forcing != 0 && par->forcing != 1) { set_error("forcing must be 0 or 1"); return SLIM_ERR_ARG; }
  if (par->forcing && par->scheme != SLIM_SCHEME_SPLIT) {
    set_error("open-boundary forcing needs the split scheme");
    return SLIM_ERR_ARG;
  }
  if (par->forcing && !(par->forcing_t_b > par->forcing_t_a)) {
    set_error("forcing_t_b must be later than forcing_t_a");
    return SLIM_ERR_ARG;
  }
  if (par->vertical != 0 && par->vertical != 1) { set_error("vertical must be 0 or 1"); return SLIM_ERR_ARG; }
  if (par->vertical == 1 && par->scheme != SLIM_SCHEME_TRACER) {
    set_error("the coupled column system (vertical = 1) is built for the tracer scheme only");
    return SLIM_ERR_UNSUPPORTED;
  }
  return SLIM_OK;
}

slim_status dev_alloc(slim_state* s, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? SLIM_ERR_OOM : SLIM_ERR_CUDA;
  }
  s->allocs.push_back(*p);
  e = cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return SLIM_ERR_CUDA; }
  return SLIM_OK;
}

void drop_graph(slim_state* s) {
  if (s->g_exec) cudaGraphExecDestroy(s->g_exec);
  if (s->g_graph) cudaGraphDestroy(s->g_graph);
  s->g_exec = nullptr;
  s->g_graph = nullptr;
  s->g_time_node = nullptr;
}

void free_state(slim_state* s) {
  if (!s) return;
  drop_graph(s);
  if (s->g_in) cudaEventDestroy(s->g_in);
  if (s->g_out) cudaEventDestroy(s->g_out);
  if (s->g_stream) cudaStreamDestroy(s->g_stream);
  split_free(s);
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  for (void* p : s->allocs) cudaFree(p);
  delete s;
}

struct FieldRef {
  void* ptr;
  bool is3d;
  bool is_double;
};

bool field_ref(slim_state* s, int field, FieldRef* r) {
  const bool dbl3 = s->prec == SLIM_FP64;
  switch (field) {
    case SLIM_FIELD_T: *r = {s->T, true, dbl3}; return true;
    case SLIM_FIELD_S: *r = {s->S, true, dbl3}; return true;
    case SLIM_FIELD_U: *r = {s->U, true, dbl3}; return true;
    case SLIM_FIELD_V: *r = {s->V, true, dbl3}; return true;
    case SLIM_FIELD_W: *r = {s->W, true, dbl3}; return true;
    case SLIM_FIELD_R_X: *r = {s->Rx, true, dbl3}; return true;
    case SLIM_FIELD_R_Y: *r = {s->Ry, true, dbl3}; return true;
    case SLIM_FIELD_T_EXT: *r = {s->Text, true, dbl3}; return true;
    case SLIM_FIELD_S_EXT: *r = {s->Sext, true, dbl3}; return true;
    case SLIM_FIELD_U_EXT: if (!s->Uxa) return false; *r = {s->Uxa, true, dbl3}; return true;
    case SLIM_FIELD_V_EXT: if (!s->Vxa) return false; *r = {s->Vxa, true, dbl3}; return true;
    case SLIM_FIELD_U_EXT_B: if (!s->Uxb) return false; *r = {s->Uxb, true, dbl3}; return true;
    case SLIM_FIELD_V_EXT_B: if (!s->Vxb) return false; *r = {s->Vxb, true, dbl3}; return true;
    case SLIM_FIELD_T_EXT_B: if (!s->Textb) return false; *r = {s->Textb, true, dbl3}; return true;
    case SLIM_FIELD_S_EXT_B: if (!s->Sextb) return false; *r = {s->Sextb, true, dbl3}; return true;
    case SLIM_FIELD_ETA: *r = {s->eta, false, true}; return true;
    case SLIM_FIELD_QX: *r = {s->Qx, false, true}; return true;
    case SLIM_FIELD_QY: *r = {s->Qy, false, true}; return true;
    case SLIM_FIELD_ETA_NEXT: *r = {s->eta_next, false, true}; return true;
    case SLIM_FIELD_QBAR_X: *r = {s->Qbx, false, true}; return true;
    case SLIM_FIELD_QBAR_Y: *r = {s->Qby, false, true}; return true;
    case SLIM_FIELD_S3_X: case SLIM_FIELD_S3_Y: case SLIM_FIELD_F2D_X: case SLIM_FIELD_F2D_Y: {
      void* p = split_field(s, field);
      if (!p) return false;
      *r = {p, false, true};
      return true;
    }
  }
  return false;
}

size_t field_len(const slim_state* s, bool is3d) {
  return is3d ? (size_t)6 * s->mesh->d.P : (size_t)3 * s->mesh->d.n_tri;
}

StageParams tracer_stage_params(const slim_state* s) {
  StageParams sp;
  sp.kappa = s->par.kappa_v;
  sp.penalty = s->par.penalty_v;
  sp.flux_top = s->par.flux_top;
  sp.flux_bot = s->par.flux_bot;
  return sp;
}

int tile_of(const slim_state* s) { return s->mesh->tile_prisms; }

#define SLIM_LAUNCH(expr)                                                     \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) {                                                  \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));          \
      return SLIM_ERR_CUDA;                                                   \
    }                                                                         \
  } while (0)

template <typename R>
slim_status tracer_step(slim_state* s, double dt, cudaStream_t st) {
  const DevMesh& m = s->mesh->d;
  const int TP = tile_of(s);
  const R* U = (const R*)s->U;
  const R* V = (const R*)s->V;
  R* T = (R*)s->T;
  R* T1 = (R*)s->tmp[0];
  R* T2 = (R*)s->tmp[1];
  R* W = (R*)s->W;
  const R* Text = (const R*)s->Text;
  const StageParams sp = tracer_stage_params(s);
  const R* st0 = (const R*)s->st_cur;
  const R* st1 = (const R*)s->st_next;
  {
    ProfScope ps(s, SLIM_PHASE_CONTINUITY, st);
      if (s->par.vertical)
      SLIM_LAUNCH(launch_continuity_cpl<R>(m, TP, U, V, s->eta, st0, s->eta_next, (R*)s->st_next, W, dt, st));
    else
      SLIM_LAUNCH(launch_continuity<R>(m, TP, U, V, s->eta, st0, s->eta_next, (R*)s->st_next, W, dt, st));
  }
  // Shu-Osher SSP-RK3: (alpha, beta) = (0, 1), (3/4, 1/4), (1/3, 2/3);
  // stage elevations eta^{n+1}, (eta^n + eta^{n+1})/2, eta^{n+1}
  const bool cpl = s->par.vertical != 0;
  auto stage = [&](const R* Tp, R* To, double th_p, double th_s, double al, double be) {
    return cpl ? launch_tracer_stage_cpl<R>(m, TP, U, V, T, Tp, Text, W, To, st0, st1, th_p, th_s, al, be, dt,
                                            sp, s->err, st)
               : launch_tracer_stage<R>(m, TP, U, V, T, Tp, Text, W, To, st0, st1, th_p, th_s, al, be, dt, sp,
                                        s->err, st);
  };
  {
    ProfScope ps(s, SLIM_PHASE_TRACER_STAGE, st);
    SLIM_LAUNCH(stage(T, T1, 0.0, 1.0, 0.0, 1.0));
  }
  {
    ProfScope ps(s, SLIM_PHASE_TRACER_STAGE, st);
    SLIM_LAUNCH(stage(T1, T2, 1.0, 0.5, 0.75, 0.25));
  }
  {
    ProfScope ps(s, SLIM_PHASE_TRACER_STAGE, st);
    SLIM_LAUNCH(stage(T2, T, 0.5, 1.0, 1.0 / 3.0, 2.0 / 3.0));
  }
  SLIM_CUDA_TRY(cudaMemcpyAsync(s->eta, s->eta_next, sizeof(double) * 3 * m.n_tri,
                                cudaMemcpyDeviceToDevice, st));
  SLIM_CUDA_TRY(cudaMemcpyAsync(s->st_cur, s->st_next, sizeof(R) * 3 * m.n_tri,
                                cudaMemcpyDeviceToDevice, st));
  return SLIM_OK;
}

slim_status refresh_stretch(slim_state* s, cudaStream_t st) {
  if (s->prec == SLIM_FP64)
    SLIM_LAUNCH(launch_stretch<double>(s->mesh->d, s->eta, (double*)s->st_cur, st));
  else
    SLIM_LAUNCH(launch_stretch<float>(s->mesh->d, s->eta, (float*)s->st_cur, st));
  return SLIM_OK;
}

}  // namespace

extern "C" slim_status slim_state_alloc(const slim_mesh* m, slim_precision prec,
                                        const slim_params* par, slim_state** out) {
  clear_error();
  if (!out) { set_error("out is null"); return SLIM_ERR_ARG; }
  *out = nullptr;
  if (!m) { set_error("mesh is null"); return SLIM_ERR_ARG; }
  if (prec != SLIM_FP64 && prec != SLIM_MIXED) { set_error("unknown precision"); return SLIM_ERR_ARG; }
  slim_status st = check_params(par);
  if (st != SLIM_OK) return st;
  if (par->vertical == 1) {
    const size_t esz = prec == SLIM_FP64 ? sizeof(double) : sizeof(float);
    if (coupled_smem_bytes(m->d, m->tile_prisms, esz) > (size_t)227 * 1024) {
      set_error("coupled column system: the tile's shared memory exceeds 227 KB (use smaller tiles)");
      return SLIM_ERR_UNSUPPORTED;
    }
  }
  slim_state* s = new slim_state();
  s->mesh = m;
  s->prec = prec;
  s->par = *par;
  s->esz = prec == SLIM_FP64 ? sizeof(double) : sizeof(float);
  const size_t n3 = (size_t)6 * m->d.P, n2 = (size_t)3 * m->d.n_tri;
  void** f3[] = {&s->T, &s->S, &s->U, &s->V, &s->W, &s->Text, &s->Sext, &s->Rx, &s->Ry,
                 &s->tmp[0], &s->tmp[1], &s->tmp[2], &s->tmp[3], &s->tmp[4], &s->tmp[5]};
  for (void** f : f3)
    if ((st = dev_alloc(s, f, n3 * s->esz)) != SLIM_OK) { free_state(s); return st; }
  double** f2[] = {&s->eta, &s->eta_next, &s->Qx, &s->Qy, &s->Qbx, &s->Qby};
  for (double** f : f2)
    if ((st = dev_alloc(s, (void**)f, n2 * sizeof(double))) != SLIM_OK) { free_state(s); return st; }
  void** fs[] = {&s->st_cur, &s->st_next};
  for (void** f : fs)
    if ((st = dev_alloc(s, f, n2 * s->esz)) != SLIM_OK) { free_state(s); return st; }
  if ((st = refresh_stretch(s, 0)) != SLIM_OK) { free_state(s); return st; }
  if (par->scheme == SLIM_SCHEME_SPLIT) {
    if (par->n_sub < 2 || par->n_sub % 2) { free_state(s); set_error("n_sub must be even"); return SLIM_ERR_ARG; }
    void** fx[] = {&s->Uxa, &s->Vxa, &s->Uxb, &s->Vxb, &s->Textb, &s->Sextb};
    for (void** f : fx) {
      if ((st = dev_alloc(s, f, n3 * s->esz)) != SLIM_OK) { free_state(s); return st; }
      cudaMemset(*f, 0, n3 * s->esz);
    }
    if ((st = split_alloc(s)) != SLIM_OK) { free_state(s); return st; }
  }
  s->aux2d_len = split_aux2d_len(m->d);
  if ((st = dev_alloc(s, (void**)&s->aux2d, s->aux2d_len * sizeof(double))) != SLIM_OK) { free_state(s); return st; }
  s->red_blocks = m->d.n_tiles;
  if ((st = dev_alloc(s, (void**)&s->red, (size_t)2 * s->red_blocks * sizeof(double))) != SLIM_OK) { free_state(s); return st; }
  if ((st = dev_alloc(s, (void**)&s->red_out, 4 * sizeof(double))) != SLIM_OK) { free_state(s); return st; }
  if ((st = dev_alloc(s, (void**)&s->err, 4 * sizeof(int))) != SLIM_OK) { free_state(s); return st; }
  if (prec == SLIM_MIXED) {
    if ((st = dev_alloc(s, (void**)&s->stage64, n3 * sizeof(double))) != SLIM_OK) { free_state(s); return st; }
  }
  *out = s;
  return SLIM_OK;
}

extern "C" void slim_state_free(slim_state* s) { free_state(s); }

extern "C" slim_status slim_state_set_params(slim_state* s, const slim_params* par) {
  clear_error();
  if (!s) { set_error("state is null"); return SLIM_ERR_ARG; }
  slim_status st = check_params(par);
  if (st != SLIM_OK) return st;
  if (par->scheme != s->par.scheme) { set_error("scheme cannot change"); return SLIM_ERR_ARG; }
  if (par->vertical != s->par.vertical) { set_error("vertical cannot change"); return SLIM_ERR_ARG; }
  if (par->scheme == SLIM_SCHEME_SPLIT && par->n_sub != s->par.n_sub) {
    set_error("n_sub cannot change");
    return SLIM_ERR_ARG;
  }
  s->par = *par;
  drop_graph(s);
  return SLIM_OK;
}

extern "C" slim_status slim_state_upload(slim_state* s, int field, const double* host, void* stream) {
  clear_error();
  if (!s || !host) { set_error("null argument"); return SLIM_ERR_ARG; }
  FieldRef r;
  if (!field_ref(s, field, &r) || field == SLIM_FIELD_W) { set_error("field cannot be uploaded"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = field_len(s, r.is3d);
  // fields that an upload also sets: the exterior tracer levels (T, S) and the
  // second forcing level of a first-level exterior field
  void* mirror[2] = {nullptr, nullptr};
  switch (field) {
    case SLIM_FIELD_T: mirror[0] = s->Text; mirror[1] = s->Textb; break;
    case SLIM_FIELD_S: mirror[0] = s->Sext; mirror[1] = s->Sextb; break;
    case SLIM_FIELD_T_EXT: mirror[0] = s->Textb; break;
    case SLIM_FIELD_S_EXT: mirror[0] = s->Sextb; break;
    case SLIM_FIELD_U_EXT: mirror[0] = s->Uxb; break;
    case SLIM_FIELD_V_EXT: mirror[0] = s->Vxb; break;
  }
  const size_t bytes = n * (r.is_double ? sizeof(double) : sizeof(float));
  if (r.is_double) {
    SLIM_CUDA_TRY(cudaMemcpyAsync(r.ptr, host, n * sizeof(double), cudaMemcpyHostToDevice, st));
  } else {
    SLIM_CUDA_TRY(cudaMemcpyAsync(s->stage64, host, n * sizeof(double), cudaMemcpyHostToDevice, st));
    SLIM_LAUNCH(launch_convert_d2f(s->stage64, (float*)r.ptr, n, st));
  }
  for (void* mp : mirror)
    if (mp) SLIM_CUDA_TRY(cudaMemcpyAsync(mp, r.ptr, bytes, cudaMemcpyDeviceToDevice, st));
  if (field == SLIM_FIELD_ETA) return refresh_stretch(s, st);
  return SLIM_OK;
}

extern "C" slim_status slim_state_download(slim_state* s, int field, double* host, void* stream) {
  clear_error();
  if (!s || !host) { set_error("null argument"); return SLIM_ERR_ARG; }
  FieldRef r;
  if (!field_ref(s, field, &r)) { set_error("unknown field"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = field_len(s, r.is3d);
  if (r.is_double) {
    SLIM_CUDA_TRY(cudaMemcpyAsync(host, r.ptr, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  } else {
    SLIM_LAUNCH(launch_convert_f2d((const float*)r.ptr, s->stage64, n, st));
    SLIM_CUDA_TRY(cudaMemcpyAsync(host, s->stage64, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  SLIM_CUDA_TRY(cudaStreamSynchronize(st));
  return SLIM_OK;
}

extern "C" slim_status slim_state_field_ptr(slim_state* s, int field, void** dev, int* elem_size) {
  clear_error();
  if (!s || !dev) { set_error("null argument"); return SLIM_ERR_ARG; }
  FieldRef r;
  if (!field_ref(s, field, &r)) { set_error("unknown field"); return SLIM_ERR_ARG; }
  *dev = r.ptr;
  if (elem_size) *elem_size = r.is_double ? 8 : 4;
  return SLIM_OK;
}

extern "C" slim_status slim_state_check(slim_state* s, void* stream) {
  clear_error();
  if (!s) { set_error("state is null"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  int flags[4] = {0, 0, 0, 0};
  SLIM_CUDA_TRY(cudaMemcpyAsync(flags, s->err, sizeof(flags), cudaMemcpyDeviceToHost, st));
  SLIM_CUDA_TRY(cudaStreamSynchronize(st));
  SLIM_CUDA_TRY(cudaMemsetAsync(s->err, 0, sizeof(flags), st));
  SLIM_CUDA_TRY(cudaStreamSynchronize(st));
  if (flags[0] & SLIM_ERRBIT_TIMEOUT) { set_error("a bounded device wait gave up"); return SLIM_ERR_TIMEOUT; }
  if (flags[0] & SLIM_ERRBIT_BOUNDS) { set_error("device index out of range"); return SLIM_ERR_BOUNDS; }
  if (flags[0] & SLIM_ERRBIT_NONFINITE) { set_error("non-finite value produced"); return SLIM_ERR_NONFINITE; }
  return SLIM_OK;
}

// ---------------------------------------------------------------------------
// operations
// ---------------------------------------------------------------------------
namespace {
template <typename R>
slim_status rhs3d_t(slim_state* s, int field, void* out, cudaStream_t st) {
  const R* T = (const R*)(field == SLIM_FIELD_T ? s->T : s->S);
  const R* Text = (const R*)(field == SLIM_FIELD_T ? s->Text : s->Sext);
  SLIM_LAUNCH(launch_rhs3d<R>(s->mesh->d, tile_of(s), (const R*)s->U, (const R*)s->V, T, Text,
                              (const R*)s->st_cur, (R*)out, st));
  return SLIM_OK;
}
}  // namespace

extern "C" slim_status slim_rhs3d(slim_state* s, int field, void* out_dev, void* stream) {
  clear_error();
  if (!s || !out_dev) { set_error("null argument"); return SLIM_ERR_ARG; }
  if (field == SLIM_FIELD_U || field == SLIM_FIELD_V) {
    if (s->par.scheme != SLIM_SCHEME_SPLIT) {
      set_error("the momentum residual needs SLIM_SCHEME_SPLIT");
      return SLIM_ERR_UNSUPPORTED;
    }
    return split_rhs3d_momentum(s, field, out_dev, (cudaStream_t)stream);
  }
  if (field != SLIM_FIELD_T && field != SLIM_FIELD_S) { set_error("field must be T, S, U or V"); return SLIM_ERR_ARG; }
  return s->prec == SLIM_FP64 ? rhs3d_t<double>(s, field, out_dev, (cudaStream_t)stream)
                              : rhs3d_t<float>(s, field, out_dev, (cudaStream_t)stream);
}

extern "C" slim_status slim_continuity(slim_state* s, double dt, void* stream) {
  clear_error();
  if (!s) { set_error("state is null"); return SLIM_ERR_ARG; }
  if (!(dt > 0)) { set_error("dt must be positive"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const bool cpl = s->par.vertical != 0;
  if (s->prec == SLIM_FP64) {
    auto f = cpl ? launch_continuity_cpl<double> : launch_continuity<double>;
    SLIM_LAUNCH(f(s->mesh->d, tile_of(s), (const double*)s->U, (const double*)s->V, s->eta,
                  (const double*)s->st_cur, s->eta_next, (double*)s->st_next, (double*)s->W, dt, st));
  } else {
    auto f = cpl ? launch_continuity_cpl<float> : launch_continuity<float>;
    SLIM_LAUNCH(f(s->mesh->d, tile_of(s), (const float*)s->U, (const float*)s->V, s->eta,
                  (const float*)s->st_cur, s->eta_next, (float*)s->st_next, (float*)s->W, dt, st));
  }
  return SLIM_OK;
}

extern "C" slim_status slim_rhs2d(slim_state* s, double t, double* out_dev, void* stream) {
  clear_error();
  if (!s || !out_dev) { set_error("null argument"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (s->par.scheme == SLIM_SCHEME_SPLIT) return split_rhs2d(s, t, out_dev, st);
  if (s->prec == SLIM_FP64)
    SLIM_LAUNCH(launch_column_divergence<double>(s->mesh->d, tile_of(s), (const double*)s->U,
                                                 (const double*)s->V, (const double*)s->st_cur, out_dev, st));
  else
    SLIM_LAUNCH(launch_column_divergence<float>(s->mesh->d, tile_of(s), (const float*)s->U,
                                                (const float*)s->V, (const float*)s->st_cur, out_dev, st));
  return SLIM_OK;
}

extern "C" slim_status slim_vertical_solve(slim_state* s, int field, double beta_dt,
                                           const void* rhs_dev, void* out_dev, void* stream) {
  clear_error();
  if (!s || !rhs_dev || !out_dev) { set_error("null argument"); return SLIM_ERR_ARG; }
  if (field < SLIM_FIELD_T || field > SLIM_FIELD_V) { set_error("field must be T, S, U or V"); return SLIM_ERR_ARG; }
  if (!(beta_dt >= 0)) { set_error("beta_dt must be >= 0"); return SLIM_ERR_ARG; }
  StageParams sp = tracer_stage_params(s);
  if (field == SLIM_FIELD_U || field == SLIM_FIELD_V) {
    sp.kappa = s->par.nu_v;
    sp.flux_top = sp.flux_bot = 0.0;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool cpl = s->par.vertical != 0;
  if (s->prec == SLIM_FP64) {
    auto f = cpl ? launch_vertical_solve_cpl<double> : launch_vertical_solve<double>;
    SLIM_LAUNCH(f(s->mesh->d, tile_of(s), (const double*)s->W, (const double*)s->st_cur,
                  (const double*)rhs_dev, (double*)out_dev, beta_dt, sp, s->err, st));
  } else {
    auto f = cpl ? launch_vertical_solve_cpl<float> : launch_vertical_solve<float>;
    SLIM_LAUNCH(f(s->mesh->d, tile_of(s), (const float*)s->W, (const float*)s->st_cur,
                  (const float*)rhs_dev, (float*)out_dev, beta_dt, sp, s->err, st));
  }
  return SLIM_OK;
}

extern "C" slim_status slim_hpg(slim_state* s, void* stream) {
  clear_error();
  if (!s) { set_error("state is null"); return SLIM_ERR_ARG; }
  if (s->par.scheme != SLIM_SCHEME_SPLIT) { set_error("slim_hpg needs SLIM_SCHEME_SPLIT"); return SLIM_ERR_UNSUPPORTED; }
  return split_hpg(s, (cudaStream_t)stream);
}

namespace {
slim_status step_launches(slim_state* s, double t, double dt, cudaStream_t st) {
  if (s->par.scheme == SLIM_SCHEME_SPLIT) return split_step(s, t, dt, st);
  return s->prec == SLIM_FP64 ? tracer_step<double>(s, dt, st) : tracer_step<float>(s, dt, st);
}

// Capture the whole step once into a graph on the state's own stream, locate the
// time kernel (first argument = start time) and replay; between replays only the
// start time of that node changes.
slim_status step_graph(slim_state* s, double t, double dt, cudaStream_t user) {
  if (!s->g_stream) {
    SLIM_CUDA_TRY(cudaStreamCreateWithFlags(&s->g_stream, cudaStreamNonBlocking));
    SLIM_CUDA_TRY(cudaEventCreateWithFlags(&s->g_in, cudaEventDisableTiming));
    SLIM_CUDA_TRY(cudaEventCreateWithFlags(&s->g_out, cudaEventDisableTiming));
  }
  if (!s->g_exec || s->g_dt != dt) {
    drop_graph(s);
    cudaGraph_t g = nullptr;
    SLIM_CUDA_TRY(cudaStreamBeginCapture(s->g_stream, cudaStreamCaptureModeThreadLocal));
    slim_status r = step_launches(s, t, dt, s->g_stream);
    cudaError_t ce = cudaStreamEndCapture(s->g_stream, &g);
    if (r != SLIM_OK) { if (g) cudaGraphDestroy(g); return r; }
    if (ce != cudaSuccess) { set_error(std::string("capture: ") + cudaGetErrorString(ce)); return SLIM_ERR_CUDA; }
    ce = cudaGraphInstantiate(&s->g_exec, g, 0);
    if (ce == cudaSuccess && s->par.scheme == SLIM_SCHEME_SPLIT) {
      size_t n = 0;
      cudaGraphGetNodes(g, nullptr, &n);
      std::vector<cudaGraphNode_t> nodes(n);
      cudaGraphGetNodes(g, nodes.data(), &n);
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        if (kp.func == split_time_kernel()) {
          s->g_time_node = nd;
          s->g_time_params = kp;
          break;
        }
      }
    }
    s->g_graph = g;
    if (ce != cudaSuccess) {
      drop_graph(s);
      set_error(std::string("instantiate: ") + cudaGetErrorString(ce));
      return SLIM_ERR_CUDA;
    }
    if (s->par.scheme == SLIM_SCHEME_SPLIT && !s->g_time_node) {
      drop_graph(s);
      set_error("time kernel not found in the captured step");
      return SLIM_ERR_CUDA;
    }
    s->g_dt = dt;
  } else if (s->g_time_node) {
    // same graph, new start time: the time kernel's one (struct) argument
    split_time_args(s, t, dt, s->g_time_args);
    void* args[1] = {s->g_time_args};
    cudaKernelNodeParams kp = s->g_time_params;
    kp.kernelParams = args;
    kp.extra = nullptr;
    SLIM_CUDA_TRY(cudaGraphExecKernelNodeSetParams(s->g_exec, s->g_time_node, &kp));
  }
  SLIM_CUDA_TRY(cudaEventRecord(s->g_in, user));
  SLIM_CUDA_TRY(cudaStreamWaitEvent(s->g_stream, s->g_in, 0));
  SLIM_CUDA_TRY(cudaGraphLaunch(s->g_exec, s->g_stream));
  SLIM_CUDA_TRY(cudaEventRecord(s->g_out, s->g_stream));
  SLIM_CUDA_TRY(cudaStreamWaitEvent(user, s->g_out, 0));
  return SLIM_OK;
}
}  // namespace

extern "C" slim_status slim_step(slim_state* s, double t, double dt, void* stream) {
  clear_error();
  if (!s) { set_error("state is null"); return SLIM_ERR_ARG; }
  if (!(dt > 0)) { set_error("dt must be positive"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  slim_status r;
  if (s->par.use_graph && !s->prof_on)
    r = step_graph(s, t, dt, st);
  else
    r = step_launches(s, t, dt, st);
  if (r != SLIM_OK) return r;
  if (s->par.check_every > 0) {
    if (++s->steps_since_check >= s->par.check_every) {
      s->steps_since_check = 0;
      return slim_state_check(s, stream);
    }
  }
  return SLIM_OK;
}

extern "C" int slim_step_kernel_count(const slim_state* s) {
  if (!s) return 0;
  if (s->par.scheme == SLIM_SCHEME_SPLIT) return split_kernel_count(s);
  return 4;
}

extern "C" slim_status slim_tracer_mass(slim_state* s, int field, double* mass_host, void* stream) {
  clear_error();
  if (!s || !mass_host) { set_error("null argument"); return SLIM_ERR_ARG; }
  if (field != SLIM_FIELD_T && field != SLIM_FIELD_S) { set_error("field must be T or S"); return SLIM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  void* T = field == SLIM_FIELD_T ? s->T : s->S;
  const bool cpl = s->par.vertical != 0;
  if (s->prec == SLIM_FP64)
    SLIM_LAUNCH(launch_mass<double>(s->mesh->d, tile_of(s), (const double*)T, s->eta, s->red, s->red_out, st, cpl));
  else
    SLIM_LAUNCH(launch_mass<float>(s->mesh->d, tile_of(s), (const float*)T, s->eta, s->red, s->red_out, st, cpl));
  SLIM_CUDA_TRY(cudaMemcpyAsync(mass_host, s->red_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  SLIM_CUDA_TRY(cudaStreamSynchronize(st));
  return SLIM_OK;
}

// ---------------------------------------------------------------------------
// phase timing
// ---------------------------------------------------------------------------
namespace slim {
ProfScope::ProfScope(slim_state* s_, int phase, cudaStream_t st_) : s(s_), idx(-1), st(st_) {
  if (!s->prof_on || s->prof_n >= s->prof_max) return;
  idx = s->prof_n++;
  s->prof_phase[idx] = phase;
  cudaEventRecord(s->prof_ev[2 * idx], st);
}
ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(s->prof_ev[2 * idx + 1], st);
}
}  // namespace slim

extern "C" slim_status slim_profile_begin(slim_state* s, int max_launches) {
  clear_error();
  if (!s || max_launches <= 0) { set_error("bad argument"); return SLIM_ERR_ARG; }
  while ((int)s->prof_ev.size() < 2 * max_launches) {
    cudaEvent_t e;
    SLIM_CUDA_TRY(cudaEventCreate(&e));
    s->prof_ev.push_back(e);
  }
  s->prof_phase.assign(max_launches, 0);
  s->prof_max = max_launches;
  s->prof_n = 0;
  s->prof_on = true;
  return SLIM_OK;
}

extern "C" slim_status slim_profile_end(slim_state* s, double* ms, int* launches) {
  clear_error();
  if (!s) { set_error("state is null"); return SLIM_ERR_ARG; }
  double acc[SLIM_PHASE_COUNT] = {0};
  int cnt[SLIM_PHASE_COUNT] = {0};
  for (int i = 0; i < s->prof_n; ++i) {
    SLIM_CUDA_TRY(cudaEventSynchronize(s->prof_ev[2 * i + 1]));
    float t = 0.f;
    SLIM_CUDA_TRY(cudaEventElapsedTime(&t, s->prof_ev[2 * i], s->prof_ev[2 * i + 1]));
    acc[s->prof_phase[i]] += t;
    cnt[s->prof_phase[i]] += 1;
  }
  s->prof_on = false;
  s->prof_n = 0;
  for (int p = 0; p < SLIM_PHASE_COUNT; ++p) {
    if (ms) ms[p] = acc[p];
    if (launches) launches[p] = cnt[p];
  }
  return SLIM_OK;
}

extern "C" const char* slim_phase_name(int phase) {
  static const char* names[SLIM_PHASE_COUNT] = {"continuity", "tracer_stage", "hpg", "mom_pred",
                                                "ext2d", "momentum", "tracers", "misc"};
  return (phase >= 0 && phase < SLIM_PHASE_COUNT) ? names[phase] : "unknown";
}
