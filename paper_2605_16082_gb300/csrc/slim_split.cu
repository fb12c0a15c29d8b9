// The split-IMEX internal step (Sec. 2, Eqs. 11-14): per stage
//   density + horizontal pressure gradient (Eqs. 7-8, Eq. 15-16, Algorithm 1)
//   -> 3D horizontal momentum prediction F_3D^h and its column sum (Sec. 2.2)
//   -> subcycled 2D external mode in FP64 with the time-averaged transport (axpy)
//   -> F2D coupling and the corrected transport (Sec. 2.2, Sec. 2.5)
//   -> vertical flux from the continuity (Eq. 17)
//   -> 3D momentum and tracers, vertically implicit (stage 1) or explicit (stage 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "slim_kernels.h"
#include "slim_split.h"
#include "slim_split_device.cuh"
#include "slim_barrier.cuh"

namespace slim {

struct SplitBufs {
  // 2D (double): running external state A and two stage buffers
  double *Ae, *AU, *AV, *Be, *BU, *BV, *Ce, *CU, *CV;
  double *S3x, *S3y, *Sqx, *Sqy, *Gb, *F2x, *F2y, *eta_half, *cw, *iw6;
  float *cw_f;
  void *Ae_r, *AU_r, *AV_r, *Be_r, *BU_r, *BV_r, *Ce_r, *CU_r, *CV_r;  // compute-type shadows
  void *S3x_r, *S3y_r;
  double* tide;  // open-boundary elevation per external stage of the step (+1 slot)
  float* tide_f;  // the same stage values in FP32 (after the doubles in the same buffer)
  // open-boundary forcing: theta per external stage slot (+ the rhs2d slot + the two
  // split-stage middles), its FP32 copy; Q_ext column sums [4][3][n_tri] (x, y at
  // t_a, x, y at t_b) in FP64 and FP32; the flag the step was built with
  double* theta;
  float* theta_f;
  double* Qext;
  float* Qext_f;
  int forcing;
  int n_tide;
  // mixed form: FP32 stage-increment sums of the 2D subcycle and FP32 1/(w/6)
  float *Dacc, *Eacc, *Gacc, *Gacc2, *iw6_f;
  // 2D adjacency in one word per edge ([3][n_tri]): neighbour << 4 | neighbour-local
  // vertices of the edge (l0 | l1 << 2), or -1 (wall) / -2 (open boundary); a quarter
  // of the bytes of the 3D adjacency, which the 2D stages re-read every stage
  int* adj2;
  // non-advective momentum terms (viscosity, Coriolis, -r/rho0, drag) of the stage's
  // evaluation state, [6][P] each: written by the prediction, read by the update
  void *Ex, *Ey;
  // lateral normal transport of a stage at the face points, [12][P]: written by the
  // continuity, read by the momentum and tracer updates of the same stage
  void* qnf;
  // persistent 2D run: grid barrier words (arrival count, generation) and grid size;
  // the block graph of the run (bit n of row b: block n owns an edge neighbour of a
  // triangle of block b; nbw words per row, null when the grid is too large for the
  // in-kernel list) and the per-block stage counters of the neighbour waits
  unsigned* bar;
  int run_blocks;
  unsigned* nbits;
  unsigned* done;
  int nbw;
  double *Qbx, *Qby;  // the state's time-averaged transport buffers
  // compute-type copies for the 3D kernels
  void *F2x_r, *F2y_r, *Dqx_r, *Dqy_r, *gcor_r, *st_half, *st_end;
  bool has_s3 = false;
};

namespace {

template <typename R, int TP>
struct MB {
  static constexpr int value = sizeof(R) == 4 ? (1024 / TP > 0 ? 1024 / TP : 1) : (512 / TP > 0 ? 512 / TP : 1);
};
// OCC: resident blocks per SM asked of the register allocator at 256 threads
// per block (scaled with the block size); the FP64 form always uses 2.
template <typename R, int TP, int OCC>
struct MBO {
  static constexpr int occ = sizeof(R) == 4 ? OCC : 2;
  static constexpr int value = (occ * 256 / TP) > 0 ? (occ * 256 / TP) : 1;
};

// Launch shapes TP x OCC.  The FP64 form has the one register budget OCC 2; the
// mixed form has OCC 2, 3, 4 (3 only for 128- and 256-thread tiles).
#define SLIM_TPO_SWITCH(R, TP, OC, ...)                                                \
  if constexpr (sizeof(R) == 8) {                                                      \
    switch (TP) {                                                                      \
      case 128: { constexpr int TPc = 128, OCc = 2; __VA_ARGS__; } break;              \
      case 256: { constexpr int TPc = 256, OCc = 2; __VA_ARGS__; } break;              \
      case 512: { constexpr int TPc = 512, OCc = 2; __VA_ARGS__; } break;              \
      default: return cudaErrorInvalidValue;                                           \
    }                                                                                  \
  } else {                                                                             \
    switch (TP * 10 + OC) {                                                            \
      case 1282: { constexpr int TPc = 128, OCc = 2; __VA_ARGS__; } break;             \
      case 1283: { constexpr int TPc = 128, OCc = 3; __VA_ARGS__; } break;             \
      case 1284: { constexpr int TPc = 128, OCc = 4; __VA_ARGS__; } break;             \
      case 2562: { constexpr int TPc = 256, OCc = 2; __VA_ARGS__; } break;             \
      case 2563: { constexpr int TPc = 256, OCc = 3; __VA_ARGS__; } break;             \
      case 2564: { constexpr int TPc = 256, OCc = 4; __VA_ARGS__; } break;             \
      case 5122: { constexpr int TPc = 512, OCc = 2; __VA_ARGS__; } break;             \
      case 5124: { constexpr int TPc = 512, OCc = 4; __VA_ARGS__; } break;             \
      default: return cudaErrorInvalidValue;                                           \
    }                                                                                  \
  }

// resident-block budget of the heavy kernels from the parameters (0 = 4; a tile of
// 512 prisms has no 3-block budget and takes 2)
inline int occ_of(const slim_params& p, int TP) {
  const int o = (p.blocks_per_sm >= 2 && p.blocks_per_sm <= 4) ? p.blocks_per_sm : 4;
  return (o == 3 && TP == 512) ? 2 : o;
}

#define SLIM_TP_SWITCH2(TP, ...)                                \
  switch (TP) {                                                 \
    case 128: { constexpr int TPc = 128; __VA_ARGS__; } break;  \
    case 256: { constexpr int TPc = 256; __VA_ARGS__; } break;  \
    case 512: { constexpr int TPc = 512; __VA_ARGS__; } break;  \
    default: return cudaErrorInvalidValue;                      \
  }

template <typename KernelT>
cudaError_t set_smem2(KernelT kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// physical parameters converted once on the host to the compute type
template <typename R>
struct PP {
  R g, rho0, irho0, f, alpha, beta, T0, S0, nu_h, kappa_h, nu_v, kappa_v, cd, pen_v, pen_h;
  double g_d;  // the 2D mode's gravity (FP64 state update)
};

// rest depth of interface k of vertex column i (0 at the surface)
template <typename R>
__device__ __forceinline__ R zhat_r(const DevMesh& m, int i, int k) {
  if (m.n_levels == 0) return -(R)k * Geo<R>::hN(m, i);
  return Geo<R>::lev(m, k);
}

// ---------------------------------------------------------------------------
// open-boundary elevation A cos(2 pi time / T) at every external stage of a step:
// stage 1 runs n/2 subcycles over dt/2, stage 2 n subcycles over dt, each
// subcycle's SSP-RK3 stages at times (0, 1, 1/2) x the subcycle length
// ---------------------------------------------------------------------------
// Time data of one step for every external stage: the open-boundary elevation
// (the analytic M2 tide) and the forcing's theta = (t - t_a)/(t_b - t_a) at each
// stage time, and theta at the middle of each split stage's 2D run.  Slot layout
// (n1 = n/2 stages of the first split stage, then n of the second, 3 stages each):
// tide [total + 1] doubles, its FP32 copy [total]; theta [total + 3] doubles (stage
// slots, the slim_rhs2d slot, the two middles), its FP32 copy.
struct TideArgs {
  double t0, dt, amp, period, ta, tb;
  int n;
  double* out;
  double* theta;
};

__global__ void k_tide(TideArgs a) {
  const int n1 = a.n / 2;
  const int total = 3 * (n1 + a.n);
  const double off[3] = {0.0, 1.0, 0.5};
  float* out_f = reinterpret_cast<float*>(a.out + total + 1);  // FP32 copies after the doubles
  float* th_f = reinterpret_cast<float*>(a.theta + total + 3);
  const double ith = 1.0 / (a.tb - a.ta);
  for (int i = threadIdx.x; i < total + 2; i += blockDim.x) {
    double time;
    if (i >= total) {  // middles of the two split stages' 2D runs
      time = a.t0 + (i == total ? 0.25 : 0.5) * a.dt;
      const double th = (time - a.ta) * ith;
      a.theta[total + 1 + (i - total)] = th;
      th_f[total + 1 + (i - total)] = (float)th;
      continue;
    }
    if (i < 3 * n1) {
      const double dts = 0.5 * a.dt / n1;
      time = a.t0 + (i / 3 + off[i % 3]) * dts;
    } else {
      const int j = i - 3 * n1;
      const double dts = a.dt / a.n;
      time = a.t0 + (j / 3 + off[j % 3]) * dts;
    }
    a.out[i] = a.amp * cos(2.0 * M_PI * time / a.period);
    out_f[i] = (float)a.out[i];
    const double th = (time - a.ta) * ith;
    a.theta[i] = th;
    th_f[i] = (float)th;
  }
}

// Column sums of the exterior layer transport (dz_rest/2) u_ext at both forcing
// times (Q_ext at the vertices of triangles with an open edge; 0 elsewhere).
template <typename R>
__global__ void k_ext_sums(DevMesh m, const R* __restrict__ Uxa, const R* __restrict__ Vxa,
                           const R* __restrict__ Uxb, const R* __restrict__ Vxb,
                           double* __restrict__ Q, float* __restrict__ Qf) {
  const int nt = m.n_tri;
  const size_t n2 = (size_t)3 * nt;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    bool open = false;
    for (int e = 0; e < 3; ++e) open |= (m.einfo[e * nt + t].x == -2);
    const int p0 = m.col_off[t], N = m.col_off[t + 1] - p0;
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      if (open) {
        for (int k = 0; k < N; ++k) {
          const double hr = 0.5 * dz_rest_r<double>(m, ia, k, N);
          const size_t i0 = (size_t)a * m.P + p0 + k, i1 = (size_t)(3 + a) * m.P + p0 + k;
          s[0] += hr * ((double)Uxa[i0] + (double)Uxa[i1]);
          s[1] += hr * ((double)Vxa[i0] + (double)Vxa[i1]);
          s[2] += hr * ((double)Uxb[i0] + (double)Uxb[i1]);
          s[3] += hr * ((double)Vxb[i0] + (double)Vxb[i1]);
        }
      }
      for (int c = 0; c < 4; ++c) {
        Q[c * n2 + ia] = s[c];
        Qf[c * n2 + ia] = (float)s[c];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// wave speed of the 2D flux at every edge point: c = sqrt(g (h^- + h^+)/2)
// ---------------------------------------------------------------------------
__global__ void k_wave_speed(DevMesh m, double g, double* __restrict__ cw, float* __restrict__ cw_f,
                             double* __restrict__ iw6, float* __restrict__ iw6_f, int* __restrict__ adj2) {
  const int nt = m.n_tri;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    iw6[t] = 6.0 / m.jh[t];
    iw6_f[t] = (float)iw6[t];
    for (int e = 0; e < 3; ++e) {
      const int4 ei = m.einfo[e * nt + t];
      adj2[e * nt + t] = ei.x >= 0 ? ((ei.x << 4) | (ei.w & 15)) : ei.x;
      const int a0 = e, a1 = (e + 1) % 3;
      for (int gs = 0; gs < 2; ++gs) {
        const double b0 = gs ? SLIM_GL2 : SLIM_GL1, b1 = gs ? SLIM_GL1 : SLIM_GL2;
        const double ho = b0 * m.h[a0 * nt + t] + b1 * m.h[a1 * nt + t];
        double hn = ho;
        if (ei.x >= 0) {
          const int l0 = ei.w & 3, l1 = (ei.w >> 2) & 3;
          hn = b0 * m.h[l0 * nt + ei.x] + b1 * m.h[l1 * nt + ei.x];
        }
        const double c = sqrt(g * 0.5 * (ho + hn));
        const int ip = (e * nt + t) * 2 + gs;
        cw[ip] = c;
        cw_f[ip] = (float)c;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// density + horizontal pressure gradient (one tile per block)
// ---------------------------------------------------------------------------
template <typename R, int TP, int OCC>
__global__ void __launch_bounds__(TP, (MBO<R, TP, OCC>::value))
    k_hpg(DevMesh m, const R* __restrict__ T, const R* __restrict__ S, const R* __restrict__ st,
          PP<R> pp, R* __restrict__ Rx, R* __restrict__ Ry) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_off = reinterpret_cast<int*>(smem);
  const int TPX = TP + m.max_tile_tris;
  R* s_F = reinterpret_cast<R*>(smem + ((TP + 1) * sizeof(int) + 15) / 16 * 16);  // [12][TPX]
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  const int nt = m.n_tri, P = m.P;
  const R rho0 = pp.rho0, al = pp.alpha, be = pp.beta, T0 = pp.T0, S0 = pp.S0;
  const R g = pp.g;
  auto rho = [&](R Tv, R Sv) { return rho0 * (-al * (Tv - T0) + be * (Sv - S0)); };
  R r[2][3];
  if (i < tl.np) {
    const int p = tl.p0 + i;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) r[c][a] = rho(T[(size_t)(c * 3 + a) * P + p], S[(size_t)(c * 3 + a) * P + p]);
  }
  load_offsets<TP>(m, tl, s_off);
  int slot = 0;
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    const int p = tl.p0 + i;
    slot = i + lt;
    const R jh = Geo<R>::jh(m, t), w24 = jh * (R)(1.0 / 24.0);
    R gx[3], gy[3], hz[3], zt[3], zb[3], stv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      gx[a] = Geo<R>::gx(m, ia); gy[a] = Geo<R>::gy(m, ia);
      stv[a] = st[ia];
      const R h = Geo<R>::h(m, ia);
      hz[a] = (R)0.5 * dz_rest_r<R>(m, ia, k, N) * stv[a];
      zt[a] = stv[a] * (zhat_r<R>(m, ia, k) + h) - h;
      zb[a] = zt[a] - (R)2 * hz[a];
    }
    const R gztx = zt[0] * gx[0] + zt[1] * gx[1] + zt[2] * gx[2];
    const R gzty = zt[0] * gy[0] + zt[1] * gy[1] + zt[2] * gy[2];
    const R gzbx = zb[0] * gx[0] + zb[1] * gx[1] + zb[2] * gx[2];
    const R gzby = zb[0] * gy[0] + zb[1] * gy[1] + zb[2] * gy[2];
    R Fx[2][3], Fy[2][3];
    // right-hand side of dr/dz = -g grad_h rho' (r is the horizontal gradient of the
    // baroclinic hydrostatic pressure g int_z^eta rho', so it grows downward)
    // volume: +g int rho' grad(phi_a) psi_c z_zeta  -  g int rho' phi_a psi_c' grad z
    {
      const R shz = hz[0] + hz[1] + hz[2];
      R A[2], Sr[2];
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        Sr[d] = r[d][0] + r[d][1] + r[d][2];
        A[d] = w24 * (Sr[d] * shz + r[d][0] * hz[0] + r[d][1] * hz[1] + r[d][2] * hz[2]);
      }
      const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
      const R tA0 = G2 * A[0] + G1 * A[1], tA1 = G1 * A[0] + G2 * A[1];
      const R Z0x = G2 * gztx + G1 * gzbx, Z0y = G2 * gzty + G1 * gzby;
      const R Z1x = G1 * gztx + G2 * gzbx, Z1y = G1 * gzty + G2 * gzby;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R m0 = w24 * (Sr[0] + r[0][a]), m1 = w24 * (Sr[1] + r[1][a]);
        const R bx = m0 * Z0x + m1 * Z1x, by = m0 * Z0y + m1 * Z1y;
        Fx[0][a] = g * (gx[a] * tA0 - (R)0.5 * bx);
        Fy[0][a] = g * (gy[a] * tA0 - (R)0.5 * by);
        Fx[1][a] = g * (gx[a] * tA1 + (R)0.5 * bx);
        Fy[1][a] = g * (gy[a] * tA1 + (R)0.5 * by);
      }
    }
    // lateral faces: - g oint v {rho'} n z_zeta dl dzeta
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int4 ei = m.einfo[e * nt + t];
      const int a0 = e, a1 = (e + 1) % 3;
      const R nxe = Geo<R>::nx(m, e * nt + t), nye = Geo<R>::ny(m, e * nt + t);
      const R half_len = (R)0.5 * Geo<R>::len(m, e * nt + t);
      R rb[2][2];
      bool has_nb = false;
      if (ei.x >= 0 && k < ei.z) {
        has_nb = true;
        const int pn = ei.y + k;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int l = j ? ((ei.w >> 2) & 3) : (ei.w & 3);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const size_t idx = (size_t)(c * 3 + l) * P + pn;
            rb[j][c] = rho(T[idx], S[idx]);
          }
        }
      }
#pragma unroll
      for (int gs = 0; gs < 2; ++gs) {
        const R b0 = gs ? (R)SLIM_GL2 : (R)SLIM_GL1, b1 = gs ? (R)SLIM_GL1 : (R)SLIM_GL2;
        const R zz = b0 * hz[a0] + b1 * hz[a1];
#pragma unroll
        for (int gz = 0; gz < 2; ++gz) {
          const R z0 = gz ? (R)SLIM_GL2 : (R)SLIM_GL1, z1 = gz ? (R)SLIM_GL1 : (R)SLIM_GL2;
          const R B00 = b0 * z0, B01 = b0 * z1, B10 = b1 * z0, B11 = b1 * z1;
          R rh = B00 * r[0][a0] + B01 * r[1][a0] + B10 * r[0][a1] + B11 * r[1][a1];
          if (has_nb) rh = (R)0.5 * (rh + (B00 * rb[0][0] + B01 * rb[0][1] + B10 * rb[1][0] + B11 * rb[1][1]));
          const R wx = -g * half_len * zz * rh * nxe, wy = -g * half_len * zz * rh * nye;
          Fx[0][a0] += wx * B00; Fx[1][a0] += wx * B01; Fx[0][a1] += wx * B10; Fx[1][a1] += wx * B11;
          Fy[0][a0] += wy * B00; Fy[1][a0] += wy * B01; Fy[0][a1] += wy * B10; Fy[1][a1] += wy * B11;
        }
      }
    }
    // top / bottom faces: central rho' with the element above / below
    R rt[3], rbt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      rt[a] = r[0][a];
      rbt[a] = r[1][a];
    }
    if (k > 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t idx = (size_t)(3 + a) * P + p - 1;
        rt[a] = (R)0.5 * (rt[a] + rho(T[idx], S[idx]));
      }
    }
    if (k + 1 < N) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t idx = (size_t)a * P + p + 1;
        rbt[a] = (R)0.5 * (rbt[a] + rho(T[idx], S[idx]));
      }
    }
    {
      const R srt = rt[0] + rt[1] + rt[2], srb = rbt[0] + rbt[1] + rbt[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R mt = w24 * (srt + rt[a]), mb = w24 * (srb + rbt[a]);
        Fx[0][a] += g * mt * gztx; Fy[0][a] += g * mt * gzty;
        Fx[1][a] -= g * mb * gzbx; Fy[1][a] -= g * mb * gzby;
      }
    }
    // surface condition r = g rho'(eta) grad(eta): F_top -= M_h r_surface (layer 0)
    if (k == 0) {
      R gex = 0, gey = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R eta = (stv[a] - (R)1) * Geo<R>::h(m, a * nt + t);
        gex += eta * gx[a]; gey += eta * gy[a];
      }
      const R sr = r[0][0] + r[0][1] + r[0][2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R mr = g * w24 * (sr + r[0][a]);
        Fx[0][a] -= mr * gex;
        Fy[0][a] -= mr * gey;
      }
    }
    // M_h^-1 per layer: f_a = (6/J_h)(4 F_a - sum F)
    const R s6 = (R)6 * rcp<R>(jh);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const R sx = Fx[c][0] + Fx[c][1] + Fx[c][2], sy = Fy[c][0] + Fy[c][1] + Fy[c][2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        s_F[(c * 3 + a) * TPX + slot] = s6 * ((R)4 * Fx[c][a] - sx);
        s_F[(6 + c * 3 + a) * TPX + slot] = s6 * ((R)4 * Fy[c][a] - sy);
      }
    }
  }
  __syncthreads();
  // Algorithm 1 per vertex column and component: s += f_t + f_b, r_t = -s + 2 f_b, r_b = -s
  for (int j = threadIdx.x; j < 6 * tl.nt; j += TP) {
    const int comp = j / (3 * tl.nt), rem = j - comp * 3 * tl.nt;
    const int a = rem / tl.nt, lt = rem - a * tl.nt;
    const int base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
    R* ft = s_F + (comp * 6 + a) * TPX + base;
    R* fb = s_F + (comp * 6 + 3 + a) * TPX + base;
    R s = 0;
    for (int k = 0; k < N; ++k) {
      s += ft[k] + fb[k];
      const R rtop = -s + (R)2 * fb[k];
      fb[k] = -s;
      ft[k] = rtop;
    }
  }
  __syncthreads();
  if (i < tl.np) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      Rx[(size_t)q * P + tl.p0 + i] = s_F[q * TPX + slot];
      Ry[(size_t)q * P + tl.p0 + i] = s_F[(6 + q) * TPX + slot];
    }
  }
}

// lumped mass apply: (M f)_c = (J_h/6) hz (G f)_c, G = [[2,1],[1,2]]/3
template <typename R>
__device__ __forceinline__ void lumped(R w6hz, R f0, R f1, R& o0, R& o1) {
  o0 = w6hz * ((R)(2.0 / 3.0) * f0 + (R)(1.0 / 3.0) * f1);
  o1 = w6hz * ((R)(1.0 / 3.0) * f0 + (R)(2.0 / 3.0) * f1);
}

// F_3D^h terms beyond advection: horizontal viscosity (unless the advection pass
// added it already: SIPG_DONE), Coriolis, -r/rho0, bed drag
template <typename R, bool SIPG_DONE = false>
__device__ __forceinline__ void momentum_extras(const DevMesh& m, int t, int k, int p, int N,
                                                const Own2<R>& own, const R* __restrict__ U,
                                                const R* __restrict__ V, const R* __restrict__ st,
                                                const R* __restrict__ Rx, const R* __restrict__ Ry,
                                                const PP<R>& pp, R Fx[2][3], R Fy[2][3]) {
  const int nt = m.n_tri, P = m.P;
  if (!SIPG_DONE && pp.nu_h > (R)0)
    prism_sipg2<R>(m, t, k, N, own.u, own.v, U, V, st, pp.nu_h, pp.pen_h, Fx, Fy);
  const R f = pp.f, irho = pp.irho0;
  const R jh = Geo<R>::jh(m, t);
  const R w6 = jh * (R)(1.0 / 6.0);
  R hz[3], rx[2][3], ry[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hz[a] = (R)0.5 * dz_rest_r<R>(m, a * nt + t, k, N) * st[a * nt + t];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      rx[c][a] = Rx[(size_t)(c * 3 + a) * P + p];
      ry[c][a] = Ry[(size_t)(c * 3 + a) * P + p];
    }
  }
  // pressure gradient integrated exactly: (1/J_h) int phi_a phi_b z_zeta dA =
  // hz_a/30 + sum/60 on the diagonal, (hz_a + hz_b + sum)/120 off it (the cubic
  // moments 1/20, 1/60, 1/120 of the P1 basis against the linear z_zeta)
  const R sh = hz[0] + hz[1] + hz[2];
  const R pj = -irho * jh;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R kx[2] = {0, 0}, ky[2] = {0, 0};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R kab = (a == b) ? hz[a] * (R)(1.0 / 30.0) + sh * (R)(1.0 / 60.0)
                             : (hz[a] + hz[b] + sh) * (R)(1.0 / 120.0);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        kx[d] += kab * rx[d][b];
        ky[d] += kab * ry[d][b];
      }
    }
    const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
    R ox0, ox1, oy0, oy1;
    lumped<R>(w6 * hz[a], f * own.v[0][a], f * own.v[1][a], ox0, ox1);
    lumped<R>(w6 * hz[a], -f * own.u[0][a], -f * own.u[1][a], oy0, oy1);
    Fx[0][a] += ox0 + pj * (G2 * kx[0] + G1 * kx[1]);
    Fx[1][a] += ox1 + pj * (G1 * kx[0] + G2 * kx[1]);
    Fy[0][a] += oy0 + pj * (G2 * ky[0] + G1 * ky[1]);
    Fy[1][a] += oy1 + pj * (G1 * ky[0] + G2 * ky[1]);
    if (k == N - 1) {
      const R ub = own.u[1][a], vb = own.v[1][a];
      const R sp = sqrt(ub * ub + vb * vb);
      Fx[1][a] -= pp.cd * w6 * sp * ub;
      Fy[1][a] -= pp.cd * w6 * sp * vb;
    }
  }
}

// ---------------------------------------------------------------------------
// 3D horizontal momentum prediction: column sums of F_3D^h and of q (FP64)
// ---------------------------------------------------------------------------
template <typename R, int TP, int OCC>
__global__ void __launch_bounds__(TP, (MBO<R, TP, OCC>::value))
    k_mompred(DevMesh m, AdvIn<R> in, const R* __restrict__ Rx, const R* __restrict__ Ry,
              PP<R> pp, double* __restrict__ S3x, double* __restrict__ S3y,
              double* __restrict__ Sqx, double* __restrict__ Sqy, R* __restrict__ S3x_r,
              R* __restrict__ S3y_r, R* __restrict__ Ex, R* __restrict__ Ey,
              R* __restrict__ Fx_out, R* __restrict__ Fy_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_off = reinterpret_cast<int*>(smem);
  const int TPX = TP + m.max_tile_tris;
  R* s_v = reinterpret_cast<R*>(smem + ((TP + 1) * sizeof(int) + 15) / 16 * 16);  // [4][3][TPX]
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  Own2<R> own;
  if (i < tl.np) load_own2<R, true>(m, tl.p0 + i, in, own);
  load_offsets<TP>(m, tl, s_off);
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    const int p = tl.p0 + i, slot = i + lt;
    R Fx[2][3] = {{0, 0, 0}, {0, 0, 0}}, Fy[2][3] = {{0, 0, 0}, {0, 0, 0}}, qx[2][3], qy[2][3];
    // the non-advective terms are the update's too (same state): kept for it; the
    // horizontal viscosity is added in the advection's pass over the faces
    R ex[2][3] = {{0, 0, 0}, {0, 0, 0}}, ey[2][3] = {{0, 0, 0}, {0, 0, 0}};
    if (pp.nu_h > (R)0)
      prism_adv<R, false, true, false>(m, t, k, p, N, own, in, Fx, Fy, qx, qy, pp.nu_h, pp.pen_h, ex, ey);
    else
      prism_adv<R, false>(m, t, k, p, N, own, in, Fx, Fy, qx, qy);
    momentum_extras<R, true>(m, t, k, p, N, own, in.U, in.V, in.st, Rx, Ry, pp, ex, ey);
    // the nodal transport of the column sums, formed again (not held through the
    // faces): q = hz u, the prediction's transport has no correction
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * m.n_tri + t;
      const R hza = (R)0.5 * dz_rest_r<R>(m, ia, k, N) * in.st[ia];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        qx[c][a] = hza * own.u[c][a];
        qy[c][a] = hza * own.v[c][a];
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Fx[c][a] += ex[c][a];
        Fy[c][a] += ey[c][a];
        Ex[(size_t)(c * 3 + a) * m.P + p] = ex[c][a];
        Ey[(size_t)(c * 3 + a) * m.P + p] = ey[c][a];
        // the whole F_3D^h per node when asked for (slim_rhs3d of a velocity)
        if (Fx_out) Fx_out[(size_t)(c * 3 + a) * m.P + p] = Fx[c][a];
        if (Fy_out) Fy_out[(size_t)(c * 3 + a) * m.P + p] = Fy[c][a];
      }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_v[(0 * 3 + a) * TPX + slot] = Fx[0][a] + Fx[1][a];
      s_v[(1 * 3 + a) * TPX + slot] = Fy[0][a] + Fy[1][a];
      s_v[(2 * 3 + a) * TPX + slot] = qx[0][a] + qx[1][a];
      s_v[(3 * 3 + a) * TPX + slot] = qy[0][a] + qy[1][a];
    }
  }
  __syncthreads();
  double* outs[4] = {S3x, S3y, Sqx, Sqy};
  for (int j = threadIdx.x; j < 12 * tl.nt; j += TP) {
    const int q = j / (3 * tl.nt), rem = j - q * 3 * tl.nt;
    const int a = rem / tl.nt, lt = rem - a * tl.nt;
    const int base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
    const R* src = s_v + (q * 3 + a) * TPX + base;
    ColSum<R> cs;
    for (int k = 0; k < N; ++k) cs.add(src[k]);
    const double v = cs.value();
    const int ia = a * m.n_tri + tl.t0 + lt;
    outs[q][ia] = v;
    if (q == 0) S3x_r[ia] = (R)v;
    if (q == 1) S3y_r[ia] = (R)v;
  }
}

// ---------------------------------------------------------------------------
// 2D external-mode stage (thread per triangle).  The state, its update and the
// accumulated averages are FP64 in both forms; the residual is evaluated in RC
// (double for the FP64 form, float for the mixed form).
//   R_eta,a = int Q.grad phi_a - oint phi_a F_eta
//   R_Q,a   = int g eta (H grad phi_a + phi_a grad H) - oint phi_a g H^- eta^ n
//   F_eta = {q} + c/2 (eta^- - eta^+),  eta^ = {eta} + (q^- - q^+)/(2c)
// Shu-Osher update (alpha, beta) from the subcycle start; the stage input is
// accumulated into Qbar and its eta flux into Gbar with weight bw.
// MODE 0: update; MODE 1: residual only (out = R_eta, R_U, R_V).
// ---------------------------------------------------------------------------
template <typename RC> struct Ext2dGeo;
template <> struct Ext2dGeo<double> {
  static __device__ __forceinline__ double c(const SplitBufs& b, int i) { return b.cw[i]; }
  static __device__ __forceinline__ const double* Q(const SplitBufs& b) { return b.Qext; }
};
template <> struct Ext2dGeo<float> {
  static __device__ __forceinline__ float c(const SplitBufs& b, int i) { return b.cw_f[i]; }
  static __device__ __forceinline__ const float* Q(const SplitBufs& b) { return b.Qext_f; }
};

// Stage buffers: FP64 state for the update plus its compute-type shadow for the
// residual (the same arrays in the FP64 form).
struct Ext2dIO {
  const double *e, *U, *V;      // stage input (FP64)
  const void *er, *Ur, *Vr;     // stage input shadow (RC)
  const double *en, *Un, *Vn;   // subcycle start (FP64)
  double *eo, *Uo, *Vo;         // stage output (FP64)
  void *eor, *Uor, *Vor;        // stage output shadow (RC); null in the FP64 form
};

// Loads of stage values: plain, or through L2 for values that other blocks of the
// same (persistent) launch wrote (the L1 caches of the SMs are not coherent).
struct LdPlain {
  template <typename T> static __device__ __forceinline__ T ld(const T* p) { return *p; }
};
struct LdL2 {
  template <typename T> static __device__ __forceinline__ T ld(const T* p) { return __ldcg(p); }
};

// Forced open boundary: the exterior normal transport Q_ext(t).n at an edge point,
// Q_ext = Q_a + theta (Q_b - Q_a) at the edge's two vertices (i0, i1) weighted b0, b1.
// Out of line: it runs on open edges only and keeps its registers off the main path.
template <typename RC>
__device__ __noinline__ RC forced_qn(const SplitBufs& bf, int nt, int i0, int i1, RC b0, RC b1, RC nx,
                                     RC ny, RC th) {
  const RC* Q = Ext2dGeo<RC>::Q(bf);
  const size_t n2 = (size_t)3 * nt;
  const RC x0 = Q[i0] + th * (Q[2 * n2 + i0] - Q[i0]), y0 = Q[n2 + i0] + th * (Q[3 * n2 + i0] - Q[n2 + i0]);
  const RC x1 = Q[i1] + th * (Q[2 * n2 + i1] - Q[i1]), y1 = Q[n2 + i1] + th * (Q[3 * n2 + i1] - Q[n2 + i1]);
  return b0 * (x0 * nx + y0 * ny) + b1 * (x1 * nx + y1 * ny);
}

// Residual of the 2D stage at the RC state (er, Ur, Vr) of triangle t; Fe
// receives the eta flux at the 6 edge points (edge-major, 2 points per edge).
template <typename RC, typename LD = LdPlain>
__device__ __forceinline__ void ext2d_residual(const DevMesh& m, const SplitBufs& bf, const RC* er,
                                               const RC* Ur, const RC* Vr, RC g, RC tide, RC th,
                                               int t, RC Re[3], RC RU[3], RC RV[3], RC Fe[6]) {
  const int nt = m.n_tri;
  RC e[3], U[3], V[3], H[3], gx[3], gy[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ia = a * nt + t;
    e[a] = LD::ld(er + ia); U[a] = LD::ld(Ur + ia); V[a] = LD::ld(Vr + ia);
    H[a] = Geo<RC>::h(m, ia) + e[a];
    gx[a] = Geo<RC>::gx(m, ia); gy[a] = Geo<RC>::gy(m, ia);
  }
  const RC jh = Geo<RC>::jh(m, t);
  const RC w6 = jh * (RC)(1.0 / 6.0), w24 = jh * (RC)(1.0 / 24.0);
  const RC sU = U[0] + U[1] + U[2], sV = V[0] + V[1] + V[2];
  const RC se = e[0] + e[1] + e[2], sH = H[0] + H[1] + H[2];
  const RC eH = w24 * (se * sH + e[0] * H[0] + e[1] * H[1] + e[2] * H[2]);
  const RC gHx = H[0] * gx[0] + H[1] * gx[1] + H[2] * gx[2];
  const RC gHy = H[0] * gy[0] + H[1] * gy[1] + H[2] * gy[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Re[a] = w6 * (sU * gx[a] + sV * gy[a]);
    const RC ea = w24 * (se + e[a]);
    RU[a] = g * (eH * gx[a] + ea * gHx);
    RV[a] = g * (eH * gy[a] + ea * gHy);
  }
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const int code = bf.adj2[ed * nt + t];
    const int nb = code >= 0 ? code >> 4 : code;
    const int a0 = ed, a1 = (ed + 1) % 3;
    const RC nx = Geo<RC>::nx(m, ed * nt + t), ny = Geo<RC>::ny(m, ed * nt + t);
    const RC hl = (RC)0.5 * Geo<RC>::len(m, ed * nt + t);
    RC en0 = 0, en1 = 0, qn0 = 0, qn1 = 0;
    if (nb >= 0) {
      const int l0 = code & 3, l1 = (code >> 2) & 3;
      const int i0 = l0 * nt + nb, i1 = l1 * nt + nb;
      en0 = LD::ld(er + i0); en1 = LD::ld(er + i1);
      qn0 = LD::ld(Ur + i0) * nx + LD::ld(Vr + i0) * ny;
      qn1 = LD::ld(Ur + i1) * nx + LD::ld(Vr + i1) * ny;
    }
    const RC qo0 = U[a0] * nx + V[a0] * ny, qo1 = U[a1] * nx + V[a1] * ny;
#pragma unroll
    for (int gs = 0; gs < 2; ++gs) {
      const RC b0 = gs ? (RC)SLIM_GL2 : (RC)SLIM_GL1, b1 = gs ? (RC)SLIM_GL1 : (RC)SLIM_GL2;
      const RC eo_ = b0 * e[a0] + b1 * e[a1];
      const RC Ho = b0 * H[a0] + b1 * H[a1];
      const RC qo = b0 * qo0 + b1 * qo1;
      RC ex, qx;
      if (nb >= 0) {
        ex = b0 * en0 + b1 * en1;
        qx = b0 * qn0 + b1 * qn1;
      } else if (nb == -2) {
        // open boundary: exterior state from data alone (tide, and the prescribed
        // transport or none), a characteristic condition that only removes energy
        ex = tide;
        qx = bf.forcing ? forced_qn<RC>(bf, nt, a0 * nt + t, a1 * nt + t, b0, b1, nx, ny, th) : (RC)0;
      } else {
        ex = eo_;
        qx = -qo;
      }
      const int ip = (ed * nt + t) * 2 + gs;
      const RC c = Ext2dGeo<RC>::c(bf, ip);
      const RC fe = (RC)0.5 * (qo + qx) + (RC)0.5 * c * (eo_ - ex);
      // 1/(2c) divided out here instead of read from a table: fewer bytes per stage
      const RC eh = (RC)0.5 * (eo_ + ex) + (qo - qx) * ((RC)0.5 / c);
      Fe[ed * 2 + gs] = fe;
      const RC gq = g * Ho * eh;
      Re[a0] -= hl * b0 * fe; Re[a1] -= hl * b1 * fe;
      RU[a0] -= hl * b0 * gq * nx; RU[a1] -= hl * b1 * gq * nx;
      RV[a0] -= hl * b0 * gq * ny; RV[a1] -= hl * b1 * gq * ny;
    }
  }
}

template <int MODE, typename RC>
__global__ void __launch_bounds__(256)
    k_ext2d(DevMesh m, SplitBufs bf, Ext2dIO io, double g_, int tide_idx, double alpha, double beta,
            double dt, double bw) {
  const int nt = m.n_tri;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  RC Re[3], RU[3], RV[3], Fe[6];
  ext2d_residual<RC>(m, bf, (const RC*)io.er, (const RC*)io.Ur, (const RC*)io.Vr, (RC)g_,
                     (RC)bf.tide[tide_idx], (RC)bf.theta[tide_idx], t, Re, RU, RV, Fe);
  if (MODE == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      io.eo[a * nt + t] = (double)Re[a];
      io.eo[(3 + a) * nt + t] = (double)RU[a];
      io.eo[(6 + a) * nt + t] = (double)RV[a];
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int ip = ((j >> 1) * nt + t) * 2 + (j & 1);
    bf.Gb[ip] += bw * (double)Fe[j];
  }
  // new = alpha start + beta stage + (beta dt / w) R, the increment in RC
  const RC bdw = (RC)(beta * dt) * (RC)bf.iw6[t];
  const RC* S3x = (const RC*)bf.S3x_r;
  const RC* S3y = (const RC*)bf.S3y_r;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ia = a * nt + t;
    const double es_ = io.e[ia], Us_ = io.U[ia], Vs_ = io.V[ia];
    bf.Qbx[ia] += bw * Us_;
    bf.Qby[ia] += bw * Vs_;
    const double e_new = alpha * io.en[ia] + beta * es_ + (double)(bdw * Re[a]);
    const double U_new = alpha * io.Un[ia] + beta * Us_ + (double)(bdw * (RU[a] + S3x[ia]));
    const double V_new = alpha * io.Vn[ia] + beta * Vs_ + (double)(bdw * (RV[a] + S3y[ia]));
    io.eo[ia] = e_new;
    io.Uo[ia] = U_new;
    io.Vo[ia] = V_new;
    if (io.eor) {
      ((RC*)io.eor)[ia] = (RC)e_new;
      ((RC*)io.Uor)[ia] = (RC)U_new;
      ((RC*)io.Vor)[ia] = (RC)V_new;
    }
  }
}

// ---------------------------------------------------------------------------
// Mixed-form 2D subcycle (thread per triangle), SSP-RK3 written with the stage
// increments D_s = dt M^-1 R(Q_s) evaluated in FP32 at FP32 stage values:
//   Q_2 = Q^n + D_1,  Q_3 = Q^n + (D_1 + D_2)/4,
//   Q^{n+1} = Q^n + (D_1 + D_2)/6 + 2 D_3/3,
// which is the Shu-Osher form of the FP64 kernel rearranged exactly.  The stage
// values only feed the FP32 residual, so they are kept in FP32; the FP64 state
// Q^n is touched once per subcycle, by the last stage.  The Butcher-weighted
// averages of the subcycle, (Q_1 + Q_2 + 4 Q_3)/6 = Q^n + (2 D_1 + D_2)/6 and
// (F_1 + F_2 + 4 F_3)/6 for the edge eta flux, are added to the FP64 sums Qbar
// and Gbar by the last stage as well.
//   KIND 0: residual at Q^n (shadow), Dacc = D_1, out = Q_2, Gacc = F_1
//   KIND 1: residual at Q_2, Dacc = D_1 + D_2, Eacc = (2 D_1 + D_2)/6 (U, V),
//           out = Q_3, Gacc2 = F_2 (a second array, so that this stage loads
//           nothing it does not need before its stores)
//   KIND 2: residual at Q_3; FP64 Q^n += Dacc/6 + 2 D_3/3, out = shadow of it;
//           Qbar += wn (Q^n + Eacc), Gbar += ((Gacc + Gacc2) + 4 F_3) wq
// ---------------------------------------------------------------------------
struct Mx2dIO {
  const float *er, *Ur, *Vr;     // stage value
  const float *en, *Un, *Vn;     // subcycle start (FP32 shadow)
  float *eo, *Uo, *Vo;           // next stage value / new shadow
  double *e, *U, *V;             // FP64 subcycle start, updated in place by KIND 2
};

// one stage for triangle t (its own accumulators and FP64 state are only touched by
// the thread that owns t).  The stage runs in three phases: every load of the
// triangle's own data, then the arithmetic, then every store.  None of these arrays
// is declared restrict, so a load written after a store could not be moved above
// it; with the loads first, the own data (stage start, increments, sums) are in
// flight together with the residual's neighbour gathers, and the FP64 sums and
// state of the last stage cost two more round trips (edge fluxes, then state and
// transport sums) instead of one per field and node.
template <int KIND, typename LD>
__device__ __forceinline__ void ext2d_mx_tri(const DevMesh& m, const SplitBufs& bf, const Mx2dIO& io,
                                             float g, float tide, float th, float dt, float wq,
                                             double wn, int t) {
  const int nt = m.n_tri;
  const size_t n2 = (size_t)3 * nt;
  const float* S3x = (const float*)bf.S3x_r;
  const float* S3y = (const float*)bf.S3y_r;
  // phase 1a: FP32 own data (before the residual, so they overlap its loads)
  float s3[2][3], q0[3][3], dacc[3][3], eacc[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ia = a * nt + t;
    s3[0][a] = S3x[ia];
    s3[1][a] = S3y[ia];
    if (KIND < 2) {
      q0[0][a] = io.en[ia]; q0[1][a] = io.Un[ia]; q0[2][a] = io.Vn[ia];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (KIND >= 1) dacc[c][a] = bf.Dacc[c * n2 + ia];
    if (KIND == 2) {
      eacc[0][a] = bf.Eacc[ia];
      eacc[1][a] = bf.Eacc[n2 + ia];
    }
  }
  float Re[3], RU[3], RV[3], Fe[6];
  ext2d_residual<float, LD>(m, bf, io.er, io.Ur, io.Vr, g, tide, th, t, Re, RU, RV, Fe);
  const float bdw = dt * ((float)6 / Geo<float>::jh(m, t));   // 1 / (J_h/6), divided out here
  // the stage increments D = (dt / (J_h/6)) R, with the column sums S3 for U, V
  float d[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[0][a] = bdw * Re[a];
    d[1][a] = bdw * (RU[a] + s3[0][a]);
    d[2][a] = bdw * (RV[a] + s3[1][a]);
  }
  double* x[3] = {io.e, io.U, io.V};
  float* o[3] = {io.eo, io.Uo, io.Vo};
  if (KIND == 0) {
#pragma unroll
    for (int j = 0; j < 6; ++j) bf.Gacc[((j >> 1) * nt + t) * 2 + (j & 1)] = Fe[j];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ia = a * nt + t;
        bf.Dacc[c * n2 + ia] = d[c][a];
        o[c][ia] = q0[c][a] + d[c][a];
      }
  } else if (KIND == 1) {
#pragma unroll
    for (int j = 0; j < 6; ++j) bf.Gacc2[((j >> 1) * nt + t) * 2 + (j & 1)] = Fe[j];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ia = a * nt + t;
        const float d1 = dacc[c][a];
        const float s12 = d1 + d[c][a];
        bf.Dacc[c * n2 + ia] = s12;
        if (c > 0) bf.Eacc[(c - 1) * n2 + ia] = (d1 + s12) * (1.0f / 6.0f);
        o[c][ia] = q0[c][a] + 0.25f * s12;
      }
  } else {
    // phase 1b: the FP64 state and sums, all loads before the first store
    double gb[6];
    float g1[6], g2[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int ip = ((j >> 1) * nt + t) * 2 + (j & 1);
      gb[j] = bf.Gb[ip];
      g1[j] = bf.Gacc[ip];
      g2[j] = bf.Gacc2[ip];
    }
#pragma unroll
    for (int j = 0; j < 6; ++j)
      bf.Gb[((j >> 1) * nt + t) * 2 + (j & 1)] = gb[j] + f2d_bits(((g1[j] + g2[j]) + 4.0f * Fe[j]) * wq);
    double xn[3][3], qb[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
#pragma unroll
      for (int c = 0; c < 3; ++c) xn[c][a] = x[c][ia];
      qb[0][a] = bf.Qbx[ia];
      qb[1][a] = bf.Qby[ia];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      // conversions on the integer pipe: the FP64 pipe keeps the three FP64 sums
      bf.Qbx[ia] = qb[0][a] + wn * (xn[1][a] + f2d_bits(eacc[0][a]));
      bf.Qby[ia] = qb[1][a] + wn * (xn[2][a] + f2d_bits(eacc[1][a]));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float inc = dacc[c][a] * (1.0f / 6.0f) + d[c][a] * (2.0f / 3.0f);
        const double qnew = xn[c][a] + f2d_bits(inc);
        x[c][ia] = qnew;
        o[c][ia] = d2f_bits(qnew);
      }
    }
  }
}

// The whole external run of the mixed form in one cooperative launch: every stage
// of every subcycle over all triangles (grid-stride, so each triangle keeps its
// thread).  Between stages a block waits only for the blocks that own the
// neighbours of its triangles (a stage reads the previous stage's values of the
// edge neighbours; the buffer it overwrites was last read two stages earlier, which
// those blocks have finished too); with no block graph, a grid barrier.
constexpr int kMaxNbBlocks = 512;
struct Mx2dRun {
  Mx2dIO io[3];
  int n_sub, tide_base;
  float g, dt, wq;
  double wn;
  unsigned* bar;
  const unsigned* nbits;
  unsigned* done;
  int nbw;
  int* err;
};

// Block graph of the persistent run: with the grid stride, triangle t belongs to
// block (t mod stride) / 256.
__global__ void k_block_graph(DevMesh m, int stride, int nbw, unsigned* __restrict__ bits) {
  const int nt = m.n_tri;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int ob = (t % stride) / 256;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int nb = m.einfo[e * nt + t].x;
    if (nb < 0) continue;
    const int on = (nb % stride) / 256;
    if (on != ob) atomicOr(bits + (size_t)ob * nbw + (on >> 5), 1u << (on & 31));
  }
}

// Stages [first, first + count) of the run (stage index 3 q + kind); a grid
// barrier between consecutive stages of one launch.  With count = 1 it is one
// ordinary launch per stage (no barrier); the whole run is one cooperative launch.
// Three blocks of 256 per SM (85 registers, a few values spilled to L1) hide more
// latency than two blocks without spills.
__global__ void __launch_bounds__(256, 3) k_ext2d_run(DevMesh m, SplitBufs bf, Mx2dRun r, int first,
                                                   int count) {
  __shared__ int s_fail;
  __shared__ int s_nn;
  __shared__ int s_nb[kMaxNbBlocks];
  const int nt = m.n_tri;
  const int stride = gridDim.x * blockDim.x;
  const bool nbw = r.nbits != nullptr && count > 1;
  if (nbw) {  // this block's neighbour blocks, from its row of the block graph
    if (threadIdx.x == 0) {
      s_nn = 0;
      s_fail = 0;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < r.nbw; w += blockDim.x) {
      unsigned x = r.nbits[(size_t)blockIdx.x * r.nbw + w];
      while (x) {
        const int n = w * 32 + __ffs(x) - 1;
        x &= x - 1;
        s_nb[atomicAdd(&s_nn, 1)] = n;
      }
    }
    __syncthreads();
  }
  for (int gs = first; gs < first + count; ++gs) {
    const int st = gs % 3;
    const float tide = bf.tide_f[r.tide_base + gs], th = bf.theta_f[r.tide_base + gs];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
      if (st == 0) ext2d_mx_tri<0, LdL2>(m, bf, r.io[0], r.g, tide, th, r.dt, r.wq, r.wn, t);
      else if (st == 1) ext2d_mx_tri<1, LdL2>(m, bf, r.io[1], r.g, tide, th, r.dt, r.wq, r.wn, t);
      else ext2d_mx_tri<2, LdL2>(m, bf, r.io[2], r.g, tide, th, r.dt, r.wq, r.wn, t);
    }
    if (gs + 1 < first + count) {
      const bool ok = nbw ? neighbour_wait(r.done, (unsigned)(gs - first + 1), s_nb, s_nn, r.err, &s_fail)
                          : grid_barrier(r.bar, gridDim.x, r.err, &s_fail);
      if (!ok) return;
    }
  }
}

// Start of a split stage's external run in one pass over the 2D nodes: the FP64
// working copies of the state (eta, Qx, Qy), their FP32 shadows (mixed form; null
// in FP64) and the zeroed time-averaged transport.
__global__ void __launch_bounds__(256)
    k_ext2d_begin(const double* __restrict__ e, const double* __restrict__ U, const double* __restrict__ V,
                  double* __restrict__ Ae, double* __restrict__ AU, double* __restrict__ AV,
                  float* __restrict__ Aer, float* __restrict__ AUr, float* __restrict__ AVr,
                  double* __restrict__ Qbx, double* __restrict__ Qby, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double ei = e[i], ui = U[i], vi = V[i];
    Ae[i] = ei; AU[i] = ui; AV[i] = vi;
    if (Aer) {
      Aer[i] = (float)ei; AUr[i] = (float)ui; AVr[i] = (float)vi;
    }
    Qbx[i] = 0.0; Qby[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// coupling after the external run (FP64, thread per triangle):
//   F2D = (Q1 - (Q0 + T S3/w))/T, Dq = Qbar - sum q, st_end = 1 + eta1/h,
//   gcor = (Gbar - {Qbar}.n) / (paired layer thickness at the edge point)
// ---------------------------------------------------------------------------
// FP64 value in the compute type (the FP32 conversion on the integer pipe)
template <typename R> __device__ __forceinline__ R to_r(double x);
template <> __device__ __forceinline__ double to_r<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_r<float>(double x) { return d2f_bits(x); }

template <typename R>
__global__ void k_couple2d(DevMesh m, const double* __restrict__ e1, const double* __restrict__ U1,
                           const double* __restrict__ V1, const double* __restrict__ U0,
                           const double* __restrict__ V0, const double* __restrict__ S3x,
                           const double* __restrict__ S3y, const double* __restrict__ Sqx,
                           const double* __restrict__ Sqy, const double* __restrict__ Qbx,
                           const double* __restrict__ Qby, const double* __restrict__ Gb,
                           const R* __restrict__ st_ev, const double* __restrict__ iw6, double T,
                           double iT, double* __restrict__ F2x,
                           double* __restrict__ F2y, R* __restrict__ F2x_r, R* __restrict__ F2y_r,
                           R* __restrict__ Dqx_r, R* __restrict__ Dqy_r, R* __restrict__ gcor_r,
                           R* __restrict__ st_end, const double* __restrict__ Qext,
                           const double* __restrict__ th_mid) {
  const int nt = m.n_tri;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double iw = iw6[t];  // 1 / (J_h/6)
  const int N = m.col_off[t + 1] - m.col_off[t];
  // the differences that cancel (F2D, Qbar - sum q, Gbar - {Qbar}.n) are FP64; in
  // the mixed form the paired thickness and the division are FP32 and the
  // conversions run on the integer pipe
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ia = a * nt + t;
    const double fx = (U1[ia] - (U0[ia] + T * (S3x[ia] * iw))) * iT;
    const double fy = (V1[ia] - (V0[ia] + T * (S3y[ia] * iw))) * iT;
    F2x[ia] = fx; F2y[ia] = fy;
    F2x_r[ia] = to_r<R>(fx); F2y_r[ia] = to_r<R>(fy);
    Dqx_r[ia] = to_r<R>(Qbx[ia] - Sqx[ia]);
    Dqy_r[ia] = to_r<R>(Qby[ia] - Sqy[ia]);
    st_end[ia] = to_r<R>(1.0 + e1[ia] * m.ih[ia]);
  }
  // paired rest thickness of vertex i of a column of N layers over its first Np layers
  auto paired = [&](int i, int Nc, int Np) -> R {
    if (Np >= Nc) return Geo<R>::h(m, i);
    if (m.n_levels == 0) return Geo<R>::hN(m, i) * (R)Np;
    return -Geo<R>::lev(m, Np);
  };
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const int4 ei = m.einfo[ed * nt + t];
    const int a0 = ed, a1 = (ed + 1) % 3;
    const double nx = m.enx[ed * nt + t], ny = m.eny[ed * nt + t];
    for (int gs = 0; gs < 2; ++gs) {
      const double b0 = gs ? SLIM_GL2 : SLIM_GL1, b1 = gs ? SLIM_GL1 : SLIM_GL2;
      const R b0r = gs ? (R)SLIM_GL2 : (R)SLIM_GL1, b1r = gs ? (R)SLIM_GL1 : (R)SLIM_GL2;
      R g = 0;
      if (ei.x != -1) {
        const int i0 = a0 * nt + t, i1 = a1 * nt + t;
        const double Qo = b0 * (Qbx[i0] * nx + Qby[i0] * ny) + b1 * (Qbx[i1] * nx + Qby[i1] * ny);
        // open boundary: the exterior transport alone (zero unforced), matching the
        // 3D open-face transport, so the face carries its layer share of Gbar
        double Qavg = 0;
        if (ei.x == -2 && Qext) {
          const double th = *th_mid;
          const size_t n2 = (size_t)3 * nt;
          auto qe = [&](int i) {
            const double x = Qext[i] + th * (Qext[2 * n2 + i] - Qext[i]);
            const double y = Qext[n2 + i] + th * (Qext[3 * n2 + i] - Qext[n2 + i]);
            return x * nx + y * ny;
          };
          Qavg = b0 * qe(i0) + b1 * qe(i1);
        }
        const int Np = ei.x >= 0 ? min(N, ei.z) : N;
        R tot = b0r * paired(i0, N, Np) * st_ev[i0] + b1r * paired(i1, N, Np) * st_ev[i1];
        if (ei.x >= 0) {
          const int l0 = ei.w & 3, l1 = (ei.w >> 2) & 3;
          const int j0 = l0 * nt + ei.x, j1 = l1 * nt + ei.x;
          const double Qn = b0 * (Qbx[j0] * nx + Qby[j0] * ny) + b1 * (Qbx[j1] * nx + Qby[j1] * ny);
          Qavg = 0.5 * (Qo + Qn);
          tot += b0r * paired(j0, ei.z, Np) * st_ev[j0] + b1r * paired(j1, ei.z, Np) * st_ev[j1];
        }
        g = to_r<R>(Gb[(ed * nt + t) * 2 + gs] - Qavg) / tot;
      }
      gcor_r[(ed * nt + t) * 2 + gs] = g;
    }
  }
}

// ---------------------------------------------------------------------------
// continuity with the corrected transport over [t0, t0 + T] (elevations given)
// ---------------------------------------------------------------------------
template <typename R, int TP>
__global__ void __launch_bounds__(TP, (MB<R, TP>::value))
    k_cont_split(DevMesh m, AdvIn<R> in, const double* __restrict__ e0, const double* __restrict__ e1,
                 double T, R* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_off = reinterpret_cast<int*>(smem);
  const int TPX = TP + m.max_tile_tris;
  R* s_F = reinterpret_cast<R*>(smem + ((TP + 1) * sizeof(int) + 15) / 16 * 16);
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  Own2<R> own;
  if (i < tl.np) load_own2<R, true>(m, tl.p0 + i, in, own);
  load_offsets<TP>(m, tl, s_off);
  int slot = 0;
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    slot = i + lt;
    R o[2][3] = {{0, 0, 0}, {0, 0, 0}}, dummy[2][3], qx[2][3], qy[2][3];
    prism_adv<R, true, false, true, 1>(m, t, k, tl.p0 + i, N, own, in, o, dummy, qx, qy);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) s_F[(c * 3 + a) * TPX + slot] = o[c][a];
  }
  __syncthreads();
  const int nt = m.n_tri;
  for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
    const int a = j / tl.nt, lt = j - a * tl.nt;
    const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
    const int ia = a * nt + t;
    R* Ft = s_F + a * TPX + base;
    R* Fb = s_F + (3 + a) * TPX + base;
    const R dm_fac = (R)((m.jh[t] / 12.0) * (e1[ia] - e0[ia]) * m.ih[ia] / T);
    R s = (R)0;
    for (int k = N - 1; k >= 0; --k) {
      const R dm = dm_fac * dz_rest_r<R>(m, ia, k, N);
      const R ft = Ft[k] - dm, fb = Fb[k] - dm;
      const R wt = ft + fb + s;
      Fb[k] = fb - ft + s;
      Ft[k] = wt;
      s = wt;
    }
  }
  __syncthreads();
  if (i < tl.np) {
#pragma unroll
    for (int r = 0; r < 6; ++r) W[(size_t)r * m.P + tl.p0 + i] = s_F[r * TPX + slot];
  }
}

// ---------------------------------------------------------------------------
// 3D update of a field pair (KIND 0: momentum u, v; KIND 1: tracers T, S)
//   M1 f1 = M0 f0 + dt (R_h(f_ev; qbar) + extras [+ M1 F2D/H1] [+ A f_ev]),
// implicit: (M1 - dt A(W, st1)) f1 = ... without A f_ev; the momentum extras (Ex,
// Ey) are the ones the prediction stored for the same state.  The outputs O0, O1
// may be the start state G0, G1 itself (the last stage updates in place): each
// thread reads its own prism's start values before writing them, and neither
// pair is declared restrict.
// ---------------------------------------------------------------------------
template <typename R>
struct UA {
  R dt;
  R kap_v;  // vertical viscosity / diffusivity
  R kap_h;  // horizontal viscosity / diffusivity
};

template <typename R, int TP, int KIND, bool IMPL, int OCC>
__global__ void __launch_bounds__(TP, (MBO<R, TP, OCC>::value))
    k_update(DevMesh m, AdvIn<R> in, const R* G0, const R* G1,
             const R* __restrict__ W, const R* __restrict__ Ex, const R* __restrict__ Ey,
             const R* __restrict__ F2x, const R* __restrict__ F2y, const R* __restrict__ st0,
             const R* __restrict__ st1, PP<R> pp, UA<R> ua, R* O0, R* O1,
             int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_off = reinterpret_cast<int*>(smem);
  const int TPX = TP + m.max_tile_tris;
  const size_t ob = ((TP + 1) * sizeof(int) + 15) / 16 * 16;
  R* s_b = reinterpret_cast<R*>(smem + ob);                 // [12][TPX]
  R* s_W = s_b + 12 * (size_t)TPX;                          // [6][TPX]
  R* s_C = s_W + 6 * (size_t)TPX;                           // [3][4][TPX]
  R* s_st = s_C + 12 * (size_t)TPX;                         // [3][TP]
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  const int nt = m.n_tri, P = m.P;
  Own2<R> own;
  if (i < tl.np) load_own2<R, KIND == 0>(m, tl.p0 + i, in, own);
  if (IMPL) {
    for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
      const int a = j / tl.nt, lt = j - a * tl.nt;
      s_st[a * TP + lt] = st1[a * nt + tl.t0 + lt];
    }
  }
  load_offsets<TP>(m, tl, s_off);
  const R dt = ua.dt;
  int slot = 0;
  R o0[2][3], o1[2][3];
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    const int p = tl.p0 + i;
    slot = i + lt;
    R F0[2][3] = {{0, 0, 0}, {0, 0, 0}}, F1[2][3] = {{0, 0, 0}, {0, 0, 0}}, qx[2][3], qy[2][3];
    // tracers: advection and horizontal SIPG in one pass over the faces
    // (the face transports come from the stage's continuity pass)
    if (KIND == 1 && ua.kap_h > (R)0)
      prism_adv<R, false, true, true, 2>(m, t, k, p, N, own, in, F0, F1, qx, qy, ua.kap_h, pp.pen_h);
    else
      prism_adv<R, false, false, true, 2>(m, t, k, p, N, own, in, F0, F1, qx, qy);
    const R w6 = Geo<R>::jh(m, t) * (R)(1.0 / 6.0);
    if (KIND == 0) {
      // viscosity, Coriolis, -r/rho0 and drag of this state, from the prediction
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          F0[c][a] += Ex[(size_t)(c * 3 + a) * P + p];
          F1[c][a] += Ey[(size_t)(c * 3 + a) * P + p];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      const R dr = dz_rest_r<R>(m, ia, k, N);
      // increment form f1 = f0 + d: rhs - M1 f0 = (M0 - M1) f0 + dt (...), with the
      // stretch difference st0 - st1 exact; the inverse mass (explicit) and the
      // column solve (implicit) then act on the increment only
      const R dhz = (R)0.5 * dr * (st0[ia] - st1[ia]);
      R b[2][2];
      const size_t i0 = (size_t)a * P + p, i1 = (size_t)(3 + a) * P + p;
      const R g00 = G0[i0], g01 = G0[i1], g10 = G1[i0], g11 = G1[i1];
      lumped<R>(w6 * dhz, g00, g01, b[0][0], b[0][1]);
      lumped<R>(w6 * dhz, g10, g11, b[1][0], b[1][1]);
      R add0 = 0, add1 = 0;
      if (KIND == 0) {  // M1 F2D / H1 = (J_h/12) dz_rest (1/h) F2D
        const R cfac = Geo<R>::jh(m, t) * (R)(1.0 / 12.0) * dr * Geo<R>::ih(m, ia);
        add0 = cfac * F2x[ia];
        add1 = cfac * F2y[ia];
      }
      R rr[2][2] = {{b[0][0] + dt * (F0[0][a] + add0), b[0][1] + dt * (F0[1][a] + add0)},
                    {b[1][0] + dt * (F1[0][a] + add1), b[1][1] + dt * (F1[1][a] + add1)}};
      if (!IMPL) {
        // + dt A(W, st_ev) f_ev, A couples the layers above and below (the implicit
        // update adds dt A f0 inside the column solve instead)
        const R kap = ua.kap_v, pen = pp.pen_v;
        const R stv = in.st[ia];
        const R dz = dr * stv, idz = rcp<R>(dz);
        R idzm = idz, idzp = idz;
        if (m.n_levels != 0) {
          if (k > 0) idzm = rcp<R>(dz_rest_r<R>(m, ia, k - 1, N) * stv);
          if (k + 1 < N) idzp = rcp<R>(dz_rest_r<R>(m, ia, k + 1, N) * stv);
        }
        const R W0 = W[(size_t)a * P + p], W1 = W[(size_t)(3 + a) * P + p];
        const R Wn = (k + 1 < N) ? W[(size_t)a * P + p + 1] : (R)0;
        R A[2][2], AL[2][2], AU[2][2];
        vertical_A<R>(k, N, w6, idzm, idz, idzp, W0, W1, Wn, kap, pen, A, AL, AU);
        const R* Fs[2] = {in.F0 ? in.F0 : in.U, in.F1 ? in.F1 : in.V};
        const R fk[2][2] = {{own.f0[0][a], own.f0[1][a]}, {own.f1[0][a], own.f1[1][a]}};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          R fm0 = 0, fm1 = 0, fp0 = 0, fp1 = 0;
          if (k > 0) { fm0 = Fs[q][i0 - 1]; fm1 = Fs[q][i1 - 1]; }
          if (k + 1 < N) { fp0 = Fs[q][i0 + 1]; fp1 = Fs[q][i1 + 1]; }
#pragma unroll
          for (int rw = 0; rw < 2; ++rw)
            rr[q][rw] += dt * (A[rw][0] * fk[q][0] + A[rw][1] * fk[q][1] + AL[rw][0] * fm0 +
                               AL[rw][1] * fm1 + AU[rw][0] * fp0 + AU[rw][1] * fp1);
        }
      }
      if (IMPL) {
        s_b[(0 * 3 + a) * TPX + slot] = rr[0][0];
        s_b[(1 * 3 + a) * TPX + slot] = rr[0][1];
        s_b[(2 * 3 + a) * TPX + slot] = rr[1][0];
        s_b[(3 * 3 + a) * TPX + slot] = rr[1][1];
      } else {
        // M1^-1: (6 / (J_h hz1)) [[2,-1],[-1,2]] per vertex-layer
        const R hz1 = (R)0.5 * dr * st1[ia];
        const R im = rcp<R>(w6 * hz1);
        o0[0][a] = g00 + im * ((R)2 * rr[0][0] - rr[0][1]);
        o0[1][a] = g01 + im * ((R)2 * rr[0][1] - rr[0][0]);
        o1[0][a] = g10 + im * ((R)2 * rr[1][0] - rr[1][1]);
        o1[1][a] = g11 + im * ((R)2 * rr[1][1] - rr[1][0]);
      }
    }
    if (IMPL) {
#pragma unroll
      for (int r = 0; r < 6; ++r) s_W[r * TPX + slot] = W[(size_t)r * P + p];
    }
  }
  if (IMPL) {
    __syncthreads();
    // increment form: every prism adds dt A(W, st1) f0 to its own rows of rhs - M1 f0
    // from the tile's shared arrays (in parallel, before the column sweeps)
    if (i < tl.np) {
      const int lt = tile_tri_of(s_off, tl.nt, i);
      const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
      const R w6 = Geo<R>::jh(m, t) * (R)(1.0 / 6.0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ia = a * nt + t;
        const R stv = s_st[a * TP + lt];
        const R dz = dz_rest_r<R>(m, ia, k, N) * stv, idz = rcp<R>(dz);
        R idzm = idz, idzp = idz;
        if (m.n_levels != 0) {
          if (k > 0) idzm = rcp<R>(dz_rest_r<R>(m, ia, k - 1, N) * stv);
          if (k + 1 < N) idzp = rcp<R>(dz_rest_r<R>(m, ia, k + 1, N) * stv);
        }
        const R W0 = s_W[a * TPX + slot], W1 = s_W[(3 + a) * TPX + slot];
        const R Wn = (k + 1 < N) ? s_W[a * TPX + slot + 1] : (R)0;
        R A[2][2], AL[2][2], AU[2][2];
        vertical_A<R>(k, N, w6, idzm, idz, idzp, W0, W1, Wn, ua.kap_v, pp.pen_v, A, AL, AU);
        const int p = tl.p0 + i;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const R* Gq = q ? G1 : G0;
          const R* xt = Gq + (size_t)a * P + p;   // top nodes of field q (global, L2)
          const R* xb = Gq + (size_t)(3 + a) * P + p;
          R fm0 = 0, fm1 = 0, fp0 = 0, fp1 = 0;
          if (k > 0) { fm0 = xt[-1]; fm1 = xb[-1]; }
          if (k + 1 < N) { fp0 = xt[1]; fp1 = xb[1]; }
          const R f0 = xt[0], f1 = xb[0];
          s_b[(2 * q * 3 + a) * TPX + slot] +=
              dt * (A[0][0] * f0 + A[0][1] * f1 + AL[0][0] * fm0 + AL[0][1] * fm1 + AU[0][0] * fp0 + AU[0][1] * fp1);
          s_b[((2 * q + 1) * 3 + a) * TPX + slot] +=
              dt * (A[1][0] * f0 + A[1][1] * f1 + AL[1][0] * fm0 + AL[1][1] * fm1 + AU[1][0] * fp0 + AU[1][1] * fp1);
        }
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
      const int a = j / tl.nt, lt = j - a * tl.nt;
      const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
      R* C = s_C + (size_t)a * 4 * TPX + base;
      column_thomas2<R>(m, t, a * nt + t, N, s_st[a * TP + lt], s_W + a * TPX + base,
                        s_W + (3 + a) * TPX + base, s_b + (0 * 3 + a) * TPX + base,
                        s_b + (1 * 3 + a) * TPX + base, s_b + (2 * 3 + a) * TPX + base,
                        s_b + (3 * 3 + a) * TPX + base, C, C + TPX, C + 2 * TPX, C + 3 * TPX,
                        ua.kap_v, pp.pen_v, dt);
    }
    __syncthreads();
    if (i < tl.np) {  // f1 = f0 + increment
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const size_t idx = (size_t)(c * 3 + a) * P + tl.p0 + i;
          o0[c][a] = G0[idx] + s_b[(c * 3 + a) * TPX + slot];
          o1[c][a] = G1[idx] + s_b[((2 + c) * 3 + a) * TPX + slot];
        }
    }
  }
  if (i < tl.np) {
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t idx = (size_t)(c * 3 + a) * P + tl.p0 + i;
        O0[idx] = o0[c][a];
        O1[idx] = o1[c][a];
        ok &= (bool)isfinite(o0[c][a]) & (bool)isfinite(o1[c][a]);
      }
    if (!ok) atomicOr(err, (int)SLIM_ERRBIT_NONFINITE);
  }
}

size_t tile_smem(const DevMesh& m, int TP, size_t esz, int rows) {
  return ((TP + 1) * sizeof(int) + 15) / 16 * 16 + (size_t)rows * (TP + m.max_tile_tris) * esz;
}
// implicit: s_b [12], s_W [6], s_C [12] x TPX, s_st [3] x TP; explicit: the offsets only
size_t update_smem(const DevMesh& m, int TP, size_t esz, bool impl) {
  // the explicit update stages nothing in shared memory (more of it stays L1 cache)
  if (!impl) return ((TP + 1) * sizeof(int) + 15) / 16 * 16;
  return ((TP + 1) * sizeof(int) + 15) / 16 * 16 + (size_t)30 * (TP + m.max_tile_tris) * esz +
         (size_t)3 * TP * esz;
}

template <typename R>
PP<R> phys(const slim_params& p) {
  PP<R> q;
  q.g = (R)p.g; q.rho0 = (R)p.rho0; q.irho0 = (R)(1.0 / p.rho0); q.f = (R)p.coriolis_f;
  q.alpha = (R)p.eos_alpha; q.beta = (R)p.eos_beta; q.T0 = (R)p.eos_T0; q.S0 = (R)p.eos_S0;
  q.nu_h = (R)p.nu_h; q.kappa_h = (R)p.kappa_h; q.nu_v = (R)p.nu_v; q.kappa_v = (R)p.kappa_v;
  q.cd = (R)p.drag_cd; q.pen_v = (R)p.penalty_v; q.pen_h = (R)p.penalty_h; q.g_d = p.g;
  return q;
}

#define SLIM_CU(expr)                                                          \
  do {                                                                         \
    cudaError_t _e = (expr);                                                   \
    if (_e != cudaSuccess) {                                                   \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));           \
      return SLIM_ERR_CUDA;                                                    \
    }                                                                          \
  } while (0)

template <typename R>
cudaError_t launch_hpg(const DevMesh& m, int TP, int occ, const R* T, const R* S, const R* st,
                       const PP<R>& pp, R* Rx, R* Ry, cudaStream_t s) {
  SLIM_TPO_SWITCH(R, TP, occ, {
    const size_t sm = tile_smem(m, TPc, sizeof(R), 12);
    cudaError_t e = set_smem2(k_hpg<R, TPc, OCc>, sm);
    if (e != cudaSuccess) return e;
    k_hpg<R, TPc, OCc><<<m.n_tiles, TPc, sm, s>>>(m, T, S, st, pp, Rx, Ry);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mompred(const DevMesh& m, int TP, int occ, const AdvIn<R>& in, const R* Rx,
                           const R* Ry, const PP<R>& pp, SplitBufs* b, cudaStream_t s,
                           R* Fx_out = nullptr, R* Fy_out = nullptr) {
  SLIM_TPO_SWITCH(R, TP, occ, {
    const size_t sm = tile_smem(m, TPc, sizeof(R), 12);
    cudaError_t e = set_smem2(k_mompred<R, TPc, OCc>, sm);
    if (e != cudaSuccess) return e;
    k_mompred<R, TPc, OCc><<<m.n_tiles, TPc, sm, s>>>(m, in, Rx, Ry, pp, b->S3x, b->S3y, b->Sqx, b->Sqy,
                                                 (R*)b->S3x_r, (R*)b->S3y_r, (R*)b->Ex, (R*)b->Ey,
                                                 Fx_out, Fy_out);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cont_split(const DevMesh& m, int TP, const AdvIn<R>& in, const double* e0,
                              const double* e1, double T, R* W, cudaStream_t s) {
  SLIM_TP_SWITCH2(TP, {
    const size_t sm = tile_smem(m, TPc, sizeof(R), 6);
    cudaError_t e = set_smem2(k_cont_split<R, TPc>, sm);
    if (e != cudaSuccess) return e;
    k_cont_split<R, TPc><<<m.n_tiles, TPc, sm, s>>>(m, in, e0, e1, T, W);
  });
  return cudaGetLastError();
}

template <typename R, int KIND, bool IMPL>
cudaError_t launch_update(const DevMesh& m, int TP, int occ, const AdvIn<R>& in, const R* G0, const R* G1,
                          const R* W, const R* Ex, const R* Ey, const R* F2x, const R* F2y,
                          const R* st0, const R* st1, const PP<R>& pp, const UA<R>& ua,
                          R* O0, R* O1, int* err, cudaStream_t s) {
  SLIM_TPO_SWITCH(R, TP, occ, {
    const size_t sm = update_smem(m, TPc, sizeof(R), IMPL);
    cudaError_t e = set_smem2(k_update<R, TPc, KIND, IMPL, OCc>, sm);
    if (e != cudaSuccess) return e;
    k_update<R, TPc, KIND, IMPL, OCc><<<m.n_tiles, TPc, sm, s>>>(m, in, G0, G1, W, Ex, Ey, F2x, F2y, st0,
                                                            st1, pp, ua, O0, O1, err);
  });
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// one stage of the split step
// ---------------------------------------------------------------------------
template <typename R>
slim_status stage(slim_state* s, double t0, double dt, int n_sub, int tide_base, bool implicit, const R* u_ev,
                  const R* v_ev, const R* T_ev, const R* S_ev, const R* st_ev, R* u_out, R* v_out,
                  R* T_out, R* S_out, cudaStream_t stm) {
  const DevMesh& m = s->mesh->d;
  SplitBufs* b = s->sp;
  const int TP = s->mesh->tile_prisms;
  const int occ = occ_of(s->par, TP);
  const PP<R> pp = phys<R>(s->par);
  const int nt = m.n_tri;
  const size_t n2 = (size_t)3 * nt;
  R* Rx = (R*)s->Rx;
  R* Ry = (R*)s->Ry;
  {
    ProfScope ps(s, SLIM_PHASE_HPG, stm);
    SLIM_CU(launch_hpg<R>(m, TP, occ, T_ev, S_ev, st_ev, pp, Rx, Ry, stm));
  }
  // open-boundary forcing: exterior state at theta of the middle of this stage's
  // 2D run (slot n_tide + 1 for the first split stage, n_tide + 2 for the second)
  const int mid = b->n_tide + (tide_base == 0 ? 1 : 2);
  const R* th_mid = sizeof(R) == 8 ? (const R*)(const void*)(b->theta + mid)
                                   : (const R*)(const void*)(b->theta_f + mid);
  const bool fx = s->par.forcing != 0;
  const R* Uxa = fx ? (const R*)s->Uxa : nullptr;
  const R* Vxa = fx ? (const R*)s->Vxa : nullptr;
  const R* Uxb = fx ? (const R*)s->Uxb : nullptr;
  const R* Vxb = fx ? (const R*)s->Vxb : nullptr;
  AdvIn<R> pin{u_ev, v_ev, nullptr, nullptr, Uxa, Vxa, st_ev, nullptr, nullptr, nullptr,
               Uxa, Vxa, Uxb, Vxb, Uxb, Vxb, th_mid};
  {
    ProfScope ps(s, SLIM_PHASE_MOM_PRED, stm);
    SLIM_CU(launch_mompred<R>(m, TP, occ, pin, Rx, Ry, pp, b, stm));
  }
  b->has_s3 = true;
  // external mode from the state at t0: working copies, FP32 shadows, zero averages
  const bool shadow = sizeof(R) != 8;
  {
    ProfScope ps(s, SLIM_PHASE_MISC, stm);
    const int blocks = (int)std::min<size_t>((n2 + 255) / 256, 4096);
    k_ext2d_begin<<<blocks, 256, 0, stm>>>(s->eta, s->Qx, s->Qy, b->Ae, b->AU, b->AV,
                                           shadow ? (float*)b->Ae_r : nullptr,
                                           shadow ? (float*)b->AU_r : nullptr,
                                           shadow ? (float*)b->AV_r : nullptr, s->Qbx, s->Qby, n2);
    SLIM_CU(cudaGetLastError());
  }
  SLIM_CU(cudaMemsetAsync(b->Gb, 0, n2 * 2 * 8, stm));
  const double dts = dt / n_sub;
  const double A_[3] = {0.0, 0.75, 1.0 / 3.0}, B_[3] = {1.0, 0.25, 2.0 / 3.0};
  const double bw_[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  const int blk = 256, grd = (nt + blk - 1) / blk;
  double* F[3][3] = {{b->Ae, b->AU, b->AV}, {b->Be, b->BU, b->BV}, {b->Ce, b->CU, b->CV}};
  void* Fr[3][3] = {{b->Ae_r, b->AU_r, b->AV_r}, {b->Be_r, b->BU_r, b->BV_r}, {b->Ce_r, b->CU_r, b->CV_r}};
  if (!shadow) {
    for (int q = 0; q < n_sub; ++q) {
      for (int st = 0; st < 3; ++st) {
        const int si = st, so = (st + 1) % 3;  // A -> B -> C -> A
        const int tide_idx = tide_base + 3 * q + st;
        Ext2dIO io;
        io.e = F[si][0]; io.U = F[si][1]; io.V = F[si][2];
        io.er = F[si][0]; io.Ur = F[si][1]; io.Vr = F[si][2];
        io.en = b->Ae; io.Un = b->AU; io.Vn = b->AV;
        io.eo = F[so][0]; io.Uo = F[so][1]; io.Vo = F[so][2];
        io.eor = io.Uor = io.Vor = nullptr;
        ProfScope ps(s, SLIM_PHASE_EXT2D, stm);
        k_ext2d<0, double><<<grd, blk, 0, stm>>>(m, *b, io, s->par.g, tide_idx, A_[st], B_[st], dts,
                                                 bw_[st] / n_sub);
        SLIM_CU(cudaGetLastError());
      }
    }
  } else {
    // mixed: FP32 stage values in the B and C shadows, FP64 state in A (updated by
    // the last stage of each subcycle); the whole run in one cooperative launch with
    // a grid barrier between stages, or one launch per stage
    Mx2dRun run;
    for (int st = 0; st < 3; ++st) {
      Mx2dIO& io = run.io[st];
      io.en = (const float*)b->Ae_r; io.Un = (const float*)b->AU_r; io.Vn = (const float*)b->AV_r;
      io.e = b->Ae; io.U = b->AU; io.V = b->AV;
      const int so = (st + 1) % 3;
      io.er = (const float*)Fr[st][0]; io.Ur = (const float*)Fr[st][1]; io.Vr = (const float*)Fr[st][2];
      io.eo = (float*)Fr[so][0]; io.Uo = (float*)Fr[so][1]; io.Vo = (float*)Fr[so][2];
    }
    run.n_sub = n_sub;
    run.tide_base = tide_base;
    run.g = (float)s->par.g;
    run.dt = (float)dts;
    run.wq = (float)(1.0 / (6.0 * n_sub));
    run.wn = 1.0 / n_sub;
    run.bar = b->bar;
    run.nbits = b->nbits;
    run.done = b->done;
    run.nbw = b->nbw;
    run.err = s->err;
    if (s->par.persistent_2d) {
      SLIM_CU(cudaMemsetAsync(b->bar, 0, sizeof(unsigned), stm));  // arrival count
      if (b->done) SLIM_CU(cudaMemsetAsync(b->done, 0, (size_t)b->run_blocks * sizeof(unsigned), stm));
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(b->run_blocks);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = stm;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      ProfScope ps(s, SLIM_PHASE_EXT2D, stm);
      SLIM_CU(cudaLaunchKernelEx(&cfg, k_ext2d_run, m, *b, run, 0, 3 * n_sub));
    } else {
      for (int gs = 0; gs < 3 * n_sub; ++gs) {
        ProfScope ps(s, SLIM_PHASE_EXT2D, stm);
        k_ext2d_run<<<grd, blk, 0, stm>>>(m, *b, run, gs, 1);
        SLIM_CU(cudaGetLastError());
      }
    }
  }
  {
    ProfScope ps(s, SLIM_PHASE_MISC, stm);
    k_couple2d<R><<<grd, blk, 0, stm>>>(m, b->Ae, b->AU, b->AV, s->Qx, s->Qy, b->S3x, b->S3y, b->Sqx,
                                        b->Sqy, s->Qbx, s->Qby, b->Gb, st_ev, b->iw6, dt, 1.0 / dt,
                                        b->F2x, b->F2y,
                                        (R*)b->F2x_r, (R*)b->F2y_r, (R*)b->Dqx_r, (R*)b->Dqy_r,
                                        (R*)b->gcor_r, (R*)b->st_end, fx ? b->Qext : nullptr,
                                        b->theta + mid);
    SLIM_CU(cudaGetLastError());
  }
  AdvIn<R> cin{u_ev, v_ev, nullptr, nullptr, Uxa, Vxa, st_ev, (const R*)b->Dqx_r,
               (const R*)b->Dqy_r, (const R*)b->gcor_r, Uxa, Vxa, Uxb, Vxb, Uxb, Vxb, th_mid};
  {
    // the continuity computes the face transports of the stage; the two updates read them
    AdvIn<R> cin_w = cin;
    cin_w.qn_out = (R*)b->qnf;
    cin.qn_in = (const R*)b->qnf;
    ProfScope ps(s, SLIM_PHASE_CONTINUITY, stm);
    SLIM_CU(launch_cont_split<R>(m, TP, cin_w, s->eta, b->Ae, dt, (R*)s->W, stm));
  }
  const R* st0 = (const R*)s->st_cur;
  const R* st1 = (const R*)b->st_end;
  UA<R> um{(R)dt, (R)s->par.nu_v, (R)s->par.nu_h};
  UA<R> ut{(R)dt, (R)s->par.kappa_v, (R)s->par.kappa_h};
  AdvIn<R> tin{u_ev, v_ev, T_ev, S_ev, (const R*)s->Text, (const R*)s->Sext, st_ev,
               (const R*)b->Dqx_r, (const R*)b->Dqy_r, (const R*)b->gcor_r, Uxa, Vxa, Uxb, Vxb,
               fx ? (const R*)s->Textb : nullptr, fx ? (const R*)s->Sextb : nullptr, th_mid, nullptr,
               (const R*)b->qnf};
  const R* U0 = (const R*)s->U;
  const R* V0 = (const R*)s->V;
  const R* T0 = (const R*)s->T;
  const R* S0 = (const R*)s->S;
  {
    ProfScope ps(s, SLIM_PHASE_MOMENTUM, stm);
    if (implicit)
      SLIM_CU((launch_update<R, 0, true>(m, TP, occ, cin, U0, V0, (const R*)s->W, (const R*)b->Ex,
                                         (const R*)b->Ey, (const R*)b->F2x_r,
                                         (const R*)b->F2y_r, st0, st1, pp, um, u_out, v_out, s->err, stm)));
    else
      SLIM_CU((launch_update<R, 0, false>(m, TP, occ, cin, U0, V0, (const R*)s->W, (const R*)b->Ex,
                                          (const R*)b->Ey, (const R*)b->F2x_r,
                                          (const R*)b->F2y_r, st0, st1, pp, um, u_out, v_out, s->err, stm)));
  }
  {
    ProfScope ps(s, SLIM_PHASE_TRACERS, stm);
    if (implicit)
      SLIM_CU((launch_update<R, 1, true>(m, TP, occ, tin, T0, S0, (const R*)s->W, nullptr, nullptr, nullptr,
                                         nullptr, st0, st1, pp, ut, T_out, S_out, s->err, stm)));
    else
      SLIM_CU((launch_update<R, 1, false>(m, TP, occ, tin, T0, S0, (const R*)s->W, nullptr, nullptr, nullptr,
                                          nullptr, st0, st1, pp, ut, T_out, S_out, s->err, stm)));
  }
  return SLIM_OK;
}

template <typename R>
slim_status step_t(slim_state* s, double t, double dt, cudaStream_t stm) {
  SplitBufs* b = s->sp;
  const DevMesh& m = s->mesh->d;
  const size_t n2 = (size_t)3 * m.n_tri;
  R* U = (R*)s->U; R* V = (R*)s->V; R* T = (R*)s->T; R* S = (R*)s->S;
  R* hu = (R*)s->tmp[0]; R* hv = (R*)s->tmp[1]; R* hT = (R*)s->tmp[2]; R* hS = (R*)s->tmp[3];
  // stage 1: t -> t + dt/2, vertically implicit, n_sub/2 external steps
  // open-boundary elevation of every external stage of the step (first kernel of the
  // step: its time argument is the only one that changes between steps)
  {
    ProfScope ps(s, SLIM_PHASE_MISC, stm);
    TideArgs ta;
    split_time_args(s, t, dt, &ta);
    k_tide<<<1, 128, 0, stm>>>(ta);
    SLIM_CU(cudaGetLastError());
  }
  b->forcing = s->par.forcing;
  if (b->forcing) {
    ProfScope ps(s, SLIM_PHASE_MISC, stm);
    const int grd = std::min((m.n_tri + 255) / 256, 2048);
    k_ext_sums<R><<<grd, 256, 0, stm>>>(m, (const R*)s->Uxa, (const R*)s->Vxa, (const R*)s->Uxb,
                                        (const R*)s->Vxb, b->Qext, b->Qext_f);
    SLIM_CU(cudaGetLastError());
  }
  slim_status r = stage<R>(s, t, 0.5 * dt, s->par.n_sub / 2, 0, true, U, V, T, S, (const R*)s->st_cur,
                           hu, hv, hT, hS, stm);
  if (r != SLIM_OK) return r;
  SLIM_CU(cudaMemcpyAsync(b->st_half, b->st_end, n2 * sizeof(R), cudaMemcpyDeviceToDevice, stm));
  SLIM_CU(cudaMemcpyAsync(b->eta_half, b->Ae, n2 * 8, cudaMemcpyDeviceToDevice, stm));
  // stage 2: t -> t + dt from the same start, horizontal terms at the stage-1 state
  r = stage<R>(s, t, dt, s->par.n_sub, 3 * (s->par.n_sub / 2), false, hu, hv, hT, hS,
               (const R*)b->st_half, U, V, T, S, stm);
  if (r != SLIM_OK) return r;
  SLIM_CU(cudaMemcpyAsync(s->eta, b->Ae, n2 * 8, cudaMemcpyDeviceToDevice, stm));
  SLIM_CU(cudaMemcpyAsync(s->Qx, b->AU, n2 * 8, cudaMemcpyDeviceToDevice, stm));
  SLIM_CU(cudaMemcpyAsync(s->Qy, b->AV, n2 * 8, cudaMemcpyDeviceToDevice, stm));
  SLIM_CU(cudaMemcpyAsync(s->st_cur, b->st_end, n2 * sizeof(R), cudaMemcpyDeviceToDevice, stm));
  SLIM_CU(cudaMemcpyAsync(s->eta_next, b->Ae, n2 * 8, cudaMemcpyDeviceToDevice, stm));
  return SLIM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// entry points used by the C ABI
// ---------------------------------------------------------------------------
size_t split_aux2d_len(const DevMesh& m) { return (size_t)16 * m.n_tri; }

const void* split_time_kernel() { return (const void*)k_tide; }
void split_time_args(const slim_state* s, double t, double dt, void* out) {
  static_assert(sizeof(TideArgs) <= 128, "time kernel argument");
  TideArgs a;
  a.t0 = t;
  a.dt = dt;
  a.amp = s->par.tide_amp;
  a.period = s->par.tide_period;
  a.ta = s->par.forcing_t_a;
  a.tb = s->par.forcing_t_b > s->par.forcing_t_a ? s->par.forcing_t_b : s->par.forcing_t_a + 1.0;
  a.n = s->par.n_sub;
  a.out = s->sp->tide;
  a.theta = s->sp->theta;
  std::memcpy(out, &a, sizeof(a));
}

slim_status split_alloc(slim_state* s) {
  if (s->sp) return SLIM_OK;
  const DevMesh& m = s->mesh->d;
  const size_t n2 = (size_t)3 * m.n_tri;
  SplitBufs* b = new SplitBufs();
  s->sp = b;
  double** d2[] = {&b->Ae, &b->AU, &b->AV, &b->Be, &b->BU, &b->BV, &b->Ce, &b->CU, &b->CV,
                   &b->S3x, &b->S3y, &b->Sqx, &b->Sqy, &b->F2x, &b->F2y, &b->eta_half};
  for (double** p : d2) {
    SLIM_CU(cudaMalloc((void**)p, n2 * 8));
    SLIM_CU(cudaMemset(*p, 0, n2 * 8));
    s->allocs.push_back(*p);
  }
  double** d6[] = {&b->Gb, &b->cw};
  for (double** p : d6) {
    SLIM_CU(cudaMalloc((void**)p, n2 * 2 * 8));
    SLIM_CU(cudaMemset(*p, 0, n2 * 2 * 8));
    s->allocs.push_back(*p);
  }
  void** r2[] = {&b->F2x_r, &b->F2y_r, &b->Dqx_r, &b->Dqy_r, &b->st_half, &b->st_end,
                 &b->Ae_r, &b->AU_r, &b->AV_r, &b->Be_r, &b->BU_r, &b->BV_r, &b->Ce_r, &b->CU_r,
                 &b->CV_r, &b->S3x_r, &b->S3y_r};
  for (void** p : r2) {
    SLIM_CU(cudaMalloc(p, n2 * s->esz));
    SLIM_CU(cudaMemset(*p, 0, n2 * s->esz));
    s->allocs.push_back(*p);
  }
  float** f6[] = {&b->cw_f};
  for (float** p : f6) {
    SLIM_CU(cudaMalloc((void**)p, n2 * 2 * sizeof(float)));
    s->allocs.push_back(*p);
  }
  const size_t n_tide = (size_t)3 * (s->par.n_sub / 2 + s->par.n_sub);
  SLIM_CU(cudaMalloc((void**)&b->tide, (n_tide + 1) * 8 + n_tide * sizeof(float)));
  SLIM_CU(cudaMemset(b->tide, 0, (n_tide + 1) * 8 + n_tide * sizeof(float)));
  s->allocs.push_back(b->tide);
  b->tide_f = reinterpret_cast<float*>(b->tide + n_tide + 1);
  b->n_tide = (int)n_tide;
  b->forcing = 0;
  SLIM_CU(cudaMalloc((void**)&b->theta, (n_tide + 3) * (8 + sizeof(float))));
  SLIM_CU(cudaMemset(b->theta, 0, (n_tide + 3) * (8 + sizeof(float))));
  s->allocs.push_back(b->theta);
  b->theta_f = reinterpret_cast<float*>(b->theta + n_tide + 3);
  SLIM_CU(cudaMalloc((void**)&b->Qext, 4 * n2 * (8 + sizeof(float))));
  SLIM_CU(cudaMemset(b->Qext, 0, 4 * n2 * (8 + sizeof(float))));
  s->allocs.push_back(b->Qext);
  b->Qext_f = reinterpret_cast<float*>(b->Qext + 4 * n2);
  SLIM_CU(cudaMalloc((void**)&b->iw6, (size_t)m.n_tri * 8));
  s->allocs.push_back(b->iw6);
  SLIM_CU(cudaMalloc((void**)&b->iw6_f, (size_t)m.n_tri * sizeof(float)));
  s->allocs.push_back(b->iw6_f);
  if (m.n_tri >= (1 << 27)) { set_error("too many triangles for the 2D adjacency word"); return SLIM_ERR_ARG; }
  SLIM_CU(cudaMalloc((void**)&b->adj2, (size_t)3 * m.n_tri * sizeof(int)));
  s->allocs.push_back(b->adj2);
  b->Dacc = b->Eacc = b->Gacc = b->Gacc2 = nullptr;
  b->bar = nullptr;
  b->run_blocks = 0;
  b->nbits = b->done = nullptr;
  b->nbw = 0;
  if (s->esz == 4) {
    SLIM_CU(cudaMalloc((void**)&b->bar, 2 * sizeof(unsigned)));
    SLIM_CU(cudaMemset(b->bar, 0, 2 * sizeof(unsigned)));
    s->allocs.push_back(b->bar);
    int dev = 0, sms = 0, per_sm = 0;
    SLIM_CU(cudaGetDevice(&dev));
    SLIM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SLIM_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ext2d_run, 256, 0));
    b->run_blocks = std::max(1, std::min(sms * per_sm, (m.n_tri + 255) / 256));
    if (b->run_blocks <= kMaxNbBlocks) {
      b->nbw = (b->run_blocks + 31) / 32;
      const size_t nbits = (size_t)b->run_blocks * b->nbw;
      SLIM_CU(cudaMalloc((void**)&b->nbits, nbits * sizeof(unsigned)));
      s->allocs.push_back(b->nbits);
      SLIM_CU(cudaMalloc((void**)&b->done, (size_t)b->run_blocks * sizeof(unsigned)));
      s->allocs.push_back(b->done);
      SLIM_CU(cudaMemset(b->nbits, 0, nbits * sizeof(unsigned)));
      SLIM_CU(cudaMemset(b->done, 0, (size_t)b->run_blocks * sizeof(unsigned)));
      k_block_graph<<<(m.n_tri + 255) / 256, 256>>>(m, b->run_blocks * 256, b->nbw, b->nbits);
      SLIM_CU(cudaGetLastError());
      SLIM_CU(cudaDeviceSynchronize());
    }
    float** fa[] = {&b->Dacc, &b->Eacc, &b->Gacc, &b->Gacc2};
    const size_t cnt[] = {3 * n2, 2 * n2, 2 * n2, 2 * n2};
    for (int j = 0; j < 4; ++j) {
      SLIM_CU(cudaMalloc((void**)fa[j], cnt[j] * sizeof(float)));
      SLIM_CU(cudaMemset(*fa[j], 0, cnt[j] * sizeof(float)));
      s->allocs.push_back(*fa[j]);
    }
  }
  b->Qbx = s->Qbx;
  b->Qby = s->Qby;
  for (void** p : {&b->Ex, &b->Ey}) {
    SLIM_CU(cudaMalloc(p, (size_t)6 * m.P * s->esz));
    SLIM_CU(cudaMemset(*p, 0, (size_t)6 * m.P * s->esz));
    s->allocs.push_back(*p);
  }
  SLIM_CU(cudaMalloc(&b->qnf, (size_t)12 * m.P * s->esz));
  SLIM_CU(cudaMemset(b->qnf, 0, (size_t)12 * m.P * s->esz));
  s->allocs.push_back(b->qnf);
  SLIM_CU(cudaMalloc(&b->gcor_r, n2 * 2 * s->esz));
  SLIM_CU(cudaMemset(b->gcor_r, 0, n2 * 2 * s->esz));
  s->allocs.push_back(b->gcor_r);
  const int grd = (m.n_tri + 255) / 256;
  k_wave_speed<<<grd, 256>>>(m, s->par.g, b->cw, b->cw_f, b->iw6, b->iw6_f, b->adj2);
  SLIM_CU(cudaGetLastError());
  return SLIM_OK;
}

void split_free(slim_state* s) {
  delete s->sp;
  s->sp = nullptr;
}

void* split_field(slim_state* s, int field) {
  if (!s->sp) return nullptr;
  switch (field) {
    case SLIM_FIELD_S3_X: return s->sp->S3x;
    case SLIM_FIELD_S3_Y: return s->sp->S3y;
    case SLIM_FIELD_F2D_X: return s->sp->F2x;
    case SLIM_FIELD_F2D_Y: return s->sp->F2y;
  }
  return nullptr;
}

slim_status split_hpg(slim_state* s, cudaStream_t st) {
  const DevMesh& m = s->mesh->d;
  if (s->prec == SLIM_FP64)
    SLIM_CU(launch_hpg<double>(m, s->mesh->tile_prisms, 2, (const double*)s->T, (const double*)s->S,
                               (const double*)s->st_cur, phys<double>(s->par), (double*)s->Rx,
                               (double*)s->Ry, st));
  else
    SLIM_CU(launch_hpg<float>(m, s->mesh->tile_prisms, occ_of(s->par, s->mesh->tile_prisms), (const float*)s->T, (const float*)s->S,
                              (const float*)s->st_cur, phys<float>(s->par), (float*)s->Rx,
                              (float*)s->Ry, st));
  return SLIM_OK;
}

// F_3D^h of the state (a velocity component into out) with r recomputed from the
// state's T, S; the column sums S3 go to the split buffers (SLIM_FIELD_S3_X/Y)
template <typename R>
slim_status rhs3d_momentum_t(slim_state* s, int field, R* out, cudaStream_t st) {
  const DevMesh& m = s->mesh->d;
  const int TP = s->mesh->tile_prisms;
  const int occ = sizeof(R) == 8 ? 2 : occ_of(s->par, TP);
  const PP<R> pp = phys<R>(s->par);
  SLIM_CU(launch_hpg<R>(m, TP, occ, (const R*)s->T, (const R*)s->S, (const R*)s->st_cur, pp, (R*)s->Rx,
                        (R*)s->Ry, st));
  AdvIn<R> pin{(const R*)s->U, (const R*)s->V, nullptr, nullptr, nullptr, nullptr, (const R*)s->st_cur,
               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  SLIM_CU(launch_mompred<R>(m, TP, occ, pin, (const R*)s->Rx, (const R*)s->Ry, pp, s->sp, st,
                            field == SLIM_FIELD_U ? out : nullptr, field == SLIM_FIELD_V ? out : nullptr));
  s->sp->has_s3 = true;
  return SLIM_OK;
}

slim_status split_rhs3d_momentum(slim_state* s, int field, void* out, cudaStream_t st) {
  if (!s->sp) { set_error("split buffers missing"); return SLIM_ERR_UNSUPPORTED; }
  if (s->par.forcing) {
    set_error("slim_rhs3d of a velocity needs forcing = 0 (the forced exterior state depends on a stage time)");
    return SLIM_ERR_UNSUPPORTED;
  }
  return s->prec == SLIM_FP64 ? rhs3d_momentum_t<double>(s, field, (double*)out, st)
                              : rhs3d_momentum_t<float>(s, field, (float*)out, st);
}

slim_status split_rhs2d(slim_state* s, double t, double* out, cudaStream_t st) {
  if (!s->sp) { set_error("split buffers missing"); return SLIM_ERR_UNSUPPORTED; }
  const DevMesh& m = s->mesh->d;
  SplitBufs* b = s->sp;
  const double tide = s->par.tide_amp * std::cos(2.0 * M_PI * t / s->par.tide_period);
  const int slot = 3 * (s->par.n_sub / 2 + s->par.n_sub);
  b->forcing = s->par.forcing;
  const double th = s->par.forcing
                        ? (t - s->par.forcing_t_a) / (s->par.forcing_t_b - s->par.forcing_t_a) : 0.0;
  SLIM_CU(cudaMemcpyAsync(b->tide + slot, &tide, sizeof(double), cudaMemcpyHostToDevice, st));
  SLIM_CU(cudaMemcpyAsync(b->theta + slot, &th, sizeof(double), cudaMemcpyHostToDevice, st));
  if (s->par.forcing) {
    const int grd = std::min((m.n_tri + 255) / 256, 2048);
    if (s->prec == SLIM_FP64)
      k_ext_sums<double><<<grd, 256, 0, st>>>(m, (const double*)s->Uxa, (const double*)s->Vxa,
                                              (const double*)s->Uxb, (const double*)s->Vxb, b->Qext,
                                              b->Qext_f);
    else
      k_ext_sums<float><<<grd, 256, 0, st>>>(m, (const float*)s->Uxa, (const float*)s->Vxa,
                                             (const float*)s->Uxb, (const float*)s->Vxb, b->Qext,
                                             b->Qext_f);
    SLIM_CU(cudaGetLastError());
  }
  SLIM_CU(cudaStreamSynchronize(st));
  const int grd = (m.n_tri + 255) / 256;
  Ext2dIO io{};
  io.e = s->eta; io.U = s->Qx; io.V = s->Qy;
  io.eo = out;
  if (s->prec == SLIM_FP64) {
    io.er = s->eta; io.Ur = s->Qx; io.Vr = s->Qy;
    k_ext2d<1, double><<<grd, 256, 0, st>>>(m, *b, io, s->par.g, slot, 0.0, 0.0, 0.0, 0.0);
  } else {
    const size_t n2 = (size_t)3 * m.n_tri;
    SLIM_CU(launch_convert_d2f(s->eta, (float*)b->Ae_r, n2, st));
    SLIM_CU(launch_convert_d2f(s->Qx, (float*)b->AU_r, n2, st));
    SLIM_CU(launch_convert_d2f(s->Qy, (float*)b->AV_r, n2, st));
    io.er = b->Ae_r; io.Ur = b->AU_r; io.Vr = b->AV_r;
    k_ext2d<1, float><<<grd, 256, 0, st>>>(m, *b, io, s->par.g, slot, 0.0, 0.0, 0.0, 0.0);
  }
  SLIM_CU(cudaGetLastError());
  return SLIM_OK;
}

slim_status split_step(slim_state* s, double t, double dt, cudaStream_t st) {
  if (!s->sp) { set_error("split buffers missing"); return SLIM_ERR_UNSUPPORTED; }
  return s->prec == SLIM_FP64 ? step_t<double>(s, t, dt, st) : step_t<float>(s, t, dt, st);
}

int split_kernel_count(const slim_state* s) {
  // time kernel; per stage: hpg, mompred, the start of the external run, 3 n_sub_stage
  // external stages, couple, continuity, momentum, tracers (the persistent mixed run
  // is one launch per stage)
  const int n = s->par.n_sub;
  const int ext = (s->prec == SLIM_MIXED && s->par.persistent_2d) ? 2 : 3 * (n / 2 + n);
  return 1 + 2 * 7 + ext;
}

}  // namespace slim
