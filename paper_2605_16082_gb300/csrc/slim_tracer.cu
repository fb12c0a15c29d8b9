// Kernels of the tracer path: continuity (vertical flux), SSP-RK3 stage with the
// fused horizontal residual + implicit vertical solve, standalone residual and
// vertical solve, compensated tracer-mass reduction.
//
// Every kernel runs one thread block per tile of whole columns (at most TP
// prisms).  Phase 1 is thread-per-prism: coalesced loads of the six node planes,
// the horizontal residual with lateral-neighbour gathers through the adjacency
// table (no atomics), results staged in shared memory.  Phase 2 is thread-per-
// vertex-column: the column recursion or the 2x2-block Thomas sweep on shared
// memory.  Phase 3 writes the six node planes back coalesced.
//
// Shared-memory slots of local prism i of local triangle lt are skewed to
// i + lt, so that the threads of phase 2 (consecutive columns, stride N + 1)
// and of phase 1 (consecutive layers, stride 1) avoid bank conflicts for even
// layer counts.
//
// The layer geometry enters only through the per-vertex-column stretch
// 1 + eta/h in the compute type (st arrays), so the mixed form runs no FP64
// arithmetic in the 3D kernels; the FP64 elevation update stays in the
// continuity kernel's column epilogue.
#include <cmath>
#include <float.h>

#include <algorithm>

#include "slim_device.cuh"
#include "slim_kernels.h"

namespace slim {

template <typename R, int TP>
struct MinBlocks {
  static constexpr int value = sizeof(R) == 4 ? (1024 / TP > 0 ? 1024 / TP : 1) : (512 / TP > 0 ? 512 / TP : 1);
};

// ---------------------------------------------------------------------------
// stretch of every vertex column: st = 1 + eta (1/h)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_stretch(DevMesh m, const double* __restrict__ eta, R* __restrict__ st) {
  const int n = 3 * m.n_tri;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    st[i] = (R)(1.0 + eta[i] * m.ih[i]);
}

// ---------------------------------------------------------------------------
// continuity: eta' (FP64) and the vertex-weighted vertical flux W
//   (J_h/6)(eta' - eta)/dt = sum_column R_h(q, 1)                        (Eq. 2)
//   F_{k,c} = R_h(q,1)_{k,c} - (J_h/12)(dz'_k - dz_k)/dt
//   bottom-up D_vd recursion (Eq. 17):  s = 0 at the bed,
//     W_{k,top} = F_top + F_bot + s,  W_{k,bot} = F_bot - F_top + s,  s = W_{k,top}
// With DIV_ONLY the kernel writes the column sums (the depth-integrated weak
// divergence) to eta_out instead and stops.
// ---------------------------------------------------------------------------
template <typename R, int TP, bool DIV_ONLY>
__global__ void __launch_bounds__(TP, (MinBlocks<R, TP>::value))
    k_continuity(DevMesh m, const R* __restrict__ U, const R* __restrict__ V,
                 const double* __restrict__ eta, const R* __restrict__ st_cur,
                 double* __restrict__ eta_out, R* __restrict__ st_out, R* __restrict__ W,
                 double dt) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_off = reinterpret_cast<int*>(smem);
  const int TPX = TP + m.max_tile_tris;
  R* s_F = reinterpret_cast<R*>(smem + ((TP + 1) * sizeof(int) + 15) / 16 * 16);
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  Own<R> own;
  if (i < tl.np) load_own<R, true>(m, tl.p0 + i, U, V, nullptr, own);
  load_offsets<TP>(m, tl, s_off);
  int slot = 0;
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    slot = i + lt;
    R out[2][3];
    prism_rh<R, true>(m, t, k, tl.p0 + i, N, own, U, V, nullptr, nullptr, st_cur, out);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) s_F[(c * 3 + a) * TPX + slot] = out[c][a];
  }
  __syncthreads();
  const int nt = m.n_tri;
  for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
    const int a = j / tl.nt, lt = j - a * tl.nt;
    const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
    R* Ft = s_F + a * TPX + base;
    R* Fb = s_F + (3 + a) * TPX + base;
    // depth integration in FP64 accuracy (each layer's two node values are added
    // in the compute type first: that rounding is of the order of the inputs' own)
    ColSum<R> cs;
    for (int k = 0; k < N; ++k) cs.add(Ft[k] + Fb[k]);
    const double D = cs.value();
    const int ia = a * nt + t;
    if (DIV_ONLY) {
      eta_out[ia] = D;
      continue;
    }
    const double jh = m.jh[t];
    const double e0 = eta[ia];
    const double e1 = e0 + dt * D / (jh / 6.0);
    eta_out[ia] = e1;
    st_out[ia] = (R)(1.0 + e1 * m.ih[ia]);
    // dz'_k - dz_k = dz_rest_k (e1 - e0) / h
    const R dm_fac = (R)((jh / 12.0) * (e1 - e0) * m.ih[ia] / dt);
    R s = (R)0;
    for (int k = N - 1; k >= 0; --k) {
      const R dm = dm_fac * dz_rest_r<R>(m, ia, k, N);
      const R ft = Ft[k] - dm, fb = Fb[k] - dm;
      const R wt = ft + fb + s;
      const R wb = fb - ft + s;
      Ft[k] = wt;
      Fb[k] = wb;
      s = wt;
    }
  }
  if (DIV_ONLY) return;
  __syncthreads();
  if (i < tl.np) {
#pragma unroll
    for (int r = 0; r < 6; ++r) W[(size_t)r * m.P + tl.p0 + i] = s_F[r * TPX + slot];
  }
}

// ---------------------------------------------------------------------------
// 2x2-block Thomas sweep of one vertex column on shared memory.
// Wt/Wb: vertex-weighted flux at the top/bottom node of every layer; bt/bb:
// right-hand side, overwritten by the solution; C0..C3: D'^-1 U of the forward
// sweep.  All indexed by layer k.  st: stretch of the column.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void column_thomas(const DevMesh& m, int t, int ia, int N, R st,
                                              const R* __restrict__ Wt, const R* __restrict__ Wb,
                                              R* __restrict__ bt, R* __restrict__ bb,
                                              R* __restrict__ C0, R* __restrict__ C1,
                                              R* __restrict__ C2, R* __restrict__ C3, R kap, R pen,
                                              R bdt, R flux_top, R flux_bot,
                                              const R* __restrict__ x0t = nullptr,
                                              const R* __restrict__ x0b = nullptr) {
  const R omega = Geo<R>::jh(m, t) * (R)(1.0 / 6.0);
  R z0 = 0, z1 = 0;
  R c00 = 0, c01 = 0, c10 = 0, c11 = 0;
  R dz = dz_rest_r<R>(m, ia, 0, N) * st;
  R idz = rcp<R>(dz);
  R idzm = idz;
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    R dzp = dz, idzp = idz;
    if (k + 1 < N && m.n_levels != 0) {
      dzp = dz_rest_r<R>(m, ia, k + 1, N) * st;
      idzp = rcp<R>(dzp);
    }
    const R Wn = (k + 1 < N) ? Wt[k + 1] : (R)0;
    Row<R> row, op;
    assemble_row<R>(k, N, omega, idzm, dz, idz, idzp, Wt[k], Wb[k], Wn, kap, pen, bdt, row, &op);
    R b0 = bt[k], b1 = bb[k];
    if (k == 0) b0 += bdt * omega * flux_top;
    if (k == N - 1) b1 -= bdt * omega * flux_bot;
    if (x0t) {  // increment form: the caller's b is rhs - M x0; add bdt A x0
      const R xt = x0t[k], xb = x0b[k];
      R a0 = op.D[0][0] * xt + op.D[0][1] * xb, a1 = op.D[1][0] * xt + op.D[1][1] * xb;
      if (k > 0) {
        const R ut = x0t[k - 1], ub = x0b[k - 1];
        a0 += op.L[0][0] * ut + op.L[0][1] * ub;
        a1 += op.L[1][0] * ut + op.L[1][1] * ub;
      }
      if (k + 1 < N) {
        const R dt_ = x0t[k + 1], db = x0b[k + 1];
        a0 += op.U[0][0] * dt_ + op.U[0][1] * db;
        a1 += op.U[1][0] * dt_ + op.U[1][1] * db;
      }
      b0 += bdt * a0;
      b1 += bdt * a1;
    }
    // D' = D - L C_{k-1},  y = b - L z_{k-1}
    R Dp[2][2];
    Dp[0][0] = row.D[0][0] - (row.L[0][0] * c00 + row.L[0][1] * c10);
    Dp[0][1] = row.D[0][1] - (row.L[0][0] * c01 + row.L[0][1] * c11);
    Dp[1][0] = row.D[1][0] - (row.L[1][0] * c00 + row.L[1][1] * c10);
    Dp[1][1] = row.D[1][1] - (row.L[1][0] * c01 + row.L[1][1] * c11);
    const R y0 = b0 - (row.L[0][0] * z0 + row.L[0][1] * z1);
    const R y1 = b1 - (row.L[1][0] * z0 + row.L[1][1] * z1);
    R Di[2][2];
    inv2<R>(Dp, Di);
    z0 = Di[0][0] * y0 + Di[0][1] * y1;
    z1 = Di[1][0] * y0 + Di[1][1] * y1;
    c00 = Di[0][0] * row.U[0][0] + Di[0][1] * row.U[1][0];
    c01 = Di[0][0] * row.U[0][1] + Di[0][1] * row.U[1][1];
    c10 = Di[1][0] * row.U[0][0] + Di[1][1] * row.U[1][0];
    c11 = Di[1][0] * row.U[0][1] + Di[1][1] * row.U[1][1];
    bt[k] = z0;
    bb[k] = z1;
    C0[k] = c00; C1[k] = c01; C2[k] = c10; C3[k] = c11;
    idzm = idz;
    dz = dzp;
    idz = idzp;
  }
  // back substitution x_k = z_k - C_k x_{k+1}
  R x0 = z0, x1 = z1;
  for (int k = N - 2; k >= 0; --k) {
    const R n0 = bt[k] - (C0[k] * x0 + C1[k] * x1);
    const R n1 = bb[k] - (C2[k] * x0 + C3[k] * x1);
    bt[k] = n0;
    bb[k] = n1;
    x0 = n0;
    x1 = n1;
  }
  if (x0t) {  // the solution is x0 + increment
    for (int k = 0; k < N; ++k) {
      bt[k] += x0t[k];
      bb[k] += x0b[k];
    }
  }
}

// shared-memory carve-up of the solve kernels (TPX = TP + most triangles per tile)
template <typename R, int TP>
struct SolveSmem {
  size_t off_b, off_W, off_C, off_x, off_st, bytes;
  __host__ __device__ SolveSmem(int TPX) {
    off_b = ((TP + 1) * sizeof(int) + 15) / 16 * 16;
    off_W = off_b + 6 * (size_t)TPX * sizeof(R);
    off_C = off_W + 6 * (size_t)TPX * sizeof(R);
    off_x = off_C + 12 * (size_t)TPX * sizeof(R);   // reference state of the increment form
    off_st = off_x + 6 * (size_t)TPX * sizeof(R);
    bytes = off_st + 3 * (size_t)TP * sizeof(R);
  }
};

template <typename R, int TP>
__device__ __forceinline__ void solve_tile_columns(const DevMesh& m, const Tile& tl,
                                                   const int* s_off, int TPX, R* s_b, R* s_W,
                                                   R* s_C, const R* s_st, const StageParams& sp,
                                                   R bdt, const R* s_x = nullptr) {
  for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
    const int a = j / tl.nt, lt = j - a * tl.nt;
    const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
    R* C = s_C + (size_t)a * 4 * TPX + base;
    // reference state of the increment form (shared memory, same layout as s_b)
    const R* x0t = s_x ? s_x + a * TPX + base : nullptr;
    const R* x0b = s_x ? s_x + (3 + a) * TPX + base : nullptr;
    column_thomas<R>(m, t, a * m.n_tri + t, N, s_st[a * TP + lt], s_W + a * TPX + base,
                     s_W + (3 + a) * TPX + base, s_b + a * TPX + base, s_b + (3 + a) * TPX + base,
                     C, C + TPX, C + 2 * TPX, C + 3 * TPX, (R)sp.kappa, (R)sp.penalty, bdt,
                     (R)sp.flux_top, (R)sp.flux_bot, x0t, x0b);
  }
}

template <typename R>
__device__ __forceinline__ void write_tile(const DevMesh& m, const Tile& tl, int TPX, int slot,
                                           const R* s_b, R* out, int* __restrict__ err) {
  const int i = threadIdx.x;
  if (i < tl.np) {
    bool ok = true;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const R x = s_b[r * TPX + slot];
      ok &= (bool)isfinite(x);
      out[(size_t)r * m.P + tl.p0 + i] = x;
    }
    if (!ok) atomicOr(err, (int)SLIM_ERRBIT_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// SSP-RK3 stage (fused): T_out solves, per vertex column,
//   (M(st_s) - beta dt A) T_out = alpha M(st_n) T_n
//                                 + beta (M(st_p) T_p + dt R_h(q(st_n), T_p)) + beta dt b
// with st_x = st_n + th_x (st_np1 - st_n) (the stretch is linear in eta) and M
// the lumped mass (J_h/12) dz [[2,1],[1,2]]/3 per vertex-layer.
// ---------------------------------------------------------------------------
template <typename R, int TP>
__global__ void __launch_bounds__(TP, (MinBlocks<R, TP>::value)) k_tracer_stage(
    DevMesh m, const R* __restrict__ U, const R* __restrict__ V, const R* Tn,
    const R* __restrict__ Tp, const R* __restrict__ Text, const R* __restrict__ W, R* Tout,
    const R* __restrict__ st_n, const R* __restrict__ st_np1, R th_p, R th_s, R alpha, R beta,
    R dt, StageParams sp, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int TPX = TP + m.max_tile_tris;
  const SolveSmem<R, TP> L(TPX);
  int* s_off = reinterpret_cast<int*>(smem);
  R* s_b = reinterpret_cast<R*>(smem + L.off_b);
  R* s_W = reinterpret_cast<R*>(smem + L.off_W);
  R* s_C = reinterpret_cast<R*>(smem + L.off_C);
  R* s_x = reinterpret_cast<R*>(smem + L.off_x);
  R* s_st = reinterpret_cast<R*>(smem + L.off_st);
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  Own<R> own;
  if (i < tl.np) load_own<R, false>(m, tl.p0 + i, U, V, Tp, own);
  const int nt = m.n_tri;
  for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
    const int a = j / tl.nt, lt = j - a * tl.nt, ia = a * nt + tl.t0 + lt;
    const R s0 = st_n[ia];
    s_st[a * TP + lt] = s0 + th_s * (st_np1[ia] - s0);
  }
  load_offsets<TP>(m, tl, s_off);
  int slot = 0;
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    const int p = tl.p0 + i;
    slot = i + lt;
    R out[2][3];
    prism_rh<R, false>(m, t, k, p, N, own, U, V, Tp, Text, st_n, out);
    const R w12 = Geo<R>::jh(m, t) * (R)(1.0 / 12.0);
    const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
    // Increment form T_out = T_p + D: the solve gets rhs - M(st_s) T_p, which with
    // alpha + beta = 1 and st_x = st_n + th_x (st_np1 - st_n) is
    //   (J_h/12) dz_rest G [alpha st_n (T_n - T_p) + (beta th_p - th_s) dst T_p]
    //   + beta dt R_h,   dst = st_np1 - st_n (an exact difference),
    // and adds beta dt A T_p itself.  The solve's own rounding then scales only the
    // increment instead of the whole state in every stage.
    const R ks = beta * th_p - th_s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      const R sn = st_n[ia];
      const R dst = st_np1[ia] - sn;
      const R dr = w12 * dz_rest_r<R>(m, ia, k, N);
      const R tn0 = Tn[(size_t)(0 * 3 + a) * m.P + p], tn1 = Tn[(size_t)(1 * 3 + a) * m.P + p];
      const R tp0 = own.T[0][a], tp1 = own.T[1][a];
      const R u0 = alpha * sn * (tn0 - tp0) + ks * dst * tp0;
      const R u1 = alpha * sn * (tn1 - tp1) + ks * dst * tp1;
      s_b[a * TPX + slot] = dr * (G2 * u0 + G1 * u1) + beta * dt * out[0][a];
      s_b[(3 + a) * TPX + slot] = dr * (G1 * u0 + G2 * u1) + beta * dt * out[1][a];
      s_x[a * TPX + slot] = tp0;
      s_x[(3 + a) * TPX + slot] = tp1;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) s_W[r * TPX + slot] = W[(size_t)r * m.P + p];
  }
  __syncthreads();
  solve_tile_columns<R, TP>(m, tl, s_off, TPX, s_b, s_W, s_C, s_st, sp, beta * dt, s_x);
  __syncthreads();
  write_tile<R>(m, tl, TPX, slot, s_b, Tout, err);
}

// standalone vertical solve: (M(st) - bdt A) x = rhs + bdt b
template <typename R, int TP>
__global__ void __launch_bounds__(TP, (MinBlocks<R, TP>::value))
    k_vertical_solve(DevMesh m, const R* __restrict__ W, const R* __restrict__ st, const R* rhs,
                     R* out, R bdt, StageParams sp, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int TPX = TP + m.max_tile_tris;
  const SolveSmem<R, TP> L(TPX);
  int* s_off = reinterpret_cast<int*>(smem);
  R* s_b = reinterpret_cast<R*>(smem + L.off_b);
  R* s_W = reinterpret_cast<R*>(smem + L.off_W);
  R* s_C = reinterpret_cast<R*>(smem + L.off_C);
  R* s_st = reinterpret_cast<R*>(smem + L.off_st);
  const Tile tl = load_tile<TP>(m, s_off);
  const int nt = m.n_tri;
  for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
    const int a = j / tl.nt, lt = j - a * tl.nt;
    s_st[a * TP + lt] = st[a * nt + tl.t0 + lt];
  }
  const int i = threadIdx.x;
  int slot = 0;
  if (i < tl.np) {
    slot = i + tile_tri_of(s_off, tl.nt, i);
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      s_b[r * TPX + slot] = rhs[(size_t)r * m.P + tl.p0 + i];
      s_W[r * TPX + slot] = W[(size_t)r * m.P + tl.p0 + i];
    }
  }
  __syncthreads();
  solve_tile_columns<R, TP>(m, tl, s_off, TPX, s_b, s_W, s_C, s_st, sp, bdt);
  __syncthreads();
  write_tile<R>(m, tl, TPX, slot, s_b, out, err);
}

// standalone horizontal residual
template <typename R, int TP>
__global__ void __launch_bounds__(TP, (MinBlocks<R, TP>::value))
    k_rhs3d(DevMesh m, const R* __restrict__ U, const R* __restrict__ V, const R* __restrict__ T,
            const R* __restrict__ Text, const R* __restrict__ st, R* __restrict__ out) {
  __shared__ int s_off[TP + 1];
  const Tile tl = tile_of_block(m);
  const int i = threadIdx.x;
  Own<R> own;
  if (i < tl.np) load_own<R, false>(m, tl.p0 + i, U, V, T, own);
  load_offsets<TP>(m, tl, s_off);
  if (i >= tl.np) return;
  const int lt = tile_tri_of(s_off, tl.nt, i);
  const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
  R o[2][3];
  prism_rh<R, false>(m, t, k, tl.p0 + i, N, own, U, V, T, Text, st, o);
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) out[(size_t)(c * 3 + a) * m.P + tl.p0 + i] = o[c][a];
}

// ---------------------------------------------------------------------------
// tracer mass sum_nodes (M T) = sum_p sum_a (J_h/12) dz_a (T_top,a + T_bot,a),
// in FP64 with a compensated pairwise (TwoSum) reduction in a fixed order:
// deterministic for a given mesh.
// ---------------------------------------------------------------------------
struct CSum {
  double s, c;
};
__device__ __forceinline__ CSum csum_add(CSum x, CSum y) {
  const double s = x.s + y.s;
  const double bp = s - x.s;
  const double err = (x.s - (s - bp)) + (y.s - bp);  // TwoSum
  return {s, x.c + y.c + err};
}

template <int TP>
__device__ __forceinline__ CSum block_csum(CSum v, double* s_s, double* s_c) {
  s_s[threadIdx.x] = v.s;
  s_c[threadIdx.x] = v.c;
  __syncthreads();
  for (int w = TP / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      CSum r = csum_add({s_s[threadIdx.x], s_c[threadIdx.x]},
                        {s_s[threadIdx.x + w], s_c[threadIdx.x + w]});
      s_s[threadIdx.x] = r.s;
      s_c[threadIdx.x] = r.c;
    }
    __syncthreads();
  }
  return {s_s[0], s_c[0]};
}

// CPL: the consistent mass of the coupled column system, whose node weights are
// sum_a K(dz/2)_ab = (J_h/48)(dz_b + sum dz) instead of the lumped (J_h/12) dz_b
template <typename R, int TP, bool CPL>
__global__ void __launch_bounds__(TP) k_mass_partial(DevMesh m, const R* __restrict__ T,
                                                     const double* __restrict__ eta,
                                                     double* __restrict__ part) {
  __shared__ int s_off[TP + 1];
  __shared__ double s_s[TP], s_c[TP];
  const Tile tl = load_tile<TP>(m, s_off);
  const int i = threadIdx.x;
  CSum v = {0.0, 0.0};
  if (i < tl.np) {
    const int lt = tile_tri_of(s_off, tl.nt, i);
    const int t = tl.t0 + lt, k = i - s_off[lt], N = s_off[lt + 1] - s_off[lt];
    const int p = tl.p0 + i, nt = m.n_tri;
    double dz[3];
    for (int a = 0; a < 3; ++a) dz[a] = dz_r<double>(m, a * nt + t, eta[a * nt + t], k, N);
    const double w12 = m.jh[t] * (1.0 / 12.0), w48 = m.jh[t] * (1.0 / 48.0);
    const double sdz = dz[0] + dz[1] + dz[2];
    for (int a = 0; a < 3; ++a) {
      const double wa = CPL ? w48 * (dz[a] + sdz) : w12 * dz[a];
      const double x = wa * ((double)T[(size_t)a * m.P + p] + (double)T[(size_t)(3 + a) * m.P + p]);
      v = csum_add(v, {x, 0.0});
    }
  }
  CSum r = block_csum<TP>(v, s_s, s_c);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r.s;
    part[2 * blockIdx.x + 1] = r.c;
  }
}

template <int TP>
__global__ void __launch_bounds__(TP) k_mass_final(const double* __restrict__ part, int n,
                                                   double* __restrict__ result) {
  __shared__ double s_s[TP], s_c[TP];
  CSum v = {0.0, 0.0};
  for (int j = threadIdx.x; j < n; j += TP) v = csum_add(v, {part[2 * j], part[2 * j + 1]});
  CSum r = block_csum<TP>(v, s_s, s_c);
  if (threadIdx.x == 0) result[0] = r.s + r.c;
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_f2d(const float* __restrict__ in, double* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define SLIM_TP_SWITCH(TP, ...)                                   \
  switch (TP) {                                                   \
    case 128: { constexpr int TPc = 128; __VA_ARGS__; } break;    \
    case 256: { constexpr int TPc = 256; __VA_ARGS__; } break;    \
    case 512: { constexpr int TPc = 512; __VA_ARGS__; } break;    \
    default: return cudaErrorInvalidValue;                        \
  }

template <typename KernelT>
static cudaError_t set_smem(KernelT kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static size_t cont_smem(const DevMesh& m, int TP, size_t esz) {
  return ((TP + 1) * sizeof(int) + 15) / 16 * 16 + 6 * (size_t)(TP + m.max_tile_tris) * esz;
}

template <typename R>
cudaError_t launch_stretch(const DevMesh& m, const double* eta, R* st, cudaStream_t stm) {
  const int n = 3 * m.n_tri;
  k_stretch<R><<<std::min((n + 255) / 256, 2048), 256, 0, stm>>>(m, eta, st);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_continuity(const DevMesh& m, int TP, const R* U, const R* V, const double* eta,
                              const R* st_cur, double* eta_out, R* st_out, R* W, double dt,
                              cudaStream_t stm) {
  SLIM_TP_SWITCH(TP, {
    const size_t sm = cont_smem(m, TPc, sizeof(R));
    cudaError_t e = set_smem(k_continuity<R, TPc, false>, sm);
    if (e != cudaSuccess) return e;
    k_continuity<R, TPc, false><<<m.n_tiles, TPc, sm, stm>>>(m, U, V, eta, st_cur, eta_out, st_out, W, dt);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_column_divergence(const DevMesh& m, int TP, const R* U, const R* V,
                                     const R* st_cur, double* out, cudaStream_t stm) {
  SLIM_TP_SWITCH(TP, {
    const size_t sm = cont_smem(m, TPc, sizeof(R));
    cudaError_t e = set_smem(k_continuity<R, TPc, true>, sm);
    if (e != cudaSuccess) return e;
    k_continuity<R, TPc, true><<<m.n_tiles, TPc, sm, stm>>>(m, U, V, nullptr, st_cur, out, nullptr, nullptr, 0.0);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_tracer_stage(const DevMesh& m, int TP, const R* U, const R* V, const R* Tn,
                                const R* Tp, const R* Text, const R* W, R* Tout, const R* st_n,
                                const R* st_np1, double th_p, double th_s, double alpha,
                                double beta, double dt, const StageParams& sp, int* err,
                                cudaStream_t stm) {
  // The weights of the convex combination in the compute type with alpha + beta = 1
  // exactly (multiples of 2^-24 in FP32, 2^-52 in FP64): weights whose sum is not one
  // scale the tracer mass by that sum in every step (1/3 and 2/3 rounded to FP32
  // sum to 1 + 3e-8).
  const double q = sizeof(R) == 4 ? 16777216.0 : 4503599627370496.0;
  const double aq = std::nearbyint(alpha * q) / q;
  const double bq = (alpha + beta == 1.0) ? 1.0 - aq : beta;
  SLIM_TP_SWITCH(TP, {
    const size_t sm = SolveSmem<R, TPc>(TPc + m.max_tile_tris).bytes;
    cudaError_t e = set_smem(k_tracer_stage<R, TPc>, sm);
    if (e != cudaSuccess) return e;
    k_tracer_stage<R, TPc><<<m.n_tiles, TPc, sm, stm>>>(m, U, V, Tn, Tp, Text, W, Tout, st_n, st_np1,
                                                        (R)th_p, (R)th_s, (R)aq, (R)bq, (R)dt,
                                                        sp, err);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_vertical_solve(const DevMesh& m, int TP, const R* W, const R* st, const R* rhs,
                                  R* out, double bdt, const StageParams& sp, int* err,
                                  cudaStream_t stm) {
  SLIM_TP_SWITCH(TP, {
    const size_t sm = SolveSmem<R, TPc>(TPc + m.max_tile_tris).bytes;
    cudaError_t e = set_smem(k_vertical_solve<R, TPc>, sm);
    if (e != cudaSuccess) return e;
    k_vertical_solve<R, TPc><<<m.n_tiles, TPc, sm, stm>>>(m, W, st, rhs, out, (R)bdt, sp, err);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rhs3d(const DevMesh& m, int TP, const R* U, const R* V, const R* T,
                         const R* Text, const R* st, R* out, cudaStream_t stm) {
  SLIM_TP_SWITCH(TP, (k_rhs3d<R, TPc><<<m.n_tiles, TPc, 0, stm>>>(m, U, V, T, Text, st, out)));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mass(const DevMesh& m, int TP, const R* T, const double* eta, double* partials,
                        double* result, cudaStream_t stm, bool consistent) {
  if (consistent)
    SLIM_TP_SWITCH(TP, (k_mass_partial<R, TPc, true><<<m.n_tiles, TPc, 0, stm>>>(m, T, eta, partials)))
  else
    SLIM_TP_SWITCH(TP, (k_mass_partial<R, TPc, false><<<m.n_tiles, TPc, 0, stm>>>(m, T, eta, partials)))
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mass_final<256><<<1, 256, 0, stm>>>(partials, m.n_tiles, result);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double* in, float* out, size_t n, cudaStream_t stm) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_d2f<<<blocks, 256, 0, stm>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_f2d(const float* in, double* out, size_t n, cudaStream_t stm) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_f2d<<<blocks, 256, 0, stm>>>(in, out, n);
  return cudaGetLastError();
}

#define SLIM_INSTANTIATE(R)                                                                         \
  template cudaError_t launch_stretch<R>(const DevMesh&, const double*, R*, cudaStream_t);          \
  template cudaError_t launch_continuity<R>(const DevMesh&, int, const R*, const R*, const double*,  \
                                            const R*, double*, R*, R*, double, cudaStream_t);        \
  template cudaError_t launch_column_divergence<R>(const DevMesh&, int, const R*, const R*,          \
                                                   const R*, double*, cudaStream_t);                 \
  template cudaError_t launch_tracer_stage<R>(const DevMesh&, int, const R*, const R*, const R*,     \
                                              const R*, const R*, const R*, R*, const R*, const R*,  \
                                              double, double, double, double, double,                \
                                              const StageParams&, int*, cudaStream_t);               \
  template cudaError_t launch_vertical_solve<R>(const DevMesh&, int, const R*, const R*, const R*,   \
                                                R*, double, const StageParams&, int*, cudaStream_t); \
  template cudaError_t launch_rhs3d<R>(const DevMesh&, int, const R*, const R*, const R*, const R*,  \
                                       const R*, R*, cudaStream_t);                                  \
  template cudaError_t launch_mass<R>(const DevMesh&, int, const R*, const double*, double*,         \
                                      double*, cudaStream_t, bool);

SLIM_INSTANTIATE(double)
SLIM_INSTANTIATE(float)

}  // namespace slim
