// Coupled (consistent-mass) column system of the tracer scheme (Sec. 2.4,
// "fully-assembled column solvers"): the consistent 2D mass M_h of Sec. 2.3
// couples the three vertices of every layer, so every prism is one 6x6 block
// row of a block-tridiagonal system per column (its top nodes couple to all six
// nodes of the prism above, its bottom nodes to all six of the prism below).
//
// Forms (the readings of the consistent column system):
//   mass       G (x) K(hz),  K(w)_ab = J_h sum_e I_abe w_e, I the exact moments
//              int phi_a phi_b phi_e / J_h (1/20, 1/60, 1/120), hz = dz/2
//   continuity (D_vd (x) M_h) Omega = R_h(q,1) - d/dt (M 1), the printed D_vd
//              pattern of Eq. 17 with M_h blocks, and M_h (eta' - eta)/dt = the
//              column sum of R_h(q,1) (consistent 2D mass)
//   advection  volume dpsi_c K(sum_f G_fd Omega_f)_ae; interface flux taken at
//              the vertices (Omega of the element below, upwind value by the
//              vertex's sign) and integrated as a P1 function: M_h F
//   diffusion  SIPG whose 1/z_zeta and penalty are integrated with the 6-point
//              degree-4 triangle rule (exact in zeta)
// The horizontal residual is the lumped path's (prism_rh: exact, consistent).
//
// Kernels (one thread block per tile of whole columns, as the 2x2-block path):
//   phase 1  thread per prism: horizontal residual and right-hand side into
//            shared memory (coalesced node planes)
//   phase 2  the column's 6x6 blocks are assembled layer by layer and
//            eliminated at once (block Thomas: a 6x6 Gauss-Jordan per layer on
//            [D' | U | b], the 36-value factor C_k kept in shared memory for the
//            back substitution); FP32: one thread per column, FP64: eight lanes
//            per column, one block row each, with shuffles (no register spills)
//   phase 3  thread per prism: coalesced write-back.
#include <algorithm>
#include <cmath>

#include "slim_device.cuh"
#include "slim_kernels.h"

namespace slim {
namespace {

// 6-point degree-4 triangle rule (Strang and Fix; Dunavant 1985): orbits
// (a, a, 1 - 2a), (b, b, 1 - 2b) with a, b = (8 - sqrt(10) +- sqrt(38 - 44 sqrt(2/5)))/18
// and weights (620 +- sqrt(213125 - 53320 sqrt(10)))/3720 (summing to 1 over the six).
__device__ __forceinline__ void rule4_point(int q, double& l0, double& l1, double& l2, double& w) {
  const double a = 0.44594849091596483, b = 0.09157621350977073;
  const double wa = 0.22338158967801144, wb = 0.10995174365532187;
  const double x = q < 3 ? a : b, y = q < 3 ? 1.0 - 2.0 * a : 1.0 - 2.0 * b;
  w = q < 3 ? wa : wb;
  const int r = q % 3;
  l0 = r == 0 ? y : x;
  l1 = r == 1 ? y : x;
  l2 = r == 2 ? y : x;
}

// K(w)_ab for vertex values w (symmetric 3x3)
template <typename R>
__device__ __forceinline__ void kmat(R jh, const R w[3], R K[3][3]) {
  const R S = w[0] + w[1] + w[2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      K[a][b] = (a == b) ? jh * (w[a] * (R)(1.0 / 30.0) + S * (R)(1.0 / 60.0))
                         : jh * (w[a] + w[b] + S) * (R)(1.0 / 120.0);
}

// (K(w) x)_a = (J_h/120)(2 w_a x_a + S x_a + w_a X + S X + P), S = sum w, X = sum x,
// P = sum w_b x_b
template <typename R>
__device__ __forceinline__ void kapply(R jh, const R w[3], const R x[3], R o[3]) {
  const R S = w[0] + w[1] + w[2], X = x[0] + x[1] + x[2];
  const R P = w[0] * x[0] + w[1] * x[1] + w[2] * x[2];
  const R f = jh * (R)(1.0 / 120.0);
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = f * ((R)2 * w[a] * x[a] + S * x[a] + w[a] * X + S * X + P);
}

// reciprocal of the P1 function with vertex values dz at the rule's six points
template <typename R>
__device__ __forceinline__ void recip_at_points(const R dz[3], R r[6]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double l0, l1, l2, w;
    rule4_point(q, l0, l1, l2, w);
    r[q] = rcp<R>((R)l0 * dz[0] + (R)l1 * dz[1] + (R)l2 * dz[2]);
  }
}

// Q(f)_ab = int phi_a phi_b f dA by the rule, f given at its points
template <typename R>
__device__ __forceinline__ void qmat(R jh, const R f[6], R Q[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Q[a][b] = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double l0, l1, l2, w;
    rule4_point(q, l0, l1, l2, w);
    const R lam[3] = {(R)l0, (R)l1, (R)l2};
    const R s = (R)0.5 * jh * (R)w * f[q];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Q[a][b] += s * lam[a] * lam[b];
  }
}

// M_h^-1 x = (6/J_h)(4 x - sum x)
template <typename R>
__device__ __forceinline__ void mh_inv(R ijh6, const R x[3], R o[3]) {
  const R s = x[0] + x[1] + x[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = ijh6 * ((R)4 * x[a] - s);
}

// ---------------------------------------------------------------------------
// continuity: eta' (FP64, consistent 2D mass) and the nodal vertical flux Omega
// ---------------------------------------------------------------------------
template <typename R, int TP>
__global__ void __launch_bounds__(TP) k_continuity_cpl(DevMesh m, const R* __restrict__ U,
                                                       const R* __restrict__ V,
                                                       const double* __restrict__ eta,
                                                       const R* __restrict__ st_cur,
                                                       double* __restrict__ eta_out,
                                                       R* __restrict__ st_out, R* __restrict__ W,
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
  for (int lt = threadIdx.x; lt < tl.nt; lt += TP) {
    const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
    // column divergence per vertex (FP64 accuracy), consistent 2D elevation update
    double D[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ColSum<R> cs;
      const R* Ft = s_F + a * TPX + base;
      const R* Fb = s_F + (3 + a) * TPX + base;
      for (int k = 0; k < N; ++k) cs.add(Ft[k] + Fb[k]);
      D[a] = cs.value();
    }
    const double jh = m.jh[t];
    const double sD = D[0] + D[1] + D[2];
    R dm[3];  // (eta' - eta)/(2 h dt) per vertex: the rate of hz per unit rest thickness
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      const double e0 = eta[ia];
      const double e1 = e0 + dt * (6.0 / jh) * (4.0 * D[a] - sD);
      eta_out[ia] = e1;
      st_out[ia] = (R)(1.0 + e1 * m.ih[ia]);
      dm[a] = (R)(0.5 * (e1 - e0) * m.ih[ia] / dt);
    }
    // per layer: f = M_h^-1 F - dhz/dt, then the bottom-up D_vd recursion per vertex
    const R ijh6 = (R)6 * rcp<R>(Geo<R>::jh(m, t));
    R s[3] = {0, 0, 0};
    for (int k = N - 1; k >= 0; --k) {
      R ft[3], fb[3], gt[3], gb[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ft[a] = s_F[a * TPX + base + k];
        fb[a] = s_F[(3 + a) * TPX + base + k];
      }
      mh_inv<R>(ijh6, ft, gt);
      mh_inv<R>(ijh6, fb, gb);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R r = dm[a] * dz_rest_r<R>(m, a * nt + t, k, N);
        const R t_ = gt[a] - r, b_ = gb[a] - r;
        const R wt = t_ + b_ + s[a];
        s_F[(3 + a) * TPX + base + k] = b_ - t_ + s[a];
        s_F[a * TPX + base + k] = wt;
        s[a] = wt;
      }
    }
  }
  __syncthreads();
  if (i < tl.np) {
#pragma unroll
    for (int r = 0; r < 6; ++r) W[(size_t)r * m.P + tl.p0 + i] = s_F[r * TPX + slot];
  }
}

// ---------------------------------------------------------------------------
// one column: (M(st) - bdt A) x = b (+ bdt Neumann), block Thomas with 6x6 blocks
// ---------------------------------------------------------------------------
// Shared-memory arrays of the tile, node row r = c*3 + a, slot base + k:
//   sb [6] right-hand side in, solution out;  sW [6] Omega;  sx [6] reference state
//   of the increment form (or null);  sC [36] the factors C_k = D'^-1 U_k.
template <typename R>
__device__ void column_solve6(const DevMesh& m, int t, int N, int base, int TPX, const R st[3],
                              R* __restrict__ sb, const R* __restrict__ sW,
                              const R* __restrict__ sx, R* __restrict__ sC, R kap, R pen, R bdt,
                              R flux_top, R flux_bot) {
  const int nt = m.n_tri;
  const R jh = Geo<R>::jh(m, t);
  const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
  R Mh[3][3];
  {
    const R one[3] = {1, 1, 1};
    kmat<R>(jh, one, Mh);
  }
  // thickness of layer k at the three vertices
  auto layer_dz = [&](int k, R dz[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) dz[a] = dz_rest_r<R>(m, a * nt + t, k, N) * st[a];
  };
  R dz_c[3], rq_c[6], rq_p[6], rq_n[6];
  layer_dz(0, dz_c);
  recip_at_points<R>(dz_c, rq_c);
#pragma unroll
  for (int q = 0; q < 6; ++q) rq_p[q] = rq_c[q];
  R yprev[6] = {0, 0, 0, 0, 0, 0};
  for (int k = 0; k < N; ++k) {
    R dz_n[3] = {dz_c[0], dz_c[1], dz_c[2]};
    if (k + 1 < N) {
      layer_dz(k + 1, dz_n);
      recip_at_points<R>(dz_n, rq_n);
    }
    // operator blocks of K = M - bdt A: D (layer k), L (layer k-1), U (layer k+1)
    R D[6][6], L[6][6], Ub[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) { D[r][c] = 0; L[r][c] = 0; Ub[r][c] = 0; }
    // advection, volume: A[(c,a),(d,e)] += dpsi_c K(sum_f G_fd Omega_f)_ae
    R Om_t[3], Om_b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Om_t[a] = sW[a * TPX + base + k];
      Om_b[a] = sW[(3 + a) * TPX + base + k];
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      R w[3], Kw[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) w[a] = d == 0 ? G2 * Om_t[a] + G1 * Om_b[a] : G1 * Om_t[a] + G2 * Om_b[a];
      kmat<R>(jh, w, Kw);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          D[a][d * 3 + e] += (R)0.5 * Kw[a][e];        // dpsi_top = 1/2
          D[3 + a][d * 3 + e] -= (R)0.5 * Kw[a][e];    // dpsi_bot = -1/2
        }
    }
    // advection, top interface (Omega of this layer's top node; surface: own value)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R Wb = Om_t[b];
      const bool own = (k == 0) || (Wb > (R)0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R cf = Mh[a][b] * Wb;
        if (own) D[a][b] -= cf; else L[a][3 + b] -= cf;
      }
    }
    // advection, bottom interface (Omega of the top node of the layer below; bed: 0)
    if (k + 1 < N) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R Wb = sW[b * TPX + base + k + 1];
        const bool below = Wb > (R)0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const R cf = Mh[a][b] * Wb;
          if (below) Ub[3 + a][b] += cf; else D[3 + a][3 + b] += cf;
        }
      }
    }
    // diffusion, element stiffness: -kappa 2 dpsi_c dpsi_d int phi_a phi_b / z_zeta
    R Qc[3][3];
    qmat<R>(jh, rq_c, Qc);   // int phi_a phi_b / dz_k
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R s = kap * Qc[a][b];      // kappa (1/2) int phi phi / hz = kappa int phi phi / dz
        D[a][b] -= s; D[3 + a][3 + b] -= s;
        D[a][3 + b] += s; D[3 + a][b] += s;
      }
    // diffusion, interface above (layer k - 1 above, this layer below)
    if (k > 0) {
      R Qa[3][3], Qs[3][3], sg[6];
      qmat<R>(jh, rq_p, Qa);
#pragma unroll
      for (int q = 0; q < 6; ++q) sg[q] = pen * kap * fmax(rq_p[q], rq_c[q]);
      qmat<R>(jh, sg, Qs);
      const R h = (R)0.5 * kap;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          // -{kappa dT/dz}[v], row (k, top, a), [v] = +1
          L[a][b] += h * Qa[a][b];
          L[a][3 + b] -= h * Qa[a][b];
          D[a][b] += h * Qc[a][b];
          D[a][3 + b] -= h * Qc[a][b];
          // + sigma [T][v]
          D[a][b] -= Qs[a][b];
          L[a][3 + b] += Qs[a][b];
          // -{kappa dv/dz}[T] for this layer's test functions (top +, bottom -)
          const R dt_ = h * Qc[a][b];
          D[a][b] += dt_;  L[a][3 + b] -= dt_;
          D[3 + a][b] -= dt_;  L[3 + a][3 + b] += dt_;
        }
    }
    // diffusion, interface below (this layer above, layer k + 1 below)
    if (k + 1 < N) {
      R Qb[3][3], Qs[3][3], sg[6];
      qmat<R>(jh, rq_n, Qb);
#pragma unroll
      for (int q = 0; q < 6; ++q) sg[q] = pen * kap * fmax(rq_c[q], rq_n[q]);
      qmat<R>(jh, sg, Qs);
      const R h = (R)0.5 * kap;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          // -{kappa dT/dz}[v], row (k, bottom, a), [v] = -1
          D[3 + a][b] -= h * Qc[a][b];
          D[3 + a][3 + b] += h * Qc[a][b];
          Ub[3 + a][b] -= h * Qb[a][b];
          Ub[3 + a][3 + b] += h * Qb[a][b];
          // + sigma [T][v]
          Ub[3 + a][b] += Qs[a][b];
          D[3 + a][3 + b] -= Qs[a][b];
          // -{kappa dv/dz}[T] for this layer's test functions
          const R dt_ = h * Qc[a][b];
          Ub[a][b] += dt_;  D[a][3 + b] -= dt_;
          Ub[3 + a][b] -= dt_;  D[3 + a][3 + b] += dt_;
        }
    }
    // right-hand side; increment form: + bdt A x0 over the three layers
    R rhs[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) rhs[r] = sb[r * TPX + base + k];
    if (sx) {
      R x0[6], xm[6], xp[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        x0[r] = sx[r * TPX + base + k];
        xm[r] = k > 0 ? sx[r * TPX + base + k - 1] : (R)0;
        xp[r] = k + 1 < N ? sx[r * TPX + base + k + 1] : (R)0;
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        R acc = 0;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc += D[r][c] * x0[c] + L[r][c] * xm[c] + Ub[r][c] * xp[c];
        rhs[r] += bdt * acc;
      }
    }
    if (k == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) rhs[a] += bdt * jh * (R)(1.0 / 6.0) * flux_top;
    }
    if (k == N - 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) rhs[3 + a] -= bdt * jh * (R)(1.0 / 6.0) * flux_bot;
    }
    // K = M - bdt A
    {
      R hz[3], Km[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) hz[a] = (R)0.5 * dz_c[a];
      kmat<R>(jh, hz, Km);
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const R g = (r < 3) == (c < 3) ? G2 : G1;
          D[r][c] = g * Km[r % 3][c % 3] - bdt * D[r][c];
          L[r][c] = -bdt * L[r][c];
          Ub[r][c] = -bdt * Ub[r][c];
        }
    }
    // D' = D - L C_{k-1},  b' = b - L y_{k-1}
    if (k > 0) {
      const R* Cp = sC + base + k - 1;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          R acc = 0;
#pragma unroll
          for (int j = 0; j < 6; ++j) acc += L[r][j] * Cp[(j * 6 + c) * TPX];
          D[r][c] -= acc;
        }
        R acc = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += L[r][j] * yprev[j];
        rhs[r] -= acc;
      }
    }
    // Gauss-Jordan on [D' | U | b'] (no pivoting: D' is the mass-dominated Schur
    // complement of a block-diagonally dominant column)
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const R ip = rcp<R>(D[p][p]);
#pragma unroll
      for (int c = 0; c < 6; ++c) { D[p][c] *= ip; Ub[p][c] *= ip; }
      rhs[p] *= ip;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        if (r == p) continue;
        const R f = D[r][p];
#pragma unroll
        for (int c = 0; c < 6; ++c) { D[r][c] -= f * D[p][c]; Ub[r][c] -= f * Ub[p][c]; }
        rhs[r] -= f * rhs[p];
      }
    }
    R* Ck = sC + base + k;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
#pragma unroll
      for (int c = 0; c < 6; ++c) Ck[(r * 6 + c) * TPX] = Ub[r][c];
      sb[r * TPX + base + k] = rhs[r];
      yprev[r] = rhs[r];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dz_c[a] = dz_n[a];
#pragma unroll
    for (int q = 0; q < 6; ++q) { rq_p[q] = rq_c[q]; rq_c[q] = rq_n[q]; }
  }
  // back substitution x_k = y_k - C_k x_{k+1}; increment form adds x0
  R xn[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) xn[r] = yprev[r];
  for (int k = N - 2; k >= 0; --k) {
    const R* Ck = sC + base + k;
    R x[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      R acc = 0;
#pragma unroll
      for (int c = 0; c < 6; ++c) acc += Ck[(r * 6 + c) * TPX] * xn[c];
      x[r] = sb[r * TPX + base + k] - acc;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      sb[r * TPX + base + k] = x[r];
      xn[r] = x[r];
    }
  }
  if (sx) {
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int r = 0; r < 6; ++r) sb[r * TPX + base + k] += sx[r * TPX + base + k];
  }
}

// ---------------------------------------------------------------------------
// The same column solve by eight lanes of a warp per column (four columns per
// warp): lane r < 6 owns block row r = (c, a) of every layer, assembles its row of
// D_k, L_k, U_k and the right-hand side, and the block-Thomas elimination runs row-
// parallel: the factor C_{k-1} and y_{k-1} of the layer above come from the other
// lanes by shuffles, the Gauss-Jordan pivot rows are broadcast by shuffles, and
// C_k is kept in shared memory for the back substitution.  Lanes 6 and 7 of a
// group and groups past the tile's last column follow the shuffles without
// touching memory.  The layer loop runs to the warp's deepest column, so every
// shuffle is executed by all 32 lanes.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R shfl(R v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

template <typename R>
__device__ void column_solve6_warp(const DevMesh& m, const Tile& tl, const int* s_off, int TPX,
                                   const R* st_tile, int TPst, R* __restrict__ sb,
                                   const R* __restrict__ sW, const R* __restrict__ sx,
                                   R* __restrict__ sC, R kap, R pen, R bdt, R flux_top, R flux_bot,
                                   int col_begin) {
  const int lane = threadIdx.x & 31, r = lane & 7, gbase = lane & ~7;
  const int col = col_begin + (lane >> 3);
  const bool active = col < tl.nt;
  const int nt = m.n_tri;
  int t = tl.t0, base = 0, N = 0;
  if (active) {
    t = tl.t0 + col;
    base = s_off[col] + col;
    N = s_off[col + 1] - s_off[col];
  }
  int Nmax = N;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Nmax = max(Nmax, __shfl_xor_sync(0xffffffffu, Nmax, o));
  const bool row_on = active && r < 6;
  const int c = (r % 6) / 3, a = r % 3;   // block row (node level, vertex); rows 6, 7 mirror 0, 1
  const R jh = Geo<R>::jh(m, t);
  const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
  const R dps = c == 0 ? (R)0.5 : (R)-0.5;
  R st[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) st[e] = active ? st_tile[e * TPst + col] : (R)1;
  auto layer_dz = [&](int k, R dz[3]) {
#pragma unroll
    for (int e = 0; e < 3; ++e) dz[e] = (k < N) ? dz_rest_r<R>(m, e * nt + t, k, N) * st[e] : (R)1;
  };
  // row a of M_h
  R Mh[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) Mh[b] = jh * (a == b ? (R)(2.0 / 24.0) : (R)(1.0 / 24.0));
  // row a of Q(f) for the rule's point values f
  auto qrow = [&](const R f[6], R out[3]) {
#pragma unroll
    for (int b = 0; b < 3; ++b) out[b] = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double l0, l1, l2, w;
      rule4_point(q, l0, l1, l2, w);
      const R lam[3] = {(R)l0, (R)l1, (R)l2};
      const R sf = (R)0.5 * jh * (R)w * f[q] * lam[a];
#pragma unroll
      for (int b = 0; b < 3; ++b) out[b] += sf * lam[b];
    }
  };
  // row a of K(w)
  auto krow = [&](const R w[3], R out[3]) {
    const R S = w[0] + w[1] + w[2];
#pragma unroll
    for (int b = 0; b < 3; ++b)
      out[b] = (a == b) ? jh * (w[a] * (R)(1.0 / 30.0) + S * (R)(1.0 / 60.0))
                        : jh * (w[a] + w[b] + S) * (R)(1.0 / 120.0);
  };
  R dz_c[3], rq_c[6], rq_p[6], rq_n[6];
  layer_dz(0, dz_c);
  recip_at_points<R>(dz_c, rq_c);
#pragma unroll
  for (int q = 0; q < 6; ++q) rq_p[q] = rq_c[q];
  R Cprev[6] = {0, 0, 0, 0, 0, 0}, yprev = 0;
  for (int k = 0; k < Nmax; ++k) {
    const bool on = k < N;          // this group's column has layer k
    const int ks = on ? k : 0;      // a safe layer index for the loads
    R dz_n[3] = {dz_c[0], dz_c[1], dz_c[2]};
    if (k + 1 < N) {
      layer_dz(k + 1, dz_n);
      recip_at_points<R>(dz_n, rq_n);
    }
    R D[6], L[6], U[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) { D[j] = 0; L[j] = 0; U[j] = 0; }
    R Om_t[3], Om_b[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      Om_t[e] = active ? sW[e * TPX + base + ks] : (R)0;
      Om_b[e] = active ? sW[(3 + e) * TPX + base + ks] : (R)0;
    }
    // advection, volume
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      R w[3], Kw[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) w[e] = d == 0 ? G2 * Om_t[e] + G1 * Om_b[e] : G1 * Om_t[e] + G2 * Om_b[e];
      krow(w, Kw);
#pragma unroll
      for (int e = 0; e < 3; ++e) D[d * 3 + e] += dps * Kw[e];
    }
    // advection, top interface (rows of the top nodes)
    if (c == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R Wb = Om_t[b];
        const R cf = Mh[b] * Wb;
        if (k == 0 || Wb > (R)0) D[b] -= cf; else L[3 + b] -= cf;
      }
    }
    // advection, bottom interface (rows of the bottom nodes)
    if (c == 1 && k + 1 < N) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R Wb = sW[b * TPX + base + k + 1];
        const R cf = Mh[b] * Wb;
        if (Wb > (R)0) U[b] += cf; else D[3 + b] += cf;
      }
    }
    // diffusion, element
    R Qc[3];
    qrow(rq_c, Qc);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R sq = kap * Qc[b];
      D[c * 3 + b] -= sq;
      D[(1 - c) * 3 + b] += sq;
    }
    const R h = (R)0.5 * kap;
    if (k > 0) {  // interface above
      R Qa[3], Qs[3], sg[6];
      qrow(rq_p, Qa);
#pragma unroll
      for (int q = 0; q < 6; ++q) sg[q] = pen * kap * fmax(rq_p[q], rq_c[q]);
      qrow(sg, Qs);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (c == 0) {
          L[b] += h * Qa[b];
          L[3 + b] -= h * Qa[b];
          D[b] += h * Qc[b];
          D[3 + b] -= h * Qc[b];
          D[b] -= Qs[b];
          L[3 + b] += Qs[b];
          D[b] += h * Qc[b];
          L[3 + b] -= h * Qc[b];
        } else {
          D[b] -= h * Qc[b];
          L[3 + b] += h * Qc[b];
        }
      }
    }
    if (k + 1 < N) {  // interface below
      R Qb[3], Qs[3], sg[6];
      qrow(rq_n, Qb);
#pragma unroll
      for (int q = 0; q < 6; ++q) sg[q] = pen * kap * fmax(rq_c[q], rq_n[q]);
      qrow(sg, Qs);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (c == 1) {
          D[b] -= h * Qc[b];
          D[3 + b] += h * Qc[b];
          U[b] -= h * Qb[b];
          U[3 + b] += h * Qb[b];
          U[b] += Qs[b];
          D[3 + b] -= Qs[b];
          U[b] -= h * Qc[b];
          D[3 + b] += h * Qc[b];
        } else {
          U[b] += h * Qc[b];
          D[3 + b] -= h * Qc[b];
        }
      }
    }
    // right-hand side of this row (+ bdt A x0 in the increment form)
    R rhs = row_on && on ? sb[r * TPX + base + k] : (R)0;
    if (sx && active && on) {
      R acc = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        acc += D[j] * sx[j * TPX + base + k];
        if (k > 0) acc += L[j] * sx[j * TPX + base + k - 1];
        if (k + 1 < N) acc += U[j] * sx[j * TPX + base + k + 1];
      }
      rhs += bdt * acc;
    }
    if (k == 0 && c == 0) rhs += bdt * jh * (R)(1.0 / 6.0) * flux_top;
    if (k == N - 1 && c == 1) rhs -= bdt * jh * (R)(1.0 / 6.0) * flux_bot;
    // K = M - bdt A (row of M: G_cd K(hz)_ab)
    {
      R hz[3], Km[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) hz[e] = (R)0.5 * dz_c[e];
      krow(hz, Km);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const R g = (j / 3 == c) ? G2 : G1;
        D[j] = g * Km[j % 3] - bdt * D[j];
        L[j] = -bdt * L[j];
        U[j] = -bdt * U[j];
      }
    }
    // D' = D - L C_{k-1},  b' = b - L y_{k-1}  (rows of C_{k-1} and y_{k-1} from the group's lanes)
#pragma unroll
    for (int mr = 0; mr < 6; ++mr) {
      const R yl = shfl<R>(yprev, gbase + mr);
      rhs -= L[mr] * yl;
#pragma unroll
      for (int j = 0; j < 6; ++j) D[j] -= L[mr] * shfl<R>(Cprev[j], gbase + mr);
    }
    // Gauss-Jordan on [D' | U | b'] across the six rows (no pivoting, as the serial form)
#pragma unroll
    for (int pv = 0; pv < 6; ++pv) {
      const R dpp = shfl<R>(D[pv], gbase + pv);
      const R ip = rcp<R>(dpp);
      if (r == pv) {
#pragma unroll
        for (int j = 0; j < 6; ++j) { D[j] *= ip; U[j] *= ip; }
        rhs *= ip;
      }
      R Dp[6], Up[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        Dp[j] = shfl<R>(D[j], gbase + pv);
        Up[j] = shfl<R>(U[j], gbase + pv);
      }
      const R rp = shfl<R>(rhs, gbase + pv);
      if (r != pv) {
        const R f = D[pv];
#pragma unroll
        for (int j = 0; j < 6; ++j) { D[j] -= f * Dp[j]; U[j] -= f * Up[j]; }
        rhs -= f * rp;
      }
    }
    if (row_on && on) {
#pragma unroll
      for (int j = 0; j < 6; ++j) sC[(r * 6 + j) * TPX + base + k] = U[j];
      sb[r * TPX + base + k] = rhs;
    }
    if (on) {  // past its last layer a group keeps that layer's factor and y
#pragma unroll
      for (int j = 0; j < 6; ++j) Cprev[j] = U[j];
      yprev = rhs;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) dz_c[e] = dz_n[e];
#pragma unroll
    for (int q = 0; q < 6; ++q) { rq_p[q] = rq_c[q]; rq_c[q] = rq_n[q]; }
  }
  // back substitution x_k = y_k - C_k x_{k+1}, from the last layer of each column up
  R xn = yprev;   // x of the layer below (each group starts at its own last layer)
  for (int k = Nmax - 2; k >= 0; --k) {
    const bool on = k + 1 < N;     // layer k exists and is not the column's last
    R acc = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const R xj = shfl<R>(xn, gbase + j);
      if (row_on && on) acc += sC[(r * 6 + j) * TPX + base + k] * xj;
    }
    if (row_on && on) {
      const R x = sb[r * TPX + base + k] - acc;
      sb[r * TPX + base + k] = x;
      xn = x;
    }
  }
  __syncwarp();
  if (sx && row_on) {
    for (int k = 0; k < N; ++k) sb[r * TPX + base + k] += sx[r * TPX + base + k];
  }
}

// shared memory: offsets | sb [6] | sW [6] | sx [6] | sC [36] (x TPX) | st [3][TP]
template <typename R>
struct CplSmem {
  size_t off_b, off_W, off_x, off_C, off_st, bytes;
  __host__ __device__ CplSmem(int TP, int TPX) {
    off_b = ((TP + 1) * sizeof(int) + 15) / 16 * 16;
    off_W = off_b + 6 * (size_t)TPX * sizeof(R);
    off_x = off_W + 6 * (size_t)TPX * sizeof(R);
    off_C = off_x + 6 * (size_t)TPX * sizeof(R);
    off_st = off_C + 36 * (size_t)TPX * sizeof(R);
    bytes = off_st + 3 * (size_t)TP * sizeof(R);
  }
};

template <typename R>
__device__ __forceinline__ void write_tile6(const DevMesh& m, const Tile& tl, int TPX, int slot,
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
// SSP-RK3 stage with the coupled column solve:
//   (M(st_s) - beta dt A) T_out = alpha M(st_n) T_n
//                                 + beta (M(st_p) T_p + dt R_h(q(st_n), T_p)) + beta dt b
// in increment form T_out = T_p + D (the right-hand side rhs - M(st_s) T_p is
// alpha M_n (T_n - T_p) + (beta th_p - th_s) dM T_p + beta dt R_h: the mass is
// linear in the stretch, dM = G (x) K((dz_rest/2)(st_np1 - st_n))).
// ---------------------------------------------------------------------------
template <typename R, int TP>
__global__ void __launch_bounds__(TP) k_tracer_stage_cpl(
    DevMesh m, const R* __restrict__ U, const R* __restrict__ V, const R* Tn,
    const R* __restrict__ Tp, const R* __restrict__ Text, const R* __restrict__ W, R* Tout,
    const R* __restrict__ st_n, const R* __restrict__ st_np1, R th_p, R th_s, R alpha, R beta,
    R dt, StageParams sp, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int TPX = TP + m.max_tile_tris;
  const CplSmem<R> L(TP, TPX);
  int* s_off = reinterpret_cast<int*>(smem);
  R* s_b = reinterpret_cast<R*>(smem + L.off_b);
  R* s_W = reinterpret_cast<R*>(smem + L.off_W);
  R* s_x = reinterpret_cast<R*>(smem + L.off_x);
  R* s_C = reinterpret_cast<R*>(smem + L.off_C);
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
    const R jh = Geo<R>::jh(m, t);
    const R ks = beta * th_p - th_s;
    R wn[3], wd[3], dn[2][3], tp[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ia = a * nt + t;
      const R hr = (R)0.5 * dz_rest_r<R>(m, ia, k, N);
      const R sn = st_n[ia];
      wn[a] = hr * sn;
      wd[a] = hr * (st_np1[ia] - sn);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        tp[c][a] = own.T[c][a];
        dn[c][a] = Tn[(size_t)(c * 3 + a) * m.P + p] - tp[c][a];
      }
    }
    R y[2][3];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      R k1[3], k2[3];
      kapply<R>(jh, wn, dn[c], k1);
      kapply<R>(jh, wd, tp[c], k2);
#pragma unroll
      for (int a = 0; a < 3; ++a) y[c][a] = alpha * k1[a] + ks * k2[a];
    }
    const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_b[a * TPX + slot] = G2 * y[0][a] + G1 * y[1][a] + beta * dt * out[0][a];
      s_b[(3 + a) * TPX + slot] = G1 * y[0][a] + G2 * y[1][a] + beta * dt * out[1][a];
      s_x[a * TPX + slot] = tp[0][a];
      s_x[(3 + a) * TPX + slot] = tp[1][a];
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) s_W[r * TPX + slot] = W[(size_t)r * m.P + p];
  }
  __syncthreads();
  if (sizeof(R) == 8) {
    // FP64: eight lanes per column, four columns per warp (the thread-per-column
    // elimination spills its FP64 blocks)
    for (int c0 = (threadIdx.x >> 5) * 4; c0 < tl.nt; c0 += (TP / 32) * 4)
      column_solve6_warp<R>(m, tl, s_off, TPX, s_st, TP, s_b, s_W, s_x, s_C, (R)sp.kappa, (R)sp.penalty,
                            beta * dt, (R)sp.flux_top, (R)sp.flux_bot, c0);
  } else {
    // FP32: one thread per column holds the blocks in registers (shorter dependence chain)
    for (int lt = threadIdx.x; lt < tl.nt; lt += TP) {
      const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
      const R st[3] = {s_st[lt], s_st[TP + lt], s_st[2 * TP + lt]};
      column_solve6<R>(m, t, N, base, TPX, st, s_b, s_W, s_x, s_C, (R)sp.kappa, (R)sp.penalty, beta * dt,
                       (R)sp.flux_top, (R)sp.flux_bot);
    }
  }
  __syncthreads();
  write_tile6<R>(m, tl, TPX, slot, s_b, Tout, err);
}

// standalone coupled vertical solve: (M(st) - bdt A) x = rhs + bdt b
template <typename R, int TP>
__global__ void __launch_bounds__(TP) k_vertical_solve_cpl(DevMesh m, const R* __restrict__ W,
                                                           const R* __restrict__ st, const R* rhs,
                                                           R* out, R bdt, StageParams sp,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int TPX = TP + m.max_tile_tris;
  const CplSmem<R> L(TP, TPX);
  int* s_off = reinterpret_cast<int*>(smem);
  R* s_b = reinterpret_cast<R*>(smem + L.off_b);
  R* s_W = reinterpret_cast<R*>(smem + L.off_W);
  R* s_C = reinterpret_cast<R*>(smem + L.off_C);
  const Tile tl = load_tile<TP>(m, s_off);
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
  const int nt = m.n_tri;
  R* s_st = reinterpret_cast<R*>(smem + L.off_st);
  for (int j = threadIdx.x; j < 3 * tl.nt; j += TP) {
    const int a = j / tl.nt, lt = j - a * tl.nt;
    s_st[a * TP + lt] = st[a * nt + tl.t0 + lt];
  }
  __syncthreads();
  if (sizeof(R) == 8) {
    for (int c0 = (threadIdx.x >> 5) * 4; c0 < tl.nt; c0 += (TP / 32) * 4)
      column_solve6_warp<R>(m, tl, s_off, TPX, s_st, TP, s_b, s_W, nullptr, s_C, (R)sp.kappa, (R)sp.penalty,
                            bdt, (R)sp.flux_top, (R)sp.flux_bot, c0);
  } else {
    for (int lt = threadIdx.x; lt < tl.nt; lt += TP) {
      const int t = tl.t0 + lt, base = s_off[lt] + lt, N = s_off[lt + 1] - s_off[lt];
      const R stv[3] = {s_st[lt], s_st[TP + lt], s_st[2 * TP + lt]};
      column_solve6<R>(m, t, N, base, TPX, stv, s_b, s_W, nullptr, s_C, (R)sp.kappa, (R)sp.penalty, bdt,
                       (R)sp.flux_top, (R)sp.flux_bot);
    }
  }
  __syncthreads();
  write_tile6<R>(m, tl, TPX, slot, s_b, out, err);
}

template <typename KernelT>
cudaError_t set_smem_cpl(KernelT kern, size_t bytes) {
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define SLIM_TP_SWITCH_CPL(TP, ...)                               \
  switch (TP) {                                                   \
    case 128: { constexpr int TPc = 128; __VA_ARGS__; } break;    \
    case 256: { constexpr int TPc = 256; __VA_ARGS__; } break;    \
    case 512: { constexpr int TPc = 512; __VA_ARGS__; } break;    \
    default: return cudaErrorInvalidValue;                        \
  }

}  // namespace

size_t coupled_smem_bytes(const DevMesh& m, int TP, size_t esz) {
  const size_t TPX = TP + m.max_tile_tris;
  return ((TP + 1) * sizeof(int) + 15) / 16 * 16 + (6 + 6 + 6 + 36) * TPX * esz + 3 * (size_t)TP * esz;
}

template <typename R>
cudaError_t launch_continuity_cpl(const DevMesh& m, int TP, const R* U, const R* V, const double* eta,
                                  const R* st_cur, double* eta_out, R* st_out, R* W, double dt,
                                  cudaStream_t stm) {
  SLIM_TP_SWITCH_CPL(TP, {
    const size_t sm = ((TPc + 1) * sizeof(int) + 15) / 16 * 16 + 6 * (size_t)(TPc + m.max_tile_tris) * sizeof(R);
    cudaError_t e = set_smem_cpl(k_continuity_cpl<R, TPc>, sm);
    if (e != cudaSuccess) return e;
    k_continuity_cpl<R, TPc><<<m.n_tiles, TPc, sm, stm>>>(m, U, V, eta, st_cur, eta_out, st_out, W, dt);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_tracer_stage_cpl(const DevMesh& m, int TP, const R* U, const R* V, const R* Tn,
                                    const R* Tp, const R* Text, const R* W, R* Tout, const R* st_n,
                                    const R* st_np1, double th_p, double th_s, double alpha,
                                    double beta, double dt, const StageParams& sp, int* err,
                                    cudaStream_t stm) {
  // stage weights with alpha + beta = 1 exactly in the compute type (see the lumped stage)
  const double q = sizeof(R) == 4 ? 16777216.0 : 4503599627370496.0;
  const double aq = std::nearbyint(alpha * q) / q;
  const double bq = (alpha + beta == 1.0) ? 1.0 - aq : beta;
  SLIM_TP_SWITCH_CPL(TP, {
    const size_t sm = CplSmem<R>(TPc, TPc + m.max_tile_tris).bytes;
    cudaError_t e = set_smem_cpl(k_tracer_stage_cpl<R, TPc>, sm);
    if (e != cudaSuccess) return e;
    k_tracer_stage_cpl<R, TPc><<<m.n_tiles, TPc, sm, stm>>>(m, U, V, Tn, Tp, Text, W, Tout, st_n, st_np1,
                                                            (R)th_p, (R)th_s, (R)aq, (R)bq, (R)dt, sp, err);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_vertical_solve_cpl(const DevMesh& m, int TP, const R* W, const R* st, const R* rhs,
                                      R* out, double bdt, const StageParams& sp, int* err,
                                      cudaStream_t stm) {
  SLIM_TP_SWITCH_CPL(TP, {
    const size_t sm = CplSmem<R>(TPc, TPc + m.max_tile_tris).bytes;
    cudaError_t e = set_smem_cpl(k_vertical_solve_cpl<R, TPc>, sm);
    if (e != cudaSuccess) return e;
    k_vertical_solve_cpl<R, TPc><<<m.n_tiles, TPc, sm, stm>>>(m, W, st, rhs, out, (R)bdt, sp, err);
  });
  return cudaGetLastError();
}

#define SLIM_INSTANTIATE_CPL(R)                                                                         \
  template cudaError_t launch_continuity_cpl<R>(const DevMesh&, int, const R*, const R*, const double*,  \
                                                const R*, double*, R*, R*, double, cudaStream_t);        \
  template cudaError_t launch_tracer_stage_cpl<R>(const DevMesh&, int, const R*, const R*, const R*,     \
                                                  const R*, const R*, const R*, R*, const R*, const R*,  \
                                                  double, double, double, double, double,                \
                                                  const StageParams&, int*, cudaStream_t);               \
  template cudaError_t launch_vertical_solve_cpl<R>(const DevMesh&, int, const R*, const R*, const R*,   \
                                                    R*, double, const StageParams&, int*, cudaStream_t);

SLIM_INSTANTIATE_CPL(double)
SLIM_INSTANTIATE_CPL(float)

}  // namespace slim
