// Device building blocks of the prismatic P1xP1 DG hot path (sm_103a).
//
// Everything here works on one prism (thread per prism) or one vertex column
// (thread per column) of a thread-block tile: a run of consecutive triangles
// whose columns hold at most TP prisms, staged in shared memory so that the
// six node planes of every field are read and written coalesced.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "slim_internal.h"

namespace slim {

// Gauss-Legendre points on [0,1]: (1 -/+ 1/sqrt(3)) / 2
#define SLIM_GL1 0.21132486540518711775
#define SLIM_GL2 0.78867513459481288225

template <typename R> struct Geo;
template <> struct Geo<double> {
  static __device__ __forceinline__ double hN(const DevMesh& m, int i) { return m.hN[i]; }
  static __device__ __forceinline__ double ih(const DevMesh& m, int i) { return m.ih[i]; }
  static __device__ __forceinline__ double h(const DevMesh& m, int i) { return m.h[i]; }
  static __device__ __forceinline__ double lev(const DevMesh& m, int k) { return m.levels[k]; }
  static __device__ __forceinline__ double jh(const DevMesh& m, int t) { return m.jh[t]; }
  static __device__ __forceinline__ double gx(const DevMesh& m, int i) { return m.gx[i]; }
  static __device__ __forceinline__ double gy(const DevMesh& m, int i) { return m.gy[i]; }
  static __device__ __forceinline__ double nx(const DevMesh& m, int i) { return m.enx[i]; }
  static __device__ __forceinline__ double ny(const DevMesh& m, int i) { return m.eny[i]; }
  static __device__ __forceinline__ double len(const DevMesh& m, int i) { return m.elen[i]; }
};
template <> struct Geo<float> {
  static __device__ __forceinline__ float hN(const DevMesh& m, int i) { return m.hN_f[i]; }
  static __device__ __forceinline__ float ih(const DevMesh& m, int i) { return m.ih_f[i]; }
  static __device__ __forceinline__ float h(const DevMesh& m, int i) { return m.h_f[i]; }
  static __device__ __forceinline__ float lev(const DevMesh& m, int k) { return m.levels_f[k]; }
  static __device__ __forceinline__ float jh(const DevMesh& m, int t) { return m.jh_f[t]; }
  static __device__ __forceinline__ float gx(const DevMesh& m, int i) { return m.gx_f[i]; }
  static __device__ __forceinline__ float gy(const DevMesh& m, int i) { return m.gy_f[i]; }
  static __device__ __forceinline__ float nx(const DevMesh& m, int i) { return m.enx_f[i]; }
  static __device__ __forceinline__ float ny(const DevMesh& m, int i) { return m.eny_f[i]; }
  static __device__ __forceinline__ float len(const DevMesh& m, int i) { return m.elen_f[i]; }
};

// Layer thickness at elevation eta in the compute type R, for the vertex column
// entry i = a*n_tri + t: the interfaces stretch with the column, z = eta + (1 + eta/h) zhat,
// so dz = dz_rest (1 + eta (1/h)) with dz_rest = h/N for sigma layers or the level
// spacing (the column's own depth at the bed) for z-levels.  Division-free.
template <typename R>
__device__ __forceinline__ R dz_rest_r(const DevMesh& m, int i, int k, int N) {
  if (m.n_levels == 0) return Geo<R>::hN(m, i);
  const R top = Geo<R>::lev(m, k);
  const R bot = (k + 1 < N) ? Geo<R>::lev(m, k + 1) : -Geo<R>::h(m, i);
  return top - bot;
}
template <typename R>
__device__ __forceinline__ R stretch_r(const DevMesh& m, int i, double eta) {
  return (R)1 + (R)eta * Geo<R>::ih(m, i);
}
template <typename R>
__device__ __forceinline__ R dz_r(const DevMesh& m, int i, double eta, int k, int N) {
  return dz_rest_r<R>(m, i, k, N) * stretch_r<R>(m, i, eta);
}

// ---------------------------------------------------------------------------
// tile bookkeeping
// ---------------------------------------------------------------------------
struct Tile {
  int t0, nt, p0, np;
};

__device__ __forceinline__ Tile tile_of_block(const DevMesh& m) {
  const int4 ti = m.tile_info[blockIdx.x];
  Tile tl;
  tl.t0 = ti.x; tl.nt = ti.y; tl.p0 = ti.z; tl.np = ti.w;
  return tl;
}

// local column offsets of the tile into shared memory (ends with a barrier)
template <int TP>
__device__ __forceinline__ void load_offsets(const DevMesh& m, const Tile& tl, int* s_off) {
  for (int i = threadIdx.x; i <= tl.nt; i += TP) s_off[i] = m.col_off[tl.t0 + i] - tl.p0;
  __syncthreads();
}

template <int TP>
__device__ __forceinline__ Tile load_tile(const DevMesh& m, int* s_off) {
  const Tile tl = tile_of_block(m);
  load_offsets<TP>(m, tl, s_off);
  return tl;
}

// Column sum returned in FP64.  FP64 form: plain FP64 accumulation.  Mixed form:
// compensated FP32 accumulation (TwoSum of every addition, the error terms summed
// separately), whose result carries about 48 bits, converted to FP64 once; this
// keeps the FP64-accurate depth integration off GB300's narrow FP64 pipe.
template <typename R> struct ColSum;
template <> struct ColSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct ColSum<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// reciprocal: fast approximate for the FP32 form, exact division in FP64
// IEEE 754 binary32 <-> binary64 conversions on the integer pipe (bit fields of
// the two formats; exact in one direction, round-to-nearest-even in the other,
// subnormals included).  The FP64 pipe of this GPU runs conversions at the FP64
// rate; these keep it for the arithmetic of the mixed-form 2D update.
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xffu, mt = u & 0x7fffffu;
  unsigned hi, lo;
  if (e != 0u && e != 255u) {                       // normal: rebias 127 -> 1023
    hi = s | ((e + 896u) << 20) | (mt >> 3);
    lo = mt << 29;
  } else if (e == 255u) {                           // infinity / NaN (payload kept)
    hi = s | 0x7ff00000u | (mt >> 3);
    lo = mt << 29;
  } else if (mt == 0u) {                            // signed zero
    hi = s;
    lo = 0u;
  } else {                                          // subnormal: normalise
    const int lz = __clz(mt) - 9;                   // leading zeros inside the 23-bit field
    const unsigned mn = (mt << (lz + 1)) & 0x7fffffu;
    hi = s | ((unsigned)(896 - lz) << 20) | (mn >> 3);
    lo = mn << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned s = hi & 0x80000000u, mh = hi & 0xfffffu;
  const int E = (int)((hi >> 20) & 0x7ffu);
  unsigned f;
  if (E > 896 && E < 1151) {                        // binary32 normal range
    f = ((unsigned)(E - 896) << 23) | (mh << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu, half = 0x10000000u;
    f += (rem > half || (rem == half && (f & 1u))) ? 1u : 0u;  // a carry may reach infinity
  } else if (E == 2047) {                           // infinity / NaN
    f = 0x7f800000u | (((mh | lo) != 0u) ? (0x400000u | (mh << 3) | (lo >> 29)) : 0u);
  } else if (E >= 1151) {                           // overflow
    f = 0x7f800000u;
  } else {                                          // binary32 subnormal or zero
    const int r = 926 - E;                          // right shift of the 53-bit significand
    if (E == 0 || r >= 64) {
      f = 0u;
    } else {
      const unsigned long long M = (1ull << 52) | ((unsigned long long)mh << 32) | lo;
      const unsigned long long k = M >> r, rem = M & ((1ull << r) - 1ull), half = 1ull << (r - 1);
      f = (unsigned)k + ((rem > half || (rem == half && (k & 1ull))) ? 1u : 0u);
    }
  }
  return __uint_as_float(s | f);
}

template <typename R> __device__ __forceinline__ R rcp(R x);
// correctly rounded (IEEE) in both forms: the approximate reciprocal is biased,
// and a biased inverse in the column solves and the inverse mass changes the tracer
// mass by the same fraction every step
template <> __device__ __forceinline__ float rcp<float>(float x) { return 1.0f / x; }
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }

// local triangle of local prism i (largest j with s_off[j] <= i)
__device__ __forceinline__ int tile_tri_of(const int* s_off, int nt, int i) {
  int lo = 0, hi = nt - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (s_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// horizontal residual of one prism
//   out[c][a] = int q T . grad(phi_a) psi_c J_h  -  sum_e int phi_a psi_c (q.n)^ T^
// q = (dz/2) u nodal, dz = dz_rest x stretch st_q of the vertex column (the stretch
// 1 + eta/h of the elevation the transport is frozen at).  UNIT: T = 1 (continuity).
// Volume term in closed form: with the P1 mass M2_be = J_h (1 + d_be)/24 and the
// triple integrals G3_dfc = int psi_d psi_f psi_c (1/2 if d = f = c, else 1/6),
//   X_c = sum_{d,f} G3_dfc sum_{b,e} M2_be q_bd T_ef,   out_vol[c][a] = grad(phi_a) . X_c
// Lateral faces: 2 x 2 Gauss points, mean transport of both sides, upwind T.
// ---------------------------------------------------------------------------
// Node values of one prism, loaded before the tile barrier so that these loads
// overlap the tile set-up.
template <typename R>
struct Own {
  R u[2][3], v[2][3], T[2][3];
};
template <typename R, bool UNIT>
__device__ __forceinline__ void load_own(const DevMesh& m, int p, const R* __restrict__ U,
                                         const R* __restrict__ V, const R* __restrict__ T,
                                         Own<R>& o) {
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t idx = (size_t)(c * 3 + a) * m.P + p;
      o.u[c][a] = U[idx];
      o.v[c][a] = V[idx];
      o.T[c][a] = UNIT ? (R)1 : T[idx];
    }
}

template <typename R, bool UNIT>
__device__ __forceinline__ void prism_rh(const DevMesh& m, int t, int k, int p, int N,
                                         const Own<R>& own, const R* __restrict__ U,
                                         const R* __restrict__ V, const R* __restrict__ T,
                                         const R* __restrict__ Text,
                                         const R* __restrict__ st_q, R out[2][3]) {
  const int nt = m.n_tri, P = m.P;
  R qx[2][3], qy[2][3], Tv[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R hz = (R)0.5 * dz_rest_r<R>(m, a * nt + t, k, N) * st_q[a * nt + t];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      qx[c][a] = hz * own.u[c][a];
      qy[c][a] = hz * own.v[c][a];
      Tv[c][a] = UNIT ? (R)1 : own.T[c][a];
    }
  }
  const R jh = Geo<R>::jh(m, t);
  // volume term
  R Xx[2], Xy[2];
  {
    R Yx[2][2], Yy[2][2];
    const R w24 = jh * (R)(1.0 / 24.0);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      R sqx = qx[d][0] + qx[d][1] + qx[d][2];
      R sqy = qy[d][0] + qy[d][1] + qy[d][2];
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        if (UNIT) {
          Yx[d][f] = (R)4 * w24 * sqx;
          Yy[d][f] = (R)4 * w24 * sqy;
        } else {
          R st = Tv[f][0] + Tv[f][1] + Tv[f][2];
          R px = qx[d][0] * Tv[f][0] + qx[d][1] * Tv[f][1] + qx[d][2] * Tv[f][2];
          R py = qy[d][0] * Tv[f][0] + qy[d][1] * Tv[f][1] + qy[d][2] * Tv[f][2];
          Yx[d][f] = w24 * (sqx * st + px);
          Yy[d][f] = w24 * (sqy * st + py);
        }
      }
    }
    const R h2 = (R)0.5, h6 = (R)(1.0 / 6.0);
    Xx[0] = h2 * Yx[0][0] + h6 * (Yx[0][1] + Yx[1][0] + Yx[1][1]);
    Xx[1] = h2 * Yx[1][1] + h6 * (Yx[0][0] + Yx[0][1] + Yx[1][0]);
    Xy[0] = h2 * Yy[0][0] + h6 * (Yy[0][1] + Yy[1][0] + Yy[1][1]);
    Xy[1] = h2 * Yy[1][1] + h6 * (Yy[0][0] + Yy[0][1] + Yy[1][0]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R gxa = Geo<R>::gx(m, a * nt + t), gya = Geo<R>::gy(m, a * nt + t);
#pragma unroll
    for (int c = 0; c < 2; ++c) out[c][a] = gxa * Xx[c] + gya * Xy[c];
  }
  // lateral faces
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int4 ei = m.einfo[e * nt + t];
    const int nb = ei.x;
    if (nb == -1) continue;  // wall
    const int a0 = e, a1 = (e + 1) % 3;
    const R nxe = Geo<R>::nx(m, e * nt + t), nye = Geo<R>::ny(m, e * nt + t);
    const R half_len = (R)0.5 * Geo<R>::len(m, e * nt + t);
    R qo[2][2], To[2][2], qb[2][2], Tb[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      qo[0][c] = qx[c][a0] * nxe + qy[c][a0] * nye;
      qo[1][c] = qx[c][a1] * nxe + qy[c][a1] * nye;
      To[0][c] = Tv[c][a0];
      To[1][c] = Tv[c][a1];
    }
    bool has_nb = false;
    if (nb >= 0) {
      const int Nn = ei.z;
      if (k >= Nn) continue;  // wall against a shallower neighbour column
      has_nb = true;
      const int pn = ei.y + k;
      const int loc = ei.w;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int l = j ? ((loc >> 2) & 3) : (loc & 3);
        const R hz = (R)0.5 * dz_rest_r<R>(m, l * nt + nb, k, Nn) * st_q[l * nt + nb];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const size_t idx = (size_t)(c * 3 + l) * P + pn;
          qb[j][c] = hz * (U[idx] * nxe + V[idx] * nye);
          Tb[j][c] = UNIT ? (R)1 : T[idx];
        }
      }
    } else {  // open boundary: interior transport, exterior tracer on inflow
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          qb[j][c] = qo[j][c];
          Tb[j][c] = (UNIT || Text == nullptr) ? To[j][c]
                                               : Text[(size_t)(c * 3 + (j ? a1 : a0)) * P + p];
        }
    }
#pragma unroll
    for (int gs = 0; gs < 2; ++gs) {
      const R b0 = gs ? (R)SLIM_GL1 : (R)SLIM_GL2;  // basis of vertex a0 along the edge
      const R b1 = gs ? (R)SLIM_GL2 : (R)SLIM_GL1;
#pragma unroll
      for (int gz = 0; gz < 2; ++gz) {
        const R z0 = gz ? (R)SLIM_GL2 : (R)SLIM_GL1;  // psi_top at the point
        const R z1 = gz ? (R)SLIM_GL1 : (R)SLIM_GL2;
        const R B00 = b0 * z0, B01 = b0 * z1, B10 = b1 * z0, B11 = b1 * z1;
        const R qno = B00 * qo[0][0] + B01 * qo[0][1] + B10 * qo[1][0] + B11 * qo[1][1];
        R qn = qno;
        if (has_nb) {
          const R qnb = B00 * qb[0][0] + B01 * qb[0][1] + B10 * qb[1][0] + B11 * qb[1][1];
          qn = (R)0.5 * (qno + qnb);
        }
        R Tup;
        if (UNIT) {
          Tup = (R)1;
        } else if (qn > (R)0) {
          Tup = B00 * To[0][0] + B01 * To[0][1] + B10 * To[1][0] + B11 * To[1][1];
        } else {
          Tup = B00 * Tb[0][0] + B01 * Tb[0][1] + B10 * Tb[1][0] + B11 * Tb[1][1];
        }
        const R f = half_len * qn * Tup;
        out[0][a0] -= f * B00;
        out[1][a0] -= f * B01;
        out[0][a1] -= f * B10;
        out[1][a1] -= f * B11;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// vertical operator: block row k of K = M - bdt A for one vertex column
// (2x2 blocks; D couples layer k to itself, L to layer k-1, U to layer k+1).
// A = vertical upwind advection by the vertex-weighted flux W (interface i
// carries W_{i,top}, 0 on the bed) + omega x SIPG diffusion; M = omega (dz/2) G.
// ---------------------------------------------------------------------------
template <typename R>
struct Row {
  R D[2][2], L[2][2], U[2][2];
};

// idzm, idz, idzp: reciprocals of the thicknesses of layers k-1, k, k+1.  With
// op given, the operator blocks A (op->D), A_{k,k-1} (op->L) and A_{k,k+1} (op->U)
// are returned as well (K = M - bdt A).
template <typename R>
__device__ __forceinline__ void assemble_row(int k, int N, R omega, R idzm, R dz, R idz, R idzp,
                                             R W0, R W1, R Wn, R kap, R pen, R bdt, Row<R>& row,
                                             Row<R>* op = nullptr) {
  R A[2][2] = {{0, 0}, {0, 0}}, AL[2][2] = {{0, 0}, {0, 0}}, AU[2][2] = {{0, 0}, {0, 0}};
  // advection, volume: A[c][d] = dpsi_c sum_e W_e G_ed
  const R g0 = (R)(1.0 / 3.0) * ((R)2 * W0 + W1);
  const R g1 = (R)(1.0 / 3.0) * (W0 + (R)2 * W1);
  A[0][0] += (R)0.5 * g0; A[0][1] += (R)0.5 * g1;
  A[1][0] -= (R)0.5 * g0; A[1][1] -= (R)0.5 * g1;
  // advection, top interface of layer k
  if (k == 0 || W0 > (R)0) A[0][0] -= W0; else AL[0][1] -= W0;
  // advection, bottom interface
  if (k + 1 < N) {
    if (Wn > (R)0) AU[1][0] += Wn; else A[1][1] += Wn;
  }
  // diffusion, element stiffness
  const R ke = omega * kap * idz;
  A[0][0] -= ke; A[0][1] += ke; A[1][0] += ke; A[1][1] -= ke;
  if (k > 0) {
    const R sg = pen * kap * fmax(idzm, idz);
    const R cm = (R)0.5 * kap * idzm, c0 = (R)0.5 * kap * idz;
    A[0][0] -= omega * (sg - (R)2 * c0);
    A[0][1] -= omega * c0;
    A[1][0] -= omega * c0;
    AL[0][0] -= omega * (-cm);
    AL[0][1] -= omega * (cm + c0 - sg);
    AL[1][1] -= omega * (-c0);
  }
  if (k + 1 < N) {
    const R sg = pen * kap * fmax(idz, idzp);
    const R c0 = (R)0.5 * kap * idz, cp = (R)0.5 * kap * idzp;
    A[0][1] -= omega * c0;
    A[1][0] -= omega * c0;
    A[1][1] -= omega * (sg - (R)2 * c0);
    AU[0][0] -= omega * (-c0);
    AU[1][0] -= omega * (c0 + cp - sg);
    AU[1][1] -= omega * (-cp);
  }
  if (op) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        op->D[i][j] = A[i][j];
        op->L[i][j] = AL[i][j];
        op->U[i][j] = AU[i][j];
      }
  }
  const R mw = omega * (R)0.5 * dz;
  const R m2 = mw * (R)(2.0 / 3.0), m1 = mw * (R)(1.0 / 3.0);
  row.D[0][0] = m2 - bdt * A[0][0];
  row.D[0][1] = m1 - bdt * A[0][1];
  row.D[1][0] = m1 - bdt * A[1][0];
  row.D[1][1] = m2 - bdt * A[1][1];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      row.L[i][j] = -bdt * AL[i][j];
      row.U[i][j] = -bdt * AU[i][j];
    }
}

// 2x2 helpers
template <typename R>
__device__ __forceinline__ void inv2(const R a[2][2], R o[2][2]) {
  const R r = rcp<R>(a[0][0] * a[1][1] - a[0][1] * a[1][0]);
  o[0][0] = a[1][1] * r; o[0][1] = -a[0][1] * r;
  o[1][0] = -a[1][0] * r; o[1][1] = a[0][0] * r;
}

}  // namespace slim
