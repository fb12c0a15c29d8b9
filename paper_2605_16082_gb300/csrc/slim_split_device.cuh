// Device building blocks of the baroclinic (split-IMEX) path: advection of two
// fields by the corrected transport, horizontal SIPG, vertical operator blocks,
// a 2x2-block Thomas sweep with two right-hand sides.
#pragma once

#include "slim_device.cuh"

namespace slim {

// Inputs of the horizontal advection residual.
template <typename R>
struct AdvIn {
  const R* U;      // transport velocity of the evaluation state
  const R* V;
  const R* F0;     // advected fields (the transport velocity itself for momentum)
  const R* F1;
  const R* E0;     // open-boundary exterior profiles (null: zero gradient)
  const R* E1;
  const R* st;     // stretch of the evaluation geometry
  const R* Dqx;    // [3][n_tri] Qbar - column sum of q (null: no correction)
  const R* Dqy;
  const R* gcor;   // [(e n_tri + t) 2 + g] face correction delta / tot (null: none)
  // open-boundary forcing (null: none): exterior velocity at the two forcing times,
  // the second time's E0/E1, and theta at the middle of the stage's 2D run
  const R* Uxa;
  const R* Vxa;
  const R* Uxb;
  const R* Vxb;
  const R* E0b;
  const R* E1b;
  const R* th;
  // lateral normal transport at the 4 points of every face of every prism, [12][P]
  // (face e, edge point gs, zeta point gz at row 4 e + 2 gs + gz): written by the
  // pass that computes it (the continuity), read instead of recomputed by the later
  // passes of the same stage over the same transport (null: none)
  R* qn_out;
  const R* qn_in;
};

template <typename R>
struct Own2 {
  R u[2][3], v[2][3], f0[2][3], f1[2][3];
};

// SELF: the advected fields are the transport velocity (momentum)
template <typename R, bool SELF>
__device__ __forceinline__ void load_own2(const DevMesh& m, int p, const AdvIn<R>& in, Own2<R>& o) {
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t idx = (size_t)(c * 3 + a) * m.P + p;
      o.u[c][a] = in.U[idx];
      o.v[c][a] = in.V[idx];
      if (SELF) {
        o.f0[c][a] = o.u[c][a];
        o.f1[c][a] = o.v[c][a];
      } else {
        o.f0[c][a] = in.F0[idx];
        o.f1[c][a] = in.F1[idx];
      }
    }
}

// Closed-form volume term of -div(q f) tested with phi_a psi_c (see prism_rh).
template <typename R>
__device__ __forceinline__ void adv_volume(const DevMesh& m, int t, const R gx[3], const R gy[3],
                                           const R qx[2][3], const R qy[2][3], const R f[2][3],
                                           R out[2][3]) {
  const int nt = m.n_tri;
  const R w24 = Geo<R>::jh(m, t) * (R)(1.0 / 24.0);
  R Yx[2][2], Yy[2][2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const R sqx = qx[d][0] + qx[d][1] + qx[d][2];
    const R sqy = qy[d][0] + qy[d][1] + qy[d][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const R sf = f[e][0] + f[e][1] + f[e][2];
      const R px = qx[d][0] * f[e][0] + qx[d][1] * f[e][1] + qx[d][2] * f[e][2];
      const R py = qy[d][0] * f[e][0] + qy[d][1] * f[e][1] + qy[d][2] * f[e][2];
      Yx[d][e] = w24 * (sqx * sf + px);
      Yy[d][e] = w24 * (sqy * sf + py);
    }
  }
  const R h2 = (R)0.5, h6 = (R)(1.0 / 6.0);
  const R Xx0 = h2 * Yx[0][0] + h6 * (Yx[0][1] + Yx[1][0] + Yx[1][1]);
  const R Xx1 = h2 * Yx[1][1] + h6 * (Yx[0][0] + Yx[0][1] + Yx[1][0]);
  const R Xy0 = h2 * Yy[0][0] + h6 * (Yy[0][1] + Yy[1][0] + Yy[1][1]);
  const R Xy1 = h2 * Yy[1][1] + h6 * (Yy[0][0] + Yy[0][1] + Yy[1][0]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    out[0][a] += gx[a] * Xx0 + gy[a] * Xy0;
    out[1][a] += gx[a] * Xx1 + gy[a] * Xy1;
  }
}

// Horizontal SIPG of two fields on coordinate surfaces (weight nu z_zeta):
//   -int nu z_zeta grad f . grad v + oint [{nu z_zeta grad f}.n v
//                                          + 1/2 nu z_zeta^- grad v.n [f] - sigma {z_zeta}[f] v]
// sigma = pen nu / min(r_in^-, r_in^+), interior faces only (natural elsewhere).
// The two fields share the geometry: the layer thicknesses, the penalty and the
// normal derivatives of both triangles' basis functions (the gradient of a P1
// field dotted with n is the sum of its nodal values times those derivatives).
// Volume part (hz: the prism's half layer thickness at its three vertices).
template <typename R>
__device__ __forceinline__ void sipg_volume2(const DevMesh& m, int t, const R gx[3], const R gy[3],
                                             const R hz[3], const R f0[2][3], const R f1[2][3], R nu,
                                             R out0[2][3], R out1[2][3]) {
  const R(*fs[2])[3] = {f0, f1};
  R(*outs[2])[3] = {out0, out1};
  // -nu (J_h/6)(sum hz) sum_d G_dc grad f_d . grad phi_a
  const R w = nu * Geo<R>::jh(m, t) * (R)(1.0 / 6.0) * (hz[0] + hz[1] + hz[2]);
  const R G2 = (R)(2.0 / 3.0), G1 = (R)(1.0 / 3.0);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    R gux[2], guy[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      gux[c] = fs[q][c][0] * gx[0] + fs[q][c][1] * gx[1] + fs[q][c][2] * gx[2];
      guy[c] = fs[q][c][0] * gy[0] + fs[q][c][1] * gy[1] + fs[q][c][2] * gy[2];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R d0 = gux[0] * gx[a] + guy[0] * gy[a];
      const R d1 = gux[1] * gx[a] + guy[1] * gy[a];
      outs[q][0][a] -= w * (G2 * d0 + G1 * d1);
      outs[q][1][a] -= w * (G1 * d0 + G2 * d1);
    }
  }
}

// Face part on lateral face e (own vertices a0 = e, a1 = e + 1) against neighbour
// triangle nb (prism pn, its vertices l0, l1 on the face and l2 the third):
// hzo / hzn the half thicknesses at the face vertices on both sides, fn0 / fn1 the
// neighbour's values of the two fields at (l_j, level c), already loaded by the
// caller (the advection reads the same values).
template <typename R>
__device__ __forceinline__ void sipg_face2(const DevMesh& m, int t, int e, int nb, int pn, int l0, int l1, R nxe,
                                           R nye, R half_len, const R gx[3], const R gy[3],
                                           const R hzo[2], const R hzn[2],
                                           const R f0[2][3], const R f1[2][3], const R fn0[2][2],
                                           const R fn1[2][2], const R* __restrict__ F0,
                                           const R* __restrict__ F1, R nu, R pen, R out0[2][3],
                                           R out1[2][3]) {
  const int nt = m.n_tri, P = m.P;
  const int a0 = e, a1 = (e + 1) % 3, l2 = 3 - l0 - l1;
  const R isig = (sizeof(R) == 4) ? (R)m.esig_f[e * nt + t] : (R)m.esig[e * nt + t];
  R dno[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) dno[b] = gx[b] * nxe + gy[b] * nye;
  const R dn0 = Geo<R>::gx(m, l0 * nt + nb) * nxe + Geo<R>::gy(m, l0 * nt + nb) * nye;
  const R dn1 = Geo<R>::gx(m, l1 * nt + nb) * nxe + Geo<R>::gy(m, l1 * nt + nb) * nye;
  const R dn2 = Geo<R>::gx(m, l2 * nt + nb) * nxe + Geo<R>::gy(m, l2 * nt + nb) * nye;
  // The face integrals are polynomials of degree <= 3 per direction, integrated
  // exactly in closed form: with the edge basis b_i and psi_c,
  //   int b_i b_j = E2_ij (2/3, 1/3), int b_i b_j b_k = 1/2 (all equal) or 1/6,
  //   int psi_d psi_c = G_dc (2/3, 1/3).
  const R t3 = (R)(1.0 / 3.0), t6 = (R)(1.0 / 6.0);
  const R Zo[2] = {t3 * ((R)2 * hzo[0] + hzo[1]), t3 * ((R)2 * hzo[1] + hzo[0])};
  const R Zn[2] = {t3 * ((R)2 * hzn[0] + hzn[1]), t3 * ((R)2 * hzn[1] + hzn[0])};
  const R hs0 = hzo[0] + hzn[0], hs1 = hzo[1] + hzn[1];
  const R M00 = (R)0.5 * hs0 + t6 * hs1, M11 = (R)0.5 * hs1 + t6 * hs0, M01 = t6 * (hs0 + hs1);
  const R hnu = half_len * (R)0.5 * nu;
  const R hsig = half_len * (R)0.5 * pen * nu * isig;
  const R(*fs[2])[3] = {f0, f1};
  const R(*fns[2])[2] = {fn0, fn1};
  const R* Fs[2] = {F0, F1};
  R(*outs[2])[3] = {out0, out1};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const R(*f)[3] = fs[q];
    R gno[2], gnn[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const R fl2 = Fs[q][(size_t)(c * 3 + l2) * P + pn];
      gno[c] = f[c][0] * dno[0] + f[c][1] * dno[1] + f[c][2] * dno[2];
      gnn[c] = fns[q][0][c] * dn0 + fns[q][1][c] * dn1 + fl2 * dn2;
    }
    const R Go[2] = {t3 * ((R)2 * gno[0] + gno[1]), t3 * ((R)2 * gno[1] + gno[0])};
    const R Gn[2] = {t3 * ((R)2 * gnn[0] + gnn[1]), t3 * ((R)2 * gnn[1] + gnn[0])};
    // jumps at the face nodes (own vertex j <-> neighbour vertex l_j), G-weighted in zeta
    R J[2][2], gJ[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      J[0][c] = f[c][a0] - fns[q][0][c];
      J[1][c] = f[c][a1] - fns[q][1][c];
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      gJ[i][0] = t3 * ((R)2 * J[i][0] + J[i][1]);
      gJ[i][1] = t3 * ((R)2 * J[i][1] + J[i][0]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const R zj = hnu * (Zo[0] * gJ[0][c] + Zo[1] * gJ[1][c]);
      // flux {nu z_zeta grad f}.n tested with the edge functions, minus the penalty
      outs[q][c][a0] += hnu * (Zo[0] * Go[c] + Zn[0] * Gn[c]) - hsig * (M00 * gJ[0][c] + M01 * gJ[1][c]);
      outs[q][c][a1] += hnu * (Zo[1] * Go[c] + Zn[1] * Gn[c]) - hsig * (M01 * gJ[0][c] + M11 * gJ[1][c]);
      // symmetry term 1/2 nu z_zeta grad v.n [f] for every own test function
#pragma unroll
      for (int a = 0; a < 3; ++a) outs[q][c][a] += dno[a] * zj;
    }
  }
}

// Both parts, face by face with its own loads (when no advection pass shares them).
template <typename R>
__device__ __forceinline__ void prism_sipg2(const DevMesh& m, int t, int k, int N, const R f0[2][3],
                                            const R f1[2][3], const R* __restrict__ F0,
                                            const R* __restrict__ F1, const R* __restrict__ st,
                                            R nu, R pen, R out0[2][3], R out1[2][3]) {
  const int nt = m.n_tri, P = m.P;
  R hz[3], gx[3], gy[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hz[a] = (R)0.5 * dz_rest_r<R>(m, a * nt + t, k, N) * st[a * nt + t];
    gx[a] = Geo<R>::gx(m, a * nt + t);
    gy[a] = Geo<R>::gy(m, a * nt + t);
  }
  sipg_volume2<R>(m, t, gx, gy, hz, f0, f1, nu, out0, out1);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int4 ei = m.einfo[e * nt + t];
    const int nb = ei.x;
    if (nb < 0) continue;
    const int Nn = ei.z;
    if (k >= Nn) continue;
    const int pn = ei.y + k;
    const int l0 = ei.w & 3, l1 = (ei.w >> 2) & 3;
    const int a0 = e, a1 = (e + 1) % 3;
    const R nxe = Geo<R>::nx(m, e * nt + t), nye = Geo<R>::ny(m, e * nt + t);
    const R half_len = (R)0.5 * Geo<R>::len(m, e * nt + t);
    const R hzo[2] = {hz[a0], hz[a1]};
    const R hzn[2] = {(R)0.5 * dz_rest_r<R>(m, l0 * nt + nb, k, Nn) * st[l0 * nt + nb],
                      (R)0.5 * dz_rest_r<R>(m, l1 * nt + nb, k, Nn) * st[l1 * nt + nb]};
    R fn0[2][2], fn1[2][2];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const size_t idx = (size_t)(c * 3 + (j ? l1 : l0)) * P + pn;
        fn0[j][c] = F0[idx];
        fn1[j][c] = F1[idx];
      }
    sipg_face2<R>(m, t, e, nb, pn, l0, l1, nxe, nye, half_len, gx, gy, hzo, hzn, f0, f1, fn0, fn1, F0, F1, nu,
                  pen, out0, out1);
  }
}

// Horizontal advection residual of two fields (NF = 2) or of T = 1 (UNIT) by the
// transport q = (dz/2) u (+ the node correction (dz_rest/h)(Qbar - sum q)/2), with
// the lateral normal transport {q}.n + (hz^- + hz^+)(s) gcor(s) on faces where a
// face correction is given.  Accumulates into out0 / out1 and returns the nodal
// transport of the prism in qxo / qyo.
// With SIPG, the horizontal SIPG of the two fields (viscosity nu, penalty pen) is
// added in the same pass: its face part shares the face's geometry and the
// neighbour's values with the advection.  It accumulates into sout0 / sout1 when
// given (the momentum prediction keeps it apart), else into out0 / out1.  GKEEP:
// the triangle's gradient coefficients and its nodal transport stay in registers
// through the faces (fewer loads; the momentum prediction, short of registers,
// re-reads the coefficients and forms the face's own transport again from the
// velocities, so qxo / qyo are only valid up to the volume term there).
// QN: 0 computes the lateral normal transport at the face points, 1 also stores it
// in in.qn_out, 2 reads it from in.qn_in (computed by an earlier pass of the stage
// over the same transport) instead of the neighbour's velocities and corrections.
template <typename R, bool UNIT, bool SIPG = false, bool GKEEP = true, int QN = 0>
__device__ __forceinline__ void prism_adv(const DevMesh& m, int t, int k, int p, int N,
                                          const Own2<R>& own, const AdvIn<R>& in, R out0[2][3],
                                          R out1[2][3], R qxo[2][3], R qyo[2][3], R nu = 0,
                                          R pen = 0, R (*sout0)[3] = nullptr, R (*sout1)[3] = nullptr) {
  R(*so0)[3] = sout0 ? sout0 : out0;
  R(*so1)[3] = sout1 ? sout1 : out1;
  const int nt = m.n_tri, P = m.P;
  R hz[3], gxo[3], gyo[3];  // gradient coefficients of the triangle
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ia = a * nt + t;
    gxo[a] = Geo<R>::gx(m, ia);
    gyo[a] = Geo<R>::gy(m, ia);
    const R dr = dz_rest_r<R>(m, ia, k, N);
    hz[a] = (R)0.5 * dr * in.st[ia];
    R cx = 0, cy = 0;
    if (in.Dqx) {
      const R f = (R)0.5 * dr * Geo<R>::ih(m, ia);
      cx = f * in.Dqx[ia];
      cy = f * in.Dqy[ia];
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      qxo[c][a] = hz[a] * own.u[c][a] + cx;
      qyo[c][a] = hz[a] * own.v[c][a] + cy;
    }
  }
  if (UNIT) {
    R one[2][3] = {{1, 1, 1}, {1, 1, 1}};
    adv_volume<R>(m, t, gxo, gyo, qxo, qyo, one, out0);
  } else {
    adv_volume<R>(m, t, gxo, gyo, qxo, qyo, own.f0, out0);
    adv_volume<R>(m, t, gxo, gyo, qxo, qyo, own.f1, out1);
    if (SIPG) sipg_volume2<R>(m, t, gxo, gyo, hz, own.f0, own.f1, nu, so0, so1);
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int4 ei = m.einfo[e * nt + t];
    const int nb = ei.x;
    if (nb == -1) continue;  // wall
    const int a0 = e, a1 = (e + 1) % 3;
    const R nxe = Geo<R>::nx(m, e * nt + t), nye = Geo<R>::ny(m, e * nt + t);
    const R half_len = (R)0.5 * Geo<R>::len(m, e * nt + t);
    constexpr bool ql = QN == 2;  // the face transport is read, not recomputed
    R qo[2][2], qb[2][2], fo0[2][2], fo1[2][2], fb0[2][2], fb1[2][2], hzb[2] = {0, 0};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (GKEEP) {
        qo[0][c] = qxo[c][a0] * nxe + qyo[c][a0] * nye;
        qo[1][c] = qxo[c][a1] * nxe + qyo[c][a1] * nye;
      } else {
        // the same products as qxo / qyo above, formed again
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int a = j ? a1 : a0;
          R cx = 0, cy = 0;
          if (in.Dqx) {
            const int ia = a * nt + t;
            const R f = (R)0.5 * dz_rest_r<R>(m, ia, k, N) * Geo<R>::ih(m, ia);
            cx = f * in.Dqx[ia];
            cy = f * in.Dqy[ia];
          }
          qo[j][c] = (hz[a] * own.u[c][a] + cx) * nxe + (hz[a] * own.v[c][a] + cy) * nye;
        }
      }
      if (!UNIT) {
        fo0[0][c] = own.f0[c][a0]; fo0[1][c] = own.f0[c][a1];
        fo1[0][c] = own.f1[c][a0]; fo1[1][c] = own.f1[c][a1];
      }
    }
    bool has_nb = false, is_open = false;
    int pn = 0, loc = 0;
    if (nb >= 0) {
      const int Nn = ei.z;
      if (k >= Nn) continue;  // wall against a shallower neighbour column
      has_nb = true;
      pn = ei.y + k;
      loc = ei.w;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int l = j ? ((loc >> 2) & 3) : (loc & 3);
        const int il = l * nt + nb;
        R dr = 0, h = 0;
        if (!ql || SIPG) {
          dr = dz_rest_r<R>(m, il, k, Nn);
          h = (R)0.5 * dr * in.st[il];
        }
        hzb[j] = h;
        R cn = 0;
        if (!ql && in.Dqx) cn = (R)0.5 * dr * Geo<R>::ih(m, il) * (in.Dqx[il] * nxe + in.Dqy[il] * nye);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const size_t idx = (size_t)(c * 3 + l) * P + pn;
          if (!ql) qb[j][c] = h * (in.U[idx] * nxe + in.V[idx] * nye) + cn;
          if (!UNIT) {
            fb0[j][c] = in.F0 ? in.F0[idx] : in.U[idx];
            fb1[j][c] = in.F1 ? in.F1[idx] : in.V[idx];
          }
        }
      }
    } else {  // open boundary
      // the face transport is the exterior one alone (the exterior state comes
      // from data): forced, (dz_rest/2) u_ext at theta of the middle of the
      // stage's 2D run, else zero; the face correction adds the layer's share of
      // the 2D flux.  Inflow values: the exterior profiles (lerped when forced).
      const R th = in.Uxa ? *in.th : (R)0;
      is_open = true;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int la = j ? a1 : a0;
        const R hr = in.Uxa ? (R)0.5 * dz_rest_r<R>(m, la * nt + t, k, N) : (R)0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const size_t idx = (size_t)(c * 3 + la) * P + p;
          if (ql) {
          } else if (in.Uxa) {
            const R ux = in.Uxa[idx] + th * (in.Uxb[idx] - in.Uxa[idx]);
            const R vx = in.Vxa[idx] + th * (in.Vxb[idx] - in.Vxa[idx]);
            qb[j][c] = hr * (ux * nxe + vx * nye);
          } else {
            qb[j][c] = (R)0;
          }
          if (!UNIT) {
            fb0[j][c] = in.E0 ? (in.E0b ? in.E0[idx] + th * (in.E0b[idx] - in.E0[idx]) : in.E0[idx]) : fo0[j][c];
            fb1[j][c] = in.E1 ? (in.E1b ? in.E1[idx] + th * (in.E1b[idx] - in.E1[idx]) : in.E1[idx]) : fo1[j][c];
          }
        }
      }
    }
    R gc[2] = {0, 0};
    if (!ql && in.gcor) {
      gc[0] = in.gcor[(e * nt + t) * 2 + 0];
      gc[1] = in.gcor[(e * nt + t) * 2 + 1];
    }
#pragma unroll
    for (int gs = 0; gs < 2; ++gs) {
      const R b0 = gs ? (R)SLIM_GL2 : (R)SLIM_GL1;  // basis of vertex a0 at edge point gs
      const R b1 = gs ? (R)SLIM_GL1 : (R)SLIM_GL2;
      const R corr = (b0 * (hz[a0] + hzb[0]) + b1 * (hz[a1] + hzb[1])) * gc[gs];
#pragma unroll
      for (int gz = 0; gz < 2; ++gz) {
        const R z0 = gz ? (R)SLIM_GL2 : (R)SLIM_GL1;  // psi_top at the zeta point
        const R z1 = gz ? (R)SLIM_GL1 : (R)SLIM_GL2;
        const R B00 = b0 * z0, B01 = b0 * z1, B10 = b1 * z0, B11 = b1 * z1;
        const size_t iq = (size_t)(e * 4 + gs * 2 + gz) * P + p;
        R qn;
        if (ql) {
          qn = in.qn_in[iq];
        } else {
          const R qno = B00 * qo[0][0] + B01 * qo[0][1] + B10 * qo[1][0] + B11 * qo[1][1];
          const R qnb = B00 * qb[0][0] + B01 * qb[0][1] + B10 * qb[1][0] + B11 * qb[1][1];
          // (the prediction, without a face correction, keeps the uncorrected own
          // transport at open faces: its estimate of the 2D flux there)
          qn = (is_open && in.gcor) ? qnb : (has_nb ? (R)0.5 * (qno + qnb) : qno);
          qn += corr;
          if (QN == 1) in.qn_out[iq] = qn;
        }
        if (UNIT) {
          const R f = half_len * qn;
          out0[0][a0] -= f * B00; out0[1][a0] -= f * B01;
          out0[0][a1] -= f * B10; out0[1][a1] -= f * B11;
        } else {
          const bool up = qn > (R)0;
          const R f0 = half_len * qn * (up ? (B00 * fo0[0][0] + B01 * fo0[0][1] + B10 * fo0[1][0] + B11 * fo0[1][1])
                                           : (B00 * fb0[0][0] + B01 * fb0[0][1] + B10 * fb0[1][0] + B11 * fb0[1][1]));
          const R f1 = half_len * qn * (up ? (B00 * fo1[0][0] + B01 * fo1[0][1] + B10 * fo1[1][0] + B11 * fo1[1][1])
                                           : (B00 * fb1[0][0] + B01 * fb1[0][1] + B10 * fb1[1][0] + B11 * fb1[1][1]));
          out0[0][a0] -= f0 * B00; out0[1][a0] -= f0 * B01;
          out0[0][a1] -= f0 * B10; out0[1][a1] -= f0 * B11;
          out1[0][a0] -= f1 * B00; out1[1][a0] -= f1 * B01;
          out1[0][a1] -= f1 * B10; out1[1][a1] -= f1 * B11;
        }
      }
    }
    if (SIPG && !UNIT && has_nb) {
      const R hzo[2] = {hz[a0], hz[a1]};
      if (!GKEEP) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          gxo[b] = Geo<R>::gx(m, b * nt + t);
          gyo[b] = Geo<R>::gy(m, b * nt + t);
        }
      }
      sipg_face2<R>(m, t, e, nb, pn, loc & 3, (loc >> 2) & 3, nxe, nye, half_len, gxo, gyo, hzo, hzb, own.f0,
                    own.f1, fb0, fb1, in.F0 ? in.F0 : in.U, in.F1 ? in.F1 : in.V, nu, pen, so0, so1);
    }
  }
}

// Vertical operator A of block row k (advection by W + omega x SIPG diffusion),
// as in assemble_row but without the mass and the time step.
template <typename R>
__device__ __forceinline__ void vertical_A(int k, int N, R omega, R idzm, R idz, R idzp, R W0, R W1,
                                           R Wn, R kap, R pen, R A[2][2], R AL[2][2], R AU[2][2]) {
  Row<R> row;
  // assemble_row computes K = M - bdt A; with bdt = -1 and the mass removed we get A
  assemble_row<R>(k, N, omega, idzm, (R)0, idz, idzp, W0, W1, Wn, kap, pen, (R)-1, row);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      A[i][j] = row.D[i][j];
      AL[i][j] = row.L[i][j];
      AU[i][j] = row.U[i][j];
    }
}

// 2x2-block Thomas sweep of one vertex column with two right-hand sides sharing
// the matrix K = M(st) - bdt A.  b?t/b?b: right-hand sides of field ? (top/bottom
// rows), overwritten by the solution; C0..C3 scratch.  Increment form when x0 is
// given (top/bottom of field 0, then of field 1, by layer): the b are rhs - M x0,
// the sweep adds bdt A x0, solves for the increment and returns x0 + increment.
template <typename R>
__device__ __forceinline__ void column_thomas2(const DevMesh& m, int t, int ia, int N, R st,
                                               const R* __restrict__ Wt, const R* __restrict__ Wb,
                                               R* __restrict__ b0t, R* __restrict__ b0b,
                                               R* __restrict__ b1t, R* __restrict__ b1b,
                                               R* __restrict__ C0, R* __restrict__ C1,
                                               R* __restrict__ C2, R* __restrict__ C3, R kap, R pen,
                                               R bdt, const R* const* x0 = nullptr) {
  const R omega = Geo<R>::jh(m, t) * (R)(1.0 / 6.0);
  R z[2][2] = {{0, 0}, {0, 0}};
  R c00 = 0, c01 = 0, c10 = 0, c11 = 0;
  R dz = dz_rest_r<R>(m, ia, 0, N) * st;
  R idz = rcp<R>(dz);
  R idzm = idz;
  for (int k = 0; k < N; ++k) {
    R dzp = dz, idzp = idz;
    if (k + 1 < N && m.n_levels != 0) {
      dzp = dz_rest_r<R>(m, ia, k + 1, N) * st;
      idzp = rcp<R>(dzp);
    }
    const R Wn = (k + 1 < N) ? Wt[k + 1] : (R)0;
    Row<R> row, op;
    assemble_row<R>(k, N, omega, idzm, dz, idz, idzp, Wt[k], Wb[k], Wn, kap, pen, bdt, row, &op);
    R ax[2][2] = {{0, 0}, {0, 0}};  // bdt A x0 of both fields
    if (x0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const R* xt = x0[2 * q];
        const R* xb = x0[2 * q + 1];
        R a0 = op.D[0][0] * xt[k] + op.D[0][1] * xb[k], a1 = op.D[1][0] * xt[k] + op.D[1][1] * xb[k];
        if (k > 0) {
          a0 += op.L[0][0] * xt[k - 1] + op.L[0][1] * xb[k - 1];
          a1 += op.L[1][0] * xt[k - 1] + op.L[1][1] * xb[k - 1];
        }
        if (k + 1 < N) {
          a0 += op.U[0][0] * xt[k + 1] + op.U[0][1] * xb[k + 1];
          a1 += op.U[1][0] * xt[k + 1] + op.U[1][1] * xb[k + 1];
        }
        ax[q][0] = bdt * a0;
        ax[q][1] = bdt * a1;
      }
    }
    R Dp[2][2];
    Dp[0][0] = row.D[0][0] - (row.L[0][0] * c00 + row.L[0][1] * c10);
    Dp[0][1] = row.D[0][1] - (row.L[0][0] * c01 + row.L[0][1] * c11);
    Dp[1][0] = row.D[1][0] - (row.L[1][0] * c00 + row.L[1][1] * c10);
    Dp[1][1] = row.D[1][1] - (row.L[1][0] * c01 + row.L[1][1] * c11);
    R Di[2][2];
    inv2<R>(Dp, Di);
    R* bt[2] = {b0t, b1t};
    R* bb[2] = {b0b, b1b};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const R y0 = (bt[q][k] + ax[q][0]) - (row.L[0][0] * z[q][0] + row.L[0][1] * z[q][1]);
      const R y1 = (bb[q][k] + ax[q][1]) - (row.L[1][0] * z[q][0] + row.L[1][1] * z[q][1]);
      z[q][0] = Di[0][0] * y0 + Di[0][1] * y1;
      z[q][1] = Di[1][0] * y0 + Di[1][1] * y1;
      bt[q][k] = z[q][0];
      bb[q][k] = z[q][1];
    }
    c00 = Di[0][0] * row.U[0][0] + Di[0][1] * row.U[1][0];
    c01 = Di[0][0] * row.U[0][1] + Di[0][1] * row.U[1][1];
    c10 = Di[1][0] * row.U[0][0] + Di[1][1] * row.U[1][0];
    c11 = Di[1][0] * row.U[0][1] + Di[1][1] * row.U[1][1];
    C0[k] = c00; C1[k] = c01; C2[k] = c10; C3[k] = c11;
    idzm = idz;
    dz = dzp;
    idz = idzp;
  }
  R* bt[2] = {b0t, b1t};
  R* bb[2] = {b0b, b1b};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    R y0 = z[q][0], y1 = z[q][1];
    for (int k = N - 2; k >= 0; --k) {
      const R n0 = bt[q][k] - (C0[k] * y0 + C1[k] * y1);
      const R n1 = bb[q][k] - (C2[k] * y0 + C3[k] * y1);
      bt[q][k] = n0;
      bb[q][k] = n1;
      y0 = n0;
      y1 = n1;
    }
    if (x0) {
      for (int k = 0; k < N; ++k) {
        bt[q][k] += x0[2 * q][k];
        bb[q][k] += x0[2 * q + 1][k];
      }
    }
  }
}

}  // namespace slim
