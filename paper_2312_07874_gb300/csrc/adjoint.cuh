// Device functions of the vector-Jacobian product (residual adjoint and projection
// adjoint kernels in kernels.cu): the adjoint of the two-point flux, of the interface
// flux, of the entropy-variable maps, and the shared-memory layout of the residual
// adjoint.  Kept apart from device.cuh so that the forward kernels do not depend on it.
#pragma once

#include "device.cuh"

namespace esd {

// The tables hold n/2.  The pair adjoint's outputs are bilinear in the direction and the
// cotangent F_b, so the residual adjoint keeps its cotangents r_b, h_b doubled instead and
// uses n/2 as stored: the same values (scaling by 2 is exact), D multiplies fewer per pair.
template <int D>
__device__ __forceinline__ void load_dir(const double* base, int slot, int T, int t, double* n) {
#pragma unroll
  for (int k = 0; k < D; ++k) n[k] = base[(slot * D + k) * T + t];
}

// ---------------------------------------------------------------------------
// Vector-Jacobian product (reverse mode, hand-derived; not in the paper)
//
// Per-node cotangents are carried for the primitive triple q = (rho, v, p); the
// derived fields beta = rho/p, ln rho, ln beta are functions of q and their
// cotangents are folded back inside the pair adjoint.
// ---------------------------------------------------------------------------

// Adjoint of the directional flux, differentiating exactly what ec_flux_fast evaluates
// (same branch decisions, same series), without divisions: reciprocals from the MUFU
// estimate plus Newton steps, as in the forward.
//   rho_ln: series branch s G(u), u = (d/s)^2, G = 1/2 - u/6 - 2u^2/45 - 22u^3/945,
//           d/da = G - 4 f b G'(u)/s, d/db = G + 4 f a G'(u)/s   (f = d/s, s = a+b, d = b-a);
//           direct branch m = d/(ln b - ln a), d/da = (m/a - 1)/(ln b - ln a),
//           d/db = (1 - m/b)/(ln b - ln a).
//   1/beta_ln: series branch H(u)/s, H = 2 + 2u/3 + 2u^2/5 + 2u^3/7,
//           d/da = -(H + 4 f b H'/s)/s^2, d/db = -(H - 4 f a H'/s)/s^2;
//           direct branch i = (ln b - ln a)/d, d/da = (i - 1/a)/d, d/db = (1/b - i)/d.
// The beta cotangent goes to (rho, p) through beta = rho/p.
// Adds (d F/d qL)^T Fb to qL and (d F/d qR)^T Fb to qR, q = (rho, v, p), F = f#(L, R, n);
// ipL, ipR = 1/p of the two states.
template <int D>
__device__ __forceinline__ void ec_flux_adj(const NodeState<D>& L, const NodeState<D>& R, const double* n,
                                            double inv_gm1, const double* Fb, double* qL, double* qR, double ipL,
                                            double ipR) {
  const unsigned active = __activemask();
  const double s1 = L.rho + R.rho, d1 = R.rho - L.rho;
  const double r1 = rcp_nr<1>(s1), f1 = d1 * r1, u1 = f1 * f1;
  const bool ser1 = below_logmean_cutoff(u1);
  const double G = fma(u1, fma(u1, fma(u1, -22.0 / 945.0, -2.0 / 45.0), -1.0 / 6.0), 0.5);
  // 4 G'(u) with the factor 4 in the coefficients (exact: a power of two)
  const double Gp4 = fma(u1, fma(u1, 4.0 * (-22.0 / 315.0), 4.0 * (-4.0 / 45.0)), 4.0 * (-1.0 / 6.0));
  const double t1 = f1 * r1 * Gp4;
  double rl = s1 * G, dra = fma(-t1, R.rho, G), drb = fma(t1, L.rho, G);
  if (__any_sync(active, !ser1)) {
    const double rln = rcp_nr<2>(R.lrho - L.lrho), m = d1 * rln;
    const double ia = rcp_nr<2>(L.rho), ibb = rcp_nr<2>(R.rho);
    if (!ser1) {
      rl = m;
      dra = fma(m, ia, -1.0) * rln;
      drb = fma(-m, ibb, 1.0) * rln;
    }
  }
  const double s2 = L.beta + R.beta, d2 = R.beta - L.beta;
  const double r2 = rcp_nr<2>(s2), f2 = d2 * r2, u2 = f2 * f2;
  const bool ser2 = below_logmean_cutoff(u2);
  const double H = fma(u2, fma(u2, fma(u2, 2.0 / 7.0, 2.0 / 5.0), 2.0 / 3.0), 2.0);
  const double Hp4 = fma(u2, fma(u2, 4.0 * (6.0 / 7.0), 4.0 * (4.0 / 5.0)), 4.0 * (2.0 / 3.0));   // 4 H'(u)
  const double t2 = f2 * r2 * Hp4, r2s = r2 * r2;
  double ib = r2 * H, dia = -r2s * fma(t2, R.beta, H), dib = -r2s * fma(-t2, L.beta, H);
  if (__any_sync(active, !ser2)) {
    const double rd = rcp_nr<2>(d2), m = (R.lbeta - L.lbeta) * rd;
    const double ia = rcp_nr<2>(L.beta), ibb = rcp_nr<2>(R.beta);
    if (!ser2) {
      ib = m;
      dia = rd * (m - ia);
      dib = rd * (ibb - m);
    }
  }
  double vnL = 0.0, vnR = 0.0, vv = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vnL = fma(n[k], L.v[k], vnL);
    vnR = fma(n[k], R.v[k], vnR);
    vv = fma(L.v[k], R.v[k], vv);
  }
  const double hvn = 0.5 * (vnL + vnR);
  const double frho = rl * hvn, hfrho = 0.5 * frho;
  const double FE = Fb[D + 1];
  double frho_b = fma(FE, fma(0.5, vv, inv_gm1 * ib), Fb[0]);
  double pavg_b = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    frho_b = fma(Fb[1 + k], 0.5 * (L.v[k] + R.v[k]), frho_b);
    pavg_b = fma(Fb[1 + k], n[k], pavg_b);
  }
  const double hFE = 0.5 * FE;
  const double vv_b = hFE * frho;
  const double ib_b = FE * frho * inv_gm1;
  double pL_b = fma(0.5, pavg_b, hFE * vnR);
  double pR_b = fma(0.5, pavg_b, hFE * vnL);
  const double rl_b = frho_b * hvn;
  const double hfr = 0.5 * frho_b * rl;
  const double vnL_b = fma(hFE, R.p, hfr);
  const double vnR_b = fma(hFE, L.p, hfr);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double vs_b = Fb[1 + k] * hfrho;
    qL[1 + k] += fma(vnL_b, n[k], fma(vv_b, R.v[k], vs_b));
    qR[1 + k] += fma(vnR_b, n[k], fma(vv_b, L.v[k], vs_b));
  }
  // beta = rho / p: d beta/d rho = 1/p, d beta/d p = -beta/p
  const double gL = ib_b * dia * ipL, gR = ib_b * dib * ipR;
  qL[0] += fma(rl_b, dra, gL);
  qR[0] += fma(rl_b, drb, gR);
  qL[D + 1] += fma(-gL, L.beta, pL_b);
  qR[D + 1] += fma(-gR, R.beta, pR_b);
}

// adjoint of the interface flux f* = f#(q-, q+, n) - lambda/2 (U+ - U-) (Eq. (num_flux),
// Eq. (wave_speed)); max/|.| use the sub-gradient with ties to the interior side.
template <int D>
__device__ __forceinline__ void iface_adj(const NodeState<D>& L, const NodeState<D>& R, const double* n,
                                          double inv_gm1, double cL, double cR, int lf, const double* fb,
                                          double* qL, double* qR) {
  ec_flux_adj<D>(L, R, n, inv_gm1, fb, qL, qR, rcp_nr<2>(L.p), rcp_nr<2>(R.p));
  if (!lf) return;
  constexpr int NC = D + 2;
  double vnL = 0.0, vnR = 0.0, vvL = 0.0, vvR = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vnL = fma(L.v[k], n[k], vnL);
    vnR = fma(R.v[k], n[k], vnR);
    vvL = fma(L.v[k], L.v[k], vvL);
    vvR = fma(R.v[k], R.v[k], vvR);
  }
  const double lam = fmax(fabs(vnL), fabs(vnR)) + fmax(cL, cR);
  double UL[NC], UR[NC];
  UL[0] = L.rho;
  UR[0] = R.rho;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    UL[1 + k] = L.rho * L.v[k];
    UR[1 + k] = R.rho * R.v[k];
  }
  UL[D + 1] = L.p * inv_gm1 + 0.5 * L.rho * vvL;
  UR[D + 1] = R.p * inv_gm1 + 0.5 * R.rho * vvR;
  double lam_b = 0.0;
#pragma unroll
  for (int c = 0; c < NC; ++c) lam_b -= 0.5 * fb[c] * (UR[c] - UL[c]);
  // U(q) adjoints with U+_b = -lam/2 fb, U-_b = +lam/2 fb
  const double hl = 0.5 * lam;
  {
    double ER = -hl * fb[D + 1], EL = hl * fb[D + 1];
    qR[0] += -hl * fb[0] + 0.5 * vvR * ER;
    qL[0] += hl * fb[0] + 0.5 * vvL * EL;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      qR[0] += -hl * fb[1 + k] * R.v[k];
      qL[0] += hl * fb[1 + k] * L.v[k];
      qR[1 + k] += -hl * fb[1 + k] * R.rho + ER * R.rho * R.v[k];
      qL[1 + k] += hl * fb[1 + k] * L.rho + EL * L.rho * L.v[k];
    }
    qR[D + 1] += ER * inv_gm1;
    qL[D + 1] += EL * inv_gm1;
  }
  if (fabs(vnL) >= fabs(vnR)) {
    const double g = lam_b * (vnL > 0.0 ? 1.0 : (vnL < 0.0 ? -1.0 : 0.0));
#pragma unroll
    for (int k = 0; k < D; ++k) qL[1 + k] += g * n[k];
  } else {
    const double g = lam_b * (vnR > 0.0 ? 1.0 : (vnR < 0.0 ? -1.0 : 0.0));
#pragma unroll
    for (int k = 0; k < D; ++k) qR[1 + k] += g * n[k];
  }
  if (cL >= cR) {
    qL[D + 1] += lam_b * cL / (2.0 * L.p);
    qL[0] -= lam_b * cL / (2.0 * L.rho);
  } else {
    qR[D + 1] += lam_b * cR / (2.0 * R.p);
    qR[0] -= lam_b * cR / (2.0 * R.rho);
  }
}

// (dq/dw)^T qb for q = (rho, v, p) = U(w) written through the entropy variables:
// b = -w_last, v = w_v/b, ln rho = -(s + ln b)/(gamma-1), s = gamma - (gamma-1)(w_1 + b|v|^2/2), p = rho/b.
template <int D>
__device__ __forceinline__ void qbar_to_wbar(const NodeState<D>& s, const double* qb, double gamma, double* wb) {
  double vv = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) vv = fma(s.v[k], s.v[k], vv);
  const double b = s.beta;
  const double Lb = qb[0] * s.rho + qb[D + 1] * s.p;   // cotangent of ln rho
  double bb = -qb[D + 1] * s.p / b + Lb * (-0.5 * vv - 1.0 / ((gamma - 1.0) * b));
#pragma unroll
  for (int k = 0; k < D; ++k) {
    bb -= qb[1 + k] * s.v[k] / b;
    wb[1 + k] = Lb * s.v[k] + qb[1 + k] / b;
  }
  wb[0] = Lb;
  wb[D + 1] = -bb;
}

// (d W/du)^T g for the entropy variables of the conservative state u (Section 7.1).
template <int D>
__device__ __forceinline__ void entropy_vars_adj(const double* u, double gamma, const double* g, double* ub) {
  const double rho = u[0];
  double v[D], vv = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = u[1 + k] / rho;
    vv = fma(v[k], v[k], vv);
  }
  const double p = (gamma - 1.0) * (u[D + 1] - 0.5 * rho * vv);
  const double b = rho / p;
  double bb = -g[D + 1] - 0.5 * vv * g[0];
  double vb[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    bb += g[1 + k] * v[k];
    vb[k] = g[1 + k] * b - g[0] * b * v[k];
  }
  const double sb = -g[0] / (gamma - 1.0);
  const double pb = sb / p - bb * b / p;
  const double rb = -sb * gamma / rho + bb / p;
  ub[D + 1] = pb * (gamma - 1.0);
  double r = rb + pb * (gamma - 1.0) * 0.5 * vv;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ub[1 + k] = vb[k] / rho - pb * (gamma - 1.0) * v[k];
    r -= vb[k] * v[k] / rho;
  }
  ub[0] = r;
}

// out (nodal, += sign * R^T in) with scratch y (tetrahedra)
template <int D>
__device__ void apply_RT(const DevRef& R, const Tile& t, int in, int y, int out, int nc, double sign) {
  const int n = R.n, Nq = R.Nq, Nfn = R.Nfn, Nqf = R.Nqf;
  if (D == 3) {
    for (int idx = threadIdx.x; idx < t.E * nc * n * n; idx += blockDim.x) {
      int e = idx / (nc * n * n), rr = idx % (nc * n * n), c = rr / (n * n), ab = rr % (n * n);
      int a = ab % n, b2 = ab / n;
      const double* hh = t.base + e * t.pe + in + c * Nfn + 3 * Nqf;
      double s = 0.0;
      for (int bp = 0; bp < n; ++bp) s = fma(R.L2J[bp * n + b2], hh[a + n * bp], s);
      t.base[e * t.pe + y + rr] = s;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < t.E * nc * Nq; idx += blockDim.x) {
    int e = idx / (nc * Nq), rr = idx % (nc * Nq), c = rr / Nq, v = rr % Nq;
    const double* hh = t.base + e * t.pe + in + c * Nfn;
    double s;
    if (D == 2) {
      int a = v % n, b = v / n;
      s = R.l2m[b] * hh[a] + R.l1p[a] * hh[Nqf + b] + R.l1m[a] * hh[2 * Nqf + b];
    } else {
      int a = v % n, b = (v / n) % n, c3 = v / (n * n);
      const double* yy = t.base + e * t.pe + y + c * n * n;
      s = R.l2m[b] * hh[a + n * c3] + R.l1p[a] * hh[Nqf + b + n * c3] + R.l1m[a] * hh[2 * Nqf + b + n * c3] +
          R.l3m[c3] * yy[a + n * b];
    }
    t.base[e * t.pe + out + rr] += sign * s;
  }
  __syncthreads();
}

// Residual adjoint: cot (cotangent of d u~/dt) -> per-node cotangents of q at own volume
// and facet nodes (qbar [E][NQ][Ntot]) and, per facet node, the cotangent of the
// neighbour's state through this element's interface flux (qext [E][NQ][Nfn]).
struct AdjLayout {
  int oReg, oM, oS1, oS2, oSv, oSf, oIp, oRb, oHb, oQv, oQf, oQvx, oQf4x, pe;
  int glob;   // 1: q_b accumulated in the global output instead of shared memory
  int conc;   // 1: the D line families run concurrently, families 1.. into their own
              //    volume-node cotangent copies at oQvx and (tetrahedra) facet-4 node
              //    cotangent copies at oQf4x, summed in a fixed order after
  // oIp: 1/p of every node ([Nq + Nfn] after the states), or -1 where it does not fit
  // (then computed per pair)
};

// Shared memory per element of the residual adjoint.  The per-node cotangents q_b are
// accumulated in shared memory when everything fits in one CTA's 227 KB; otherwise
// (tetrahedra of the highest degrees) they are accumulated in place in the global output
// q_b (`glob`).
constexpr int kAdjSmemBudget = 227 * 1024;

template <int D>
__host__ __device__ inline AdjLayout adj_layout_with(int Nq, int Nfn, int Np, int n, bool glob, bool ip,
                                                     bool conc) {
  constexpr int NC = D + 2, NF = D + 5, NQ = D + 2;
  AdjLayout L;
  L.oReg = 0;
  L.oS1 = 0;
  L.oS2 = NC * Nq;
  L.oM = 2 * NC * Nq;
  L.oSv = 0;
  L.oSf = NF * Nq;
  L.oIp = ip ? NF * (Nq + Nfn) : -1;
  int r0 = 2 * NC * Nq + NC * Np;
  const int rs = (NF + (ip ? 1 : 0)) * (Nq + Nfn);
  if (rs > r0) r0 = rs;
  L.oRb = r0;
  L.oHb = L.oRb + NC * Nq;
  L.glob = glob ? 1 : 0;
  L.conc = (!glob && conc) ? 1 : 0;
  L.oQvx = L.oQf4x = -1;
  if (!glob) {
    L.oQv = L.oHb + NC * Nfn;
    L.oQf = L.oQv + NQ * Nq;
    L.pe = L.oQf + NQ * Nfn;
    if (L.conc) {
      L.oQvx = L.pe;
      L.pe += (D - 1) * NQ * Nq;
      if (D == 3) {
        L.oQf4x = L.pe;
        L.pe += (D - 1) * NQ * n * n;
      }
    }
  } else {
    L.oQv = L.oQf = -1;
    L.pe = L.oHb + NC * Nfn;
  }
  return L;
}

// Threads of a residual-adjoint CTA of e elements: the e*T line tasks of one family,
// rounded up to whole warps, times D when the families run concurrently (family-major, so
// that no warp mixes two families' code paths).
template <int D>
__host__ __device__ inline int adj_block_threads(const AdjLayout& L, int T, int e) {
  const int per_family = ((e * T + 31) / 32) * 32;
  return L.conc ? D * per_family : per_family;
}

// The first layout that fits one CTA (and, for concurrent families, leaves room for at least
// two elements per SM): q_b in shared memory with concurrent families and 1/p, then without
// 1/p, then sequential families with and without 1/p, then q_b in global memory.
template <int D>
__host__ __device__ inline AdjLayout adj_layout(int Nq, int Nfn, int Np, int n) {
  const bool glob[6] = {false, false, false, false, true, true};
  const bool ip[6] = {true, false, true, false, true, false};
  const bool conc[6] = {true, true, false, false, false, false};
  for (int k = 0; k < 6; ++k) {
    const AdjLayout L = adj_layout_with<D>(Nq, Nfn, Np, n, glob[k], ip[k], conc[k]);
    const long long lim = conc[k] ? kAdjSmemBudget / 2 : kAdjSmemBudget;
    if ((long long)L.pe * 8 <= lim) return L;
  }
  return adj_layout_with<D>(Nq, Nfn, Np, n, true, false, false);
}

}  // namespace esd
