// The skew-symmetric nodal form of Section 4.4, Eq. (rhs_skew):
//
//   r = 1/2 sum_l ( Q^(l)T sum_m G^(l,m) f_m - sum_m G^(l,m) Q^(l) f_m )
//       - sum_zeta R^(zeta)T B^(zeta) J^zeta ( f* - 1/2 sum_m N^(zeta,m) R^(zeta) f_m )
//
// with the fluxes f_m evaluated at the nodal solution u = V u~ (no entropy projection, no
// two-point flux) and d u~/dt = M~^{-1} V^T r (Eq. (modal), weight-adjusted inverse).
// Q^(l) = W D^(l) couples only nodes on a common collapsed-coordinate line, so the volume
// term is a sum over line pairs:
//
//   r_i += sum_{j on a line through i, j != i} sum_m c^m_ij f_m(u_j),
//   c^m_ij = 1/2 sum_l ( Q^(l)_ji G_lm(x_j) - G_lm(x_i) Q^(l)_ij )   (c^m_ii = 0),
//
// with the mesh-static coefficients c^m_ij stored per element (HBM, task-fastest like the
// entropy-stable pair directions).  A line task owns one line of N nodes per phase, forms
// f_m at its nodes on the fly and accumulates its nodes' residuals in registers; it also
// owns the facet nodes attached to its line (faces 1-3: trace R f_m along the line,
// interface flux, lift; face 4 of tetrahedra: two barrier-separated steps, as in the
// entropy-stable kernel).  Two models: the compressible Euler equations (Section 7.1, the
// interface flux of Eq. (num_flux)) and scalar linear advection f_m(u) = a_m u with the
// central or upwind interface flux.  Internal to the library.
#pragma once

#include "device.cuh"

namespace esd {

struct SkewModel {
  double gamma;   // Euler (the interface flux's dissipation follows the mesh's flux choice)
  double a[3];    // advection velocity
  double sigma;   // advection: 0 central, 1 upwind
};

// f_m(u) at one node, m = 0..D-1.  NC == D + 2: Euler (Eq. (euler)); NC == 1: a_m u.
template <int D, int NC>
__device__ __forceinline__ void node_flux(const double* u, const SkewModel& P, double (&f)[D][NC]) {
  if constexpr (NC == 1) {
#pragma unroll
    for (int m = 0; m < D; ++m) f[m][0] = P.a[m] * u[0];
  } else {
    const double ir = rcp_nr<2>(u[0]);
    double v[D], mv = 0.0;   // mv = rho |v|^2
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = u[1 + k] * ir;
      mv = fma(u[1 + k], v[k], mv);
    }
    const double p = (P.gamma - 1.0) * fma(-0.5, mv, u[D + 1]);
    const double ep = u[D + 1] + p;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      f[m][0] = u[1 + m];
#pragma unroll
      for (int k = 0; k < D; ++k) f[m][1 + k] = k == m ? fma(u[1 + k], v[m], p) : u[1 + k] * v[m];
      f[m][D + 1] = v[m] * ep;
    }
  }
}

// h = B J^zeta ( f* - 1/2 sum_m n_m (R f_m) ) at facet node f of element eg, given the
// trace rf[m][c] = (R f_m)_c.  Traces of both sides are read from the mesh workspace
// (written by the trace kernel): NodeStates for Euler, field 0 for advection.
template <int D, int NC>
__device__ __forceinline__ void skew_facet_term(const DevRef& R, const DevMesh& M, const SkewModel& P,
                                                const FluxK& K, int64_t eg, int f, const double (&rf)[D][NC],
                                                double (&h)[NC]) {
  constexpr int NF = D + 5;
  const int Nq = R.Nq, Nfn = R.Nfn, Ntot = R.Ntot;
  const double bj = M.bj[eg * Nfn + f];
  double nn[D];
#pragma unroll
  for (int k = 0; k < D; ++k) nn[k] = M.nrm[(eg * D + k) * Nfn + f];
  if constexpr (NC == 1) {
    const int64_t e2 = M.nbr_e[eg * Nfn + f];
    const int f2 = M.nbr_f[eg * Nfn + f];
    const double uL = M.states[eg * NF * Ntot + Nq + f], uR = M.states[e2 * NF * Ntot + Nq + f2];
    double an = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) an = fma(P.a[k], nn[k], an);
    const double fs = 0.5 * an * (uL + uR) - 0.5 * P.sigma * fabs(an) * (uR - uL);
    double fn = 0.0;
#pragma unroll
    for (int m = 0; m < D; ++m) fn = fma(nn[m], rf[m][0], fn);
    h[0] = bj * fma(-0.5, fn, fs);
  } else {
    double F[NC];
    interface_flux<D>(M, Nq, Nfn, Ntot, eg, f, M.states + eg * NF * Ntot + Nq, K, F);   // B J f*
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double fn = 0.0;
#pragma unroll
      for (int m = 0; m < D; ++m) fn = fma(nn[m], rf[m][c], fn);
      h[c] = fma(-0.5 * bj, fn, F[c]);
    }
  }
}

template <int D, int NC>
__device__ __forceinline__ void load_u(const double* U, int Nq, int v, double (&u)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) u[c] = U[c * Nq + v];
}

// Line task t of phase ph of the skew-symmetric residual (phases as in line_task of the
// entropy-stable kernel).  U: nodal u [NC][Nq] (shared); r: [NC][Nq] (shared); e3:
// [D*NC][n^2], h4: [NC][n^2] (tetrahedra, shared); sd: this element's coefficient table.
// Every thread of the block calls this (phase 2 of tetrahedra has barriers).
template <int D, int N, int NC>
__device__ __forceinline__ void skew_line_task(int ph, int t, bool act, const DevRef& R, const DevMesh& M,
                                               const SkewModel& P, const FluxK& K, int64_t eg,
                                               const double* __restrict__ U, double* r, double* e3, double* h4,
                                               const double* __restrict__ sd) {
  const int Nq = R.Nq, Nqf = R.Nqf, T = R.T;
  int base, stride;
  if (D == 2) {
    base = ph == 0 ? N * t : t;
    stride = ph == 0 ? 1 : N;
  } else {
    if (ph == 0) { base = N * t; stride = 1; }
    else if (ph == 1) { base = (t % N) + N * N * (t / N); stride = N; }
    else { base = t; stride = N * N; }
  }
  double acc[N][NC];
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[a][c] = 0.0;
  if (act) {
    // volume line pairs: r_a += sum_m c^m_ab f_m(u_b), b != a; ordered pair (a, b) is
    // slot b (N-1) + (a < b ? a : a - 1) of the phase
    const double* cd = sd + (size_t)ph * N * (N - 1) * D * T + t;
#pragma unroll 1
    for (int b = 0; b < N; ++b) {
      double u[NC], f[D][NC];
      load_u<D, NC>(U, Nq, base + b * stride, u);
      node_flux<D, NC>(u, P, f);
#pragma unroll
      for (int a = 0; a < N; ++a) {
        if (a == b) continue;
        const int slot = b * (N - 1) + (a < b ? a : a - 1);
#pragma unroll
        for (int m = 0; m < D; ++m) {
          const double cm = cd[(slot * D + m) * T];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[a][c] = fma(cm, f[m][c], acc[a][c]);
        }
      }
    }
    // facets on this line: trace R f_m along the line, facet term, lift
    const int nfac = (ph == 0) ? 2 : (ph == 1 ? 1 : 0);
#pragma unroll 1
    for (int zz = 0; zz < nfac; ++zz) {
      const double* l = ph == 0 ? (zz == 0 ? R.l1p : R.l1m) : R.l2m;
      const int f = ph == 0 ? (1 + zz) * Nqf + t : t;
      double rf[D][NC];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int c = 0; c < NC; ++c) rf[m][c] = 0.0;
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        double u[NC], fa[D][NC];
        load_u<D, NC>(U, Nq, base + a * stride, u);
        node_flux<D, NC>(u, P, fa);
        const double la = l[a];
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int c = 0; c < NC; ++c) rf[m][c] = fma(la, fa[m][c], rf[m][c]);
      }
      double h[NC];
      skew_facet_term<D, NC>(R, M, P, K, eg, f, rf, h);
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const double la = l[a];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[a][c] = fma(-la, h[c], acc[a][c]);
      }
    }
  }
  if (D == 3 && ph == 2) {
    // face 4 (eta3 = -1): (R4 g)(a1, b') = sum_a2 L2J[b'][a2] sum_a3 l3m[a3] g(a1, a2, a3)
    const int a1 = t % N, a2 = t / N;
    if (act) {   // step 1: eta3-extrapolated fluxes of this task's line
      double e[D][NC];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int c = 0; c < NC; ++c) e[m][c] = 0.0;
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        double u[NC], fa[D][NC];
        load_u<D, NC>(U, Nq, base + a * stride, u);
        node_flux<D, NC>(u, P, fa);
        const double la = R.l3m[a];
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int c = 0; c < NC; ++c) e[m][c] = fma(la, fa[m][c], e[m][c]);
      }
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int c = 0; c < NC; ++c) e3[(m * NC + c) * Nqf + t] = e[m][c];
    }
    __syncthreads();
    if (act) {   // step 2: facet-4 node j = (a1, b' = a2) owned by this task
      double rf[D][NC];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int c = 0; c < NC; ++c) rf[m][c] = 0.0;
#pragma unroll 1
      for (int q = 0; q < N; ++q) {
        const double w = R.L2J[a2 * N + q];
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int c = 0; c < NC; ++c) rf[m][c] = fma(w, e3[(m * NC + c) * Nqf + a1 + N * q], rf[m][c]);
      }
      double h[NC];
      skew_facet_term<D, NC>(R, M, P, K, eg, 3 * Nqf + t, rf, h);
#pragma unroll
      for (int c = 0; c < NC; ++c) h4[c * Nqf + t] = h[c];
    }
    __syncthreads();
    if (act) {   // step 3: lift of facet 4 along this task's eta3-line
      double y[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = 0.0;
#pragma unroll 1
      for (int bp = 0; bp < N; ++bp) {
        const double w = R.L2J[bp * N + a2];
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c] = fma(w, h4[c * Nqf + a1 + N * bp], y[c]);
      }
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const double la = R.l3m[a];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[a][c] = fma(-la, y[c], acc[a][c]);
      }
    }
  }
  if (act) {
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int c = 0; c < NC; ++c) r[c * Nq + base + a * stride] += acc[a][c];
  }
}

// Shared memory per element of the skew-symmetric residual (doubles, even count):
//   Mod[NC*Np] | A[NC*Nq] | B[NC*Nq] | C[max(NC*Nq, (D+1)*NC*n^2 for tetrahedra)]
// u = V u~ lands in A; r accumulates in B; C holds e3/h4 during the phases and is
// transform scratch before and after them.
struct SkewLayout {
  int oMod, oA, oB, oC, pe;
};

template <int D>
__host__ __device__ inline SkewLayout skew_layout(int nc, int Nq, int Np, int n) {
  SkewLayout L;
  L.oMod = 0;
  L.oA = nc * Np;
  L.oB = L.oA + nc * Nq;
  L.oC = L.oB + nc * Nq;
  int c = nc * Nq;
  if (D == 3 && (D + 1) * nc * n * n > c) c = (D + 1) * nc * n * n;
  L.pe = L.oC + c;
  L.pe += L.pe & 1;
  return L;
}

// d u~/dt of Eq. (rhs_skew) for a tile of E elements starting at e0.
template <int D, int N, int NC>
__device__ void skew_residual_tile(const DevRef& R, const DevMesh& M, const SkewModel& P,
                                   const double* __restrict__ sdir, int64_t e0, int E, const double* __restrict__ u,
                                   double* __restrict__ dudt) {
  extern __shared__ double sm[];
  const int Nq = R.Nq, Np = R.Np, T = R.T, n = R.n;
  const SkewLayout Ly = skew_layout<D>(NC, Nq, Np, n);
  const int pe = Ly.pe;
  Tile tile{sm, pe, E};
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    const int e = idx / (NC * Np), rr = idx % (NC * Np);
    sm[e * pe + Ly.oMod + rr] = u[(e0 + e) * NC * Np + rr];
  }
  __syncthreads();
  // 1. u = V u~ into A (tetrahedra: s1 = A, s2 = B, out = A; triangles: s1 = B, out = A)
  if (D == 3)
    apply_V<D>(R, tile, Ly.oMod, Ly.oA, Ly.oB, Ly.oA, NC);
  else
    apply_V<D>(R, tile, Ly.oMod, Ly.oB, Ly.oC, Ly.oA, NC);
  for (int idx = threadIdx.x; idx < E * NC * Nq; idx += blockDim.x) {
    const int e = idx / (NC * Nq);
    sm[e * pe + Ly.oB + idx % (NC * Nq)] = 0.0;
  }
  __syncthreads();
  // 2. line tasks: volume line pairs, facet terms, lift
  {
    const FluxK K = make_fluxk(P.gamma);
    const int el = threadIdx.x / T, t = threadIdx.x % T;
    const bool act = el < E;
    const int elc = act ? el : 0;
    const int64_t eg = e0 + elc;
    const double* sd = act ? sdir + eg * (int64_t)D * T * N * (N - 1) * D : sdir;
    double* base = sm + elc * pe;
#pragma unroll 1
    for (int ph = 0; ph < D; ++ph) {
      skew_line_task<D, N, NC>(ph, t, act, R, M, P, K, eg, base + Ly.oA, base + Ly.oB, base + Ly.oC,
                               base + Ly.oC + D * NC * R.Nqf, sd);
      __syncthreads();
    }
  }
  // 3. d u~/dt = [V^T (W/J) V] (V^T r)
  apply_VT<D>(R, tile, Ly.oB, Ly.oA, Ly.oC, Ly.oMod, NC);
  apply_minv<D>(R, M, tile, e0, Ly.oMod, Ly.oA, Ly.oC, Ly.oB, Ly.oB, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    const int e = idx / (NC * Np), rr = idx % (NC * Np);
    dudt[(e0 + e) * NC * Np + rr] = sm[e * pe + Ly.oB + rr];
  }
}

// Facet traces of u = V u~ for a tile (the cross-element input of the facet terms):
// Euler: the NodeState of the trace (rho, v, p, beta, ln rho, ln beta) and the sound
// speed, stored like the entropy-stable kernel's facet states; advection: u itself.
// Shared layout per element: Mod[NC*Np] | A | B | C [NC*Nq] | F[NC*Nfn].
template <int D, int NC>
__device__ void skew_trace_tile(const DevRef& R, const DevMesh& M, const SkewModel& P, int64_t e0, int E,
                                const double* __restrict__ u) {
  extern __shared__ double sm[];
  constexpr int NF = D + 5;
  const int Np = R.Np, Nq = R.Nq, Nfn = R.Nfn, Ntot = R.Ntot;
  const int oM = 0, oA = NC * Np, oB = oA + NC * Nq, oC = oB + NC * Nq, oF = oC + NC * Nq;
  const int pe = oF + NC * Nfn;
  Tile t{sm, pe, E};
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    const int e = idx / (NC * Np), rr = idx % (NC * Np);
    sm[e * pe + oM + rr] = u[(e0 + e) * NC * Np + rr];
  }
  __syncthreads();
  apply_V<D>(R, t, oM, oB, oC, oA, NC);
  apply_R<D>(R, t, oA, oB, oF, NC);
  int lbad = 0;
  const double sqrt_gamma = sqrt(P.gamma);
  for (int idx = threadIdx.x; idx < E * Nfn; idx += blockDim.x) {
    const int e = idx / Nfn, f = idx % Nfn;
    const int64_t eg = e0 + e;
    double* S = M.states + eg * NF * Ntot + Nq;
    if constexpr (NC == 1) {
      S[f] = sm[e * pe + oF + f];
    } else {
      double w[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) w[c] = sm[e * pe + oF + c * Nfn + f];
      NodeState<D> st;
      st.rho = w[0];
      const double ir = rcp_nr<2>(w[0]);
      double mv = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        st.v[k] = w[1 + k] * ir;
        mv = fma(w[1 + k], st.v[k], mv);
      }
      st.p = (P.gamma - 1.0) * fma(-0.5, mv, w[D + 1]);
      if (!finite_pos(st.rho) || !finite_pos(st.p)) {
        lbad = 1;
        st.rho = st.p = 1.0;   // keep the arithmetic finite; reported as non-admissible
      }
      st.beta = st.rho * rcp_nr<2>(st.p);
      st.lrho = log_tab(st.rho, R.mtab);
      st.lbeta = log_tab(st.beta, R.mtab);
      store_state<D>(S, Ntot, f, st);
      M.cfac[eg * Nfn + f] = sqrt_gamma * rsqrt_nr(st.beta);   // sqrt(gamma p / rho)
    }
  }
  if (lbad) atomicOr(M.flag, kFlagState);
}

template <int D, int NC>
__global__ void skew_trace_kernel(DevRef R, DevMesh M, SkewModel P, int epc, const double* __restrict__ u) {
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  skew_trace_tile<D, NC>(R, M, P, e0, E, u);
}

template <int D, int N, int NC>
__global__ void skew_residual_kernel(DevRef R, DevMesh M, SkewModel P, const double* __restrict__ sdir, int epc,
                                     const double* __restrict__ u, double* __restrict__ dudt) {
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  skew_residual_tile<D, N, NC>(R, M, P, sdir, e0, E, u, dudt);
}

}  // namespace esd
