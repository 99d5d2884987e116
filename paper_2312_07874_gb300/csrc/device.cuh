// Device-side building blocks shared by the kernel translation units: per-node
// states, the two-point flux, table-driven log/exp, sum-factorised transforms, the
// projection and residual tiles (the adjoint pieces are in adjoint.cuh).  Internal to
// the library.
#pragma once

#include <cmath>
#include <cstdint>

#include "esd_internal.h"

namespace esd {

// ---------------------------------------------------------------------------
// Per-node state and the two-point flux (Section 7.2)
// ---------------------------------------------------------------------------
template <int D>
struct NodeState {
  double rho, v[D], p, beta, lrho, lbeta;
};

// fields are stored SoA: S[field*stride + idx]
template <int D>
__device__ __forceinline__ NodeState<D> load_state(const double* S, int stride, int idx) {
  NodeState<D> s;
  s.rho = S[idx];
#pragma unroll
  for (int k = 0; k < D; ++k) s.v[k] = S[(1 + k) * stride + idx];
  s.p = S[(D + 1) * stride + idx];
  s.beta = S[(D + 2) * stride + idx];
  s.lrho = S[(D + 3) * stride + idx];
  s.lbeta = S[(D + 4) * stride + idx];
  return s;
}

// ---------------------------------------------------------------------------
// The directional entropy-conservative flux f#(U^-, U^+, n) = sum_m n_m f_m^#
// (Eq. (ranocha_flux); the printed one-half is read as multiplying v^-.v^+ alone, since
// the printed placement would make the flux inconsistent, so the energy component is
// rho_ln {{v}}.n (v^-.v^+/2 + 1/((gamma-1) {{rho/p}}_ln)) + (p^- v^+.n + p^+ v^-.n)/2),
// evaluated FP64-lean for the pair loops:
//
// * Reciprocals come from the MUFU approximation (rcp.approx.ftz.f64, another pipe)
//   refined by Newton-Raphson steps x <- x + x (1 - a x), each of which squares the
//   relative error: one step is enough where the result only enters a series
//   correction, two steps give full double precision.
// * The log-mean branch is chosen by an integer comparison of the bit patterns of
//   u >= 0 and 1e-4 (same decision as the floating-point comparison, off the FP64 pipe).
// * Logarithmic means {{a}}_ln = (b-a)/(ln b - ln a) use the per-node logarithms; for
//   u = f^2 < 1e-4, f = (b-a)/(b+a), the series of ln(b/a) = 2 artanh f gives
//   {{a}}_ln = (a+b)/(2F(u)), F(u) = artanh(f)/f = 1 + u/3 + u^2/5 + u^3/7 + ...
// * In the series branch, rho_ln = (a+b) G(u) with G = 1/(2F(u)) expanded to the same
//   order, G = 1/2 - u/6 - 2u^2/45 - 22u^3/945 (differs from (a+b)/(2F) by < 1e-17
//   relative for u < 1e-4); 1/((gamma-1) beta_ln) = K(u)/(a+b) with K = 2F/(gamma-1).
// * Pair directions are stored halved (n/2), which absorbs the arithmetic means.
// ---------------------------------------------------------------------------
// 1/sqrt(a), a > 0 normal: hardware estimate, then two Newton steps y <- y (3 - a y^2)/2
__device__ __forceinline__ double rsqrt_nr(double a) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double h = 0.5 * a * y;
    y = fma(y, fma(-h, y, 0.5), y);
  }
  return y;
}

template <int NR>
__device__ __forceinline__ double rcp_nr(double a) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(a));
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const double e = fma(-a, x, 1.0);
    x = fma(x, e, x);
  }
  return x;
}

__device__ __forceinline__ bool below_logmean_cutoff(double u) {
  return __double_as_longlong(u) < 0x3F1A36E2EB1C432DLL;   // bit pattern of 1.0e-4
}

// Table-driven logarithm (after Tang, 1990): x = 2^k m, F = 1 + j/128 nearest to m,
// ln x = k ln2 + ln F + log1p((m - F)/F), with log1p(r) = r + r^2 q(r) to degree 7
// (|r| <= 2^-8).  For positive normal x; ~1 ulp.
__device__ __forceinline__ double log_tab(double x, const double* __restrict__ T) {
  const long long b = __double_as_longlong(x);
  const long long k = (b >> 52) - 1023;
  const long long mb = b & 0x000FFFFFFFFFFFFFLL;
  const int j = (int)((mb + (1LL << 44)) >> 45);
  const double m = __longlong_as_double(mb | 0x3FF0000000000000LL);
  const double F = __longlong_as_double(0x3FF0000000000000LL + ((long long)j << 45));
  const double r = (m - F) * __ldg(T + j);
  const double r2 = r * r;
  const double q = fma(r, fma(r, fma(r, fma(r, fma(r, 1.0 / 7.0, -1.0 / 6.0), 1.0 / 5.0), -1.0 / 4.0), 1.0 / 3.0),
                       -0.5);
  const double kd = __longlong_as_double(0x4338000000000000LL + k) - 6755399441055744.0;
  const double hi = fma(kd, __ldg(T + 451), __ldg(T + 129 + j));
  const double lo = fma(kd, __ldg(T + 452), __ldg(T + 258 + j));
  return hi + (lo + fma(r2, q, r));
}

// Table-driven exponential (after Tang, 1989): x = (32 m + j) ln2/32 + r, |r| <= ln2/64,
// e^x = 2^m 2^(j/32) (1 + expm1(r)), expm1 to degree 6.  For results in the normal range.
__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ T) {
  const double magic = 6755399441055744.0;   // 1.5 * 2^52
  const double t = fma(x, __ldg(T + 455), magic);
  const long long n = __double_as_longlong(t) - 0x4338000000000000LL;
  const double nd = t - magic;
  double r = fma(-nd, __ldg(T + 453), x);
  r = fma(-nd, __ldg(T + 454), r);
  const int j = (int)(n & 31);
  const long long me = n >> 5;
  const double r2 = r * r;
  const double p = fma(r2, fma(r, fma(r, fma(r, fma(r, 1.0 / 720.0, 1.0 / 120.0), 1.0 / 24.0), 1.0 / 6.0), 0.5), r);
  const double s = __ldg(T + 387 + j);
  const double res = s + fma(s, p, __ldg(T + 419 + j));
  return __longlong_as_double(__double_as_longlong(res) + (me << 52));
}

struct FluxK {
  double inv_gm1;
  double k0, k1, k2, k3;   // (2, 2/3, 2/5, 2/7) / (gamma - 1)
};

__device__ __forceinline__ FluxK make_fluxk(double gamma) {
  FluxK K;
  K.inv_gm1 = 1.0 / (gamma - 1.0);
  K.k0 = 2.0 * K.inv_gm1;
  K.k1 = (2.0 / 3.0) * K.inv_gm1;
  K.k2 = (2.0 / 5.0) * K.inv_gm1;
  K.k3 = (2.0 / 7.0) * K.inv_gm1;
  return K;
}

// F = f#(L, R, 2 nh): the directional flux for the direction 2*nh.
template <int D>
__device__ __forceinline__ void ec_flux_fast(const NodeState<D>& L, const NodeState<D>& R, const double* nh,
                                             const FluxK& K, double* F) {
  // {{rho}}_ln.  The direct (log) formula is evaluated only when some lane of the warp
  // needs it: for smooth states whole warps stay on the series, and the compiler cannot
  // turn the rare branch into always-executed predicated code.
  const unsigned active = __activemask();
  const double s1 = L.rho + R.rho, d1 = R.rho - L.rho;
  const double f1 = d1 * rcp_nr<1>(s1), u1 = f1 * f1;
  const bool ser1 = below_logmean_cutoff(u1);
  double rho_ln = s1 * fma(u1, fma(u1, fma(u1, -22.0 / 945.0, -2.0 / 45.0), -1.0 / 6.0), 0.5);
  if (__any_sync(active, !ser1)) {
    const double direct = d1 * rcp_nr<2>(R.lrho - L.lrho);
    rho_ln = ser1 ? rho_ln : direct;
  }
  // 1 / ((gamma-1) {{rho/p}}_ln)
  const double s2 = L.beta + R.beta, d2 = R.beta - L.beta;
  const double r2 = rcp_nr<2>(s2);
  const double f2 = d2 * r2, u2 = f2 * f2;
  const bool ser2 = below_logmean_cutoff(u2);
  double ibc = r2 * fma(u2, fma(u2, fma(u2, K.k3, K.k2), K.k1), K.k0);
  if (__any_sync(active, !ser2)) {
    const double direct = K.inv_gm1 * (R.lbeta - L.lbeta) * rcp_nr<2>(d2);
    ibc = ser2 ? ibc : direct;
  }
  double vnL = 0.0, vnR = 0.0, vv = 0.0;   // vn = v.n/2
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vnL = fma(nh[k], L.v[k], vnL);
    vnR = fma(nh[k], R.v[k], vnR);
    vv = fma(L.v[k], R.v[k], vv);
  }
  const double frho = rho_ln * (vnL + vnR);
  const double hf = 0.5 * frho, ps = L.p + R.p;
  F[0] = frho;
#pragma unroll
  for (int k = 0; k < D; ++k) F[1 + k] = fma(hf, L.v[k] + R.v[k], ps * nh[k]);
  F[D + 1] = fma(frho, fma(0.5, vv, ibc), fma(L.p, vnR, R.p * vnL));
}

// ---------------------------------------------------------------------------
// Sum-factorised PKD transforms (Section 5.2) on a tile of E elements.
// Buffers are per element with stride `pe` (doubles); each holds N_c variables.
// ---------------------------------------------------------------------------
struct Tile {
  double* base;   // shared memory
  int pe;         // doubles per element
  int E;          // elements in this tile
};

// A contraction output: dst = sum_{j < len} c[j cs] x[j xs].
struct Dot {
  const double* c;
  int cs;
  const double* x;
  int xs;
  double* dst;
};

// Evaluates the tot outputs described by setup(idx) (all of length len), four per thread at
// a time: each output is a chain of dependent FMAs (a 64-cycle latency apiece on this
// FP64 pipe), and four independent chains interleave.  The summation order of every output
// is the plain j = 0, 1, ... order.
template <class F>
__device__ __forceinline__ void contract4(int tot, int len, F&& setup) {
  const int bd = blockDim.x;
  for (int i0 = threadIdx.x; i0 < tot; i0 += 4 * bd) {
    Dot d[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = i0 + u * bd;
      ok[u] = idx < tot;
      d[u] = setup(ok[u] ? idx : i0);
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < len; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(d[u].c[j * d[u].cs], d[u].x[j * d[u].xs], acc[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) *d[u].dst = acc[u];
  }
}

// out = V in  (modal -> nodal), using scratch s1 (and s2 for tetrahedra).  All buffers
// distinct, except that for tetrahedra `out` may equal s1.
// The stages whose sums run over a triangular index range are enumerated with the
// (element, variable) index fastest and, for the alpha3 stage, the (alpha1, alpha2)
// pairs by decreasing sum length: neighbouring threads then run loops of equal length
// (an FP64 instruction costs the same whatever the number of active lanes).
template <int D>
__device__ void apply_V(const DevRef& R, const Tile& t, int in, int s1, int s2, int out, int nc) {
  const int n = R.n, p = R.p;
  const int EV = t.E * nc;
  if (D == 2) {
    int rows = (p + 1) * n, tot = t.E * nc * rows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      int row = idx / EV, ev = idx % EV, var = ev % nc, e = ev / nc;
      int a1 = row / n, c2 = row % n;
      const double* x = t.base + e * t.pe + in + var * R.Np;
      int m0 = R.off1[a1];
      double acc = 0.0;
      for (int a2 = 0; a2 <= p - a1; ++a2) acc = fma(R.psi2[(m0 + a2) * n + c2], x[m0 + a2], acc);
      t.base[e * t.pe + s1 + var * R.Nq + row] = acc;
    }
    __syncthreads();
    rows = R.Nq;
    tot = t.E * nc * rows;
    contract4(tot, p + 1, [&](int idx) {
      const int v = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int c1 = v % n, c2 = v / n;
      return Dot{R.psi1 + c1, n, t.base + e * t.pe + s1 + var * R.Nq + c2, n, t.base + e * t.pe + out + var * R.Nq + v};
    });
    __syncthreads();
  } else {
    // stage 1: contract alpha3 -> [s12][c3]   (into s1)
    int rows = R.S12 * n, tot = t.E * nc * rows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int rank = idx / EV, ev = idx % EV, var = ev % nc, e = ev / nc;
      const int s = R.s12len[rank / n], c3 = rank % n, row = s * n + c3;
      int a1 = R.s12a1[s], a2 = s - R.off1[a1], m0 = R.moff[s];
      const double* x = t.base + e * t.pe + in + var * R.Np;
      double acc = 0.0;
      for (int a3 = 0; a3 <= p - a1 - a2; ++a3) acc = fma(R.psi3[(m0 + a3) * n + c3], x[m0 + a3], acc);
      t.base[e * t.pe + s1 + var * R.Nq + row] = acc;
    }
    __syncthreads();
    // stage 2: contract alpha2 -> [a1][c2][c3]  (into s2)
    rows = (p + 1) * n * n;
    tot = t.E * nc * rows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      int row = idx / EV, ev = idx % EV, var = ev % nc, e = ev / nc;
      int c3 = row % n, c2 = (row / n) % n, a1 = row / (n * n);
      const double* y = t.base + e * t.pe + s1 + var * R.Nq;
      int s0 = R.off1[a1];
      double acc = 0.0;
      for (int a2 = 0; a2 <= p - a1; ++a2) acc = fma(R.psi2[(s0 + a2) * n + c2], y[(s0 + a2) * n + c3], acc);
      t.base[e * t.pe + s2 + var * R.Nq + row] = acc;
    }
    __syncthreads();
    // stage 3: contract alpha1 -> nodal
    rows = R.Nq;
    tot = t.E * nc * rows;
    contract4(tot, p + 1, [&](int idx) {
      const int v = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int c1 = v % n, c2 = (v / n) % n, c3 = v / (n * n);
      return Dot{R.psi1 + c1, n, t.base + e * t.pe + s2 + var * R.Nq + c2 * n + c3, n * n,
                 t.base + e * t.pe + out + var * R.Nq + v};
    });
    __syncthreads();
  }
}

// out = V^T in (nodal -> modal) with scratch s1, s2 (nodal-sized).
template <int D>
__device__ void apply_VT(const DevRef& R, const Tile& t, int in, int s1, int s2, int out, int nc) {
  const int n = R.n, p = R.p;
  if (D == 2) {
    int rows = (p + 1) * n, tot = t.E * nc * rows;
    contract4(tot, n, [&](int idx) {
      const int row = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int a1 = row / n, c2 = row % n;
      return Dot{R.psi1 + a1 * n, 1, t.base + e * t.pe + in + var * R.Nq + n * c2, 1,
                 t.base + e * t.pe + s1 + var * R.Nq + row};
    });
    __syncthreads();
    rows = R.Np;
    tot = t.E * nc * rows;
    contract4(tot, n, [&](int idx) {
      const int m = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int a1 = R.mode[m];
      return Dot{R.psi2 + m * n, 1, t.base + e * t.pe + s1 + var * R.Nq + a1 * n, 1,
                 t.base + e * t.pe + out + var * R.Np + m};
    });
    __syncthreads();
  } else {
    int rows = (p + 1) * n * n, tot = t.E * nc * rows;
    contract4(tot, n, [&](int idx) {
      const int row = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int c3 = row % n, c2 = (row / n) % n, a1 = row / (n * n);
      return Dot{R.psi1 + a1 * n, 1, t.base + e * t.pe + in + var * R.Nq + n * (c2 + n * c3), 1,
                 t.base + e * t.pe + s1 + var * R.Nq + row};
    });
    __syncthreads();
    rows = R.S12 * n;
    tot = t.E * nc * rows;
    contract4(tot, n, [&](int idx) {
      const int row = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int s = row / n, c3 = row % n, a1 = R.s12a1[s];
      return Dot{R.psi2 + s * n, 1, t.base + e * t.pe + s1 + var * R.Nq + a1 * n * n + c3, n,
                 t.base + e * t.pe + s2 + var * R.Nq + row};
    });
    __syncthreads();
    rows = R.Np;
    tot = t.E * nc * rows;
    contract4(tot, n, [&](int idx) {
      const int m = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      const int s = R.mode[m];
      return Dot{R.psi3 + m * n, 1, t.base + e * t.pe + s2 + var * R.Nq + s * n, 1,
                 t.base + e * t.pe + out + var * R.Np + m};
    });
    __syncthreads();
  }
}

// facet values wf = R^(zeta) w (Eq. (r_2d), Eq. (r_3d)); `y` is nodal scratch (tetrahedra).
template <int D>
__device__ void apply_R(const DevRef& R, const Tile& t, int in, int y, int out, int nc) {
  const int n = R.n;
  if (D == 3) {
    const int rows = n * n, tot = t.E * nc * rows;
    contract4(tot, n, [&](int idx) {   // face 4: extrapolate eta3 -> -1
      const int row = idx % rows, ev = idx / rows, var = ev % nc, e = ev / nc;
      return Dot{R.l3m, 1, t.base + e * t.pe + in + var * R.Nq + row, n * n, t.base + e * t.pe + y + var * R.Nq + row};
    });
    __syncthreads();
  }
  const int tot = t.E * nc * R.Nfn;
  contract4(tot, n, [&](int idx) {
    const int f = idx % R.Nfn, ev = idx / R.Nfn, var = ev % nc, e = ev / nc;
    const int z = f / R.Nqf, j = f % R.Nqf;
    const double* w = t.base + e * t.pe + in + var * R.Nq;
    double* dst = t.base + e * t.pe + out + var * R.Nfn + f;
    if (D == 2) {
      if (z == 0) return Dot{R.l2m, 1, w + j, n, dst};
      return Dot{z == 1 ? R.l1p : R.l1m, 1, w + n * j, 1, dst};
    }
    const int a = j % n, b = j / n;
    if (z == 0) return Dot{R.l2m, 1, w + a + n * n * b, n, dst};
    if (z < 3) return Dot{z == 1 ? R.l1p : R.l1m, 1, w + n * j, 1, dst};
    return Dot{R.L2J + b * n, 1, t.base + e * t.pe + y + var * R.Nq + a, n, dst};
  });
  __syncthreads();
}

// out = V^T (W/J) V in (modal -> modal), the weight-adjusted inverse of
// Eq. (weight_adjusted_inverse) with M = I: the stored symmetric per-element matrix when
// R.dense_minv, else sum-factorised through nodal scratch s1, s2, s3.  `out` must differ
// from `in`, s1 and s2; it may equal s3.
template <int D>
__device__ void apply_minv(const DevRef& R, const DevMesh& M, const Tile& t, int64_t e0, int in, int s1, int s2,
                           int s3, int out, int nc) {
  const int Np = R.Np, Nq = R.Nq;
  if (R.dense_minv) {
    const int tot = t.E * nc * Np;
    contract4(tot, Np, [&](int idx) {
      const int i = idx % Np, ev = idx / Np, var = ev % nc, e = ev / nc;
      // column i == row i (symmetric): consecutive threads read consecutive addresses
      return Dot{M.minv + (e0 + e) * (int64_t)Np * Np + i, Np, t.base + e * t.pe + in + var * Np, 1,
                 t.base + e * t.pe + out + var * Np + i};
    });
    __syncthreads();
    return;
  }
  apply_V<D>(R, t, in, s1, s2, s3, nc);
  for (int idx = threadIdx.x; idx < t.E * nc * Nq; idx += blockDim.x) {
    const int e = idx / (nc * Nq), v = idx % Nq;
    t.base[e * t.pe + s3 + idx % (nc * Nq)] *= M.wdj[(e0 + e) * Nq + v];
  }
  __syncthreads();
  apply_VT<D>(R, t, s3, s1, s2, out, nc);
}

// ---------------------------------------------------------------------------
// Pointwise maps
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool finite_pos(double x) { return x > 0.0 && x < 1.0e300; }

// entropy variables W(u) = grad_U S (Section 7.1), times the weight W J
template <int D>
__device__ __forceinline__ void entropy_vars(const double* u, double gamma, double scale, double* w, int* bad,
                                             const double* __restrict__ mt) {
  double rho = u[0];
  double ir = rcp_nr<2>(rho), vv = 0.0, v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = u[1 + k] * ir;
    vv = fma(v[k], v[k], vv);
  }
  double p = (gamma - 1.0) * (u[D + 1] - 0.5 * rho * vv);
  if (!finite_pos(rho) || !finite_pos(p)) {
    *bad = 1;
    p = rho = 1.0;   // keep the arithmetic finite; the state is reported as non-admissible
  }
  double s = log_tab(p, mt) - gamma * log_tab(rho, mt);
  double b = rho * rcp_nr<2>(p);
  w[0] = scale * ((gamma - s) * (1.0 / (gamma - 1.0)) - 0.5 * b * vv);
#pragma unroll
  for (int k = 0; k < D; ++k) w[1 + k] = scale * b * v[k];
  w[D + 1] = -scale * b;
}

// conservative variables U(w) (inverse of the entropy-variable map) returned as the
// flux state: b = -w_last = rho/p, v = w_v/b, s = gamma - (gamma-1)(w_1 + b|v|^2/2),
// ln rho = -(s + ln b)/(gamma-1), p = rho/b.
template <int D>
__device__ __forceinline__ NodeState<D> state_from_entropy(const double* w, double gamma, int* bad,
                                                           const double* __restrict__ mt) {
  NodeState<D> st;
  double b = -w[D + 1];
  if (!finite_pos(b)) {
    *bad = 1;
    b = 1.0;
  }
  double ib = rcp_nr<2>(b), vv = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    st.v[k] = w[1 + k] * ib;
    vv = fma(st.v[k], st.v[k], vv);
  }
  double s = gamma - (gamma - 1.0) * (w[0] + 0.5 * b * vv);
  double lb = log_tab(b, mt);
  st.lrho = -(s + lb) * (1.0 / (gamma - 1.0));
  st.rho = (st.lrho > -700.0 && st.lrho < 700.0) ? exp_tab(st.lrho, mt) : exp(st.lrho);
  st.p = st.rho * ib;
  st.beta = b;
  st.lbeta = lb;
  if (!finite_pos(st.rho) || !finite_pos(st.p)) *bad = 1;
  return st;
}

template <int D>
__device__ __forceinline__ void store_state(double* S, int stride, int idx, const NodeState<D>& s) {
  S[idx] = s.rho;
#pragma unroll
  for (int k = 0; k < D; ++k) S[(1 + k) * stride + idx] = s.v[k];
  S[(D + 1) * stride + idx] = s.p;
  S[(D + 2) * stride + idx] = s.beta;
  S[(D + 3) * stride + idx] = s.lrho;
  S[(D + 4) * stride + idx] = s.lbeta;
}

// ---------------------------------------------------------------------------
// Projection kernel
// shared layout per element (doubles): M[nc*Np] | A[nc*Nq] | B[nc*Nq] | C[nc*Nq] | F[nc*Nfn]
// ---------------------------------------------------------------------------
template <int D>
__device__ void project_tile(const DevRef& R, const DevMesh& M, int64_t e0, int E, const double* __restrict__ u,
                             double* __restrict__ w_modal) {
  extern __shared__ double sm[];
  constexpr int NC = D + 2, NF = D + 5;
  const int Np = R.Np, Nq = R.Nq, Nfn = R.Nfn, Ntot = R.Ntot;
  const int oM = 0, oA = NC * Np, oB = oA + NC * Nq, oC = oB + NC * Nq, oF = oC + NC * Nq;
  const int pe = oF + NC * Nfn;
  Tile t{sm, pe, E};
  // 1. load u~
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np), r = idx % (NC * Np);
    sm[e * pe + oM + r] = u[(e0 + e) * NC * Np + r];
  }
  __syncthreads();
  // 2. u = V u~
  apply_V<D>(R, t, oM, oB, oC, oA, NC);
  // 3. W J W(u)
  int lbad = 0;
  for (int idx = threadIdx.x; idx < E * Nq; idx += blockDim.x) {
    int e = idx / Nq, v = idx % Nq;
    double uu[NC], ww[NC];
    double* A = sm + e * pe + oA;
#pragma unroll
    for (int c = 0; c < NC; ++c) uu[c] = A[c * Nq + v];
    entropy_vars<D>(uu, M.gamma, M.wj[(e0 + e) * Nq + v], ww, &lbad, R.mtab);
#pragma unroll
    for (int c = 0; c < NC; ++c) A[c * Nq + v] = ww[c];
  }
  __syncthreads();
  // 4-6. w~ = [V^T (W/J) V] V^T (W J W)
  apply_VT<D>(R, t, oA, oB, oC, oM, NC);
  apply_minv<D>(R, M, t, e0, oM, oB, oC, oA, oA, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np);
    sm[e * pe + oM + idx % (NC * Np)] = sm[e * pe + oA + idx % (NC * Np)];
  }
  __syncthreads();
  if (w_modal) {
    for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
      int e = idx / (NC * Np), r = idx % (NC * Np);
      w_modal[(e0 + e) * NC * Np + r] = sm[e * pe + oM + r];
    }
    if (lbad) atomicOr(M.flag, kFlagState);
    return;
  }
  // 7-8. w = V w~, facet values R w
  apply_V<D>(R, t, oM, oB, oC, oA, NC);
  apply_R<D>(R, t, oA, oB, oF, NC);
  // 9. entropy-projected conservative states at volume and facet nodes
  const double sqrt_gamma = sqrt(M.gamma);
  for (int idx = threadIdx.x; idx < E * Ntot; idx += blockDim.x) {
    int e = idx / Ntot, k = idx % Ntot;
    double ww[NC];
    const double* src = k < Nq ? sm + e * pe + oA + k : sm + e * pe + oF + (k - Nq);
    const int str = k < Nq ? Nq : Nfn;
#pragma unroll
    for (int c = 0; c < NC; ++c) ww[c] = src[c * str];
    NodeState<D> st = state_from_entropy<D>(ww, M.gamma, &lbad, R.mtab);
    store_state<D>(M.states + (e0 + e) * NF * Ntot, Ntot, k, st);
    if (k >= Nq) M.cfac[(e0 + e) * Nfn + (k - Nq)] = sqrt_gamma * rsqrt_nr(st.beta);   // sqrt(gamma p / rho)
  }
  if (lbad) atomicOr(M.flag, kFlagState);
}

// ---------------------------------------------------------------------------
// Bulk copies global -> shared memory by the TMA unit (cp.async.bulk), completing on an
// mbarrier in shared memory; waits are bounded (about a second), after which the kernel
// reports the failure through the mesh's flag instead of spinning.
// ---------------------------------------------------------------------------
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// true once phase `parity` of the barrier has completed; false after `limit` clock cycles
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// ---------------------------------------------------------------------------
// Residual kernel
// dynamic shared memory: 16 bytes for the staging mbarrier, then per element (doubles,
// an even count so that every element starts 16-byte aligned):
//   states S[NF][Ntot] (volume nodes then facet nodes, the global layout; one bulk copy)
//   -- reused as transform scratch S1, S2, Mod after the pair phases --
//   r[NC*Nq] | h4[NC*n^2] (tetrahedra: facet-4 node accumulators)
// ---------------------------------------------------------------------------
struct ResLayout {
  int oS, oS1, oS2, oMod, oR, oH4, pe;
};

template <int D>
__host__ __device__ inline ResLayout res_layout(int Nq, int Nfn, int Np, int n) {
  constexpr int NC = D + 2, NF = D + 5;
  ResLayout L;
  L.oS = 0;
  int r0 = NF * (Nq + Nfn);
  L.oS1 = 0;
  L.oS2 = NC * Nq;
  L.oMod = 2 * NC * Nq;
  const int r0b = L.oMod + NC * Np;
  if (r0b > r0) r0 = r0b;
  L.oR = r0;
  L.oH4 = L.oR + NC * Nq;
  L.pe = L.oH4 + (D == 3 ? NC * n * n : 0);
  L.pe += L.pe & 1;
  return L;
}
constexpr int kResSmemHeader = 2;   // doubles before the first element (the mbarrier)

// F = B J f* at facet node f of element eg (Eq. (interface_flux), Eq. (num_flux),
// Eq. (wave_speed)): own trace from shared memory, the neighbour's from its stored states.
template <int D>
__device__ __forceinline__ void interface_flux(const DevMesh& M, int Nq, int Nfn, int Ntot, int64_t eg, int f,
                                               const double* __restrict__ Sf, const FluxK& K, double* F) {
  constexpr int NF = D + 5;
  const NodeState<D> L = load_state<D>(Sf, Ntot, f);
  const int64_t e2 = M.nbr_e[eg * Nfn + f];
  const int f2 = M.nbr_f[eg * Nfn + f];
  const NodeState<D> Rr = load_state<D>(M.states + e2 * NF * Ntot + Nq, Ntot, f2);
  double nn[D], nh[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    nn[k] = M.nrm[(eg * D + k) * Nfn + f];
    nh[k] = 0.5 * nn[k];
  }
  ec_flux_fast<D>(L, Rr, nh, K, F);
  if (M.lf) {
    double vnL = 0.0, vnR = 0.0, vvL = 0.0, vvR = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      vnL = fma(L.v[k], nn[k], vnL);
      vnR = fma(Rr.v[k], nn[k], vnR);
      vvL = fma(L.v[k], L.v[k], vvL);
      vvR = fma(Rr.v[k], Rr.v[k], vvR);
    }
    const double lam = fmax(fabs(vnL), fabs(vnR)) + fmax(M.cfac[eg * Nfn + f], M.cfac[e2 * Nfn + f2]);
    const double hl = 0.5 * lam;
    F[0] -= hl * (Rr.rho - L.rho);
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] -= hl * (Rr.rho * Rr.v[k] - L.rho * L.v[k]);
    const double EL = L.p * K.inv_gm1 + 0.5 * L.rho * vvL, ER = Rr.p * K.inv_gm1 + 0.5 * Rr.rho * vvR;
    F[D + 1] -= hl * (ER - EL);
  }
  const double bj = M.bj[eg * Nfn + f];
#pragma unroll
  for (int c = 0; c < D + 2; ++c) F[c] *= bj;
}

// Pair directions formed on the fly from per-node metric terms (meshes created with
// ESD_MESH_METRICS_ON_THE_FLY), the same quantities the stored tables hold:
//   volume pair (i at a, j at b) of an eta_k-line:
//     n_ij / 2 = 1/4 sum_l (Q^(l)_ij - Q^(l)_ji) (G_l.(x_i) + G_l.(x_j)),
//     Q^(l)_ij = w_i (d eta_k / d xi_l)(xi_i) ell'_{k,b}(eta_{k,a})       (Eq. (avg_volume_metric))
//   facet pair (volume node i, facet node f of face z):
//     {{J n}}_if [R^T B]_if / 2 = [R^T B]_if / 4 (G(x_i)^T nhat_z + J^z n(x_f))   (Eq. (facet_correction))
// G: the element's metric terms [dim*dim][Nq] (component l*dim + m).
template <int D>
__device__ __forceinline__ void otf_vol_dir(const DevRef& R, const double* __restrict__ G, int Nq, int k, int a,
                                            int b, int vi, int vj, double* nh) {
  const int n = R.n;
  const double dab = R.dk4[(k * n + a) * n + b], dba = R.dk4[(k * n + b) * n + a];
  const double* __restrict__ aw = R.aw + (size_t)k * D * Nq;
  double c[D];
#pragma unroll
  for (int l = 0; l < D; ++l) c[l] = fma(dab, aw[l * Nq + vi], -dba * aw[l * Nq + vj]);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) s = fma(c[l], G[(l * D + m) * Nq + vi] + G[(l * D + m) * Nq + vj], s);
    nh[m] = s;
  }
}

// rbq = [R^T B]_if / 4; nz = the face's reference normal; jn = J^z n at the facet node
template <int D>
__device__ __forceinline__ void otf_fac_dir(const double* __restrict__ G, int Nq, const double* nz, int vi,
                                            const double* jn, double rbq, double* nh) {
#pragma unroll
  for (int m = 0; m < D; ++m) {
    double s = jn[m];
#pragma unroll
    for (int l = 0; l < D; ++l) s = fma(nz[l], G[(l * D + m) * Nq + vi], s);
    nh[m] = rbq * s;
  }
}

// N facet-correction pairs between facet node f (state Sj) and the line's volume nodes,
// direction of pair a from dir(a, nh): acc[a] -= F_a, hs -= F_a (register accumulators,
// unrolled over the line).
template <int D, int N, class Dir>
__device__ __forceinline__ void facet_strip(const double* __restrict__ Sv, int Ntot, int base, int stride,
                                            const NodeState<D>& Sj, Dir&& dir, const FluxK& K,
                                            double (&acc)[N][D + 2], double* hs) {
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const NodeState<D> Si = load_state<D>(Sv, Ntot, base + a * stride);
    double nh[D], F[D + 2];
    dir(a, nh);
    ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
    for (int c = 0; c < D + 2; ++c) {
      acc[a][c] -= F[c];
      hs[c] -= F[c];
    }
  }
}

// The same with the line's residuals in shared memory, r[c * Nq + base + a * stride]
// (a loop over the line).
template <int D, int N, class Dir>
__device__ __forceinline__ void facet_strip_shared(const double* __restrict__ Sv, int Ntot, int base, int stride,
                                                   const NodeState<D>& Sj, Dir&& dir, const FluxK& K, double* r,
                                                   int Nq, double* hs) {
#pragma unroll 1
  for (int a = 0; a < N; ++a) {
    const NodeState<D> Si = load_state<D>(Sv, Ntot, base + a * stride);
    double nh[D], F[D + 2];
    dir(a, nh);
    ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
    for (int c = 0; c < D + 2; ++c) {
      r[c * Nq + base + a * stride] -= F[c];
      hs[c] -= F[c];
    }
  }
}

// The line task with the line's node residuals in the shared residual r (which the task
// owns for its line in this phase) instead of registers; node a's running sum over its
// pairs stays in registers.  Used by line_task for large N.
template <int D, int N, bool OTF>
__device__ __forceinline__ void line_task_shared(int ph, int t, bool act, const DevRef& R, const DevMesh& M, int64_t eg,
                                          const double* __restrict__ Sv, const double* __restrict__ Sf, double* r,
                                          double* h4, const double* __restrict__ vdir,
                                          const double* __restrict__ fdir, const FluxK& K) {
  constexpr int NC = D + 2;
  // on-the-fly directions: the element's metric terms and facet normals
  const double* __restrict__ G = OTF ? M.gvol + eg * (int64_t)D * D * R.Nq : nullptr;
  const double* __restrict__ JN = OTF ? M.jnf + eg * (int64_t)D * R.Nfn : nullptr;
  auto jn_at = [&](int f, double* jn) {
#pragma unroll
    for (int m = 0; m < D; ++m) jn[m] = JN[m * R.Nfn + f];
  };
  const int Nq = R.Nq, Nfn = R.Nfn, Nqf = R.Nqf, T = R.T, Ntot = R.Ntot;
  int base, stride;
  if (D == 2) {
    base = ph == 0 ? N * t : t;
    stride = ph == 0 ? 1 : N;
  } else {
    if (ph == 0) { base = N * t; stride = 1; }
    else if (ph == 1) { base = (t % N) + N * N * (t / N); stride = N; }
    else { base = t; stride = N * N; }
  }
  // Node residuals of the line: in registers (acc, unrolled pair loops), or -- where N
  // accumulators no longer fit in registers beside the flux (tetrahedra N >= 6), or where
  // the register path's 160-255 registers cap an SM's warps while the tiles would allow
  // more (triangles N >= 3, tetrahedra N <= 3) -- directly in the shared residual r, which
  // this task owns for its line in this phase, with node a's running sum over its pairs in
  // registers (about 96 registers).
  constexpr bool SACC = D == 3 ? (N >= 6 || N <= 3) : N >= 3;
  double acc[N][NC];
  if constexpr (!SACC) {
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[a][c] = 0.0;
  }
  auto strip = [&](const NodeState<D>& Sj, auto&& dir, double* hs) {
    if constexpr (SACC)
      facet_strip_shared<D, N>(Sv, Ntot, base, stride, Sj, dir, K, r, Nq, hs);
    else
      facet_strip<D, N>(Sv, Ntot, base, stride, Sj, dir, K, acc, hs);
  };
  if (act) {
    constexpr int Lv = N * (N - 1) / 2;
    const double* vd = vdir + (size_t)ph * Lv * D * T + t;
    if constexpr (SACC) {
      int m = 0;
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        const NodeState<D> Si = load_state<D>(Sv, Ntot, base + a * stride);
        double ra[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ra[c] = 0.0;
#pragma unroll 1
        for (int b = a + 1; b < N; ++b, ++m) {
          const NodeState<D> Sj = load_state<D>(Sv, Ntot, base + b * stride);
          double nh[D], F[NC];
          if constexpr (OTF) {
            otf_vol_dir<D>(R, G, Nq, ph, a, b, base + a * stride, base + b * stride, nh);
          } else {
#pragma unroll
            for (int k = 0; k < D; ++k) nh[k] = vd[(m * D + k) * T];
          }
          ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            ra[c] -= F[c];
            r[c * Nq + base + b * stride] += F[c];
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) r[c * Nq + base + a * stride] += ra[c];
      }
    } else {
#pragma unroll
      for (int a = 0, m = 0; a < N; ++a) {
#pragma unroll
        for (int b = a + 1; b < N; ++b, ++m) {
          const NodeState<D> Si = load_state<D>(Sv, Ntot, base + a * stride);
          const NodeState<D> Sj = load_state<D>(Sv, Ntot, base + b * stride);
          double nh[D], F[NC];
          if constexpr (OTF) {
            otf_vol_dir<D>(R, G, Nq, ph, a, b, base + a * stride, base + b * stride, nh);
          } else {
#pragma unroll
            for (int k = 0; k < D; ++k) nh[k] = vd[(m * D + k) * T];
          }
          ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            acc[a][c] -= F[c];
            acc[b][c] += F[c];
          }
        }
      }
    }
    if (ph == 0) {
#pragma unroll
      for (int zz = 0; zz < 2; ++zz) {
        const int f = (1 + zz) * Nqf + t;
        double hs[NC];
        interface_flux<D>(M, Nq, Nfn, Ntot, eg, f, Sf, K, hs);
        const NodeState<D> Sj = load_state<D>(Sf, Ntot, f);
        const double* l = zz == 0 ? R.l1p : R.l1m;   // R entries along the eta1-line (and the lift)
        if constexpr (OTF) {
          double jn[D];
          jn_at(f, jn);
          const double wq = 0.25 * R.wfac[f];
          strip(Sj, [&](int a, double* nh) {
            otf_fac_dir<D>(G, Nq, R.nhat[1 + zz], base + a * stride, jn, wq * l[a], nh);
          }, hs);
        } else {
          const double* fd = fdir + R.fph_off[0] + (size_t)zz * N * D * T + t;
          strip(Sj, [&](int a, double* nh) {
#pragma unroll
            for (int k = 0; k < D; ++k) nh[k] = fd[(a * D + k) * T];
          }, hs);
        }
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const double la = l[a];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
          if constexpr (SACC) {
            double& ra = r[c * Nq + base + a * stride];
            ra = fma(-la, hs[c], ra);
          } else {
            acc[a][c] = fma(-la, hs[c], acc[a][c]);
          }
        }
        }
      }
    } else if (ph == 1) {
      const int f = t;
      double hs[NC];
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, f, Sf, K, hs);
      const NodeState<D> Sj = load_state<D>(Sf, Ntot, f);
      if constexpr (OTF) {
        double jn[D];
        jn_at(f, jn);
        const double wq = 0.25 * R.wfac[f];
        strip(Sj, [&](int a, double* nh) {
          otf_fac_dir<D>(G, Nq, R.nhat[0], base + a * stride, jn, wq * R.l2m[a], nh);
        }, hs);
      } else {
        const double* fd = fdir + R.fph_off[1] + t;
        strip(Sj, [&](int a, double* nh) {
#pragma unroll
          for (int k = 0; k < D; ++k) nh[k] = fd[(a * D + k) * T];
        }, hs);
      }
#pragma unroll
      for (int a = 0; a < N; ++a) {   // lift of facet 1 along the eta2-line
        const double la = R.l2m[a];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if constexpr (SACC) {
            double& ra = r[c * Nq + base + a * stride];
            ra = fma(-la, hs[c], ra);
          } else {
            acc[a][c] = fma(-la, hs[c], acc[a][c]);
          }
        }
      }
    } else if (D == 3) {
      double hs[NC];
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, 3 * Nqf + t, Sf, K, hs);
#pragma unroll
      for (int c = 0; c < NC; ++c) h4[c * Nqf + t] = hs[c];
    }
  }
  if (D == 3 && ph == 2) {
    const int a1 = t % N, a2 = t / N;
    const double* fd4 = (act && !OTF) ? fdir + R.fph_off[3] + t : nullptr;
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      if (act) {
        const int bp = a2 + k < N ? a2 + k : a2 + k - N;
        const int j = a1 + N * bp;
        const NodeState<D> Sj = load_state<D>(Sf, Ntot, 3 * Nqf + j);
        double hs[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) hs[c] = 0.0;
        if constexpr (OTF) {
          double jn[D];
          jn_at(3 * Nqf + j, jn);
          const double wq = 0.25 * R.wfac[3 * Nqf + j] * R.L2J[bp * N + a2];
          strip(Sj, [&](int a, double* nh) {
            otf_fac_dir<D>(G, Nq, R.nhat[3], base + a * stride, jn, wq * R.l3m[a], nh);
          }, hs);
        } else {
          const double* fd = fd4 + (size_t)bp * N * D * T;
          strip(Sj, [&](int a, double* nh) {
#pragma unroll
            for (int kk = 0; kk < D; ++kk) nh[kk] = fd[(a * D + kk) * T];
          }, hs);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) h4[c * Nqf + j] += hs[c];
      }
      __syncthreads();
    }
    if (act) {   // lift of facet 4: y = sum_b' L2J[b'][a2] h4(a1, b'), along the eta3-line
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
        for (int c = 0; c < NC; ++c) {
          if constexpr (SACC) {
            double& ra = r[c * Nq + base + a * stride];
            ra = fma(-la, y[c], ra);
          } else {
            acc[a][c] = fma(-la, y[c], acc[a][c]);
          }
        }
      }
    }
  }
  if constexpr (!SACC) {
    if (act) {
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) r[c * Nq + base + a * stride] += acc[a][c];
    }
  }
}

// Tetrahedra with N >= 8: one element's tile (72-175 KB) leaves 1-2 warps per SM scheduler,
// too few to hide the FP64 latency of one line task per thread.  Here two threads (adjacent
// lanes, h = 0, 1) share each line task, accumulating in the shared residual r:
//  * volume pairs in round-robin rounds (the circle method): with MO = N (N odd) or N - 1
//    (N even), round s leaves out node u (2u = s mod MO) and pairs u + d with u - d (mod MO),
//    d = 1 .. (MO - 1) / 2, and for even N also u with node N - 1 -- every node in at most one
//    pair, every pair in exactly one round; the round's pairs alternate between the two
//    threads, and __syncwarp() between rounds orders the two threads' updates of a node;
//  * facet pairs split by the parity of the line node (each thread updates only its own
//    nodes), the facet node's two partial sums combined by a lane exchange (p0 + p1 in both
//    lanes, so both hold the same value);
//  * interface fluxes computed by one lane and exchanged.
// Every thread of the block calls this (the rounds, lane exchanges and the facet-4 steps
// synchronise); `act` marks the threads that own a task.
// threads per line task of the residual kernel (the host's residual_line_lanes gives the same)
template <int D, int N>
constexpr int kLineLanes = (D == 3 && N >= 8) ? 2 : 1;

template <int D, int N>
struct LineRounds {
  static constexpr bool EVEN = N % 2 == 0;
  static constexpr int MO = EVEN ? N - 1 : N;      // odd circle; node N - 1 of even N stays fixed
  static constexpr int HALF = (MO - 1) / 2;        // circle pairs per round
  static constexpr int D0 = EVEN ? 0 : 1;          // d = 0: the pair (u, N - 1) of even N
  static constexpr int INV2 = (MO + 1) / 2;        // 2 * INV2 = 1 (mod MO)
};

template <int D, int N, bool OTF>
__device__ __forceinline__ void line_task_split(int ph, int t, int h, bool act, const DevRef& R, const DevMesh& M,
                                                int64_t eg, const double* __restrict__ Sv,
                                                const double* __restrict__ Sf, double* r, double* h4,
                                                const double* __restrict__ vdir, const double* __restrict__ fdir,
                                                const FluxK& K) {
  static_assert(D == 3, "two threads per line task: tetrahedra");
  constexpr int NC = D + 2;
  using RR = LineRounds<D, N>;
  const double* __restrict__ G = OTF ? M.gvol + eg * (int64_t)D * D * R.Nq : nullptr;
  const double* __restrict__ JN = OTF ? M.jnf + eg * (int64_t)D * R.Nfn : nullptr;
  auto jn_at = [&](int f, double* jn) {
#pragma unroll
    for (int m = 0; m < D; ++m) jn[m] = JN[m * R.Nfn + f];
  };
  const int Nq = R.Nq, Nfn = R.Nfn, Nqf = R.Nqf, T = R.T, Ntot = R.Ntot;
  const unsigned full = 0xffffffffu;
  const int lane0 = (threadIdx.x & 31) & ~1;   // the task's first lane
  int base, stride;
  if (ph == 0) { base = N * t; stride = 1; }
  else if (ph == 1) { base = (t % N) + N * N * (t / N); stride = N; }
  else { base = t; stride = N * N; }
  auto node = [&](int a) { return base + a * stride; };
  // facet pairs of facet node f (state Sj) with this thread's line nodes a = h, h + 2, ...:
  // r[a] -= F, part -= F
  auto strip = [&](const NodeState<D>& Sj, auto&& dir, double* part) {
#pragma unroll 1
    for (int a = h; a < N; a += 2) {
      const NodeState<D> Si = load_state<D>(Sv, Ntot, node(a));
      double nh[D], F[NC];
      dir(a, nh);
      ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        r[c * Nq + node(a)] -= F[c];
        part[c] -= F[c];
      }
    }
  };
  auto combine = [&](double* part) {   // part := p0 + p1 in both lanes
#pragma unroll
    for (int c = 0; c < NC; ++c) part[c] += __shfl_xor_sync(full, part[c], 1);
  };
  auto lift = [&](const double* l, const double* hs) {   // r[a] -= l[a] hs for this thread's a
#pragma unroll 1
    for (int a = h; a < N; a += 2) {
      const double la = l[a];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double& ra = r[c * Nq + node(a)];
        ra = fma(-la, hs[c], ra);
      }
    }
  };
  // 1. volume pairs, round by round
  constexpr int Lv = N * (N - 1) / 2;
  const double* vd = act && !OTF ? vdir + (size_t)ph * Lv * D * T + t : nullptr;
#pragma unroll 1
  for (int s = 0; s < RR::MO; ++s) {
    if (act) {
      const int u = (s * RR::INV2) % RR::MO;   // left out of the circle pairs in this round
#pragma unroll 1
      for (int d = RR::D0 + ((h + s) & 1); d <= RR::HALF; d += 2) {
        int i, j;
        if (d == 0) {   // even N: u with the fixed node
          i = u;
          j = N - 1;
        } else {
          i = u + d;
          j = u - d;
          if (i >= RR::MO) i -= RR::MO;
          if (j < 0) j += RR::MO;
        }
        const int a = i < j ? i : j, b = i < j ? j : i;
        const int m = a * (2 * N - a - 1) / 2 + (b - a - 1);   // the pair's index in the line's table
        const NodeState<D> Si = load_state<D>(Sv, Ntot, node(a));
        const NodeState<D> Sj = load_state<D>(Sv, Ntot, node(b));
        double nh[D], F[NC];
        if constexpr (OTF) {
          otf_vol_dir<D>(R, G, Nq, ph, a, b, node(a), node(b), nh);
        } else {
#pragma unroll
          for (int k = 0; k < D; ++k) nh[k] = vd[(m * D + k) * T];
        }
        ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          r[c * Nq + node(a)] -= F[c];
          r[c * Nq + node(b)] += F[c];
        }
      }
    }
    __syncwarp();
  }
  // 2. facets attached to the line
  if (ph == 0) {
    // faces 2 and 3 (f = (1 + zz) Nqf + t): lane h computes the interface flux of face 2 + h
    double own[NC];
    const int fo = (1 + h) * Nqf + t;
    if (act) {
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, fo, Sf, K, own);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) own[c] = 0.0;
    }
#pragma unroll 1
    for (int zz = 0; zz < 2; ++zz) {
      double hs[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double v = __shfl_sync(full, own[c], lane0 + zz);
        hs[c] = h == 0 ? v : 0.0;   // lane 0 carries B J f*, lane 1 only its pair sums
      }
      if (act) {
        const int f = (1 + zz) * Nqf + t;
        const NodeState<D> Sj = load_state<D>(Sf, Ntot, f);
        const double* l = zz == 0 ? R.l1p : R.l1m;
        if constexpr (OTF) {
          double jn[D];
          jn_at(f, jn);
          const double wq = 0.25 * R.wfac[f];
          strip(Sj, [&](int a, double* nh) { otf_fac_dir<D>(G, Nq, R.nhat[1 + zz], node(a), jn, wq * l[a], nh); },
                hs);
        } else {
          const double* fd = fdir + R.fph_off[0] + (size_t)zz * N * D * T + t;
          strip(Sj, [&](int a, double* nh) {
#pragma unroll
            for (int k = 0; k < D; ++k) nh[k] = fd[(a * D + k) * T];
          }, hs);
        }
      }
      combine(hs);
      if (act) lift(zz == 0 ? R.l1p : R.l1m, hs);
    }
  } else if (ph == 1) {
    // face 1 (f = t): lane 0 computes the interface flux
    const int f = t;
    double own[NC], hs[NC];
    if (act && h == 0) {
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, f, Sf, K, own);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) own[c] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) hs[c] = own[c];
    if (act) {
      const NodeState<D> Sj = load_state<D>(Sf, Ntot, f);
      if constexpr (OTF) {
        double jn[D];
        jn_at(f, jn);
        const double wq = 0.25 * R.wfac[f];
        strip(Sj, [&](int a, double* nh) { otf_fac_dir<D>(G, Nq, R.nhat[0], node(a), jn, wq * R.l2m[a], nh); }, hs);
      } else {
        const double* fd = fdir + R.fph_off[1] + t;
        strip(Sj, [&](int a, double* nh) {
#pragma unroll
          for (int k = 0; k < D; ++k) nh[k] = fd[(a * D + k) * T];
        }, hs);
      }
    }
    combine(hs);
    if (act) lift(R.l2m, hs);
  } else {
    // face 4: h4 = B J f* of node t (lane 0), then N barrier-separated steps of the diagonal
    // schedule (task (a1, a2) handles column b' = (a2 + k) mod N), then the lift along the
    // eta3-line
    if (act && h == 0) {
      double hs[NC];
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, 3 * Nqf + t, Sf, K, hs);
#pragma unroll
      for (int c = 0; c < NC; ++c) h4[c * Nqf + t] = hs[c];
    }
    __syncthreads();
    const int a1 = t % N, a2 = t / N;
    const double* fd4 = (act && !OTF) ? fdir + R.fph_off[3] + t : nullptr;
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      const int bp = a2 + k < N ? a2 + k : a2 + k - N;
      const int j = a1 + N * bp;
      double hs[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) hs[c] = 0.0;
      if (act) {
        const NodeState<D> Sj = load_state<D>(Sf, Ntot, 3 * Nqf + j);
        if constexpr (OTF) {
          double jn[D];
          jn_at(3 * Nqf + j, jn);
          const double wq = 0.25 * R.wfac[3 * Nqf + j] * R.L2J[bp * N + a2];
          strip(Sj, [&](int a, double* nh) { otf_fac_dir<D>(G, Nq, R.nhat[3], node(a), jn, wq * R.l3m[a], nh); },
                hs);
        } else {
          const double* fd = fd4 + (size_t)bp * N * D * T;
          strip(Sj, [&](int a, double* nh) {
#pragma unroll
            for (int kk = 0; kk < D; ++kk) nh[kk] = fd[(a * D + kk) * T];
          }, hs);
        }
      }
      combine(hs);
      if (act && h == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) h4[c * Nqf + j] += hs[c];
      }
      __syncthreads();
    }
    if (act) {   // y = sum_b' L2J[b'][a2] h4(a1, b'), lifted along the eta3-line
      double y[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = 0.0;
#pragma unroll 1
      for (int bp = 0; bp < N; ++bp) {
        const double w = R.L2J[bp * N + a2];
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c] = fma(w, h4[c * Nqf + a1 + N * bp], y[c]);
      }
      lift(R.l3m, y);
    }
  }
}

// Line task t of phase ph (Section 5.1, along collapsed-coordinate lines, Remark 4): the
// pairs of one eta_{ph+1}-line of N nodes, the facet nodes attached to it -- their
// interface fluxes, facet-correction pairs and lift -- accumulated in registers.
//   tetrahedra: phase 0 = eta1-lines + facets 2, 3; phase 1 = eta2-lines + facet 1;
//               phase 2 = eta3-lines + facet 4;
//   triangles:  phase 0 = eta1-lines + facets 2, 3; phase 1 = eta2-lines + facet 1.
// A facet node of faces 1-3 couples only with the N volume nodes of its line, so its
// h = B J f* - C^T 1 is complete inside the task and its lift R^T h (a 1D extrapolation
// along the line) goes straight into the line's accumulators.  Facet-4 node (a1, b')
// couples with all volume nodes (a1, ., .): task (a1, a2) writes h4 = B J f* of node
// (a1, a2), then in N barrier-separated steps handles column b' = (a2 + k) mod N -- the
// tasks sharing a1 update distinct facet nodes in every step -- and finally lifts
// y = L2J h4 along its eta3-line.  Every thread of the block calls this (phase 2 has
// barriers); `act` marks the threads that own a task.
template <int D, int N, bool OTF = false>
__device__ __forceinline__ void line_task(int ph, int t, bool act, const DevRef& R, const DevMesh& M, int64_t eg,
                                          const double* __restrict__ Sv, const double* __restrict__ Sf, double* r,
                                          double* h4, const double* __restrict__ vdir,
                                          const double* __restrict__ fdir, const FluxK& K) {
  constexpr int NC = D + 2;
  // Tetrahedra N >= 6 (N accumulators no longer fit in registers beside the flux), and
  // triangles N >= 3 and tetrahedra N <= 3 (occupancy): the line's residuals accumulate in
  // shared memory instead.
  if constexpr (D == 3 ? (N >= 6 || N <= 3) : N >= 3) {
    line_task_shared<D, N, OTF>(ph, t, act, R, M, eg, Sv, Sf, r, h4, vdir, fdir, K);
    return;
  }
  // on-the-fly directions: the element's metric terms and facet normals
  const double* __restrict__ G = OTF ? M.gvol + eg * (int64_t)D * D * R.Nq : nullptr;
  const double* __restrict__ JN = OTF ? M.jnf + eg * (int64_t)D * R.Nfn : nullptr;
  auto jn_at = [&](int f, double* jn) {
#pragma unroll
    for (int m = 0; m < D; ++m) jn[m] = JN[m * R.Nfn + f];
  };
  const int Nq = R.Nq, Nfn = R.Nfn, Nqf = R.Nqf, T = R.T, Ntot = R.Ntot;
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
    constexpr int Lv = N * (N - 1) / 2;
    const double* vd = vdir + (size_t)ph * Lv * D * T + t;
#pragma unroll
    for (int a = 0, m = 0; a < N; ++a) {
#pragma unroll
      for (int b = a + 1; b < N; ++b, ++m) {
        const NodeState<D> Si = load_state<D>(Sv, Ntot, base + a * stride);
        const NodeState<D> Sj = load_state<D>(Sv, Ntot, base + b * stride);
        double nh[D], F[NC];
        if constexpr (OTF) {
          otf_vol_dir<D>(R, G, Nq, ph, a, b, base + a * stride, base + b * stride, nh);
        } else {
#pragma unroll
          for (int k = 0; k < D; ++k) nh[k] = vd[(m * D + k) * T];
        }
        ec_flux_fast<D>(Si, Sj, nh, K, F);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          acc[a][c] -= F[c];
          acc[b][c] += F[c];
        }
      }
    }
    if (ph == 0) {
#pragma unroll
      for (int zz = 0; zz < 2; ++zz) {
        const int f = (1 + zz) * Nqf + t;
        double hs[NC];
        interface_flux<D>(M, Nq, Nfn, Ntot, eg, f, Sf, K, hs);
        const NodeState<D> Sj = load_state<D>(Sf, Ntot, f);
        const double* l = zz == 0 ? R.l1p : R.l1m;   // R entries along the eta1-line (and the lift)
        if constexpr (OTF) {
          double jn[D];
          jn_at(f, jn);
          const double wq = 0.25 * R.wfac[f];
          facet_strip<D, N>(Sv, Ntot, base, stride, Sj, [&](int a, double* nh) {
            otf_fac_dir<D>(G, Nq, R.nhat[1 + zz], base + a * stride, jn, wq * l[a], nh);
          }, K, acc, hs);
        } else {
          const double* fd = fdir + R.fph_off[0] + (size_t)zz * N * D * T + t;
          facet_strip<D, N>(Sv, Ntot, base, stride, Sj, [&](int a, double* nh) {
#pragma unroll
            for (int k = 0; k < D; ++k) nh[k] = fd[(a * D + k) * T];
          }, K, acc, hs);
        }
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const double la = l[a];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[a][c] = fma(-la, hs[c], acc[a][c]);
        }
      }
    } else if (ph == 1) {
      const int f = t;
      double hs[NC];
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, f, Sf, K, hs);
      const NodeState<D> Sj = load_state<D>(Sf, Ntot, f);
      if constexpr (OTF) {
        double jn[D];
        jn_at(f, jn);
        const double wq = 0.25 * R.wfac[f];
        facet_strip<D, N>(Sv, Ntot, base, stride, Sj, [&](int a, double* nh) {
          otf_fac_dir<D>(G, Nq, R.nhat[0], base + a * stride, jn, wq * R.l2m[a], nh);
        }, K, acc, hs);
      } else {
        const double* fd = fdir + R.fph_off[1] + t;
        facet_strip<D, N>(Sv, Ntot, base, stride, Sj, [&](int a, double* nh) {
#pragma unroll
          for (int k = 0; k < D; ++k) nh[k] = fd[(a * D + k) * T];
        }, K, acc, hs);
      }
#pragma unroll
      for (int a = 0; a < N; ++a) {   // lift of facet 1 along the eta2-line
        const double la = R.l2m[a];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[a][c] = fma(-la, hs[c], acc[a][c]);
      }
    } else if (D == 3) {
      double hs[NC];
      interface_flux<D>(M, Nq, Nfn, Ntot, eg, 3 * Nqf + t, Sf, K, hs);
#pragma unroll
      for (int c = 0; c < NC; ++c) h4[c * Nqf + t] = hs[c];
    }
  }
  if (D == 3 && ph == 2) {
    const int a1 = t % N, a2 = t / N;
    const double* fd4 = (act && !OTF) ? fdir + R.fph_off[3] + t : nullptr;
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      if (act) {
        const int bp = a2 + k < N ? a2 + k : a2 + k - N;
        const int j = a1 + N * bp;
        const NodeState<D> Sj = load_state<D>(Sf, Ntot, 3 * Nqf + j);
        double hs[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) hs[c] = 0.0;
        if constexpr (OTF) {
          double jn[D];
          jn_at(3 * Nqf + j, jn);
          const double wq = 0.25 * R.wfac[3 * Nqf + j] * R.L2J[bp * N + a2];
          facet_strip<D, N>(Sv, Ntot, base, stride, Sj, [&](int a, double* nh) {
            otf_fac_dir<D>(G, Nq, R.nhat[3], base + a * stride, jn, wq * R.l3m[a], nh);
          }, K, acc, hs);
        } else {
          const double* fd = fd4 + (size_t)bp * N * D * T;
          facet_strip<D, N>(Sv, Ntot, base, stride, Sj, [&](int a, double* nh) {
#pragma unroll
            for (int kk = 0; kk < D; ++kk) nh[kk] = fd[(a * D + kk) * T];
          }, K, acc, hs);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) h4[c * Nqf + j] += hs[c];
      }
      __syncthreads();
    }
    if (act) {   // lift of facet 4: y = sum_b' L2J[b'][a2] h4(a1, b'), along the eta3-line
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

template <int D, int N, bool OTF = false>
__device__ void residual_tile(const DevRef& R, const DevMesh& M, int64_t e0, int E, const Epilogue& ep) {
  extern __shared__ double sm_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm_raw);
  double* const sm = sm_raw + kResSmemHeader;
  constexpr int NC = D + 2, NF = D + 5;
  const int n = R.n, Nq = R.Nq, Nfn = R.Nfn, Ntot = R.Ntot, Np = R.Np, T = R.T;
  const ResLayout Ly = res_layout<D>(Nq, Nfn, Np, n);
  const int pe = Ly.pe;
  const double inv_gm1 = 1.0 / (M.gamma - 1.0);
  Tile tile{sm, pe, E};

  // 1. stage the elements' states with one bulk copy each (TMA), zero the residual
  //    accumulators meanwhile
  // (NF*Ntot*8 bytes per element is a multiple of 16; elements start 16-byte aligned)
  const unsigned bytes = (unsigned)(NF * Ntot * sizeof(double));
  const bool tma = ((smem_addr(sm) & 15u) | (unsigned)(reinterpret_cast<uintptr_t>(M.states) & 15)) == 0;
  if (tma) {
    if (threadIdx.x == 0) mbar_init(bar);
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier shared writes before the copies
      mbar_arrive_expect_tx(bar, bytes * (unsigned)E);
      for (int e = 0; e < E; ++e) bulk_copy_g2s(sm + e * pe + Ly.oS, M.states + (e0 + e) * NF * Ntot, bytes, bar);
    }
  } else {
    for (int idx = threadIdx.x; idx < E * NF * Ntot; idx += blockDim.x) {
      const int e = idx / (NF * Ntot);
      sm[e * pe + Ly.oS + idx % (NF * Ntot)] = M.states[e0 * NF * Ntot + idx];
    }
  }
  for (int idx = threadIdx.x; idx < E * NC * Nq; idx += blockDim.x) {
    int e = idx / (NC * Nq);
    sm[e * pe + Ly.oR + idx % (NC * Nq)] = 0.0;
  }
  if (tma) {
    const bool staged = mbar_wait(bar, 0, kWaitCycles);
    if (!__syncthreads_and(staged)) {
      if (threadIdx.x == 0) {
        atomicOr(M.flag, kFlagTimeout);
        mbar_wait(bar, 0, kWaitCycles);   // let copies still in flight land before the block exits
      }
      return;
    }
    if (threadIdx.x == 0) mbar_inval(bar);
  } else {
    __syncthreads();
  }
  // 2. interface fluxes, line-based flux differencing, facet correction and lift
  //    (Eq. (entropy_stable)), one line task per thread and phase
  {
    const FluxK K = make_fluxk(M.gamma);
    constexpr int LPL = kLineLanes<D, N>;   // threads per line task
    const int task = (int)threadIdx.x / LPL, h = (int)threadIdx.x % LPL;
    const int el = task / T, t = task % T;
    const bool act = el < E;
    const int elc = act ? el : 0;
    const int64_t eg = e0 + elc;
    const double* vdir = (act && !OTF) ? M.vdir + eg * (int64_t)R.nvp * D : nullptr;
    const double* fdir = (act && !OTF) ? M.fdir + eg * (int64_t)R.nfp * D : nullptr;
    double* base = sm + elc * pe;
#pragma unroll 1
    for (int ph = 0; ph < D; ++ph) {
      if constexpr (LPL == 2)
        line_task_split<D, N, OTF>(ph, t, h, act, R, M, eg, base + Ly.oS, base + Ly.oS + Nq, base + Ly.oR,
                                   base + Ly.oH4, vdir, fdir, K);
      else
        line_task<D, N, OTF>(ph, t, act, R, M, eg, base + Ly.oS, base + Ly.oS + Nq, base + Ly.oR, base + Ly.oH4,
                             vdir, fdir, K);
      __syncthreads();
    }
  }
  if (ep.mode == 2) {
    // diagnostics: per element sum_i r_i (per variable), sum w.r, sum |w r|
    for (int e = threadIdx.x / 32; e < E; e += blockDim.x / 32) {
      const int lane = threadIdx.x % 32;
      double acc[NC + 2];
#pragma unroll
      for (int c = 0; c < NC + 2; ++c) acc[c] = 0.0;
      for (int v = lane; v < Nq; v += 32) {
        NodeState<D> s = load_state<D>(sm + e * pe + Ly.oS, Ntot, v);
        double vv = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) vv += s.v[k] * s.v[k];
        double sent = (1.0 - M.gamma) * s.lrho - s.lbeta;   // ln(p / rho^gamma)
        double w[NC];
        w[0] = (M.gamma - sent) * inv_gm1 - 0.5 * s.beta * vv;
#pragma unroll
        for (int k = 0; k < D; ++k) w[1 + k] = s.beta * s.v[k];
        w[D + 1] = -s.beta;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double rv = sm[e * pe + Ly.oR + c * Nq + v];
          acc[c] += rv;
          acc[NC] += w[c] * rv;
          acc[NC + 1] += fabs(w[c] * rv);
        }
      }
#pragma unroll
      for (int c = 0; c < NC + 2; ++c) {
        double x = acc[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) ep.diag[(e0 + e) * (NC + 2) + c] = x;
      }
    }
    return;
  }
  // 5. d u~/dt = [V^T (W/J) V] (V^T r)   (Eq. (matvec_dudt), M = I)
  apply_VT<D>(R, tile, Ly.oR, Ly.oS1, Ly.oS2, Ly.oMod, NC);
  apply_minv<D>(R, M, tile, e0, Ly.oMod, Ly.oS1, Ly.oS2, Ly.oR, Ly.oR, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {   // result to oMod
    int e = idx / (NC * Np);
    sm[e * pe + Ly.oMod + idx % (NC * Np)] = sm[e * pe + Ly.oR + idx % (NC * Np)];
  }
  __syncthreads();
  // 6. epilogue
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np), rr = idx % (NC * Np);
    const int64_t g = (e0 + e) * NC * Np + rr;
    double k = sm[e * pe + Ly.oMod + rr];
    if (ep.mode == 0) {
      ep.dudt[g] = k;
    } else {
      double acc = ep.acc_in[g] + ep.cb * k;
      if (ep.stage_out) ep.stage_out[g] = ep.u0[g] + ep.ca * k;
      ep.acc_out[g] = acc;
    }
  }
}

}  // namespace esd
