// Host-side construction of the reference-element tables (Sections 2.5, 3, 4.3)
// and of the per-element geometric data (Sections 4.1, 4.2, 4.5, 5.1, 6) used by
// the CUDA kernels.  Runs once per mesh in esd_mesh_create; not on the hot path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <sstream>
#include <thread>

#include "esd_internal.h"

namespace esd {
namespace {

// ---------------------------------------------------------------------------
// One-dimensional building blocks (Section 2.5)
// ---------------------------------------------------------------------------

// Orthonormal Jacobi polynomials P_0..P_n^{(a,b)}(x) for the weight
// (1-x)^a (1+x)^b, from the three-term recurrence of the monic family:
// alpha_k = (b^2-a^2)/((2k+a+b)(2k+a+b+2)),
// beta_k  = 4k(k+a)(k+b)(k+a+b)/((2k+a+b)^2 (2k+a+b+1)(2k+a+b-1)),
// beta_0  = 2^(a+b+1) Gamma(a+1)Gamma(b+1)/Gamma(a+b+2).
struct JacobiRec {
  std::vector<double> al, sb;  // alpha_k, sqrt(beta_k)
  JacobiRec(int n, double a, double b) : al(n + 2), sb(n + 2) {
    for (int k = 0; k < n + 2; ++k) {
      double s = 2.0 * k + a + b;
      if (k == 0) {
        al[0] = (b - a) / (a + b + 2.0);
        sb[0] = std::sqrt(std::exp((a + b + 1.0) * std::log(2.0) + std::lgamma(a + 1.0) +
                                   std::lgamma(b + 1.0) - std::lgamma(a + b + 2.0)));
      } else {
        al[k] = (b * b - a * a) / (s * (s + 2.0));
        sb[k] = std::sqrt(4.0 * k * (k + a) * (k + b) * (k + a + b) / (s * s * (s + 1.0) * (s - 1.0)));
      }
    }
  }
  // values of P_0..P_n at x
  void eval(int n, double x, double* P) const {
    P[0] = 1.0 / sb[0];
    if (n >= 1) P[1] = (x - al[0]) * P[0] / sb[1];
    for (int k = 1; k < n; ++k) P[k + 1] = ((x - al[k]) * P[k] - sb[k] * P[k - 1]) / sb[k + 1];
  }
};

double jacobi_value(int n, double a, double b, double x) {
  JacobiRec r(n, a, b);
  std::vector<double> P(n + 1);
  r.eval(n, x, P.data());
  return P[n];
}

// Gauss rule with q+1 nodes for (1-x)^a(1+x)^b: nodes are the roots of P_{q+1},
// found by Newton's method with Maehly's deflation from Chebyshev starting
// guesses; weights are the Christoffel numbers 1 / sum_{k<=q} P_k(x_i)^2.
void gauss_rule(int q, double a, double b, std::vector<double>* x, std::vector<double>* w) {
  const int N = q + 1;
  JacobiRec rec(N, a, b);
  JacobiRec drec(N, a + 1.0, b + 1.0);
  std::vector<double> P(N + 1), dP(N + 1);
  x->assign(N, 0.0);
  w->assign(N, 0.0);
  for (int k = 0; k < N; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * N));
    if (k > 0) r = 0.5 * (r + (*x)[k - 1]);
    for (int it = 0; it < 200; ++it) {
      rec.eval(N, r, P.data());
      drec.eval(N - 1, r, dP.data());
      double f = P[N];
      double df = std::sqrt((double)N * (N + a + b + 1.0)) * dP[N - 1];
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (r - (*x)[j]);
      double delta = f / (df - f * s);
      r -= delta;
      if (std::fabs(delta) < 1e-16 * std::max(1.0, std::fabs(r))) break;
    }
    (*x)[k] = r;
  }
  std::sort(x->begin(), x->end());
  for (int i = 0; i < N; ++i) {
    rec.eval(q, (*x)[i], P.data());
    double s = 0.0;
    for (int k = 0; k <= q; ++k) s += P[k] * P[k];
    (*w)[i] = 1.0 / s;
  }
}

// Lagrange polynomial ell_j (nodes x) at t, product form of Eq. (lagrange).
double lag(const std::vector<double>& x, int j, double t) {
  double v = 1.0;
  for (size_t k = 0; k < x.size(); ++k)
    if ((int)k != j) v *= (t - x[k]) / (x[j] - x[k]);
  return v;
}

// Differentiation matrix on the nodes: D[a*n+b] = ell_b'(x_a), from the
// barycentric weights c_j = 1/prod_{k!=j}(x_j-x_k): D_ab = (c_b/c_a)/(x_a-x_b),
// D_aa = -sum_{b!=a} D_ab.
std::vector<double> diff_matrix(const std::vector<double>& x) {
  int n = (int)x.size();
  std::vector<double> c(n, 1.0), D(n * n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) c[j] /= (x[j] - x[k]);
  for (int a = 0; a < n; ++a) {
    double s = 0.0;
    for (int b = 0; b < n; ++b)
      if (b != a) {
        D[a * n + b] = (c[b] / c[a]) / (x[a] - x[b]);
        s += D[a * n + b];
      }
    D[a * n + a] = -s;
  }
  return D;
}

// ---------------------------------------------------------------------------
// Collapsed coordinates (Section 3)
// ---------------------------------------------------------------------------
void collapse(int dim, const double* e, double* xi) {
  if (dim == 2) {
    xi[0] = 0.5 * (1.0 + e[0]) * (1.0 - e[1]) - 1.0;
    xi[1] = e[1];
  } else {
    xi[0] = 0.25 * (1.0 + e[0]) * (1.0 - e[1]) * (1.0 - e[2]) - 1.0;
    xi[1] = 0.5 * (1.0 + e[1]) * (1.0 - e[2]) - 1.0;
    xi[2] = e[2];
  }
}

// d eta_k / d xi_l at a point given in collapsed coordinates (chain rule of the
// collapsed map; reproduces the factors of Eq. (d_2d) and Eq. (d_3d)).
void deta_dxi(int dim, const double* e, double c[3][3]) {
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) c[k][l] = 0.0;
  if (dim == 2) {
    c[0][0] = 2.0 / (1.0 - e[1]);
    c[0][1] = (1.0 + e[0]) / (1.0 - e[1]);
    c[1][1] = 1.0;
  } else {
    double d23 = (1.0 - e[1]) * (1.0 - e[2]);
    c[0][0] = 4.0 / d23;
    c[0][1] = 2.0 * (1.0 + e[0]) / d23;
    c[0][2] = 2.0 * (1.0 + e[0]) / d23;
    c[1][1] = 2.0 / (1.0 - e[2]);
    c[1][2] = (1.0 + e[1]) / (1.0 - e[2]);
    c[2][2] = 1.0;
  }
}

// ---------------------------------------------------------------------------
// Equispaced simplex lattice and its Lagrange basis (mapping of Eq. (poly_mapping))
// ---------------------------------------------------------------------------
struct Lattice {
  int dim, P;
  std::vector<int> bary;  // [n][dim+1] barycentric integer indices (sum P)
  std::vector<double> xi; // [n][dim]
  int size() const { return (int)xi.size() / dim; }
};

Lattice make_lattice(int dim, int P) {
  Lattice L{dim, P, {}, {}};
  if (dim == 2) {
    for (int j = 0; j <= P; ++j)
      for (int i = 0; i <= P - j; ++i) {
        L.bary.insert(L.bary.end(), {P - i - j, i, j});
        L.xi.insert(L.xi.end(), {-1.0 + 2.0 * i / P, -1.0 + 2.0 * j / P});
      }
  } else {
    for (int k = 0; k <= P; ++k)
      for (int j = 0; j <= P - k; ++j)
        for (int i = 0; i <= P - j - k; ++i) {
          L.bary.insert(L.bary.end(), {P - i - j - k, i, j, k});
          L.xi.insert(L.xi.end(), {-1.0 + 2.0 * i / P, -1.0 + 2.0 * j / P, -1.0 + 2.0 * k / P});
        }
  }
  return L;
}

// Values val[i] and xi-gradients grad[i*dim+s] of every lattice Lagrange
// polynomial at the reference point xi.  For the equispaced lattice the basis is
// a product of linear factors in the barycentric coordinates lambda:
// ell_I(lambda) = prod_k prod_{m<I_k} (P lambda_k - m) / (I_k - m).
void lattice_basis(const Lattice& L, const double* xi, double* val, double* grad) {
  const int d = L.dim, P = L.P, nb = L.size();
  double lam[4];
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    lam[k + 1] = 0.5 * (xi[k] + 1.0);
    s += lam[k + 1];
  }
  lam[0] = 1.0 - s;
  for (int i = 0; i < nb; ++i) {
    double f[4], df[4];
    for (int k = 0; k <= d; ++k) {
      int I = L.bary[i * (d + 1) + k];
      double v = 1.0, dv = 0.0;
      for (int m = 0; m < I; ++m) {
        double t = (P * lam[k] - m) / (double)(I - m);
        dv = dv * t + v * P / (double)(I - m);
        v *= t;
      }
      f[k] = v;
      df[k] = dv;
    }
    double prod = 1.0;
    for (int k = 0; k <= d; ++k) prod *= f[k];
    val[i] = prod;
    if (grad) {
      double dl[4];
      for (int k = 0; k <= d; ++k) {
        double g = df[k];
        for (int k2 = 0; k2 <= d; ++k2)
          if (k2 != k) g *= f[k2];
        dl[k] = g;
      }
      // lambda_0 = 1 - sum (xi+1)/2, lambda_{s+1} = (xi_s+1)/2
      for (int sdir = 0; sdir < d; ++sdir) grad[i * d + sdir] = 0.5 * (dl[sdir + 1] - dl[0]);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Reference tables
// ---------------------------------------------------------------------------
esd_status build_ref(int dim, int p, RefTables* R, std::string* err) {
  if (dim != 2 && dim != 3) {
    *err = "dim must be 2 or 3";
    return ESD_ERR_ARG;
  }
  int pmax = dim == 2 ? kMaxPTri : kMaxPTet;
  if (p < 1 || p > pmax) {
    std::ostringstream o;
    o << "degree p=" << p << " outside 1.." << pmax << " for dim " << dim;
    *err = o.str();
    return ESD_ERR_UNSUPPORTED;
  }
  RefTables& r = *R;
  r.dim = dim;
  r.p = p;
  const int q = p, n = q + 1;
  r.n = n;
  r.Nq = dim == 2 ? n * n : n * n * n;
  r.Np = dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
  r.Nf = dim + 1;
  r.Nqf = dim == 2 ? n : n * n;
  r.Nfn = r.Nf * r.Nqf;
  r.Ntot = r.Nq + r.Nfn;
  r.T = dim == 2 ? n : n * n;
  r.Lv = q * (q + 1) / 2;
  r.S12 = (p + 1) * (p + 2) / 2;
  r.nvp = dim * r.T * r.Lv;
  // 1D rules: LG in eta1, eta2 and on facets; Gauss-Jacobi(1,0) in eta3 (Eq. (tet_quadrature))
  gauss_rule(q, 0.0, 0.0, &r.eta[0], &r.w1[0]);
  gauss_rule(q, 0.0, 0.0, &r.eta[1], &r.w1[1]);
  if (dim == 3) gauss_rule(q, 1.0, 0.0, &r.eta[2], &r.w1[2]);
  for (int k = 0; k < dim; ++k) r.dl[k] = diff_matrix(r.eta[k]);
  r.l1m.resize(n); r.l1p.resize(n); r.l2m.resize(n); r.l3m.assign(n, 0.0); r.L2J.assign(n * n, 0.0);
  for (int a = 0; a < n; ++a) {
    r.l1m[a] = lag(r.eta[0], a, -1.0);
    r.l1p[a] = lag(r.eta[0], a, 1.0);
    r.l2m[a] = lag(r.eta[1], a, -1.0);
    if (dim == 3) {
      r.l3m[a] = lag(r.eta[2], a, -1.0);
      for (int bp = 0; bp < n; ++bp) r.L2J[bp * n + a] = lag(r.eta[1], a, r.eta[2][bp]);
    }
  }
  // PKD principal functions (Eq. (principal_functions)) at the 1D nodes
  r.psi1.assign((p + 1) * n, 0.0);
  for (int a1 = 0; a1 <= p; ++a1)
    for (int c = 0; c < n; ++c) r.psi1[a1 * n + c] = std::sqrt(2.0) * jacobi_value(a1, 0.0, 0.0, r.eta[0][c]);
  std::vector<int> off1(p + 1), s12a1, moff, mode;
  {
    int s = 0;
    for (int a1 = 0; a1 <= p; ++a1) {
      off1[a1] = s;
      s += p + 1 - a1;
    }
  }
  if (dim == 2) {
    r.psi2.assign(r.Np * n, 0.0);
    int m = 0;
    for (int a1 = 0; a1 <= p; ++a1)
      for (int a2 = 0; a2 <= p - a1; ++a2, ++m) {
        mode.push_back(a1);
        for (int c = 0; c < n; ++c)
          r.psi2[m * n + c] = std::pow(1.0 - r.eta[1][c], a1) * jacobi_value(a2, 2.0 * a1 + 1.0, 0.0, r.eta[1][c]);
      }
  } else {
    r.psi2.assign(r.S12 * n, 0.0);
    r.psi3.assign(r.Np * n, 0.0);
    int s12 = 0, m = 0;
    for (int a1 = 0; a1 <= p; ++a1)
      for (int a2 = 0; a2 <= p - a1; ++a2, ++s12) {
        s12a1.push_back(a1);
        moff.push_back(m);
        for (int c = 0; c < n; ++c)
          r.psi2[s12 * n + c] = std::pow(1.0 - r.eta[1][c], a1) * jacobi_value(a2, 2.0 * a1 + 1.0, 0.0, r.eta[1][c]);
        for (int a3 = 0; a3 <= p - a1 - a2; ++a3, ++m) {
          mode.push_back(s12);
          for (int c = 0; c < n; ++c)
            r.psi3[m * n + c] = 2.0 * std::pow(1.0 - r.eta[2][c], a1 + a2) *
                                jacobi_value(a3, 2.0 * a1 + 2.0 * a2 + 2.0, 0.0, r.eta[2][c]);
        }
      }
  }
  r.ints.clear();
  r.i_off1 = 0;
  r.ints.insert(r.ints.end(), off1.begin(), off1.end());
  r.i_s12a1 = (int)r.ints.size();
  r.ints.insert(r.ints.end(), s12a1.begin(), s12a1.end());
  r.i_moff = (int)r.ints.size();
  r.ints.insert(r.ints.end(), moff.begin(), moff.end());
  r.i_mode = (int)r.ints.size();
  r.ints.insert(r.ints.end(), mode.begin(), mode.end());
  // (alpha1, alpha2) pairs ordered by decreasing length p + 1 - alpha1 - alpha2 of their
  // alpha3 sums, so that neighbouring threads of the first V stage run equal loops
  r.i_s12len = (int)r.ints.size();
  if (dim == 3) {
    std::vector<int> ord(r.S12);
    for (int s = 0; s < r.S12; ++s) ord[s] = s;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const int la = p - s12a1[a] - (a - off1[s12a1[a]]), lb = p - s12a1[b] - (b - off1[s12a1[b]]);
      return la > lb;
    });
    r.ints.insert(r.ints.end(), ord.begin(), ord.end());
  }
  r.ints.push_back(0);
  // volume nodes, weights (Eq. (tri_quadrature), Eq. (tet_quadrature)), chain-rule factors
  r.wvol.assign(r.Nq, 0.0);
  r.xi_vol.assign(r.Nq * dim, 0.0);
  r.deta.assign(r.Nq * 9, 0.0);
  for (int v = 0; v < r.Nq; ++v) {
    int c[3] = {v % n, (v / n) % n, dim == 3 ? v / (n * n) : 0};
    double e[3] = {r.eta[0][c[0]], r.eta[1][c[1]], dim == 3 ? r.eta[2][c[2]] : 0.0};
    if (dim == 2)
      r.wvol[v] = 0.5 * (1.0 - e[1]) * r.w1[0][c[0]] * r.w1[1][c[1]];
    else
      r.wvol[v] = (1.0 - e[1]) * (1.0 - e[2]) / 8.0 * r.w1[0][c[0]] * r.w1[1][c[1]] * r.w1[2][c[2]];
    collapse(dim, e, &r.xi_vol[v * dim]);
    double cc[3][3];
    deta_dxi(dim, e, cc);
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) r.deta[v * 9 + k * 3 + l] = cc[k][l];
  }
  // facet nodes and weights (Eq. (tri_facet_quadrature_nodes), Eq. (tet_facet_quadrature_nodes),
  // Eq. (tet_facet_quadrature_weights)); outward reference normals
  r.wfac.assign(r.Nfn, 0.0);
  r.xi_fac.assign(r.Nfn * dim, 0.0);
  if (dim == 2) {
    const double s2 = std::sqrt(2.0);
    double nh[3][2] = {{0, -1}, {1 / s2, 1 / s2}, {-1, 0}};
    for (int z = 0; z < 3; ++z) {
      r.nhat[z][0] = nh[z][0];
      r.nhat[z][1] = nh[z][1];
      for (int j = 0; j < n; ++j) {
        double e[2];
        if (z == 0) { e[0] = r.eta[0][j]; e[1] = -1.0; r.wfac[j] = r.w1[0][j]; }
        if (z == 1) { e[0] = 1.0; e[1] = r.eta[1][j]; r.wfac[n + j] = s2 * r.w1[1][j]; }
        if (z == 2) { e[0] = -1.0; e[1] = r.eta[1][j]; r.wfac[2 * n + j] = r.w1[1][j]; }
        collapse(2, e, &r.xi_fac[(z * n + j) * 2]);
      }
    }
  } else {
    const double s3 = std::sqrt(3.0);
    double nh[4][3] = {{0, -1, 0}, {1 / s3, 1 / s3, 1 / s3}, {-1, 0, 0}, {0, 0, -1}};
    for (int z = 0; z < 4; ++z) {
      for (int k = 0; k < 3; ++k) r.nhat[z][k] = nh[z][k];
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          int j = a + n * b, f = z * r.Nqf + j;
          double e[3];
          double wj = r.w1[2][b];  // second facet coordinate uses the GJ(1,0) rule
          switch (z) {
            case 0: e[0] = r.eta[0][a]; e[1] = -1.0; e[2] = r.eta[2][b]; r.wfac[f] = 0.5 * r.w1[0][a] * wj; break;
            case 1: e[0] = 1.0; e[1] = r.eta[1][a]; e[2] = r.eta[2][b]; r.wfac[f] = 0.5 * s3 * r.w1[1][a] * wj; break;
            case 2: e[0] = -1.0; e[1] = r.eta[1][a]; e[2] = r.eta[2][b]; r.wfac[f] = 0.5 * r.w1[1][a] * wj; break;
            default: e[0] = r.eta[0][a]; e[1] = r.eta[2][b]; e[2] = -1.0; r.wfac[f] = 0.5 * r.w1[0][a] * wj; break;
          }
          collapse(3, e, &r.xi_fac[f * 3]);
        }
    }
  }
  // dense generalized Vandermonde V[v][m] = phi_m(xi_v) from the principal functions, and
  // the choice between a stored per-element V^T (W/J) V (Np^2 FMAs) and its
  // sum-factorised application (V, scaling, V^T)
  r.Vd.assign((size_t)r.Nq * r.Np, 0.0);
  for (int v = 0; v < r.Nq; ++v) {
    const int c1 = v % n, c2 = (v / n) % n, c3 = v / (n * n);
    int m = 0;
    for (int a1 = 0; a1 <= p; ++a1)
      for (int a2 = 0; a2 <= p - a1; ++a2) {
        if (dim == 2) {
          r.Vd[(size_t)v * r.Np + m] = r.psi1[a1 * n + c1] * r.psi2[m * n + c2];
          ++m;
        } else {
          const int s12 = off1[a1] + a2;
          for (int a3 = 0; a3 <= p - a1 - a2; ++a3, ++m)
            r.Vd[(size_t)v * r.Np + m] = r.psi1[a1 * n + c1] * r.psi2[s12 * n + c2] * r.psi3[m * n + c3];
        }
      }
  }
  {
    const long V = dim == 2 ? (long)r.Np * n + (long)r.Nq * (p + 1)
                            : (long)r.Np * n + (long)r.S12 * n * n + (long)r.Nq * (p + 1);
    r.dense_minv = (long)r.Np * r.Np <= 2 * V + r.Nq ? 1 : 0;
  }
  // facet pair phases (the line-task structure of device.cuh: line_task)
  if (dim == 2) {
    r.fph_len[0] = 2 * n;  // faces 2 and 3 along eta1-lines
    r.fph_len[1] = n;      // face 1 along eta2-lines
    r.fph_off[0] = 0;
    r.fph_off[1] = r.fph_len[0] * dim * r.T;
    r.nfp = (r.fph_len[0] + r.fph_len[1]) * r.T;
  } else {
    r.fph_len[0] = 2 * n;  // faces 2, 3 along eta1-lines
    r.fph_len[1] = n;      // face 1 along eta2-lines
    r.fph_len[2] = 0;      // eta3-lines carry no facet pairs
    r.fph_len[3] = n * n;  // face 4: (eta2, eta3) planes
    r.fph_off[0] = 0;
    r.fph_off[1] = r.fph_len[0] * dim * r.T;
    r.fph_off[2] = r.fph_off[1] + r.fph_len[1] * dim * r.T;
    r.fph_off[3] = r.fph_off[2];
    r.nfp = (r.fph_len[0] + r.fph_len[1] + r.fph_len[3]) * r.T;
  }
  return ESD_OK;
}

// ---------------------------------------------------------------------------
// Per-element geometry and pair coefficients
// ---------------------------------------------------------------------------
namespace {

struct BasisAt {  // lattice basis values/gradients at a list of points
  int npts = 0, nb = 0, dim = 0;
  std::vector<double> val, grad;  // [npts][nb], [npts][nb][dim]
};

BasisAt basis_at(const Lattice& L, const std::vector<double>& pts) {
  BasisAt B;
  B.dim = L.dim;
  B.nb = L.size();
  B.npts = (int)pts.size() / L.dim;
  B.val.resize((size_t)B.npts * B.nb);
  B.grad.resize((size_t)B.npts * B.nb * L.dim);
  for (int t = 0; t < B.npts; ++t)
    lattice_basis(L, &pts[t * L.dim], &B.val[(size_t)t * B.nb], &B.grad[(size_t)t * B.nb * L.dim]);
  return B;
}

void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

double det(int d, const double* A) {  // A[m*d+k] = d x_m / d xi_k
  if (d == 2) return A[0] * A[3] - A[1] * A[2];
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

}  // namespace

esd_status build_host_mesh(const esd_mesh_desc& d, HostMesh* H, std::string* err, int tables, int64_t n_ghost) {
  const bool es = (tables & kTablesEntropyStable) != 0, skew = (tables & kTablesSkew) != 0;
  const bool metrics = (tables & kTablesMetrics) != 0;
  esd_status st = build_ref(d.dim, d.p, &H->ref, err);
  if (st != ESD_OK) return st;
  const RefTables& r = H->ref;
  const int dim = r.dim, n = r.n, Nq = r.Nq, Nfn = r.Nfn, Nqf = r.Nqf, T = r.T;
  const int64_t E = d.n_elem;
  // partition meshes: the last n_ghost elements are ghosts; their geometry is computed (their
  // facet nodes are matched against the local elements') but only local elements are kept
  if (n_ghost < 0 || n_ghost >= E) {
    *err = "n_ghost must be in [0, n_elem)";
    return ESD_ERR_ARG;
  }
  const int64_t El = E - n_ghost;
  H->E = El;
  Lattice Lmap = make_lattice(dim, d.p);
  const int nmap = Lmap.size();
  // points: volume nodes, facet nodes, mapping lattice nodes, (3D) curl interpolation nodes
  std::vector<double> pts(r.xi_vol);
  pts.insert(pts.end(), r.xi_fac.begin(), r.xi_fac.end());
  pts.insert(pts.end(), Lmap.xi.begin(), Lmap.xi.end());
  Lattice Lint = make_lattice(dim, d.p + 1);
  if (dim == 3) pts.insert(pts.end(), Lint.xi.begin(), Lint.xi.end());
  BasisAt Bm = basis_at(Lmap, pts);
  const int o_fac = Nq, o_lat = Nq + Nfn, o_int = Nq + Nfn + nmap;
  std::vector<double> tgt(r.xi_vol);
  tgt.insert(tgt.end(), r.xi_fac.begin(), r.xi_fac.end());
  BasisAt Bi;
  if (dim == 3) Bi = basis_at(Lint, tgt);
  const int nint = dim == 3 ? Lint.size() : 0;

  H->vdir.assign(es ? (size_t)E * r.nvp * dim : 0, 0.0);
  H->fdir.assign(es ? (size_t)E * r.nfp * dim : 0, 0.0);
  H->sdir.assign(skew ? (size_t)E * dim * T * n * (n - 1) * dim : 0, 0.0);
  H->gvol.assign(metrics ? (size_t)E * dim * dim * Nq : 0, 0.0);
  H->jnf.assign(metrics ? (size_t)E * dim * Nfn : 0, 0.0);
  H->wj.assign((size_t)E * Nq, 0.0);
  H->wdj.assign((size_t)E * Nq, 0.0);
  H->bj.assign((size_t)E * Nfn, 0.0);
  H->nrm.assign((size_t)E * dim * Nfn, 0.0);
  H->nbr_e.assign((size_t)E * Nfn, 0);
  H->nbr_f.assign((size_t)E * Nfn, 0);
  H->xvol.assign((size_t)E * Nq * dim, 0.0);
  H->minv.assign(r.dense_minv ? (size_t)E * r.Np * r.Np : 0, 0.0);
  std::vector<double> xfac((size_t)E * Nfn * dim);   // physical facet node positions (matching)
  std::vector<double> Jnfac((size_t)E * Nfn * dim);  // G^T nhat at facet nodes
  std::vector<double> hsize(E);
  std::vector<std::string> errs(E);
  std::vector<int> bad(E, 0);

  auto work = [&](int64_t e0, int64_t e1) {
    std::vector<double> X(nmap * dim), A((Nq + Nfn) * 9), G((Nq + Nfn) * 9);
    std::vector<double> detl(nmap), rv((size_t)nint * 9);
    for (int64_t e = e0; e < e1; ++e) {
      const double* Xg = d.map_nodes + (size_t)e * nmap * dim;
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int i = 0; i < nmap; ++i)
        for (int k = 0; k < dim; ++k) {
          X[i * dim + k] = Xg[i * dim + k] - Xg[k];  // element-local translation
          lo[k] = std::min(lo[k], Xg[i * dim + k]);
          hi[k] = std::max(hi[k], Xg[i * dim + k]);
        }
      double hs = 0.0;
      for (int k = 0; k < dim; ++k) hs = std::max(hs, hi[k] - lo[k]);
      hsize[e] = hs;
      // positions and Jacobians at volume and facet nodes
      for (int t = 0; t < Nq + Nfn; ++t) {
        const double* val = &Bm.val[(size_t)t * nmap];
        const double* gr = &Bm.grad[(size_t)t * nmap * dim];
        double x[3] = {0, 0, 0}, Ad[9] = {0};
        for (int i = 0; i < nmap; ++i)
          for (int m = 0; m < dim; ++m) {
            x[m] += val[i] * Xg[i * dim + m];
            for (int k = 0; k < dim; ++k) Ad[m * dim + k] += gr[i * dim + k] * X[i * dim + m];
          }
        for (int m = 0; m < 9; ++m) A[t * 9 + m] = Ad[m];
        if (t < Nq)
          for (int m = 0; m < dim; ++m) H->xvol[((size_t)e * Nq + t) * dim + m] = x[m];
        else
          for (int m = 0; m < dim; ++m) xfac[((size_t)e * Nfn + (t - Nq)) * dim + m] = x[m];
      }
      // metric terms G_lm = J d xi_l / d x_m (stored G[t*9 + l*3 + m])
      if (dim == 2) {
        for (int t = 0; t < Nq + Nfn; ++t) {
          const double* Ad = &A[t * 9];  // Ad[m*2+k] = d x_m/d xi_k
          double* Gt = &G[t * 9];
          Gt[0 * 3 + 0] = Ad[1 * 2 + 1];
          Gt[0 * 3 + 1] = -Ad[0 * 2 + 1];
          Gt[1 * 3 + 0] = -Ad[1 * 2 + 0];
          Gt[1 * 3 + 1] = Ad[0 * 2 + 0];
        }
      } else {
        // conservative curl form, Eq. (metric_interpolants) and Eq. (conservative_curl):
        // r1 = x3 grad x2, r2 = x3 grad x1, r3 = x1 grad x2 at the degree-(q+1) lattice,
        // G(:, m) = (-curl r1, curl r2, curl r3)_m of the interpolant
        for (int i = 0; i < nint; ++i) {
          const double* val = &Bm.val[(size_t)(o_int + i) * nmap];
          const double* gr = &Bm.grad[(size_t)(o_int + i) * nmap * 3];
          double x[3] = {0, 0, 0}, g[3][3] = {{0}};
          for (int a = 0; a < nmap; ++a)
            for (int m = 0; m < 3; ++m) {
              x[m] += val[a] * X[a * 3 + m];
              for (int k = 0; k < 3; ++k) g[m][k] += gr[a * 3 + k] * X[a * 3 + m];
            }
          for (int k = 0; k < 3; ++k) {
            rv[i * 9 + 0 * 3 + k] = x[2] * g[1][k];
            rv[i * 9 + 1 * 3 + k] = x[2] * g[0][k];
            rv[i * 9 + 2 * 3 + k] = x[0] * g[1][k];
          }
        }
        for (int t = 0; t < Nq + Nfn; ++t) {
          const double* gr = &Bi.grad[(size_t)t * nint * 3];
          double c[3][3] = {{0}};
          for (int i = 0; i < nint; ++i)
            for (int col = 0; col < 3; ++col) {
              double cr[3];
              cross3(&gr[i * 3], &rv[i * 9 + col * 3], cr);
              for (int l = 0; l < 3; ++l) c[col][l] += cr[l];
            }
          for (int l = 0; l < 3; ++l) {
            G[t * 9 + l * 3 + 0] = -c[0][l];
            G[t * 9 + l * 3 + 1] = c[1][l];
            G[t * 9 + l * 3 + 2] = c[2][l];
          }
        }
      }
      // interpolated Jacobian determinant (Eq. (jacobian_approx)) and weights
      for (int i = 0; i < nmap; ++i) {
        const double* gr = &Bm.grad[(size_t)(o_lat + i) * nmap * dim];
        double Ad[9] = {0};
        for (int a = 0; a < nmap; ++a)
          for (int m = 0; m < dim; ++m)
            for (int k = 0; k < dim; ++k) Ad[m * dim + k] += gr[a * dim + k] * X[a * dim + m];
        detl[i] = det(dim, Ad);
        if (!(detl[i] > 0.0)) bad[e] = 1;
      }
      for (int v = 0; v < Nq; ++v) {
        double J = 0.0;
        const double* val = &Bm.val[(size_t)v * nmap];
        for (int i = 0; i < nmap; ++i) J += val[i] * detl[i];
        if (!(J > 0.0)) bad[e] = 1;
        H->wj[(size_t)e * Nq + v] = r.wvol[v] * J;
        H->wdj[(size_t)e * Nq + v] = r.wvol[v] / J;
      }
      if (r.dense_minv) {   // weight-adjusted inverse V^T (W/J) V, Eq. (weight_adjusted_inverse)
        const int Np = r.Np;
        double* Mi = &H->minv[(size_t)e * Np * Np];
        const double* wd = &H->wdj[(size_t)e * Nq];
        for (int i = 0; i < Np; ++i)
          for (int j = i; j < Np; ++j) {
            double s = 0.0;
            for (int v = 0; v < Nq; ++v) s += r.Vd[(size_t)v * Np + i] * wd[v] * r.Vd[(size_t)v * Np + j];
            Mi[i * Np + j] = s;
            Mi[j * Np + i] = s;
          }
      }
      // facet normals and weights (Eq. (nanson))
      for (int f = 0; f < Nfn; ++f) {
        int z = f / Nqf;
        double Jn[3] = {0, 0, 0}, nn = 0.0;
        for (int m = 0; m < dim; ++m) {
          for (int l = 0; l < dim; ++l) Jn[m] += G[(Nq + f) * 9 + l * 3 + m] * r.nhat[z][l];
          nn += Jn[m] * Jn[m];
        }
        nn = std::sqrt(nn);
        for (int m = 0; m < dim; ++m) {
          Jnfac[((size_t)e * Nfn + f) * dim + m] = Jn[m];
          if (metrics) H->jnf[((size_t)e * dim + m) * Nfn + f] = Jn[m];
          H->nrm[((size_t)e * dim + m) * Nfn + f] = Jn[m] / nn;
        }
        H->bj[(size_t)e * Nfn + f] = r.wfac[f] * nn;
      }
      if (metrics)   // metric terms at the volume nodes, component-major
        for (int v = 0; v < Nq; ++v)
          for (int l = 0; l < dim; ++l)
            for (int mm = 0; mm < dim; ++mm)
              H->gvol[((size_t)e * dim * dim + l * dim + mm) * Nq + v] = G[v * 9 + l * 3 + mm];
      // line node indices: node a of line t of phase ph
      auto line_node = [&](int ph, int t, int a) {
        if (dim == 2) return ph == 0 ? a + n * t : t + n * a;
        if (ph == 0) return a + n * t;
        if (ph == 1) return (t % n) + n * (a + n * (t / n));
        return t + n * n * a;
      };
      // skew-symmetric form (Eq. (rhs_skew)) as line pairs: for nodes i (index a) and j
      // (index b) of an eta_k-line, c^m_ij = 1/2 sum_l (Q^(l)_ji G_lm(x_j) - G_lm(x_i) Q^(l)_ij),
      // stored [phase][slot b (n-1) + (a < b ? a : a - 1)][m][task]
      if (skew) {
        double* sd = &H->sdir[(size_t)e * dim * T * n * (n - 1) * dim];
        for (int ph = 0; ph < dim; ++ph)
          for (int t = 0; t < T; ++t)
            for (int b = 0; b < n; ++b)
              for (int a = 0; a < n; ++a) {
                if (a == b) continue;
                const int vi = line_node(ph, t, a), vj = line_node(ph, t, b);
                const double* Dk = r.dl[ph].data();
                const int slot = b * (n - 1) + (a < b ? a : a - 1);
                for (int mm = 0; mm < dim; ++mm) {
                  double c = 0.0;
                  for (int l = 0; l < dim; ++l) {
                    const double Qij = r.wvol[vi] * r.deta[vi * 9 + ph * 3 + l] * Dk[a * n + b];
                    const double Qji = r.wvol[vj] * r.deta[vj * 9 + ph * 3 + l] * Dk[b * n + a];
                    c += Qji * G[vj * 9 + l * 3 + mm] - G[vi * 9 + l * 3 + mm] * Qij;
                  }
                  sd[(((size_t)ph * n * (n - 1) + slot) * dim + mm) * T + t] = 0.5 * c;
                }
              }
      }
      if (!es) continue;
      // volume pair directions: n_ij = sum_l S^(l)_ij (G_l.(xi_i) + G_l.(xi_j)), with the
      // line entries of S^(l) from Q^(l)_ij = w_i (d eta_k/d xi_l)(xi_i) ell'_{k,b}(eta_{k,a})
      double* vd = &H->vdir[(size_t)e * r.nvp * dim];
      for (int ph = 0; ph < dim; ++ph)
        for (int t = 0; t < T; ++t) {
          int m = 0;
          for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b, ++m) {
              int vi, vj;
              if (dim == 2) {
                vi = ph == 0 ? a + n * t : t + n * a;
                vj = ph == 0 ? b + n * t : t + n * b;
              } else {
                int t0 = t % n, t1 = t / n;
                if (ph == 0) { vi = a + n * t; vj = b + n * t; }
                else if (ph == 1) { vi = t0 + n * (a + n * t1); vj = t0 + n * (b + n * t1); }
                else { vi = t + n * n * a; vj = t + n * n * b; }
              }
              const double* Dk = r.dl[ph].data();
              double nij[3] = {0, 0, 0};
              for (int l = 0; l < dim; ++l) {
                double Qij = r.wvol[vi] * r.deta[vi * 9 + ph * 3 + l] * Dk[a * n + b];
                double Qji = r.wvol[vj] * r.deta[vj * 9 + ph * 3 + l] * Dk[b * n + a];
                double S = 0.5 * (Qij - Qji);
                for (int mm = 0; mm < dim; ++mm) nij[mm] += S * (G[vi * 9 + l * 3 + mm] + G[vj * 9 + l * 3 + mm]);
              }
              // stored halved: the kernels use n/2 (device.cuh, ec_flux_fast)
              for (int mm = 0; mm < dim; ++mm) vd[((size_t)(ph * r.Lv + m) * dim + mm) * T + t] = 0.5 * nij[mm];
            }
        }
      // facet pair directions: [R^T B]_ij * (G(xi_i)^T nhat + G(xi_j^zeta)^T nhat) / 2
      double* fd = &H->fdir[(size_t)e * r.nfp * dim];
      auto facet_pair = [&](int off, int m, int t, int vi, int f, double RB) {
        int z = f / Nqf;
        for (int mm = 0; mm < dim; ++mm) {
          double a = 0.0, b = 0.0;
          for (int l = 0; l < dim; ++l) {
            a += G[vi * 9 + l * 3 + mm] * r.nhat[z][l];
            b += G[(Nq + f) * 9 + l * 3 + mm] * r.nhat[z][l];
          }
          fd[off + ((size_t)m * dim + mm) * T + t] = 0.5 * (RB * 0.5 * (a + b));   // stored halved
        }
      };
      for (int t = 0; t < T; ++t) {
        // phase 1: eta1-line t with facet 2 (eta1 = +1) and facet 3 (eta1 = -1) nodes
        for (int a = 0; a < n; ++a) {
          int vi = a + n * t;
          facet_pair(r.fph_off[0], a, t, vi, 1 * Nqf + t, r.l1p[a] * r.wfac[1 * Nqf + t]);
          facet_pair(r.fph_off[0], n + a, t, vi, 2 * Nqf + t, r.l1m[a] * r.wfac[2 * Nqf + t]);
        }
        // phase 2: eta2-line with facet 1 (eta2 = -1) node
        for (int b = 0; b < n; ++b) {
          int vi, f;
          if (dim == 2) { vi = t + n * b; f = t; }
          else { vi = (t % n) + n * (b + n * (t / n)); f = t; }
          facet_pair(r.fph_off[1], b, t, vi, f, r.l2m[b] * r.wfac[f]);
        }
        if (dim == 3) {
          // phase 4: task t = a + n*b2 owns volume nodes (a, b2, b3); facet-4 nodes (a, b')
          int a = t % n, b2 = t / n;
          int m = 0;
          for (int bp = 0; bp < n; ++bp)
            for (int b3 = 0; b3 < n; ++b3, ++m) {
              int vi = a + n * (b2 + n * b3);
              int f = 3 * Nqf + a + n * bp;
              facet_pair(r.fph_off[3], m, t, vi, f, r.L2J[bp * n + b2] * r.l3m[b3] * r.wfac[f]);
            }
        }
      }
    }
  };
  {
    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    int64_t chunk = (E + nth - 1) / nth;
    for (unsigned i = 0; i < nth; ++i) {
      int64_t a = i * chunk, b = std::min<int64_t>(E, a + chunk);
      if (a < b) th.emplace_back(work, a, b);
    }
    for (auto& t : th) t.join();
  }
  for (int64_t e = 0; e < E; ++e)
    if (bad[e]) {
      std::ostringstream o;
      o << "element " << e << " has a non-positive Jacobian determinant";
      *err = o.str();
      return ESD_ERR_MESH;
    }
  // facet matching (Assumption 2): identity or reversal of the first facet coordinate,
  // positions equal up to one constant shift; normals opposite, B J equal.
  std::vector<int> perm_id(Nqf), perm_rev(Nqf);
  for (int j = 0; j < Nqf; ++j) {
    perm_id[j] = j;
    int a = j % n, b = j / n;
    perm_rev[j] = dim == 2 ? n - 1 - j : (n - 1 - a) + n * b;
  }
  std::vector<int> fail(El, 0);
  auto match = [&](int64_t e0, int64_t e1) {   // local elements only: ghosts are not computed
    for (int64_t e = e0; e < e1; ++e)
      for (int z = 0; z < r.Nf; ++z) {
        int64_t e2 = d.nbr_elem[e * r.Nf + z];
        int z2 = d.nbr_face[e * r.Nf + z];
        if (e2 < 0 || e2 >= E || z2 < 0 || z2 >= r.Nf || (e2 == e && z2 == z)) {
          fail[e] = 1;
          continue;
        }
        if (d.nbr_elem[e2 * r.Nf + z2] != e || d.nbr_face[e2 * r.Nf + z2] != z) {
          fail[e] = 2;
          continue;
        }
        const std::vector<int>* found = nullptr;
        for (const std::vector<int>* P : {&perm_id, &perm_rev}) {
          double d0[3], worst = 0.0;
          for (int j = 0; j < Nqf; ++j) {
            for (int m = 0; m < dim; ++m) {
              double dd = xfac[((size_t)e * Nfn + z * Nqf + j) * dim + m] -
                          xfac[((size_t)e2 * Nfn + z2 * Nqf + (*P)[j]) * dim + m];
              if (j == 0) d0[m] = dd;
              worst = std::max(worst, std::fabs(dd - d0[m]));
            }
          }
          if (worst < 1e-9 * hsize[e]) {
            found = P;
            break;
          }
        }
        if (!found) {
          fail[e] = 3;
          continue;
        }
        for (int j = 0; j < Nqf; ++j) {
          int f = z * Nqf + j, f2 = z2 * Nqf + (*found)[j];
          double sn = 0.0;
          for (int m = 0; m < dim; ++m)
            sn = std::max(sn, std::fabs(H->nrm[((size_t)e * dim + m) * Nfn + f] + H->nrm[((size_t)e2 * dim + m) * Nfn + f2]));
          double b1 = H->bj[(size_t)e * Nfn + f], b2 = H->bj[(size_t)e2 * Nfn + f2];
          if (sn > 1e-8 || std::fabs(b1 - b2) > 1e-8 * std::fabs(b1)) fail[e] = 4;
          H->nbr_e[(size_t)e * Nfn + f] = (int32_t)e2;
          H->nbr_f[(size_t)e * Nfn + f] = f2;
        }
      }
  };
  {
    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    int64_t chunk = (El + nth - 1) / nth;
    for (unsigned i = 0; i < nth; ++i) {
      int64_t a = i * chunk, b = std::min<int64_t>(El, a + chunk);
      if (a < b) th.emplace_back(match, a, b);
    }
    for (auto& t : th) t.join();
  }
  for (int64_t e = 0; e < El; ++e)
    if (fail[e]) {
      static const char* why[] = {"", "neighbour index out of range", "connectivity not symmetric",
                                  "facet nodes do not coincide with the neighbour's",
                                  "normals/weights differ from the neighbour's"};
      std::ostringstream o;
      o << "element " << e << ": " << why[fail[e]];
      *err = o.str();
      return ESD_ERR_MESH;
    }
  if (n_ghost > 0) {   // keep the local elements' tables ([E][...] arrays, element-major)
    auto keep = [&](auto& v) { v.resize(v.size() / (size_t)E * (size_t)El); };
    keep(H->vdir); keep(H->fdir); keep(H->sdir); keep(H->gvol); keep(H->jnf); keep(H->wj); keep(H->wdj);
    keep(H->bj); keep(H->nrm); keep(H->nbr_e); keep(H->nbr_f); keep(H->xvol); keep(H->minv);
  }
  return ESD_OK;
}

// Tables of the table-driven log (after Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", 1990) and exp (after Tang,
// "Table-driven implementation of the exponential function in IEEE floating-point
// arithmetic", 1989), computed in long double.  High parts carry trailing zeros so that
// k * ln2_hi + (ln F)_hi and n * (ln2/32)_hi are exact in double.
void build_math_table(double* t) {
  auto round_to = [](long double v, int bits_after_point) {   // v rounded to a multiple of 2^-bits
    long double s = std::ldexp(1.0L, bits_after_point);
    return (double)(std::nearbyint(v * s) / s);
  };
  const long double ln2 = std::log(2.0L);
  for (int j = 0; j <= 128; ++j) {
    const long double F = 1.0L + j / 128.0L;
    t[j] = (double)(1.0L / F);
    const long double L = std::log(F);
    const double hi = round_to(L, 42);
    t[129 + j] = hi;
    t[258 + j] = (double)(L - (long double)hi);
  }
  for (int j = 0; j < 32; ++j) {
    const long double S = std::exp2((long double)j / 32.0L);
    const double hi = (double)S;
    t[387 + j] = hi;
    t[419 + j] = (double)(S - (long double)hi);
  }
  const double ln2_hi = round_to(ln2, 32);
  t[451] = ln2_hi;
  t[452] = (double)(ln2 - (long double)ln2_hi);
  // F_128 = 2: store ln 2 split exactly like the k ln 2 term, so that for x just below 1
  // (k = -1, j = 128) both halves cancel exactly and only the polynomial remains.
  t[129 + 128] = t[451];
  t[258 + 128] = t[452];
  const long double l32 = ln2 / 32.0L;
  const double l32_hi = round_to(l32, 46);
  t[453] = l32_hi;
  t[454] = (double)(l32 - (long double)l32_hi);
  t[455] = (double)(32.0L / ln2);
}

}  // namespace esd
