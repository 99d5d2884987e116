// CUDA kernels (sm_103a, FP64) for the entropy-stable tensor-product DSEM.
//
//   project_kernel   : u~ -> u = V u~ -> W(u) -> weight-adjusted entropy projection
//                      (Eq. (matvec_entropy_projection)) -> w, R w -> entropy-projected
//                      conservative states U(w) at volume and facet nodes, stored with
//                      the per-node quantities the two-point flux needs.
//   residual_kernel  : interface flux (Eq. (interface_flux)), line-based volume flux
//                      differencing and facet correction (Eq. (entropy_stable) evaluated
//                      along collapsed-coordinate lines, Remark 4), lift R^T, and the
//                      weight-adjusted inverse (Eq. (matvec_dudt)), with an RK4 epilogue.
//
// One CTA owns a tile of elements; every per-element working array lives in
// shared memory.  All arithmetic is FP64: GB300 issues FP64 at 1/64 of the FP32
// rate, so the kernels are organised to keep the FP64 pipe busy with useful
// lanes (uniform per-thread work within a phase) and to move everything that is
// mesh-static (pair directions, weights, normals) to precomputed tables in HBM.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <string>

#include "adjoint.cuh"

namespace esd {

template <int D>
__global__ void project_kernel(DevRef R, DevMesh M, int epc, const double* __restrict__ u,
                               double* __restrict__ w_modal) {
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  project_tile<D>(R, M, e0, E, u, w_modal);
}

// ---------------------------------------------------------------------------
// Volume integrals of the conserved variables and of the entropy function
// S(u) = -rho s / (gamma - 1), s = ln(p / rho^gamma) (Section 7.1), with the quadrature of
// the mass matrix (W J, interpolated J): per element sum_i (W J)_i u_i and
// sum_i (W J)_i S(u_i) at the volume nodes, u = V u~.  part: [E][N_c + 1].
// ---------------------------------------------------------------------------
template <int D>
__global__ void integrals_kernel(DevRef R, DevMesh M, int epc, const double* __restrict__ u,
                                 double* __restrict__ part) {
  extern __shared__ double sm[];
  constexpr int NC = D + 2;
  const int Np = R.Np, Nq = R.Nq;
  const int oM = 0, oA = NC * Np, oB = oA + NC * Nq, oC = oB + NC * Nq;
  const int pe = oC + NC * Nq;
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  Tile t{sm, pe, E};
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    const int e = idx / (NC * Np), r = idx % (NC * Np);
    sm[e * pe + oM + r] = u[(e0 + e) * NC * Np + r];
  }
  __syncthreads();
  apply_V<D>(R, t, oM, oB, oC, oA, NC);
  const double gamma = M.gamma, inv_gm1 = 1.0 / (gamma - 1.0);
  const int lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int e = threadIdx.x / 32; e < E; e += nw) {
    double acc[NC + 1];
#pragma unroll
    for (int c = 0; c <= NC; ++c) acc[c] = 0.0;
    for (int v = lane; v < Nq; v += 32) {
      const double wj = M.wj[(e0 + e) * Nq + v];
      double uc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        uc[c] = sm[e * pe + oA + c * Nq + v];
        acc[c] = fma(wj, uc[c], acc[c]);
      }
      double vv = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) vv = fma(uc[1 + k], uc[1 + k], vv);
      const double rho = uc[0];
      const double p = (gamma - 1.0) * (uc[D + 1] - 0.5 * vv * rcp_nr<2>(rho));
      const double sent = log_tab(p, R.mtab) - gamma * log_tab(rho, R.mtab);
      acc[NC] = fma(wj, -rho * sent * inv_gm1, acc[NC]);
    }
#pragma unroll
    for (int c = 0; c <= NC; ++c) {
      double x = acc[c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) part[(e0 + e) * (NC + 1) + c] = x;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched execution of many meshes (one launch per kernel and dimension): a
// persistent grid walks a list of (mesh, element tile) items; each item runs the
// same tile code with that mesh's tables, layout and epilogue.
// ---------------------------------------------------------------------------
template <int D>
__global__ void project_batch_kernel(const BatchMesh* __restrict__ meshes, const BatchItem* __restrict__ items,
                                     int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem w = items[it];
    const BatchMesh& bm = meshes[w.mesh];
    project_tile<D>(bm.R, bm.M, w.e0, w.E, bm.u, nullptr);
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Reference L2 projection u~ = V^T W u of nodal input data (input preparation)
// ---------------------------------------------------------------------------
template <int D>
__global__ void l2_project_kernel(DevRef R, DevMesh M, int epc, const double* __restrict__ un,
                                  double* __restrict__ um) {
  extern __shared__ double sm[];
  constexpr int NC = D + 2;
  const int Nq = R.Nq, Np = R.Np;
  const int pe = 3 * NC * Nq + NC * Np;
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  Tile t{sm, pe, E};
  for (int idx = threadIdx.x; idx < E * NC * Nq; idx += blockDim.x) {
    int e = idx / (NC * Nq), rr = idx % (NC * Nq);
    sm[e * pe + rr] = un[(e0 + e) * NC * Nq + rr] * R.wvol[rr % Nq];
  }
  __syncthreads();
  apply_VT<D>(R, t, 0, NC * Nq, 2 * NC * Nq, 3 * NC * Nq, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np), rr = idx % (NC * Np);
    um[(e0 + e) * NC * Np + rr] = sm[e * pe + 3 * NC * Nq + rr];
  }
}

template <int D>
__global__ void residual_adjoint_kernel(DevRef R, DevMesh M, int epc, const double* __restrict__ cot,
                                        double* qbar, double* __restrict__ qext) {
  extern __shared__ double sm[];
  constexpr int NC = D + 2, NF = D + 5, NQ = D + 2;
  const int n = R.n, Nq = R.Nq, Nfn = R.Nfn, Ntot = R.Ntot, Np = R.Np, T = R.T, Nqf = R.Nqf;
  const AdjLayout Ly = adj_layout<D>(Nq, Nfn, Np, n);
  const int pe = Ly.pe;
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  const double inv_gm1 = 1.0 / (M.gamma - 1.0);
  Tile tile{sm, pe, E};
  // 1. r_b = V V^T (W/J) V cot   (transpose of d u~/dt = V^T (W/J) V V^T r)
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np), r = idx % (NC * Np);
    sm[e * pe + Ly.oM + r] = cot[(e0 + e) * NC * Np + r];
  }
  __syncthreads();
  apply_minv<D>(R, M, tile, e0, Ly.oM, Ly.oS1, Ly.oS2, Ly.oRb, Ly.oRb, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np);
    sm[e * pe + Ly.oM + idx % (NC * Np)] = sm[e * pe + Ly.oRb + idx % (NC * Np)];
  }
  __syncthreads();
  apply_V<D>(R, tile, Ly.oM, Ly.oS1, Ly.oS2, Ly.oRb, NC);
  // 2. h_b = -R r_b  (r -= R^T h in the forward).  From here on r_b and h_b are held doubled
  //    (the pair tables hold n/2; see load_dir), exactly: scaling by 2 rounds nothing.
  apply_R<D>(R, tile, Ly.oRb, Ly.oS1, Ly.oHb, NC);
  for (int idx = threadIdx.x; idx < E * NC * Nfn; idx += blockDim.x) {
    int e = idx / (NC * Nfn);
    sm[e * pe + Ly.oHb + idx % (NC * Nfn)] *= -2.0;
  }
  for (int idx = threadIdx.x; idx < E * NC * Nq; idx += blockDim.x) {
    int e = idx / (NC * Nq);
    sm[e * pe + Ly.oRb + idx % (NC * Nq)] *= 2.0;
  }
  // 3. states, zero cotangents
  for (int idx = threadIdx.x; idx < E * NF * Ntot; idx += blockDim.x) {
    int e = idx / (NF * Ntot), r = idx % (NF * Ntot), f = r / Ntot, k = r % Ntot;
    double val = M.states[(e0 + e) * NF * Ntot + r];
    if (k < Nq)
      sm[e * pe + Ly.oSv + f * Nq + k] = val;
    else
      sm[e * pe + Ly.oSf + f * Nfn + (k - Nq)] = val;
  }
  __syncthreads();
  // 1/p at every node, once, where the layout has room for it (else per pair)
  if (Ly.oIp >= 0)
    for (int idx = threadIdx.x; idx < E * Ntot; idx += blockDim.x) {
      const int e = idx / Ntot, k = idx % Ntot;
      const double pk = k < Nq ? sm[e * pe + Ly.oSv + (D + 1) * Nq + k] : sm[e * pe + Ly.oSf + (D + 1) * Nfn + (k - Nq)];
      sm[e * pe + Ly.oIp + k] = rcp_nr<2>(pk);
    }
  // q_b of element e: volume node v of variable c at qv_e[c * qvs + v], facet node f at
  // qf_e[c * qfs + f] (shared memory, or the global output itself when it does not fit)
  const int qvs = Ly.glob ? Ntot : Nq, qfs = Ly.glob ? Ntot : Nfn;
  auto qv_of = [&](int e) { return Ly.glob ? qbar + (e0 + e) * NQ * Ntot : sm + e * pe + Ly.oQv; };
  auto qf_of = [&](int e) { return Ly.glob ? qbar + (e0 + e) * NQ * Ntot + Nq : sm + e * pe + Ly.oQf; };
  for (int idx = threadIdx.x; idx < E * NQ * Ntot; idx += blockDim.x) {
    int e = idx / (NQ * Ntot);
    if (Ly.glob)
      qbar[e0 * NQ * Ntot + idx] = 0.0;
    else
      sm[e * pe + Ly.oQv + idx % (NQ * Ntot)] = 0.0;   // qv and qf are contiguous
  }
  if (Ly.conc) {   // the families' copies (volume nodes, facet-4 nodes) are contiguous
    const int nx = (D - 1) * NQ * (Nq + (D == 3 ? n * n : 0));
    for (int idx = threadIdx.x; idx < E * nx; idx += blockDim.x) {
      const int e = idx / nx;
      sm[e * pe + Ly.oQvx + idx % nx] = 0.0;
    }
  }
  __syncthreads();
  // 4. interface flux adjoint: f*_b = B J h_b
  for (int idx = threadIdx.x; idx < E * Nfn; idx += blockDim.x) {
    int e = idx / Nfn, f = idx % Nfn;
    const int64_t eg = e0 + e;
    NodeState<D> L = load_state<D>(sm + e * pe + Ly.oSf, Nfn, f);
    const int64_t e2 = M.nbr_e[eg * Nfn + f];
    const int f2 = M.nbr_f[eg * Nfn + f];
    NodeState<D> Rr = load_state<D>(M.states + e2 * NF * Ntot + Nq, Ntot, f2);
    double nn[D];
#pragma unroll
    for (int k = 0; k < D; ++k) nn[k] = M.nrm[(eg * D + k) * Nfn + f];
    const double bj = 0.5 * M.bj[eg * Nfn + f];   // h_b is held doubled
    double fb[NC], qL[NQ], qR[NQ];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      fb[c] = bj * sm[e * pe + Ly.oHb + c * Nfn + f];
      qL[c] = 0.0;
      qR[c] = 0.0;
    }
    iface_adj<D>(L, Rr, nn, inv_gm1, M.cfac[eg * Nfn + f], M.cfac[e2 * Nfn + f2], M.lf, fb, qL, qR);
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
      qf_of(e)[c * qfs + f] = qL[c];
      qext[(eg * NQ + c) * Nfn + f] = qR[c];
    }
  }
  __syncthreads();
  // 5. pair adjoints, same task structure as the forward phases.  With `conc` the D line
  //    families run at once (D x T tasks per element), family k > 0 adding its volume-node
  //    cotangents to its own copy; the copies are summed in a fixed order afterwards, so the
  //    result does not depend on timing.  Facet nodes of faces 1-3 belong to one family each.
  const int tid = threadIdx.x;
  const int tpf = ((epc * T + 31) / 32) * 32;   // threads per family (whole warps)
  const int fam = Ly.conc ? tid / tpf : 0, rem = Ly.conc ? tid % tpf : tid;
  const int el = rem / T, t = rem % T;
  const bool active = el < E && fam < D;
  const int64_t eg = e0 + el;
  const double* vdir = active ? M.vdir + eg * (int64_t)R.nvp * D : nullptr;
  const double* fdir = active ? M.fdir + eg * (int64_t)R.nfp * D : nullptr;
  const double* Sv = sm + el * pe + Ly.oSv;
  const double* Sf = sm + el * pe + Ly.oSf;
  const double* rb = sm + el * pe + Ly.oRb;
  const double* hb = sm + el * pe + Ly.oHb;
  double* qv = !active ? nullptr : (fam > 0 ? sm + el * pe + Ly.oQvx + (fam - 1) * NQ * Nq : qv_of(el));
  double* qf = active ? qf_of(el) : nullptr;
  const double* ipn = sm + el * pe + (Ly.oIp >= 0 ? Ly.oIp : 0);   // [Nq volume | Nfn facet]
  const bool have_ip = Ly.oIp >= 0;
  auto ip_v = [&](const NodeState<D>& S, int v) { return have_ip ? ipn[v] : rcp_nr<2>(S.p); };
  auto ip_f = [&](const NodeState<D>& S, int f) { return have_ip ? ipn[Nq + f] : rcp_nr<2>(S.p); };
  const int ph_begin = Ly.conc ? fam : 0, ph_end = Ly.conc ? fam + 1 : D;
  for (int ph = ph_begin; ph < ph_end; ++ph) {
    if (active) {
      int base, stride;
      if (D == 2) {
        base = ph == 0 ? n * t : t;
        stride = ph == 0 ? 1 : n;
      } else {
        if (ph == 0) { base = n * t; stride = 1; }
        else if (ph == 1) { base = (t % n) + n * n * (t / n); stride = n; }
        else { base = t; stride = n * n; }
      }
      int m = 0;
      for (int a = 0; a < n; ++a) {
        const int vi = base + a * stride;
        NodeState<D> Si = load_state<D>(Sv, Nq, vi);
        const double ipi = ip_v(Si, vi);
        // node a's cotangent accumulates in registers over its pairs (one shared-memory
        // update per node instead of a read-modify-write chain through every pair)
        double qa[NQ], rbi[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          qa[c] = 0.0;
          rbi[c] = rb[c * Nq + vi];
        }
        for (int b = a + 1; b < n; ++b, ++m) {
          const int vj = base + b * stride;
          NodeState<D> Sj = load_state<D>(Sv, Nq, vj);
          double nn[D], Fb[NC], qb[NQ];
          load_dir<D>(vdir, ph * R.Lv + m, T, t, nn);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            Fb[c] = rb[c * Nq + vj] - rbi[c];
            qb[c] = 0.0;
          }
          ec_flux_adj<D>(Si, Sj, nn, inv_gm1, Fb, qa, qb, ipi, ip_v(Sj, vj));
#pragma unroll
          for (int c = 0; c < NQ; ++c) qv[c * qvs + vj] += qb[c];
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) qv[c * qvs + vi] += qa[c];
      }
      auto facet_pairs = [&](const double* fd, int slot0, int f, int cnt) {
        NodeState<D> Sfj = load_state<D>(Sf, Nfn, f);
        const double ipj = ip_f(Sfj, f);
        double acc[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) acc[c] = 0.0;
        for (int a = 0; a < cnt; ++a) {
          const int vi = base + a * stride;
          NodeState<D> Si = load_state<D>(Sv, Nq, vi);
          double nn[D], Fb[NC], qa[NQ];
          load_dir<D>(fd, slot0 + a, T, t, nn);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            Fb[c] = -rb[c * Nq + vi] - hb[c * Nfn + f];
            qa[c] = 0.0;
          }
          ec_flux_adj<D>(Si, Sfj, nn, inv_gm1, Fb, qa, acc, ip_v(Si, vi), ipj);
#pragma unroll
          for (int c = 0; c < NQ; ++c) qv[c * qvs + vi] += qa[c];
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) qf[c * qfs + f] += acc[c];
      };
      if (ph == 0) {
        facet_pairs(fdir + R.fph_off[0], 0, 1 * Nqf + t, n);
        facet_pairs(fdir + R.fph_off[0], n, 2 * Nqf + t, n);
      } else if (ph == 1) {
        facet_pairs(fdir + R.fph_off[1], 0, t, n);
      }
    }
    if (!Ly.conc) __syncthreads();
  }
  if (Ly.conc) __syncthreads();
  // facet 4 on the forward's diagonal schedule: task (a, b2) owns the volume nodes
  // (a, b2, .); in step k it handles facet-4 node (a, b') with b' = (b2 + k) mod n, whose
  // cotangent only it updates in that step (the tasks sharing a hold distinct b'), so no
  // partial sums are kept; a barrier separates the steps.  With concurrent families the
  // volume nodes (a, b2, b3) of a task are split by b3 among the families (b3 = fam,
  // fam + D, ...), each adding its facet-node sums to its own copy.
  if (D == 3) {
    const int a = t % n, b2 = t / n;
    const bool act4 = active;
    double* qv4 = qv;
    double* qf4 = !act4 ? nullptr : (fam > 0 ? sm + el * pe + Ly.oQf4x + (fam - 1) * NQ * n * n : qf + 3 * Nqf);
    const int qf4s = fam > 0 ? n * n : qfs;
    const int b3_0 = Ly.conc ? fam : 0, b3_step = Ly.conc ? D : 1;
    const double* fd = act4 ? fdir + R.fph_off[3] : nullptr;
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
      if (act4) {
        const int bp = b2 + k < n ? b2 + k : b2 + k - n;
        const int f = 3 * Nqf + a + n * bp;
        NodeState<D> Sfj = load_state<D>(Sf, Nfn, f);
        const double ipj = ip_f(Sfj, f);
        double acc[NQ], hbf[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          acc[c] = 0.0;
          hbf[c] = hb[c * Nfn + f];
        }
        for (int b3 = b3_0; b3 < n; b3 += b3_step) {
          const int vi = a + n * (b2 + n * b3);
          NodeState<D> Si = load_state<D>(Sv, Nq, vi);
          double nn[D], Fb[NC], qa[NQ];
          load_dir<D>(fd, bp * n + b3, T, t, nn);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            Fb[c] = -rb[c * Nq + vi] - hbf[c];
            qa[c] = 0.0;
          }
          ec_flux_adj<D>(Si, Sfj, nn, inv_gm1, Fb, qa, acc, ip_v(Si, vi), ipj);
#pragma unroll
          for (int c = 0; c < NQ; ++c) qv4[c * qvs + vi] += qa[c];
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) qf4[c * qf4s + (f - 3 * Nqf)] += acc[c];
      }
      __syncthreads();
    }
  }
  if (Ly.conc) {   // sum the families' copies in a fixed order
    const int nv = NQ * Nq, nf4 = D == 3 ? NQ * n * n : 0;
    for (int idx = threadIdx.x; idx < E * (nv + nf4); idx += blockDim.x) {
      const int e = idx / (nv + nf4), r = idx % (nv + nf4);
      double* dst;
      const double* src;
      int str;
      if (r < nv) {
        dst = sm + e * pe + Ly.oQv + r;
        src = sm + e * pe + Ly.oQvx + r;
        str = nv;
      } else {
        const int c = (r - nv) / (n * n), j = (r - nv) % (n * n);
        dst = sm + e * pe + Ly.oQf + c * Nfn + 3 * Nqf + j;
        src = sm + e * pe + Ly.oQf4x + (r - nv);
        str = nf4;
      }
      double v = *dst;
#pragma unroll
      for (int k = 0; k < D - 1; ++k) v += src[k * str];
      *dst = v;
    }
    __syncthreads();
  }
  // 6. store q cotangents (already in place when accumulated in global memory)
  if (Ly.glob) return;
  for (int idx = threadIdx.x; idx < E * NQ * Ntot; idx += blockDim.x) {
    int e = idx / (NQ * Ntot), r = idx % (NQ * Ntot), c = r / Ntot, k = r % Ntot;
    double val = k < Nq ? sm[e * pe + Ly.oQv + c * Nq + k] : sm[e * pe + Ly.oQf + c * Nfn + (k - Nq)];
    qbar[(e0 + e) * NQ * Ntot + r] = val;
  }
}

// Projection adjoint: q cotangents (own + neighbours' interface contributions) -> grad.
// shared layout per element: M[nc*Np] | A[nc*Nq] | B[nc*Nq] | C[nc*Nq] | F[nc*Nfn]
template <int D>
__global__ void project_adjoint_kernel(DevRef R, DevMesh M, int epc, const double* __restrict__ u,
                                       const double* __restrict__ qbar, const double* __restrict__ qext,
                                       double* __restrict__ grad) {
  extern __shared__ double sm[];
  constexpr int NC = D + 2, NF = D + 5, NQ = D + 2;
  const int Np = R.Np, Nq = R.Nq, Nfn = R.Nfn, Ntot = R.Ntot;
  const int oM = 0, oA = NC * Np, oB = oA + NC * Nq, oC = oB + NC * Nq, oF = oC + NC * Nq;
  const int pe = oF + NC * Nfn;
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  Tile t{sm, pe, E};
  // 1. w_b at volume (A) and facet (F) nodes
  for (int idx = threadIdx.x; idx < E * Ntot; idx += blockDim.x) {
    int e = idx / Ntot, k = idx % Ntot;
    const int64_t eg = e0 + e;
    double qb[NQ], wb[NC];
#pragma unroll
    for (int c = 0; c < NQ; ++c) qb[c] = qbar[(eg * NQ + c) * Ntot + k];
    if (k >= Nq) {
      const int f = k - Nq;
      const int64_t e2 = M.nbr_e[eg * Nfn + f];
      const int f2 = M.nbr_f[eg * Nfn + f];
#pragma unroll
      for (int c = 0; c < NQ; ++c) qb[c] += qext[(e2 * NQ + c) * Nfn + f2];
    }
    NodeState<D> s = load_state<D>(M.states + eg * NF * Ntot, Ntot, k);
    qbar_to_wbar<D>(s, qb, M.gamma, wb);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (k < Nq)
        sm[e * pe + oA + c * Nq + k] = wb[c];
      else
        sm[e * pe + oF + c * Nfn + (k - Nq)] = wb[c];
    }
  }
  __syncthreads();
  // 2. w_b += R^T w_b^f ; 3. w~_b = V^T w_b
  apply_RT<D>(R, t, oF, oB, oA, NC, 1.0);
  apply_VT<D>(R, t, oA, oB, oC, oM, NC);
  // 4. g = V [V^T (W/J) V] w~_b   (transpose of w~ = V^T (W/J) V V^T g)
  apply_minv<D>(R, M, t, e0, oM, oB, oC, oA, oA, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np);
    sm[e * pe + oM + idx % (NC * Np)] = sm[e * pe + oA + idx % (NC * Np)];
  }
  __syncthreads();
  apply_V<D>(R, t, oM, oB, oC, oA, NC);
  // 5. u = V u~ (apply_V's output must differ from s1 for triangles, from s2 for tetrahedra)
  const int oU = D == 2 ? oC : oB, oUb = D == 2 ? oB : oC;
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np), r = idx % (NC * Np);
    sm[e * pe + oM + r] = u[(e0 + e) * NC * Np + r];
  }
  __syncthreads();
  apply_V<D>(R, t, oM, oB, oC, oU, NC);
  // 6. u_b = W J (dW/du)^T g
  for (int idx = threadIdx.x; idx < E * Nq; idx += blockDim.x) {
    int e = idx / Nq, v = idx % Nq;
    double uu[NC], g[NC], ub[NC];
    const double wj = M.wj[(e0 + e) * Nq + v];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      uu[c] = sm[e * pe + oU + c * Nq + v];
      g[c] = wj * sm[e * pe + oA + c * Nq + v];
    }
    entropy_vars_adj<D>(uu, M.gamma, g, ub);
#pragma unroll
    for (int c = 0; c < NC; ++c) sm[e * pe + oUb + c * Nq + v] = ub[c];
  }
  __syncthreads();
  // 7. grad = V^T u_b
  apply_VT<D>(R, t, oUb, oA, oU, oM, NC);
  for (int idx = threadIdx.x; idx < E * NC * Np; idx += blockDim.x) {
    int e = idx / (NC * Np), r = idx % (NC * Np);
    grad[(e0 + e) * NC * Np + r] = sm[e * pe + oM + r];
  }
}

// RK4 adjoint combination: out = a*x + b*y (+ c*z), elementwise
__global__ void axpby_kernel(double* __restrict__ out, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

__global__ void reduce_diag_kernel(const double* __restrict__ part, int64_t E, int ncol, double* out) {
  // one block; column c reduced by warp c (deterministic order)
  const int lane = threadIdx.x % 32, c = threadIdx.x / 32;
  if (c >= ncol) return;
  double s = 0.0;
  for (int64_t e = lane; e < E; e += 32) s += part[e * ncol + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}

__global__ void copy_kernel(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// evaluates log_tab (which = 0) or exp_tab (which = 1) elementwise (accuracy tests)
__global__ void math_probe_kernel(int which, const double* __restrict__ mt, const double* __restrict__ x,
                                  double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = which == 0 ? log_tab(x[i], mt) : exp_tab(x[i], mt);
}

// Failure-path check of the bounded staging wait: an mbarrier expecting a transaction
// that no copy will complete; the wait gives up after `limit` cycles and sets the flag.
__global__ void staging_timeout_probe_kernel(int* flag, long long limit) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    mbar_arrive_expect_tx(&bar, 16);
    if (!mbar_wait(&bar, 0, limit)) atomicOr(flag, kFlagTimeout);
  }
}

__global__ void fp64_fma_kernel(double* out, int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-9 * (tid + k);
  const double b = 0.999999999, c = 1e-9;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[tid] = s;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
size_t smem_project(const RefTables& r, int e) {
  const int nc = r.dim + 2;
  return (size_t)e * nc * (r.Np + 3 * r.Nq + r.Nfn) * sizeof(double);
}

size_t smem_residual(const RefTables& r, int e) {
  ResLayout L = r.dim == 2 ? res_layout<2>(r.Nq, r.Nfn, r.Np, r.n) : res_layout<3>(r.Nq, r.Nfn, r.Np, r.n);
  return ((size_t)e * L.pe + kResSmemHeader) * sizeof(double);
}

static constexpr size_t kSmemBudget = 227 * 1024;   // opt-in maximum per CTA
size_t smem_residual_adj(const RefTables& r, int e);
int adj_threads_host(const RefTables& r, int e);

LaunchCfg choose_launch(const RefTables& r) {
  LaunchCfg L;
  // projection: as many elements as fit, 256 threads
  int ea = std::max(1, (int)(kSmemBudget / smem_project(r, 1)));
  ea = std::min(ea, 32);
  L.ea = ea;
  L.ta = 256;
  L.sa = smem_project(r, ea);
  L.eq = L.ea;
  L.tq = L.ta;
  L.sq = L.sa;
  // residual: E*T threads for the pair phases.  The kernels use up to ~255 registers, so an SM
  // holds at most 256 of their threads; pick E to maximise the threads doing pair work per SM
  // (CTAs per SM x E*T, limited by shared memory and registers), then lane utilisation.
  const int lanes = residual_line_lanes(r.dim, r.n);
  int emax = std::max(1, (int)(kSmemBudget / smem_residual(r, 1)));
  emax = std::min(emax, std::max(1, 1024 / (lanes * r.T)));
  int best = 1;
  double best_score = -1.0;
  for (int e = 1; e <= emax; ++e) {
    const int thr = residual_threads(r.dim, r.n, r.T, e);
    const int by_smem = (int)(kSmemBudget / smem_residual(r, e));
    const int by_regs = std::max(1, 256 / thr);
    const int ctas = std::max(1, std::min(by_smem, by_regs));
    if (thr > 256 && e > 1) break;
    const double useful = (double)ctas * e * r.T * lanes;   // lanes with pair work per SM
    const double score = useful + 1e-3 * (double)(e * r.T * lanes) / thr;
    if (score > best_score) {
      best_score = score;
      best = e;
    }
  }
  L.eb = best;
  L.tb = residual_threads(r.dim, r.n, r.T, best);
  L.sb = smem_residual(r, best);
  // residual adjoint: same task structure, larger shared footprint
  // (the adjoint kernel uses up to 128 registers per thread: at most 512 threads per block)
  int evmax = std::max(1, (int)(kSmemBudget / smem_residual_adj(r, 1)));
  best = 1;
  best_score = -1.0;
  for (int e = 1; e <= evmax; ++e) {
    const int thr = adj_threads_host(r, e);
    if (thr > 512) break;
    const double util = (double)(e * r.T) / ((e * r.T + 31) / 32 * 32);
    const int ctas = std::max(1, std::min((int)(kSmemBudget / smem_residual_adj(r, e)), 2048 / thr));
    const double score = util * std::min(1.0, ctas * thr / 384.0) + 1e-3 * e;
    if (score > best_score) {
      best_score = score;
      best = e;
    }
  }
  L.ev = best;
  L.tv = std::max(64, adj_threads_host(r, best));
  L.sv = smem_residual_adj(r, best);
  return L;
}

// Host-side audit of the shared-memory layouts and default launch shapes of every
// supported (dim, p): regions in bounds and disjoint where they are live together, bulk
// copies 16-byte sized and aligned, footprints within one CTA.  No device involved.
bool audit_layouts(std::string* err) {
  char msg[256];
  auto bad = [&](int dim, int p, const char* what) {
    std::snprintf(msg, sizeof msg, "layout audit failed: dim %d p %d: %s", dim, p, what);
    *err = msg;
    return false;
  };
  for (int dim = 2; dim <= 3; ++dim) {
    const int pmax = dim == 2 ? kMaxPTri : kMaxPTet;
    for (int p = 1; p <= pmax; ++p) {
      RefTables r;
      std::string e2;
      if (build_ref(dim, p, &r, &e2) != ESD_OK) return bad(dim, p, "reference tables");
      const int NC = dim + 2, NF = dim + 5, NQ = dim + 2;
      // residual kernel
      const ResLayout L = dim == 2 ? res_layout<2>(r.Nq, r.Nfn, r.Np, r.n) : res_layout<3>(r.Nq, r.Nfn, r.Np, r.n);
      if (L.pe % 2) return bad(dim, p, "residual element stride not 16-byte aligned");
      if ((NF * r.Ntot * 8) % 16) return bad(dim, p, "state block not a multiple of 16 bytes");
      if (L.oS + NF * r.Ntot > L.oR) return bad(dim, p, "states overlap the accumulators");
      if (L.oMod + NC * r.Np > L.oR || L.oS2 + NC * r.Nq > L.oMod) return bad(dim, p, "transform scratch");
      if (L.oR + NC * r.Nq > L.oH4 || L.oH4 + (dim == 3 ? NC * r.Nqf : 0) > L.pe) return bad(dim, p, "r / h4");
      const LaunchCfg C = choose_launch(r);
      if (smem_residual(r, C.eb) > kSmemBudget || smem_project(r, C.ea) > kSmemBudget)
        return bad(dim, p, "default shape exceeds the shared-memory budget");
      if (C.tb < C.eb * r.T * residual_line_lanes(r.dim, r.n) || C.tb > 1024 || C.tb % 32)
        return bad(dim, p, "residual threads");
      // residual adjoint
      const AdjLayout A = dim == 2 ? adj_layout<2>(r.Nq, r.Nfn, r.Np, r.n) : adj_layout<3>(r.Nq, r.Nfn, r.Np, r.n);
      if ((size_t)A.pe * 8 > kSmemBudget) return bad(dim, p, "adjoint footprint");
      const int states_end = A.oSf + NF * r.Nfn;
      if (states_end > A.oRb || (A.oIp >= 0 && A.oIp < states_end) ||
          (A.oIp >= 0 && A.oIp + r.Nq + r.Nfn > A.oRb) || A.oM + NC * r.Np > A.oRb)
        return bad(dim, p, "adjoint states / scratch");
      if (A.oHb + NC * r.Nfn > (A.glob ? A.pe : A.oQv)) return bad(dim, p, "adjoint h_b");
      if (!A.glob && (A.oQf + NQ * r.Nfn > A.pe)) return bad(dim, p, "adjoint q_b");
      if (C.tv > 512 || C.tv < adj_threads_host(r, C.ev)) return bad(dim, p, "adjoint threads");
    }
  }
  return true;
}

cudaError_t set_smem_limits(const LaunchCfg& L, int dim) {
  (void)L;
  const int lim = 227 * 1024;
  cudaError_t e;
  if (dim == 2) {
    e = cudaFuncSetAttribute(project_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(l2_project_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(residual_adjoint_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(project_adjoint_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(project_batch_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(integrals_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = set_residual_smem_d2(lim);
    if (!e) e = set_residual_otf_smem_d2(lim);
  } else {
    e = cudaFuncSetAttribute(project_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(l2_project_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(residual_adjoint_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(project_adjoint_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(project_batch_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(integrals_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = set_residual_smem_d3(lim);
    if (!e) e = set_residual_otf_smem_d3(lim);
  }
  return e;
}

cudaError_t launch_project(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u,
                           double* w_modal, cudaStream_t s) {
  const unsigned grid = (unsigned)((M.E + L.ea - 1) / L.ea);
  if (R.dim == 2)
    project_kernel<2><<<grid, L.ta, L.sa, s>>>(R, M, L.ea, u, w_modal);
  else
    project_kernel<3><<<grid, L.ta, L.sa, s>>>(R, M, L.ea, u, w_modal);
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                            cudaStream_t s) {
  if (M.gvol)   // pair directions formed on the fly (ESD_MESH_METRICS_ON_THE_FLY)
    return R.dim == 2 ? launch_residual_otf_d2(R, M, L, ep, s) : launch_residual_otf_d3(R, M, L, ep, s);
  return R.dim == 2 ? launch_residual_d2(R, M, L, ep, s) : launch_residual_d3(R, M, L, ep, s);
}

cudaError_t launch_l2_project(const DevRef& R, const DevMesh& M, const double* un, double* um, cudaStream_t s) {
  const int nc = R.dim + 2;
  const size_t pe = (size_t)(3 * nc * R.Nq + nc * R.Np) * sizeof(double);
  int epc = std::max(1, (int)(kSmemBudget / pe));
  epc = std::min(epc, 16);
  const unsigned grid = (unsigned)((M.E + epc - 1) / epc);
  if (R.dim == 2)
    l2_project_kernel<2><<<grid, 256, pe * epc, s>>>(R, M, epc, un, um);
  else
    l2_project_kernel<3><<<grid, 256, pe * epc, s>>>(R, M, epc, un, um);
  return cudaGetLastError();
}

int adj_threads_host(const RefTables& r, int e) {
  if (r.dim == 2) return adj_block_threads<2>(adj_layout<2>(r.Nq, r.Nfn, r.Np, r.n), r.T, e);
  return adj_block_threads<3>(adj_layout<3>(r.Nq, r.Nfn, r.Np, r.n), r.T, e);
}

size_t smem_residual_adj(const RefTables& r, int e) {
  AdjLayout L = r.dim == 2 ? adj_layout<2>(r.Nq, r.Nfn, r.Np, r.n) : adj_layout<3>(r.Nq, r.Nfn, r.Np, r.n);
  return (size_t)e * L.pe * sizeof(double);
}

cudaError_t launch_residual_adjoint(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* cot,
                                    double* qbar, double* qext, cudaStream_t s) {
  const unsigned gb = (unsigned)((M.E + L.ev - 1) / L.ev);
  if (R.dim == 2)
    residual_adjoint_kernel<2><<<gb, L.tv, L.sv, s>>>(R, M, L.ev, cot, qbar, qext);
  else
    residual_adjoint_kernel<3><<<gb, L.tv, L.sv, s>>>(R, M, L.ev, cot, qbar, qext);
  return cudaGetLastError();
}

cudaError_t launch_project_adjoint(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u,
                                   const double* qbar, const double* qext, double* grad, cudaStream_t s) {
  const unsigned ga = (unsigned)((M.E + L.eq - 1) / L.eq);
  if (R.dim == 2)
    project_adjoint_kernel<2><<<ga, L.tq, L.sq, s>>>(R, M, L.eq, u, qbar, qext, grad);
  else
    project_adjoint_kernel<3><<<ga, L.tq, L.sq, s>>>(R, M, L.eq, u, qbar, qext, grad);
  return cudaGetLastError();
}

cudaError_t launch_vjp(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u, const double* cot,
                       double* grad, double* qbar, double* qext, cudaStream_t s, bool project_first) {
  cudaError_t e;
  if (project_first && (e = launch_project(R, M, L, u, nullptr, s))) return e;
  if ((e = launch_residual_adjoint(R, M, L, cot, qbar, qext, s))) return e;
  return launch_project_adjoint(R, M, L, u, qbar, qext, grad, s);
}

// Trace messages of a partition mesh (esd_part_export / esd_part_import), per element:
// kind 0 (forward), the facet-node columns of the states [nfields][Nfn] then the facet sound
// speeds [Nfn]; kind 1 (VJP), the interface cotangents [nc][Nfn] of the residual adjoint.
// Export reads local elements elems[0..n); an index outside [0, E) sets kFlagIndex and sends
// zeros.  Import writes ghost rows E + first .. E + first + n - 1 (range checked on the host).
__global__ void trace_export_kernel(DevRef R, DevMesh M, const double* __restrict__ qext, int kind,
                                    const int64_t* __restrict__ elems, int64_t n, double* __restrict__ buf) {
  const int nf = R.dim + 5, nc = R.dim + 2, Nfn = R.Nfn, Nq = R.Nq, Ntot = R.Ntot;
  const int per = kind == 0 ? (nf + 1) * Nfn : nc * Nfn;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * per; idx += stride) {
    const int64_t i = idx / per;
    const int r = (int)(idx - i * per);
    const int64_t e = elems[i];
    double v = 0.0;
    if (e < 0 || e >= M.E) {
      if (r == 0) atomicOr(M.flag, kFlagIndex);
    } else if (kind == 0) {
      const int c = r / Nfn, k = r - c * Nfn;
      v = c < nf ? M.states[(e * nf + c) * Ntot + Nq + k] : M.cfac[e * Nfn + k];
    } else {
      v = qext[e * (int64_t)(nc * Nfn) + r];
    }
    buf[idx] = v;
  }
}

__global__ void trace_import_kernel(DevRef R, DevMesh M, double* __restrict__ qext, int kind,
                                    const double* __restrict__ buf, int64_t first, int64_t n) {
  const int nf = R.dim + 5, nc = R.dim + 2, Nfn = R.Nfn, Nq = R.Nq, Ntot = R.Ntot;
  const int per = kind == 0 ? (nf + 1) * Nfn : nc * Nfn;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * per; idx += stride) {
    const int64_t i = idx / per;
    const int r = (int)(idx - i * per);
    const int64_t e = M.E + first + i;   // ghost row
    const double v = buf[idx];
    if (kind == 0) {
      const int c = r / Nfn, k = r - c * Nfn;
      if (c < nf)
        M.states[(e * nf + c) * Ntot + Nq + k] = v;
      else
        M.cfac[e * Nfn + k] = v;
    } else {
      qext[e * (int64_t)(nc * Nfn) + r] = v;
    }
  }
}

cudaError_t launch_trace_export(const DevRef& R, const DevMesh& M, const double* qext, int kind,
                                const int64_t* elems, int64_t n, double* buf, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  trace_export_kernel<<<152 * 4, 256, 0, s>>>(R, M, qext, kind, elems, n, buf);
  return cudaGetLastError();
}

cudaError_t launch_trace_import(const DevRef& R, const DevMesh& M, double* qext, int kind, const double* buf,
                                int64_t first, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  trace_import_kernel<<<152 * 4, 256, 0, s>>>(R, M, qext, kind, buf, first, n);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* out, double a, const double* x, double b, const double* y, int64_t n,
                         cudaStream_t s) {
  axpby_kernel<<<152 * 4, 256, 0, s>>>(out, a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_batch(int dim, int n, int stage, const BatchMesh* meshes, const BatchItem* items, int nitems,
                         int grid, int threads, size_t smem, cudaStream_t s) {
  if (stage == 0) {
    if (dim == 2)
      project_batch_kernel<2><<<grid, threads, smem, s>>>(meshes, items, nitems);
    else
      project_batch_kernel<3><<<grid, threads, smem, s>>>(meshes, items, nitems);
    return cudaGetLastError();
  }
  return dim == 2 ? launch_residual_batch_d2(n, meshes, items, nitems, grid, threads, smem, s)
                  : launch_residual_batch_d3(n, meshes, items, nitems, grid, threads, smem, s);
}

cudaError_t launch_integrals(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u, double* part,
                             cudaStream_t s) {
  // same shared footprint as the projection tile without its facet block
  const unsigned grid = (unsigned)((M.E + L.ea - 1) / L.ea);
  const int nc = R.dim + 2;
  const size_t smem = (size_t)L.ea * nc * (R.Np + 3 * R.Nq) * sizeof(double);
  const int threads = L.ta < 64 ? 64 : L.ta;
  if (R.dim == 2)
    integrals_kernel<2><<<grid, threads, smem, s>>>(R, M, L.ea, u, part);
  else
    integrals_kernel<3><<<grid, threads, smem, s>>>(R, M, L.ea, u, part);
  return cudaGetLastError();
}

cudaError_t launch_reduce_diag(const double* part, int64_t E, int ncol, double* out, cudaStream_t s) {
  reduce_diag_kernel<<<1, 32 * ncol, 0, s>>>(part, E, ncol, out);
  return cudaGetLastError();
}

cudaError_t launch_copy(const double* src, double* dst, int64_t n, cudaStream_t s) {
  copy_kernel<<<152 * 4, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_math_probe(int which, const double* mtab, const double* x, double* y, int64_t n, cudaStream_t s) {
  math_probe_kernel<<<152 * 4, 256, 0, s>>>(which, mtab, x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_staging_timeout_probe(int* flag, double seconds, cudaStream_t s) {
  int dev = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (e) return e;
  const long long limit = (long long)(seconds * 1e3 * (khz > 0 ? khz : 2000000));
  staging_timeout_probe_kernel<<<1, 32, 0, s>>>(flag, limit);
  return cudaGetLastError();
}

cudaError_t measure_fp64(double* flops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return e;
  const int blocks = sms * 8, threads = 256, iters = 8192;
  double* buf = nullptr;
  e = cudaMallocAsync(&buf, (size_t)blocks * threads * sizeof(double), s);
  if (e) return e;
  fp64_fma_kernel<<<blocks, threads, 0, s>>>(buf, 64);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s);
  fp64_fma_kernel<<<blocks, threads, 0, s>>>(buf, iters);
  cudaEventRecord(b, s);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(buf, s);
  cudaStreamSynchronize(s);
  *flops = 2.0 * 8.0 * (double)blocks * threads * iters / (ms * 1e-3);
  return e ? e : cudaGetLastError();
}

}  // namespace esd
