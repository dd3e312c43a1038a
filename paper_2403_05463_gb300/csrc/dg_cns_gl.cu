// dg_cns_gl.cu -- sm_103a kernels of the compressible form (arXiv 2403.05463, App. A) on
// Gauss-Legendre element nodes (App. B, the paper's quadrature), FP64.
//
// The passes of the compressible Gauss-Lobatto kernels with the face handling of the
// incompressible Gauss-Legendre ones: every face quantity is the interpolant along the line of
// nodes normal to the face (l_i(+-1) the Lagrange basis at the ends) and every face term is
// lifted back onto that line with l_i(+-1) / w_i:
//   traces   : the 5 conservative face values for the neighbours;
//   viscous  (NS elements): BR1 gradient of phi = (v, T), J G = sum_d D_d (Ja^d phi)
//              + sum_faces l_i/w_i (phi* S - sigma (Ja^d phi)_face), phi* = {{phi}} of the face
//              states (interpolated own state, the neighbour's trace or the boundary ghost) or
//              the projected mortar value (the face terms evaluated once per face point in
//              shared memory, then lifted onto every node); eddy viscosity, stress, heat flux,
//              contravariant viscous flux, its divergence J r_v and the outward traces
//              sigma (Ja^d . Fv)_face;
//   inviscid (all elements): J R = -sum_d D_d Ftil^d - sum_faces l_i/w_i [(F_e* - F_v*) . S
//              - sigma (Ftil_e - Ftil_v)_face] + J r_v, Roe/LLF on the interpolated states, the
//              RK update and the interpolated next-stage traces.
// With Gauss quadrature exact to degree 2N+1 this strong form equals the weak form of Eq. NS4,
// (.)_face being the interpolant of the nodal product as the weak form's boundary term needs.
// Boundary faces take the ghost states of the Gauss-Lobatto compressible path; p-nonconforming
// faces take the results of the five-variable mortar kernels on the Gauss points.
#include "dg_device.cuh"
#include "dg_cns_phys.cuh"

namespace dgk {

__constant__ double c_Dgc[NP][NP * NP];  // D[N][i*n+m] on the Gauss points
__constant__ double c_wgc[NP][NP];       // Gauss weights
__constant__ double c_lbc[NP][2][NP];    // l_i(-1), l_i(+1)
// Williamson 2N-storage RK3 (the paper's low-storage third-order scheme, Sec. 2.3)
__constant__ double c_rkAgc[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
__constant__ double c_rkBgc[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

cudaError_t upload_ops_cns_gl(const Ops1D& ops) {
  cudaError_t r = cudaMemcpyToSymbol(c_Dgc, ops.Dg, sizeof(ops.Dg));
  if (r == cudaSuccess) r = cudaMemcpyToSymbol(c_wgc, ops.wg, sizeof(ops.wg));
  if (r == cudaSuccess) r = cudaMemcpyToSymbol(c_lbc, ops.lbg, sizeof(ops.lbg));
  return r;
}

// the element's face coordinates (a, b) of a volume node on faces normal to direction d
__device__ __forceinline__ void face_ab(int d, const int ii[3], int& a, int& b) {
  a = d == 0 ? ii[1] : ii[0];
  b = d == 2 ? ii[1] : ii[2];
}

// the ghost state behind a boundary face of kind `kind` for the interior face state uf and the
// outward face metric S: mirror states at walls, the far field at an inflow, the interior
// density and momentum with the far-field pressure at an outflow
__device__ __forceinline__ void cns_ghost(const DevMesh& M, int kind, const double uf[5], const double S[3],
                                          double up[5]) {
  const double gm1 = M.gamma - 1.0;
  if (kind == FK_WALL || kind == FK_SLIP) {
    const double mo[3] = {uf[1], uf[2], uf[3]};
    double jw[3];
    wall_jump<double>(kind, mo, S, jw);
    up[0] = uf[0];
    up[4] = uf[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) up[1 + c] = uf[1 + c] + jw[c];
  } else if (kind == FK_INFLOW) {
    const double r = M.inflow[0];
    up[0] = r;
#pragma unroll
    for (int c = 0; c < 3; ++c) up[1 + c] = r * M.inflow[1 + c];
    up[4] = M.p_inf / gm1 + 0.5 * r * (M.inflow[1] * M.inflow[1] + M.inflow[2] * M.inflow[2] + M.inflow[3] * M.inflow[3]);
  } else {  // outflow
    up[0] = uf[0];
#pragma unroll
    for (int c = 0; c < 3; ++c) up[1 + c] = uf[1 + c];
    up[4] = M.p_inf / gm1 + 0.5 * (uf[1] * uf[1] + uf[2] * uf[2] + uf[3] * uf[3]) / uf[0];
  }
}

__device__ __forceinline__ void phi_of(const double u[5], double gamma, double ph[4]) {
  const Prim P = prim(u, gamma);
  ph[0] = P.v[0], ph[1] = P.v[1], ph[2] = P.v[2], ph[3] = P.p / P.rho;
}

// ---------------------------------------------------------------------------------------
// traces: interpolated conservative face values
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void k_traces_cns_gl(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ u) {
  constexpr int n = N + 1, n2 = n * n, per = 6 * n2;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)count * per) return;
  const int le = (int)(gid / per), r = (int)(gid % per);
  const int f = r / n2, ab = r % n2, a = ab % n, b = ab / n;
  const int e = list[le];
  const int64_t off = M.elem_off[e], dst = M.tr_off[e] + f * n2 + ab;
  const double* l = c_lbc[N][f & 1];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) s += l[i] * __ldg(&u[v * M.total + off + line_node(f, n, a, b, i)]);
    M.Tq[v * M.tr_total + dst] = s;
  }
}

// ---------------------------------------------------------------------------------------
// viscous pass (NS elements)
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_viscous_cns_gl(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ u) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;                                 // n*n
  double* sU = sD + NP * NP;                       // EPB * 5 * n3: u
  double* sP = sU + EPB * 5 * n3;                  // EPB * 4 * n3: phi = (v, T)
  double* sJa = sP + EPB * 4 * n3;                 // EPB * 9 * n3 (curved only)
  double* sF = sJa + (CURVED ? EPB * 9 * n3 : 0);  // EPB * 12 * n3: Ftil_v[d][4]
  double* sT = sF + EPB * 12 * n3;                 // EPB * 72 * n2: face terms [f*n2+ab][c*3+k]
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_Dgc[N][t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* U = sU + le * 5 * n3;
  double* P = sP + le * 4 * n3;
  double* JA = sJa + le * 9 * n3;
  double* F = sF + le * 12 * n3;
  double* TG = sT + le * 72 * n2;
  const double gamma = M.gamma;
  double Ja[9], invJ = 0.0, uu[5] = {1.0, 0.0, 0.0, 0.0, 1.0}, ph[4] = {0.0, 0.0, 0.0, 0.0};
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      uu[v] = __ldg(&u[v * M.total + off + p]);
      U[v * n3 + p] = uu[v];
    }
    phi_of(uu, gamma, ph);
#pragma unroll
    for (int c = 0; c < 4; ++c) P[c * n3 + p] = ph[c];
    if (CURVED) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        Ja[k] = __ldg(&M.geo[k * M.total + off + p]);
        JA[k * n3 + p] = Ja[k];
      }
      invJ = 1.0 / __ldg(&M.geo[9 * M.total + off + p]);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = M.ec[e].Ja[k];
      invJ = M.ec[e].invJ;
    }
  }
  __syncthreads();
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  double G[4][3];  // G[c][k] = d phi_c / d x_k
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) G[c][k] = 0.0;
  if (active) {
    // volume part: J G_ck = sum_d D_d (Ja^d_k phi_c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double dm = sD[ii[d] * n + m];
        const int pm = base + m * str[d];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double dj = dm * (CURVED ? JA[(d * 3 + k) * n3 + pm] : Ja[d * 3 + k]);
#pragma unroll
          for (int c = 0; c < 4; ++c) G[c][k] += dj * P[c * n3 + pm];
        }
      }
    }
    // face phase, one item per face point of the element's 6 n^2:
    // TG = phi* S - sigma (Ja^d phi)_face, S outward (the mortar's projected phi* S there)
    for (int t = p; t < 6 * n2; t += n3) {
      const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n, d = f >> 1;
      const double* l = c_lbc[N][f & 1];
      const double sg = (f & 1) ? 1.0 : -1.0;
      const FaceLink L = M.link[e * 6 + f];
      double uf[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, Sv[3] = {0.0, 0.0, 0.0}, JP[4][3];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) JP[c][k] = 0.0;
      double pf[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const int pm = line_node(f, n, a, b, m);
#pragma unroll
        for (int v = 0; v < 5; ++v) uf[v] += l[m] * U[v * n3 + pm];
        if (CURVED) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double jk = JA[(d * 3 + k) * n3 + pm];
            Sv[k] += l[m] * jk;
#pragma unroll
            for (int c = 0; c < 4; ++c) JP[c][k] += l[m] * jk * P[c * n3 + pm];
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) pf[c] += l[m] * P[c * n3 + pm];
        }
      }
      if (!CURVED) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Sv[k] = M.ec[e].Ja[d * 3 + k];  // d varies at run time here
#pragma unroll
          for (int c = 0; c < 4; ++c) JP[c][k] = Sv[k] * pf[c];
        }
      }
      double* tg = TG + t * 12;
      if (L.kind == FK_MORTAR) {
        const int64_t ms = M.tr_off[e] + t;
#pragma unroll
        for (int ck = 0; ck < 12; ++ck) tg[ck] = M.LU[ck * M.tr_total + ms] - sg * JP[ck / 3][ck % 3];
        continue;
      }
      const double So[3] = {sg * Sv[0], sg * Sv[1], sg * Sv[2]};
      double up[5];  // the neighbour's face state, or the ghost's behind a boundary face
      if (L.kind == FK_CONF) {
        int a1, b1;
        inv_orient(L.orient, N, a, b, a1, b1);
        const int64_t ns = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
        for (int v = 0; v < 5; ++v) up[v] = M.Tq[v * M.tr_total + ns];
      } else {
        cns_ghost(M, L.kind, uf, So, up);
      }
      double pm_[4], pp_[4];
      phi_of(uf, gamma, pm_);
      phi_of(up, gamma, pp_);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double ps = 0.5 * (pm_[c] + pp_[c]);
#pragma unroll
        for (int k = 0; k < 3; ++k) tg[c * 3 + k] = sg * (ps * Sv[k] - JP[c][k]);
      }
    }
  }
  __syncthreads();
  if (active) {
    // lifting from both faces of every direction: l_i(+-1) / w_i times the face term
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int a, b;
      face_ab(d, ii, a, b);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const double cf = c_lbc[N][s][ii[d]] / c_wgc[N][ii[d]];
        const double* tg = TG + ((2 * d + s) * n2 + a + n * b) * 12;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += cf * tg[c * 3 + k];
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[c][k] *= invJ;
    // eddy viscosity, stress, heat flux, contravariant viscous flux Ftil_v^d = sum_k Ja^d_k fv_k
    const double Gv[3][3] = {{G[0][0], G[0][1], G[0][2]}, {G[1][0], G[1][1], G[1][2]}, {G[2][0], G[2][1], G[2][2]}};
    const double mut = uu[0] * eddy_visc(Gv, M.ec[e].delta, M.closure, M.cs, M.cv);
    const double mu = M.nu + mut;
    const double kappa = gamma / (gamma - 1.0) * (M.nu / M.prandtl + mut / M.prandtl_t);
    const double tr = Gv[0][0] + Gv[1][1] + Gv[2][2];
    double fv[4][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) fv[c][k] = mu * (Gv[c][k] + Gv[k][c]) - (c == k ? (2.0 / 3.0) * mu * tr : 0.0);
#pragma unroll
    for (int k = 0; k < 3; ++k) fv[3][k] = ph[0] * fv[0][k] + ph[1] * fv[1][k] + ph[2] * fv[2][k] + kappa * G[3][k];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 4; ++v) F[(d * 4 + v) * n3 + p] = Ja[d * 3] * fv[v][0] + Ja[d * 3 + 1] * fv[v][1] + Ja[d * 3 + 2] * fv[v][2];
  }
  __syncthreads();
  if (active) {
    // J r_v = sum_d D_d Ftil_v^d
    double V[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double dm = sD[ii[d] * n + m];
        const int pm = base + m * str[d];
#pragma unroll
        for (int v = 0; v < 4; ++v) V[v] += dm * F[(d * 4 + v) * n3 + pm];
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) M.rv[v * M.total + off + p] = V[v];
    // outward viscous traces sigma (Ftil_v^d)_face at the element's 6 n^2 face points
    for (int t = p; t < 6 * n2; t += n3) {
      const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n, d = f >> 1;
      const double* l = c_lbc[N][f & 1];
      const double sg = (f & 1) ? 1.0 : -1.0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += l[m] * F[(d * 4 + v) * n3 + line_node(f, n, a, b, m)];
        M.Tv[v * M.tr_total + M.tr_off[e] + t] = sg * s;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// inviscid pass + assembly + (optional) RK update
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED>
struct CnsGlSmem {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = Shape<N>::EPB;
  // per element: Ftil_e[d][v] (15 n3), u[v] (5 n3), Ja (9 n3, curved), face terms [6 n2][5]
  static constexpr int per = 15 * n3 + 5 * n3 + (CURVED ? 9 * n3 : 0) + 30 * n2;
  static constexpr size_t bytes = sizeof(double) * (NP * NP + EPB * per);
};

template <int N, bool CURVED, int MODE>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_inviscid_cns_gl(DevMesh M, const int32_t* __restrict__ list, int count, const double* uin, double* out,
                      double* g, int stage, double dt, int write_tr) {
  using S = Shape<N>;
  using SM = CnsGlSmem<N, CURVED>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_Dgc[N][t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* F = sD + NP * NP + le * SM::per;  // Ftil_e[d][v]
  double* Q = F + 15 * n3;                  // u[v]
  double* JA = Q + 5 * n3;                  // Ja (curved)
  double* T = JA + (CURVED ? 9 * n3 : 0);   // face terms [f*n2+ab][v]
  const double gamma = M.gamma;
  double uu[5] = {1.0, 0.0, 0.0, 0.0, 1.0}, Ja[9], invJ = 0.0;
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      uu[v] = uin[v * M.total + off + p];
      Q[v * n3 + p] = uu[v];
    }
    if (CURVED) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        Ja[k] = __ldg(&M.geo[k * M.total + off + p]);
        JA[k * n3 + p] = Ja[k];
      }
      invJ = 1.0 / __ldg(&M.geo[9 * M.total + off + p]);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = M.ec[e].Ja[k];
      invJ = M.ec[e].invJ;
    }
    const Prim Pq = prim(uu, gamma);
    double fl[5][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      fl[0][k] = uu[1 + k];
#pragma unroll
      for (int c = 0; c < 3; ++c) fl[1 + c][k] = uu[1 + c] * Pq.v[k] + (c == k ? Pq.p : 0.0);
      fl[4][k] = (uu[4] + Pq.p) * Pq.v[k];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v)
        F[(d * 5 + v) * n3 + p] = Ja[d * 3] * fl[v][0] + Ja[d * 3 + 1] * fl[v][1] + Ja[d * 3 + 2] * fl[v][2];
  }
  __syncthreads();
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  double JR[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const bool ns = active && M.flag[e] != 0;
  if (active) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double dm = sD[ii[d] * n + m];
        const int pm = base + m * str[d];
#pragma unroll
        for (int v = 0; v < 5; ++v) JR[v] -= dm * F[(d * 5 + v) * n3 + pm];
      }
    }
    // face terms at the element's 6 n^2 face points:
    // T = (F_e* - F_v*) . S - sigma (Ftil_e - Ftil_v)_face
    for (int t = p; t < 6 * n2; t += n3) {
      const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n, d = f >> 1;
      const double* l = c_lbc[N][f & 1];
      const double sg = (f & 1) ? 1.0 : -1.0;
      const FaceLink L = M.link[e * 6 + f];
      const int64_t ms = M.tr_off[e] + t;
      double uf[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, Ff[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, Sv[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const int pm = line_node(f, n, a, b, m);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          uf[v] += l[m] * Q[v * n3 + pm];
          Ff[v] += l[m] * F[(d * 5 + v) * n3 + pm];
        }
        if (CURVED) {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sv[k] += l[m] * JA[(d * 3 + k) * n3 + pm];
        }
      }
      double tv[5];
      if (L.kind == FK_MORTAR) {
        // the projected (F_e* - F_v*) . S from the mortar minus the own outward flux (Euler,
        // and viscous for NS elements)
#pragma unroll
        for (int v = 0; v < 5; ++v) tv[v] = M.LH[v * M.tr_total + ms] - sg * Ff[v] + (v > 0 && ns ? M.Tv[(v - 1) * M.tr_total + ms] : 0.0);
      } else {
        if (!CURVED) {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sv[k] = M.ec[e].Ja[d * 3 + k];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) Sv[k] *= sg;
        const double s = sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
        const double nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
        double up[5];  // the neighbour's face state, or the ghost's behind a boundary face
        int64_t nsl = 0;
        if (L.kind == FK_CONF) {
          int a1, b1;
          inv_orient(L.orient, N, a, b, a1, b1);
          nsl = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
          for (int v = 0; v < 5; ++v) up[v] = M.Tq[v * M.tr_total + nsl];
        } else {
          cns_ghost(M, L.kind, uf, Sv, up);
        }
        double Fn[5], fx[5];
        cns_normal_flux(uf, nh, gamma, Fn);
        cns_fluct(uf, up, nh, gamma, M.riemann, fx);
#pragma unroll
        for (int v = 0; v < 5; ++v) tv[v] = s * (Fn[v] + fx[v]) - sg * Ff[v];
        if (L.kind == FK_CONF && (ns || L.nflag)) {
          // BR1: sigma Ftil_v,face - F_v* . S = wo Fv_own . S + wn Fv_nbr . S_nbr
          float wo, wn;
          visc_face_weights(M.mixed_face, ns, L.nflag != 0, wo, wn);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            if (ns) tv[1 + v] += (double)wo * M.Tv[v * M.tr_total + ms];
            if (L.nflag) tv[1 + v] += (double)wn * M.Tv[v * M.tr_total + nsl];
          }
        } else if (ns && (L.kind == FK_WALL || L.kind == FK_SLIP)) {
          // adiabatic walls: F_v* . S is the own traction (no-slip) or its normal part
          // (free-slip) with no energy, leaving nothing or the tangential traction in momentum
          // and the own energy trace; at inflow and outflow F_v* is the own flux: nothing
          if (L.kind == FK_SLIP) {
            const double tw[3] = {M.Tv[ms], M.Tv[M.tr_total + ms], M.Tv[2 * M.tr_total + ms]};
            double tt[3];
            slip_visc_term<double>(tw, Sv, tt);
#pragma unroll
            for (int c = 0; c < 3; ++c) tv[1 + c] += tt[c];
          }
          tv[4] += M.Tv[3 * M.tr_total + ms];
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) T[t * 5 + v] = tv[v];
    }
  }
  __syncthreads();
  if (active) {
    // lift the face terms onto the node: l_i(+-1) / w_i along each direction
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int a, b;
      face_ab(d, ii, a, b);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const double cf = c_lbc[N][s][ii[d]] / c_wgc[N][ii[d]];
        const double* tt = T + ((2 * d + s) * n2 + a + n * b) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) JR[v] -= cf * tt[v];
      }
    }
    if (ns) {
#pragma unroll
      for (int v = 0; v < 4; ++v) JR[1 + v] += M.rv[v * M.total + off + p];
    }
    if (MODE == MODE_RESIDUAL) {
#pragma unroll
      for (int v = 0; v < 5; ++v) out[v * M.total + off + p] = JR[v] * invJ;
    } else {
      const double A = c_rkAgc[stage], B = c_rkBgc[stage];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int64_t ix = v * M.total + off + p;
        double gi = dt * (JR[v] * invJ);
        if (stage > 0) gi = fma(A, g[ix], gi);  // explicit FMAs: one rounding order in every code path
        g[ix] = gi;
        const double qn = fma(B, gi, uu[v]);
        out[ix] = qn;
        Q[v * n3 + p] = qn;  // every read of the old state ended at the barrier above
      }
    }
  }
  if (MODE == MODE_RK && write_tr) {
    __syncthreads();
    if (active) {
      // next-stage traces: the new state interpolated to the face points
      for (int t = p; t < 6 * n2; t += n3) {
        const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n;
        const double* l = c_lbc[N][f & 1];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) s += l[m] * Q[v * n3 + line_node(f, n, a, b, m)];
          M.Tq_next[v * M.tr_total + M.tr_off[e] + t] = s;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------------------
template <int N, bool C>
static size_t visc_smem_cns_gl() {
  return sizeof(double) * (NP * NP + Shape<N>::EPB * ((5 + 4 + (C ? 9 : 0) + 12) * Shape<N>::n3 + 72 * Shape<N>::n2));
}

template <int N>
static cudaError_t prep_cns_gl() {
  cudaError_t r;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((r = cudaFuncSetAttribute(k_viscous_cns_gl<N, false>, attr, (int)visc_smem_cns_gl<N, false>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous_cns_gl<N, true>, attr, (int)visc_smem_cns_gl<N, true>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_cns_gl<N, false, MODE_RESIDUAL>, attr, (int)CnsGlSmem<N, false>::bytes)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_cns_gl<N, true, MODE_RESIDUAL>, attr, (int)CnsGlSmem<N, true>::bytes)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_cns_gl<N, false, MODE_RK>, attr, (int)CnsGlSmem<N, false>::bytes)) != cudaSuccess) return r;
  return cudaFuncSetAttribute(k_inviscid_cns_gl<N, true, MODE_RK>, attr, (int)CnsGlSmem<N, true>::bytes);
}

cudaError_t prepare_kernels_cns_gl() {
  cudaError_t r;
  if ((r = prep_cns_gl<1>()) != cudaSuccess) return r;
  if ((r = prep_cns_gl<2>()) != cudaSuccess) return r;
  if ((r = prep_cns_gl<3>()) != cudaSuccess) return r;
  if ((r = prep_cns_gl<4>()) != cudaSuccess) return r;
  if ((r = prep_cns_gl<5>()) != cudaSuccess) return r;
  if ((r = prep_cns_gl<6>()) != cudaSuccess) return r;
  return prep_cns_gl<7>();
}

cudaError_t launch_traces_cns_gl(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * 6 * (NN + 1) * (NN + 1);
    k_traces_cns_gl<NN><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, b.list, b.count, u);
  });
  return cudaGetLastError();
}

cudaError_t launch_viscous_cns_gl(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (b.curved)
      k_viscous_cns_gl<NN, true><<<grid, SH::threads, visc_smem_cns_gl<NN, true>(), s>>>(M, b.list, b.count, u);
    else
      k_viscous_cns_gl<NN, false><<<grid, SH::threads, visc_smem_cns_gl<NN, false>(), s>>>(M, b.list, b.count, u);
  });
  return cudaGetLastError();
}

cudaError_t launch_inviscid_cns_gl(const DevMesh& M, const Bucket& b, const double* u, double* out, double* g,
                                   int mode, int stage, double dt, int write_tr, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (mode == MODE_RESIDUAL) {
      if (b.curved)
        k_inviscid_cns_gl<NN, true, MODE_RESIDUAL><<<grid, SH::threads, CnsGlSmem<NN, true>::bytes, s>>>(
            M, b.list, b.count, u, out, g, stage, dt, write_tr);
      else
        k_inviscid_cns_gl<NN, false, MODE_RESIDUAL><<<grid, SH::threads, CnsGlSmem<NN, false>::bytes, s>>>(
            M, b.list, b.count, u, out, g, stage, dt, write_tr);
    } else {
      if (b.curved)
        k_inviscid_cns_gl<NN, true, MODE_RK><<<grid, SH::threads, CnsGlSmem<NN, true>::bytes, s>>>(
            M, b.list, b.count, u, out, g, stage, dt, write_tr);
      else
        k_inviscid_cns_gl<NN, false, MODE_RK><<<grid, SH::threads, CnsGlSmem<NN, false>::bytes, s>>>(
            M, b.list, b.count, u, out, g, stage, dt, write_tr);
    }
  });
  return cudaGetLastError();
}

}  // namespace dgk
