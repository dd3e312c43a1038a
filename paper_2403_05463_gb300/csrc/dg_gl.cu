// dg_gl.cu -- sm_103a kernels of the incompressible form on Gauss-Legendre element nodes
// (arXiv 2403.05463, App. B: the paper's quadrature), FP64.
//
// The nodes of an element do not lie on its faces, so every face quantity is interpolated
// along the line of nodes normal to the face, with l_i(+-1) the Lagrange basis at the ends,
// and every face term is lifted back onto that line with l_i(+-1) / w_i:
//   traces   : q at the face points, sum_i l_i(+-1) q_i, for the neighbours;
//   viscous  (NS elements): BR1 gradient J G = sum_d D_d (Ja^d u) + sum_faces l_i/w_i
//              (u* S - sigma (Ja^d u)_face), u* = ({u}_face + u_nbr)/2, S the interpolated face
//              metric (the face terms evaluated once per face point in shared memory, then
//              lifted onto every node); eddy viscosity, stress, contravariant viscous flux, its divergence J r_v
//              and the outward viscous traces sigma (Ja^d . tau)_face;
//   inviscid (all elements): J R = -sum_d D_d Ftil^d - sum_faces l_i/w_i [F* . S - sigma
//              Ftil^d_face + BR1 viscous face terms] + J r_v, Roe/LLF on the interpolated states;
//              the RK update and the interpolated next-stage traces.
// With Gauss quadrature exact to degree 2N+1, this strong form equals the weak form of Eq. NS4
// (the integration by parts is exact for the degree-2N-1 products), face terms included:
// (.)_face is the interpolant of the nodal product, as the weak form's boundary term requires.
// p-nonconforming faces (Sec. 3.2) take the mortar results of the shared mortar kernels (the
// projected u* S and (F_e* - F_v*) . S on the Gauss points); boundary faces take the ghost
// states of the Gauss-Lobatto path (inflow, outflow, no-slip and free-slip walls).
#include "dg_device.cuh"

namespace dgk {

__constant__ double c_Dg[NP][NP * NP];  // D[N][i*n+m] on the Gauss points
__constant__ double c_wg[NP][NP];       // Gauss weights
__constant__ double c_lb[NP][2][NP];    // l_i(-1), l_i(+1)
// Williamson 2N-storage RK3 (the paper's low-storage third-order scheme, Sec. 2.3)
__constant__ double c_rkAg[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
__constant__ double c_rkBg[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

cudaError_t upload_ops_gl(const Ops1D& ops) {
  cudaError_t r = cudaMemcpyToSymbol(c_Dg, ops.Dg, sizeof(ops.Dg));
  if (r == cudaSuccess) r = cudaMemcpyToSymbol(c_wg, ops.wg, sizeof(ops.wg));
  if (r == cudaSuccess) r = cudaMemcpyToSymbol(c_lb, ops.lbg, sizeof(ops.lbg));
  return r;
}

// the element's face coordinates (a, b) of a volume node on faces normal to direction d
__device__ __forceinline__ void face_coords(int d, const int ii[3], int& a, int& b) {
  a = d == 0 ? ii[1] : ii[0];
  b = d == 2 ? ii[1] : ii[2];
}

// ---------------------------------------------------------------------------------------
// traces: interpolated face values
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void k_traces_gl(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ q) {
  constexpr int n = N + 1, n2 = n * n, per = 6 * n2;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)count * per) return;
  const int le = (int)(gid / per), r = (int)(gid % per);
  const int f = r / n2, ab = r % n2, a = ab % n, b = ab / n;
  const int e = list[le];
  const int64_t off = M.elem_off[e], dst = M.tr_off[e] + f * n2 + ab;
  const double* l = c_lb[N][f & 1];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) s += l[i] * __ldg(&q[v * M.total + off + line_node(f, n, a, b, i)]);
    M.Tq[v * M.tr_total + dst] = s;
  }
}

// ---------------------------------------------------------------------------------------
// viscous pass (NS elements)
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_viscous_gl(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ q) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;                                // n*n
  double* sU = sD + NP * NP;                      // EPB * 3 * n3
  double* sJa = sU + EPB * 3 * n3;                // EPB * 9 * n3 (curved only)
  double* sF = sJa + (CURVED ? EPB * 9 * n3 : 0); // EPB * 9 * n3: Ftil_v[d][c]
  double* sT = sF + EPB * 9 * n3;                 // EPB * 54 * n2: face terms [f*n2+ab][c*3+k]
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_Dg[N][t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* U = sU + le * 3 * n3;
  double* JA = sJa + le * 9 * n3;
  double* F = sF + le * 9 * n3;
  double* TG = sT + le * 54 * n2;
  double Ja[9], invJ = 0.0;
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c * n3 + p] = __ldg(&q[(1 + c) * M.total + off + p]);
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
  double G[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  if (active) {
    // volume part: J G_ck = sum_d D_d (Ja^d_k u_c)
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
          for (int c = 0; c < 3; ++c) G[c][k] += dj * U[c * n3 + pm];
        }
      }
    }
    // face phase, one item per face point of the element's 6 n^2:
    // TG = u* S - sigma (Ja^d u)_face, S outward (the mortar's projected u* S there)
    for (int t = p; t < 6 * n2; t += n3) {
      const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n, d = f >> 1;
      const double* l = c_lb[N][f & 1];
      const double sg = (f & 1) ? 1.0 : -1.0;
      const FaceLink L = M.link[e * 6 + f];
      double uf[3] = {0.0, 0.0, 0.0}, Sv[3] = {0.0, 0.0, 0.0}, JU[3][3];  // JU[c][k] = (Ja^d_k u_c)_face
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) JU[c][k] = 0.0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const int pm = line_node(f, n, a, b, m);
#pragma unroll
        for (int c = 0; c < 3; ++c) uf[c] += l[m] * U[c * n3 + pm];
        if (CURVED) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double jk = JA[(d * 3 + k) * n3 + pm];
            Sv[k] += l[m] * jk;
#pragma unroll
            for (int c = 0; c < 3; ++c) JU[c][k] += l[m] * jk * U[c * n3 + pm];
          }
        }
      }
      if (!CURVED) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Sv[k] = M.ec[e].Ja[d * 3 + k];  // d varies at run time here
#pragma unroll
          for (int c = 0; c < 3; ++c) JU[c][k] = Sv[k] * uf[c];
        }
      }
      double* tg = TG + t * 9;
      if (L.kind == FK_MORTAR) {  // u*_c S_k projected from the mortar, S outward
        const int64_t ms = M.tr_off[e] + t;
#pragma unroll
        for (int ck = 0; ck < 9; ++ck) tg[ck] = M.LU[ck * M.tr_total + ms] - sg * JU[ck / 3][ck % 3];
        continue;
      }
      double up[3];  // the neighbour's face velocity, or the ghost's behind a boundary face
      if (L.kind == FK_CONF) {
        int a1, b1;
        inv_orient(L.orient, N, a, b, a1, b1);
        const int64_t ns = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
        for (int c = 0; c < 3; ++c) up[c] = M.Tq[(1 + c) * M.tr_total + ns];
      } else if (L.kind == FK_INFLOW) {
#pragma unroll
        for (int c = 0; c < 3; ++c) up[c] = M.inflow[1 + c];
      } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {
        double jw[3];
        wall_jump<double>(L.kind, uf, Sv, jw);
#pragma unroll
        for (int c = 0; c < 3; ++c) up[c] = uf[c] + jw[c];
      } else {  // outflow: the interior velocity
#pragma unroll
        for (int c = 0; c < 3; ++c) up[c] = uf[c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double us = 0.5 * (uf[c] + up[c]);
#pragma unroll
        for (int k = 0; k < 3; ++k) tg[c * 3 + k] = sg * (us * Sv[k] - JU[c][k]);
      }
    }
  }
  __syncthreads();
  if (active) {
    // lifting from both faces of every direction: l_i(+-1) / w_i times the face term
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int a, b;
      face_coords(d, ii, a, b);
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const double cf = c_lb[N][s2][ii[d]] / c_wg[N][ii[d]];
        const double* tg = TG + ((2 * d + s2) * n2 + a + n * b) * 9;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += cf * tg[c * 3 + k];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[c][k] *= invJ;
    // eddy viscosity, stress, contravariant viscous flux Ftil_v^d_c = sum_k Ja^d_k tau_ck
    const double mu = M.nu + eddy_visc(G, M.ec[e].delta, M.closure, M.cs, M.cv);
    const double tr = G[0][0] + G[1][1] + G[2][2];
    double tau[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) tau[c][k] = mu * (G[c][k] + G[k][c]) - (c == k ? (2.0 / 3.0) * mu * tr : 0.0);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        F[(d * 3 + c) * n3 + p] = Ja[d * 3] * tau[c][0] + Ja[d * 3 + 1] * tau[c][1] + Ja[d * 3 + 2] * tau[c][2];
  }
  __syncthreads();
  if (active) {
    // J r_v = sum_d D_d Ftil_v^d
    double V[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double dm = sD[ii[d] * n + m];
        const int pm = base + m * str[d];
#pragma unroll
        for (int c = 0; c < 3; ++c) V[c] += dm * F[(d * 3 + c) * n3 + pm];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) M.rv[c * M.total + off + p] = V[c];
    // outward viscous traces sigma (Ftil_v^d)_face at the element's 6 n^2 face points
    for (int t = p; t < 6 * n2; t += n3) {
      const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n, d = f >> 1;
      const double* l = c_lb[N][f & 1];
      const double sg = (f & 1) ? 1.0 : -1.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += l[m] * F[(d * 3 + c) * n3 + line_node(f, n, a, b, m)];
        M.Tv[c * M.tr_total + M.tr_off[e] + t] = sg * s;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// inviscid pass + assembly + (optional) RK update
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED>
struct GlSmem {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = Shape<N>::EPB;
  // per element: Ftil_e[d][v] (12 n3), q[v] (4 n3), Ja (9 n3, curved), face terms [6 n2][4]
  static constexpr int per = 12 * n3 + 4 * n3 + (CURVED ? 9 * n3 : 0) + 24 * n2;
  static constexpr size_t bytes = sizeof(double) * (NP * NP + EPB * per);
};

template <int N, bool CURVED, int MODE>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_inviscid_gl(DevMesh M, const int32_t* __restrict__ list, int count, const double* qin, double* out,
                  double* g, int stage, double dt, int write_tr) {
  using S = Shape<N>;
  using SM = GlSmem<N, CURVED>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_Dg[N][t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* F = sD + NP * NP + le * SM::per;  // Ftil_e[d][v]
  double* Q = F + 12 * n3;                  // q[v]
  double* JA = Q + 4 * n3;                  // Ja (curved)
  double* T = JA + (CURVED ? 9 * n3 : 0);   // face terms [f*n2+ab][v]
  double qq[4] = {0.0, 0.0, 0.0, 0.0}, Ja[9], invJ = 0.0;
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qq[v] = qin[v * M.total + off + p];
      Q[v * n3 + p] = qq[v];
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
    double fl[4][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      fl[0][k] = M.c0sq * qq[1 + k];
#pragma unroll
      for (int c = 0; c < 3; ++c) fl[1 + c][k] = qq[1 + c] * qq[1 + k] + (c == k ? qq[0] : 0.0);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        F[(d * 4 + v) * n3 + p] = Ja[d * 3] * fl[v][0] + Ja[d * 3 + 1] * fl[v][1] + Ja[d * 3 + 2] * fl[v][2];
  }
  __syncthreads();
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  double JR[4] = {0.0, 0.0, 0.0, 0.0};
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
        for (int v = 0; v < 4; ++v) JR[v] -= dm * F[(d * 4 + v) * n3 + pm];
      }
    }
    // face terms at the element's 6 n^2 face points:
    // T = F*(q_face, q_nbr) . S - sigma Ftil_e^d_face + wo Tv_own + wn Tv_nbr
    for (int t = p; t < 6 * n2; t += n3) {
      const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n, d = f >> 1;
      const double* l = c_lb[N][f & 1];
      const double sg = (f & 1) ? 1.0 : -1.0;
      const FaceLink L = M.link[e * 6 + f];
      double qf[4] = {0.0, 0.0, 0.0, 0.0}, Ff[4] = {0.0, 0.0, 0.0, 0.0}, Sv[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const int pm = line_node(f, n, a, b, m);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          qf[v] += l[m] * Q[v * n3 + pm];
          Ff[v] += l[m] * F[(d * 4 + v) * n3 + pm];
        }
        if (CURVED) {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sv[k] += l[m] * JA[(d * 3 + k) * n3 + pm];
        }
      }
      if (L.kind == FK_MORTAR) {
        // the projected (F_e* - F_v*) . S from the mortar minus the own outward flux
        // (inviscid, and viscous for NS elements)
        const int64_t ms = M.tr_off[e] + t;
#pragma unroll
        for (int v = 0; v < 4; ++v)
          T[t * 4 + v] = M.LH[v * M.tr_total + ms] - sg * Ff[v] + (v > 0 && ns ? M.Tv[(v - 1) * M.tr_total + ms] : 0.0);
        continue;
      }
      if (!CURVED) {
#pragma unroll
        for (int k = 0; k < 3; ++k) Sv[k] = M.ec[e].Ja[d * 3 + k];  // d varies at run time here
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) Sv[k] *= sg;
      const double s = sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
      const double nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
      double qp[4];  // the neighbour's face state, or the ghost's behind a boundary face
      int64_t nsl = 0;
      if (L.kind == FK_CONF) {
        int a1, b1;
        inv_orient(L.orient, N, a, b, a1, b1);
        nsl = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
        for (int v = 0; v < 4; ++v) qp[v] = M.Tq[v * M.tr_total + nsl];
      } else if (L.kind == FK_INFLOW) {  // prescribed velocity, interior pressure
        qp[0] = qf[0];
#pragma unroll
        for (int c = 0; c < 3; ++c) qp[1 + c] = M.inflow[1 + c];
      } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {  // mirror states
        const double uo[3] = {qf[1], qf[2], qf[3]};
        double jw[3];
        wall_jump<double>(L.kind, uo, Sv, jw);
        qp[0] = qf[0];
#pragma unroll
        for (int c = 0; c < 3; ++c) qp[1 + c] = qf[1 + c] + jw[c];
      } else {  // outflow: interior velocity, zero pressure
        qp[0] = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) qp[1 + c] = qf[1 + c];
      }
      double fx[4];
      flux_fluct(qf, qp, nh, M.c0sq, M.riemann, fx);
      const double un = qf[1] * nh[0] + qf[2] * nh[1] + qf[3] * nh[2];
      double tv[4];
      tv[0] = s * (M.c0sq * un + fx[0]) - sg * Ff[0];
#pragma unroll
      for (int c = 0; c < 3; ++c) tv[1 + c] = s * (qf[1 + c] * un + qf[0] * nh[c] + fx[1 + c]) - sg * Ff[1 + c];
      if (L.kind == FK_CONF && (ns || L.nflag)) {
        float wo, wn;
        visc_face_weights(M.mixed_face, ns, L.nflag != 0, wo, wn);
        const int64_t ms = M.tr_off[e] + t;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (ns) tv[1 + c] += (double)wo * M.Tv[c * M.tr_total + ms];
          if (L.nflag) tv[1 + c] += (double)wn * M.Tv[c * M.tr_total + nsl];
        }
      } else if (L.kind == FK_SLIP && ns) {
        // free-slip wall: F_v* keeps the normal traction, leaving the tangential part of the
        // own trace; at the other boundaries F_v* is the own (interior) flux and nothing remains
        const int64_t ms = M.tr_off[e] + t;
        const double tw[3] = {M.Tv[ms], M.Tv[M.tr_total + ms], M.Tv[2 * M.tr_total + ms]};
        double tt[3];
        slip_visc_term<double>(tw, Sv, tt);
#pragma unroll
        for (int c = 0; c < 3; ++c) tv[1 + c] += tt[c];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) T[t * 4 + v] = tv[v];
    }
  }
  __syncthreads();
  if (active) {
    // lift the face terms onto the node: l_i(+-1) / w_i along each direction
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int a, b;
      face_coords(d, ii, a, b);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const double cf = c_lb[N][s][ii[d]] / c_wg[N][ii[d]];
        const double* tt = T + ((2 * d + s) * n2 + a + n * b) * 4;
#pragma unroll
        for (int v = 0; v < 4; ++v) JR[v] -= cf * tt[v];
      }
    }
    if (ns) {
#pragma unroll
      for (int c = 0; c < 3; ++c) JR[1 + c] += M.rv[c * M.total + off + p];
    }
    if (MODE == MODE_RESIDUAL) {
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v * M.total + off + p] = JR[v] * invJ;
    } else {
      const double A = c_rkAg[stage], B = c_rkBg[stage];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int64_t ix = v * M.total + off + p;
        double gi = dt * (JR[v] * invJ);
        if (stage > 0) gi = fma(A, g[ix], gi);  // explicit FMAs: one rounding order in every code path
        g[ix] = gi;
        const double qn = fma(B, gi, qq[v]);
        out[ix] = qn;
        Q[v * n3 + p] = qn;  // every read of the old Q ended at the barrier above
      }
    }
  }
  if (MODE == MODE_RK && write_tr) {
    __syncthreads();
    if (active) {
      // next-stage traces: the new state interpolated to the face points
      for (int t = p; t < 6 * n2; t += n3) {
        const int f = t / n2, ab = t % n2, a = ab % n, b = ab / n;
        const double* l = c_lb[N][f & 1];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
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
static size_t visc_smem_gl() {
  return sizeof(double) * (NP * NP + Shape<N>::EPB * ((3 + (C ? 9 : 0) + 9) * Shape<N>::n3 + 54 * Shape<N>::n2));
}

template <int N>
static cudaError_t prep_gl() {
  cudaError_t r;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((r = cudaFuncSetAttribute(k_viscous_gl<N, false>, attr, (int)visc_smem_gl<N, false>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous_gl<N, true>, attr, (int)visc_smem_gl<N, true>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_gl<N, false, MODE_RESIDUAL>, attr, (int)GlSmem<N, false>::bytes)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_gl<N, true, MODE_RESIDUAL>, attr, (int)GlSmem<N, true>::bytes)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_gl<N, false, MODE_RK>, attr, (int)GlSmem<N, false>::bytes)) != cudaSuccess) return r;
  return cudaFuncSetAttribute(k_inviscid_gl<N, true, MODE_RK>, attr, (int)GlSmem<N, true>::bytes);
}

cudaError_t prepare_kernels_gl() {
  cudaError_t r;
  if ((r = prep_gl<1>()) != cudaSuccess) return r;
  if ((r = prep_gl<2>()) != cudaSuccess) return r;
  if ((r = prep_gl<3>()) != cudaSuccess) return r;
  if ((r = prep_gl<4>()) != cudaSuccess) return r;
  if ((r = prep_gl<5>()) != cudaSuccess) return r;
  if ((r = prep_gl<6>()) != cudaSuccess) return r;
  return prep_gl<7>();
}


cudaError_t launch_traces_gl(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * 6 * (NN + 1) * (NN + 1);
    k_traces_gl<NN><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

cudaError_t launch_viscous_gl(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (b.curved)
      k_viscous_gl<NN, true><<<grid, SH::threads, visc_smem_gl<NN, true>(), s>>>(M, b.list, b.count, q);
    else
      k_viscous_gl<NN, false><<<grid, SH::threads, visc_smem_gl<NN, false>(), s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

cudaError_t launch_inviscid_gl(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                               int mode, int stage, double dt, int write_tr, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (mode == MODE_RESIDUAL) {
      if (b.curved)
        k_inviscid_gl<NN, true, MODE_RESIDUAL><<<grid, SH::threads, GlSmem<NN, true>::bytes, s>>>(
            M, b.list, b.count, q, out, g, stage, dt, write_tr);
      else
        k_inviscid_gl<NN, false, MODE_RESIDUAL><<<grid, SH::threads, GlSmem<NN, false>::bytes, s>>>(
            M, b.list, b.count, q, out, g, stage, dt, write_tr);
    } else {
      if (b.curved)
        k_inviscid_gl<NN, true, MODE_RK><<<grid, SH::threads, GlSmem<NN, true>::bytes, s>>>(
            M, b.list, b.count, q, out, g, stage, dt, write_tr);
      else
        k_inviscid_gl<NN, false, MODE_RK><<<grid, SH::threads, GlSmem<NN, false>::bytes, s>>>(
            M, b.list, b.count, q, out, g, stage, dt, write_tr);
    }
  });
  return cudaGetLastError();
}

}  // namespace dgk
