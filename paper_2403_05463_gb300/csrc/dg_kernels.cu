// dg_kernels.cu -- sm_103a kernels of the flagged Euler / NS-LES DGSEM residual (FP64 path).
//
// Per residual evaluation (one Runge-Kutta stage):
//   traces   : every element copies q at its 6 n^2 face nodes into a face-major trace buffer
//              (neighbours read only traces, never q, so the last pass may update q in place).
//   mortar_lift (p-nonconforming faces of NS elements): BR1 lifting u* S projected from the
//              mortar of the larger order.
//   viscous  (NS elements only, Sec. 2.3): BR1 gradient of the velocity, eddy viscosity,
//              stress, contravariant viscous flux, its divergence (stored as J r_v) and the
//              outward viscous flux traces tau . S on the 6 faces.
//   mortar_flux: total projected flux (F_e* - F_v*) . S on p-nonconforming faces.
//   inviscid (all elements): contravariant Euler flux, its divergence by sum-factorised
//              derivative contractions staged in shared memory, surface terms (Roe/LLF
//              fluctuation on conforming faces, BR1 average of viscous traces), + J r_v,
//              then R = (1/J)(...) or the in-place low-storage RK3 update.
// Strong form on Gauss-Lobatto nodes (equal to the weak form of App. B, Eq. NS4, by the
// summation-by-parts property of the Lobatto quadrature):
//   J R = -sum_d D_d (Ftil_e^d - Ftil_v^d) - sum_faces (1/w_end) [(F_e* - F_v*) . S - (Ftil_e - Ftil_v)_out]
#include "dg_device.cuh"

#include <algorithm>
#include <cstdio>

namespace dgk {

__constant__ Ops1D c_ops;

// Williamson 2N-storage RK3 (the paper's low-storage third-order scheme, Sec. 2.3).
__constant__ double c_rkA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
__constant__ double c_rkB[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

// Full numerical flux F*(q-, q+) (mortar faces): F_n(q-) + fluctuation.
__device__ __forceinline__ void flux_full(const double qm[4], const double qp[4], const double nh[3],
                                          double c0sq, int riemann, double out[4]) {
  double fl[4];
  flux_fluct(qm, qp, nh, c0sq, riemann, fl);
  double un = qm[1] * nh[0] + qm[2] * nh[1] + qm[3] * nh[2];
  out[0] = c0sq * un + fl[0];
#pragma unroll
  for (int c = 0; c < 3; ++c) out[1 + c] = qm[1 + c] * un + qm[0] * nh[c] + fl[1 + c];
}

// ---------------------------------------------------------------------------------------
// traces
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void k_traces(DevMesh M, const int32_t* __restrict__ list, int count,
                         const double* __restrict__ q) {
  constexpr int n = N + 1, n2 = n * n, per = 6 * n2;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)count * per) return;
  int le = (int)(gid / per), r = (int)(gid % per);
  int f = r / n2, ab = r % n2;
  int e = list[le];
  int64_t src = M.elem_off[e] + face_node(f, n, ab % n, ab / n);
  int64_t dst = M.tr_off[e] + f * n2 + ab;
#pragma unroll
  for (int v = 0; v < 4; ++v) M.Tq[v * M.tr_total + dst] = __ldg(&q[v * M.total + src]);
}

// ---------------------------------------------------------------------------------------
// viscous pass (NS elements)
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED>
__global__ void __launch_bounds__(Shape<N>::threads) k_viscous(DevMesh M, const int32_t* __restrict__ list,
                                                               int count, const double* __restrict__ q) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;                                // n*n
  double* sU = sD + NP * NP;                      // EPB * 3 * n3
  double* sJa = sU + EPB * 3 * n3;                // EPB * 9 * n3 (curved only)
  double* sF = sJa + (CURVED ? EPB * 9 * n3 : 0); // EPB * 9 * n3
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_ops.D[N][t];
  int le = tid / n3, p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* U = sU + le * 3 * n3;
  double* JA = sJa + le * 9 * n3;
  double* F = sF + le * 9 * n3;
  double Ja[9], invJ = 0.0, u[3] = {0.0, 0.0, 0.0};
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = __ldg(&q[(1 + c) * M.total + off + p]);
      U[c * n3 + p] = u[c];
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
  }
  __syncthreads();
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  double G[3][3];
  if (active) {
    // volume part: J G_ck = sum_d D_d (Ja^d_k u_c)
    if (!CURVED) {
      double du[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int base = p - ii[d] * str[d];
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          double dm = sD[ii[d] * n + m];
          int pm = base + m * str[d];
          s0 += dm * U[pm];
          s1 += dm * U[n3 + pm];
          s2 += dm * U[2 * n3 + pm];
        }
        du[0][d] = s0;
        du[1][d] = s1;
        du[2][d] = s2;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[c][k] = Ja[k] * du[c][0] + Ja[3 + k] * du[c][1] + Ja[6 + k] * du[c][2];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[c][k] = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int base = p - ii[d] * str[d];
#pragma unroll
        for (int m = 0; m < n; ++m) {
          double dm = sD[ii[d] * n + m];
          int pm = base + m * str[d];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            double dj = dm * JA[(d * 3 + k) * n3 + pm];
#pragma unroll
            for (int c = 0; c < 3; ++c) G[c][k] += dj * U[c * n3 + pm];
          }
        }
      }
    }
    // BR1 lifting on the faces this node lies on: (1/w_end) (u* - u) S
    const double invw = 1.0 / c_ops.w[N][0];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
      const double sg = side ? 1.0 : -1.0;
      const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
      const FaceLink L = M.link[e * 6 + f];
      double Sv[3] = {sg * Ja[d * 3], sg * Ja[d * 3 + 1], sg * Ja[d * 3 + 2]};
      if (L.kind == FK_MORTAR) {
        const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += invw * (M.LU[(c * 3 + k) * M.tr_total + ms] - u[c] * Sv[k]);
      } else {
        double jump[3] = {0.0, 0.0, 0.0};
        if (L.kind == FK_CONF) {
          int a1, b1;
          inv_orient(L.orient, N, a, b, a1, b1);
          const int64_t ns = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
          for (int c = 0; c < 3; ++c) jump[c] = M.Tq[(1 + c) * M.tr_total + ns] - u[c];
        } else if (L.kind == FK_INFLOW) {
#pragma unroll
          for (int c = 0; c < 3; ++c) jump[c] = M.inflow[1 + c] - u[c];
        } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {
          const double Sd[3] = {Sv[0], Sv[1], Sv[2]};
          wall_jump<double>(L.kind, u, Sd, jump);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += invw * 0.5 * jump[c] * Sv[k];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[c][k] *= invJ;
    // eddy viscosity and stress
    const double mu = M.nu + eddy_visc(G, M.ec[e].delta, M.closure, M.cs, M.cv);
    const double tr = G[0][0] + G[1][1] + G[2][2];
    double tau[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) tau[c][k] = mu * (G[c][k] + G[k][c]) - (c == k ? (2.0 / 3.0) * mu * tr : 0.0);
    // contravariant viscous flux Fv^d_c = sum_k Ja^d_k tau_ck
    double Fv[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Fv[d][c] = Ja[d * 3] * tau[c][0] + Ja[d * 3 + 1] * tau[c][1] + Ja[d * 3 + 2] * tau[c][2];
        F[(d * 3 + c) * n3 + p] = Fv[d][c];
      }
    // outward viscous flux traces tau . S = sigma Fv^d
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
      const double sg = side ? 1.0 : -1.0;
      const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
      const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
#pragma unroll
      for (int c = 0; c < 3; ++c) M.Tv[c * M.tr_total + ms] = sg * Fv[d][c];
    }
  }
  __syncthreads();
  if (active) {
    // J r_v = sum_d D_d Fv^d
    double V[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        double dm = sD[ii[d] * n + m];
        int pm = base + m * str[d];
#pragma unroll
        for (int c = 0; c < 3; ++c) V[c] += dm * F[(d * 3 + c) * n3 + pm];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) M.rv[c * M.total + off + p] = V[c];
  }
}

// ---------------------------------------------------------------------------------------
// inviscid pass + assembly + (optional) RK update
// ---------------------------------------------------------------------------------------
// KEP: the split form's volume term, sum_m 2 D_im F#(q_i, q_m) along each direction; the
// element's state [4][n3] (and, curved, its metric [9][n3]) is kept in shared memory instead
// of the contravariant fluxes.
template <int N, bool CURVED, int MODE, bool KEP>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_inviscid(DevMesh M, const int32_t* __restrict__ list, int count, const double* qin, double* out,
               double* g, int stage, double dt, int write_tr) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB, PER = KEP ? 13 : 12;
  extern __shared__ double sm[];
  double* sD = sm;
  double* sF = sD + NP * NP;  // EPB * PER * n3: Ftil_e[d][v], or (KEP) q[v] and Ja[9]
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_ops.D[N][t];
  int le = tid / n3, p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* F = sF + le * PER * n3;
  double qq[4] = {0.0, 0.0, 0.0, 0.0}, Ja[9], invJ = 0.0, fl[4][3];
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) qq[v] = qin[v * M.total + off + p];
    if (CURVED) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = __ldg(&M.geo[k * M.total + off + p]);
      invJ = 1.0 / __ldg(&M.geo[9 * M.total + off + p]);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = M.ec[e].Ja[k];
      invJ = M.ec[e].invJ;
    }
    // physical Euler flux f_v,k
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      fl[0][k] = M.c0sq * qq[1 + k];
#pragma unroll
      for (int c = 0; c < 3; ++c) fl[1 + c][k] = qq[1 + c] * qq[1 + k] + (c == k ? qq[0] : 0.0);
    }
    if (!KEP) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          F[(d * 4 + v) * n3 + p] = Ja[d * 3] * fl[v][0] + Ja[d * 3 + 1] * fl[v][1] + Ja[d * 3 + 2] * fl[v][2];
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) F[v * n3 + p] = qq[v];
      if (CURVED) {
#pragma unroll
        for (int k = 0; k < 9; ++k) F[(4 + k) * n3 + p] = Ja[k];
      }
    }
  }
  __syncthreads();
  if (!active) return;
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  double JR[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int base = p - ii[d] * str[d];
#pragma unroll
    for (int m = 0; m < n; ++m) {
      double dm = sD[ii[d] * n + m];
      int pm = base + m * str[d];
      if (!KEP) {
#pragma unroll
        for (int v = 0; v < 4; ++v) JR[v] -= dm * F[(d * 4 + v) * n3 + pm];
      } else {
        // two-point flux between this node and node m of the line: averages of u, p, Ja^d
        double ja[3], u[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          ja[k] = CURVED ? 0.5 * (Ja[d * 3 + k] + F[(4 + d * 3 + k) * n3 + pm]) : Ja[d * 3 + k];
          u[k] = 0.5 * (qq[1 + k] + F[(1 + k) * n3 + pm]);
        }
        const double pa = 0.5 * (qq[0] + F[pm]);
        const double U = ja[0] * u[0] + ja[1] * u[1] + ja[2] * u[2];
        const double d2 = 2.0 * dm;
        JR[0] -= d2 * M.c0sq * U;
#pragma unroll
        for (int c = 0; c < 3; ++c) JR[1 + c] -= d2 * (u[c] * U + pa * ja[c]);
      }
    }
  }
  const bool ns = M.flag[e] != 0;
  if (ns) {
#pragma unroll
    for (int c = 0; c < 3; ++c) JR[1 + c] += M.rv[c * M.total + off + p];
  }
  const double invw = 1.0 / c_ops.w[N][0];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (ii[d] != 0 && ii[d] != N) continue;
    const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
    const double sg = side ? 1.0 : -1.0;
    const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
    const FaceLink L = M.link[e * 6 + f];
    const double Sv[3] = {sg * Ja[d * 3], sg * Ja[d * 3 + 1], sg * Ja[d * 3 + 2]};
    const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
    if (L.kind == FK_MORTAR) {
      // projected (F_e* - F_v*) . S from the mortar, minus the own outward flux
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double own = Sv[0] * fl[v][0] + Sv[1] * fl[v][1] + Sv[2] * fl[v][2];
        if (v > 0 && ns) own -= M.Tv[(v - 1) * M.tr_total + ms];
        JR[v] -= invw * (M.LH[v * M.tr_total + ms] - own);
      }
      continue;
    }
    const double s = sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
    const double nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
    double qp[4];
    int64_t nsl = 0;
    if (L.kind == FK_CONF) {
      int a1, b1;
      inv_orient(L.orient, N, a, b, a1, b1);
      nsl = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
      for (int v = 0; v < 4; ++v) qp[v] = M.Tq[v * M.tr_total + nsl];
    } else if (L.kind == FK_INFLOW) {
      qp[0] = qq[0];
#pragma unroll
      for (int c = 0; c < 3; ++c) qp[1 + c] = M.inflow[1 + c];
    } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {
      const double uo[3] = {qq[1], qq[2], qq[3]};
      double jw[3];
      wall_jump<double>(L.kind, uo, Sv, jw);
      qp[0] = qq[0];
#pragma unroll
      for (int c = 0; c < 3; ++c) qp[1 + c] = qq[1 + c] + jw[c];
    } else {
      qp[0] = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) qp[1 + c] = qq[1 + c];
    }
    double fx[4];
    flux_fluct(qq, qp, nh, M.c0sq, M.riemann, fx);
#pragma unroll
    for (int v = 0; v < 4; ++v) JR[v] -= invw * s * fx[v];
    if (L.kind == FK_CONF && (ns || L.nflag)) {
      // BR1: Ftil_v,out - F_v* . S = wo tau_own . S_own + wn tau_nbr . S_nbr
      float wo, wn;
      visc_face_weights(M.mixed_face, ns, L.nflag != 0, wo, wn);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double t = 0.0;
        if (ns) t += (double)wo * M.Tv[c * M.tr_total + ms];
        if (L.nflag) t += (double)wn * M.Tv[c * M.tr_total + nsl];
        JR[1 + c] -= invw * t;
      }
    } else if (L.kind == FK_SLIP && ns) {
      const double tv[3] = {M.Tv[ms], M.Tv[M.tr_total + ms], M.Tv[2 * M.tr_total + ms]};
      double tt[3];
      slip_visc_term<double>(tv, Sv, tt);
#pragma unroll
      for (int c = 0; c < 3; ++c) JR[1 + c] -= invw * tt[c];
    }
  }
  if (MODE == MODE_RESIDUAL) {
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v * M.total + off + p] = JR[v] * invJ;
  } else {
    const double A = c_rkA[stage], B = c_rkB[stage];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t ix = v * M.total + off + p;
      double gi = dt * (JR[v] * invJ);
      if (stage > 0) gi = fma(A, g[ix], gi);  // explicit FMAs: one rounding order in every code path
      g[ix] = gi;
      const double qn = fma(B, gi, qq[v]);
      out[ix] = qn;
      if (write_tr) {  // traces of the new state for the next stage
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (ii[d] != 0 && ii[d] != N) continue;
          const int f = 2 * d + (ii[d] == N ? 1 : 0);
          const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
          M.Tq_next[v * M.tr_total + M.tr_off[e] + f * n2 + a + n * b] = qn;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// mortars (p-nonconforming faces): one block per (element, face) slot. They serve both node
// sets: on Gauss-Legendre nodes the traces are already the interpolated face values, S is the
// interpolated face metric and the tables interpolate and project between Gauss point sets.
// ---------------------------------------------------------------------------------------
// the tables of the context's node set: Gauss-Lobatto, or Gauss-Legendre points (nodes = 1)
__device__ __forceinline__ const double* interp_tab(const DevMesh& M, int Ns, int Nd) {
  return (M.nodes == 1 ? M.interp_g : M.interp) + (Ns * NP + Nd) * NP * NP;
}
__device__ __forceinline__ const double* proj_tab(const DevMesh& M, int Nh, int Nl) {
  return (M.nodes == 1 ? M.proj_g : M.proj) + (Nh * NP + Nl) * NP * NP;
}


__device__ __forceinline__ void node_metric(const DevMesh& M, int e, int64_t node, double Ja[9]) {
  if (M.ec[e].curved != 0.0) {
    for (int k = 0; k < 9; ++k) Ja[k] = M.geo[k * M.total + node];
  } else {
    for (int k = 0; k < 9; ++k) Ja[k] = M.ec[e].Ja[k];
  }
}

// outward face metric S = sigma Ja^d at face point (a, b) of face f of element e (order n - 1):
// the face node's metric on Gauss-Lobatto nodes; on Gauss-Legendre nodes the interpolant of
// Ja^d along the normal line, sum_i l_i(+-1) Ja^d_i (exact: constant on affine elements)
__device__ __forceinline__ void face_metric(const DevMesh& M, int e, int f, int n, int a, int b, double S[3]) {
  const int d = f >> 1;
  const double sg = (f & 1) ? 1.0 : -1.0;
  const int64_t off = M.elem_off[e];
  double Ja[9];
  if (M.nodes == 1 && M.ec[e].curved != 0.0) {
    const double* l = M.lb_g + ((n - 1) * 2 + (f & 1)) * NP;
    S[0] = S[1] = S[2] = 0.0;
    for (int i = 0; i < n; ++i) {
      const int64_t node = off + line_node(f, n, a, b, i);
      for (int k = 0; k < 3; ++k) S[k] += l[i] * M.geo[(d * 3 + k) * M.total + node];
    }
    for (int k = 0; k < 3; ++k) S[k] *= sg;
    return;
  }
  node_metric(M, e, off + face_node(f, n, a, b), Ja);
  for (int k = 0; k < 3; ++k) S[k] = sg * Ja[d * 3 + k];
}

// trace value of variable v at trace slot `slot`: FP64 planes [4][tr_total], or with precision 1
// FP32 (hi, lo) pairs interleaved per slot, [tr_total][4]
__device__ __forceinline__ double tq_load(const DevMesh& M, int v, int64_t slot) {
  if (M.precision == 1) {
    // exact widening with integer instructions, one FP64 add (the mortar kernels are
    // FP64-pipe bound)
    const float2 t = reinterpret_cast<const float2*>(M.Tq)[slot * 4 + v];
    return widen_f32(t.x) + widen_f32(t.y);
  }
  return M.Tq[v * M.tr_total + slot];
}

// viscous trace component c at `slot`: FP64 planes [3][tr_total], or FP32 [tr_total][3]
__device__ __forceinline__ double tv_load(const DevMesh& M, int c, int64_t slot) {
  return M.precision == 1 ? widen_f32(reinterpret_cast<const float*>(M.Tv)[slot * 3 + c]) : M.Tv[c * M.tr_total + slot];
}

// ---------------------------------------------------------------------------------------
// p-nonconforming faces: one warp per mortar side (element e, local face f)
// ---------------------------------------------------------------------------------------
// Launches are grouped by mortar order MO = max(N_e, N_nbr), so a warp's shared-memory planes
// hold PS = (MO + 1)^2 values. Face fields go to the mortar and back with sum-factorised
// tensor products (one direction at a time through a scratch plane), lanes over the points.
constexpr int kMortarWarps = 4;  // warps (mortar sides) per block

template <int MO>
struct MortarW {
  static constexpr int nM = MO + 1, PS = nM * nM;
  static constexpr int LIFT_PLANES = 21;  // A[9] B[3] T[9]
  static constexpr int FLUX_PLANES = 27;  // A[10] B[7] T[10]
};

// dst = (T x T) src for nv planes of stride PS: src is ns x ns, dst nd x nd, T the 1D table
// (row a: T[a * NP + aa]). tmp holds nv planes of nd x ns. When `o` >= 0 the result at
// (a, b), coordinates of the neighbour's mortar, is stored at my coordinates fwd_orient(o).
// src and dst may be the same planes (src is read only in the first step). ns == nd with T the
// identity is a (permuted) copy.
__device__ __forceinline__ void tensor2_warp(const double* __restrict__ T, bool identity, int ns, int nd, int nv,
                                             const double* src, double* tmp, double* dst, int PS, int o, int Mo,
                                             int lane) {
  if (identity) {
    for (int idx = lane; idx < nv * nd * nd; idx += 32) {
      const int v = idx / (nd * nd), r = idx % (nd * nd);
      tmp[v * PS + r] = src[v * PS + r];
    }
  } else {
    for (int idx = lane; idx < nv * nd * ns; idx += 32) {
      const int v = idx / (nd * ns), r = idx % (nd * ns), a = r % nd, bb = r / nd;
      const double* Ta = T + a * NP;
      const double* sv = src + v * PS + ns * bb;
      double acc = 0.0;
      for (int aa = 0; aa < ns; ++aa) acc = fma(__ldg(Ta + aa), sv[aa], acc);
      tmp[v * PS + r] = acc;
    }
  }
  __syncwarp();
  for (int idx = lane; idx < nv * nd * nd; idx += 32) {
    const int v = idx / (nd * nd), r = idx % (nd * nd), a = r % nd, b = r / nd;
    double acc;
    if (identity) {
      acc = tmp[v * PS + r];
    } else {
      const double* Tb = T + b * NP;
      const double* tv = tmp + v * PS + a;
      acc = 0.0;
      for (int bb = 0; bb < ns; ++bb) acc = fma(__ldg(Tb + bb), tv[nd * bb], acc);
    }
    int dr = r;
    if (o >= 0) {
      int a0, b0;
      fwd_orient(o, Mo, a, b, a0, b0);
      dr = a0 + nd * b0;
    }
    dst[v * PS + dr] = acc;
  }
  __syncwarp();
}

template <int MO>
static size_t mortar_smem(bool flux) {
  return sizeof(double) * kMortarWarps * MortarW<MO>::PS * (flux ? MortarW<MO>::FLUX_PLANES : MortarW<MO>::LIFT_PLANES);
}

// Projected BR1 lifting data of an NS element's mortar face: u*_c S_k on the mortar
// (u* = the average of both sides' interpolated velocity traces, S my interpolated face
// metric), L2-projected to my order, [9][tr_total] at my trace slots.
template <int MO>
__global__ void __launch_bounds__(32 * kMortarWarps) k_mortar_lift_w(DevMesh M, const int32_t* __restrict__ slots,
                                                                      int count) {
  using W = MortarW<MO>;
  constexpr int nM = W::nM, PS = W::PS;
  extern __shared__ double smd[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kMortarWarps + warp;
  if (item >= count) return;  // the whole warp leaves together
  double* A = smd + warp * W::LIFT_PLANES * PS;
  double* B = A + 9 * PS;
  double* T = B + 3 * PS;
  const int es = slots[item], e = es / 6, f = es % 6;
  const FaceLink L = M.link[es];
  const int Nm = M.order[e], Nn = M.order[L.nbr];
  const int nm = Nm + 1, nn = Nn + 1;
  // my velocity trace (planes 0..2) and face metric (3..5), the neighbour's velocity trace
  for (int t = lane; t < nm * nm; t += 32) {
    double Sv[3];
    face_metric(M, e, f, nm, t % nm, t / nm, Sv);
    const int64_t s0 = M.tr_off[e] + f * nm * nm + t;
    for (int c = 0; c < 3; ++c) {
      A[c * PS + t] = tq_load(M, 1 + c, s0);
      A[(3 + c) * PS + t] = Sv[c];
    }
  }
  for (int t = lane; t < nn * nn; t += 32) {
    const int64_t s1 = M.tr_off[L.nbr] + L.nface * nn * nn + t;
    for (int c = 0; c < 3; ++c) B[c * PS + t] = tq_load(M, 1 + c, s1);
  }
  __syncwarp();
  tensor2_warp(interp_tab(M, Nm, MO), nm == nM, nm, nM, 6, A, T, A, PS, -1, MO, lane);
  tensor2_warp(interp_tab(M, Nn, MO), nn == nM, nn, nM, 3, B, T, B, PS, L.orient, MO, lane);
  for (int t = lane; t < PS; t += 32)
    for (int c = 0; c < 3; ++c) {
      const double us = 0.5 * (A[c * PS + t] + B[c * PS + t]);
      for (int k = 0; k < 3; ++k) T[(c * 3 + k) * PS + t] = us * A[(3 + k) * PS + t];
    }
  __syncwarp();
  // project to my order (A is free: it takes the first step), then store
  tensor2_warp(proj_tab(M, MO, Nm), nm == nM, nM, nm, 9, T, A, T, PS, -1, MO, lane);
  for (int t = lane; t < nm * nm; t += 32)
    for (int ck = 0; ck < 9; ++ck) M.LU[ck * M.tr_total + M.tr_off[e] + f * nm * nm + t] = T[ck * PS + t];
}

// Projected total numerical flux of a mortar face, once per face: the warp takes the side of
// the larger order (element e, its order is the mortar order MO), evaluates (F_e* - F_v*) . S on
// the mortar in e's face coordinates (Roe/LLF of both sides' states, the neighbour's interpolated
// to the mortar; the BR1 average of both sides' outward viscous traces, or the NS side alone on
// an NS/Euler face with the one-sided choice), stores it for e (its own order: no projection)
// and, with the sign reversed, L2-projected to the neighbour's order in the neighbour's face
// coordinates: seen from the neighbour the states swap and S turns, F*(q+, q-, -n) = -F*(q-, q+, n)
// for Roe and LLF and the viscous average changes sign, so its value is -H. [4][tr_total] at
// both sides' trace slots.
template <int MO>
__global__ void __launch_bounds__(32 * kMortarWarps) k_mortar_flux_w(DevMesh M, const int32_t* __restrict__ slots,
                                                                      int count) {
  using W = MortarW<MO>;
  constexpr int nM = W::nM, PS = W::PS;
  extern __shared__ double smd[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kMortarWarps + warp;
  if (item >= count) return;
  double* A = smd + warp * W::FLUX_PLANES * PS;
  double* B = A + 10 * PS;
  double* T = B + 7 * PS;
  const int es = slots[item], e = es / 6, f = es % 6;
  const FaceLink L = M.link[es];
  const int Nn = M.order[L.nbr], nn = Nn + 1;  // M.order[e] == MO
  const bool vm = M.flag[e] != 0, vn = L.nflag != 0;
  // planes 0..3 q, 4..6 outward viscous traces, 7..9 (mine only) the face metric; mine is at the
  // mortar order already
  for (int t = lane; t < PS; t += 32) {
    double Sv[3];
    face_metric(M, e, f, nM, t % nM, t / nM, Sv);
    const int64_t s0 = M.tr_off[e] + f * PS + t;
    for (int v = 0; v < 4; ++v) A[v * PS + t] = tq_load(M, v, s0);
    for (int c = 0; c < 3; ++c) {
      A[(4 + c) * PS + t] = vm ? tv_load(M, c, s0) : 0.0;
      A[(7 + c) * PS + t] = Sv[c];
    }
  }
  for (int t = lane; t < nn * nn; t += 32) {
    const int64_t s1 = M.tr_off[L.nbr] + L.nface * nn * nn + t;
    for (int v = 0; v < 4; ++v) B[v * PS + t] = tq_load(M, v, s1);
    for (int c = 0; c < 3; ++c) B[(4 + c) * PS + t] = vn ? tv_load(M, c, s1) : 0.0;
  }
  __syncwarp();
  // the viscous traces (planes 4..6) only where a side is NS; between Euler elements they are 0
  tensor2_warp(interp_tab(M, Nn, MO), nn == nM, nn, nM, (vm || vn) ? 7 : 4, B, T, B, PS, L.orient, MO, lane);
  if (!(vm || vn))
    for (int t = lane; t < 3 * PS; t += 32) B[4 * PS + t] = 0.0;
  __syncwarp();
  // F_v* . S = wm (mine) - wp (neighbour's outward): the average, or the NS side alone
  const bool one = M.mixed_face == 1 && vm != vn;
  const double wm = one ? (vm ? 1.0 : 0.0) : 0.5, wp = one ? (vm ? 0.0 : 1.0) : 0.5;
  const int64_t my0 = M.tr_off[e] + f * PS;
  for (int t = lane; t < PS; t += 32) {
    const double Sv[3] = {A[7 * PS + t], A[8 * PS + t], A[9 * PS + t]};
    const double s = sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
    const double nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
    double qm[4], qp[4], Fs[4], H[4];
    for (int v = 0; v < 4; ++v) {
      qm[v] = A[v * PS + t];
      qp[v] = B[v * PS + t];
    }
    flux_full(qm, qp, nh, M.c0sq, M.riemann, Fs);
    H[0] = s * Fs[0];
    for (int c = 0; c < 3; ++c) H[1 + c] = s * Fs[1 + c] - (wm * A[(4 + c) * PS + t] - wp * B[(4 + c) * PS + t]);
    for (int v = 0; v < 4; ++v) {
      M.LH[v * M.tr_total + my0 + t] = H[v];
      T[v * PS + t] = H[v];
    }
  }
  __syncwarp();
  // the neighbour's side: -H at its mortar coordinates (a1, b1), i.e. at my fwd_orient(a1, b1)
  for (int idx = lane; idx < 4 * PS; idx += 32) {
    const int v = idx / PS, r = idx % PS;
    int a0, b0;
    fwd_orient(L.orient, MO, r % nM, r / nM, a0, b0);
    A[v * PS + r] = -T[v * PS + a0 + nM * b0];
  }
  __syncwarp();
  tensor2_warp(proj_tab(M, MO, Nn), nn == nM, nM, nn, 4, A, B, A, PS, -1, MO, lane);
  const int64_t nb0 = M.tr_off[L.nbr] + L.nface * nn * nn;
  for (int t = lane; t < nn * nn; t += 32)
    for (int v = 0; v < 4; ++v) M.LH[v * M.tr_total + nb0 + t] = A[v * PS + t];
}

// ---------------------------------------------------------------------------------------
// state re-projection after a change of orders (Sec. 3.2): one block per element
// ---------------------------------------------------------------------------------------
// The element's state at its previous order, re-laid out at its current order by a 1D operator
// applied along each direction in turn: Lagrange interpolation when the order grows or stays,
// the L2 projection when it drops. Two shared buffers of nvar n^3 doubles ping-pong between
// the three passes (nvar = 4, or 5 for the compressible form).
__global__ void __launch_bounds__(256) k_project_state(DevMesh M, const int8_t* __restrict__ old_order,
                                                       const int64_t* __restrict__ old_off, int64_t total_old,
                                                       const double* __restrict__ qo, double* __restrict__ qn) {
  __shared__ double A[5 * NP * NP * NP], X[5 * NP * NP * NP];
  const int nv = M.model == 1 ? 5 : 4;
  const int e = blockIdx.x;
  const int No = old_order[e], Nn = M.order[e], no = No + 1, nn = Nn + 1;
  const double* T = Nn >= No ? interp_tab(M, No, Nn) : proj_tab(M, No, Nn);  // T[i * NP + j]: new i, old j
  const int64_t oo = old_off[e], on = M.elem_off[e];
  const int no3 = no * no * no;
  for (int t = threadIdx.x; t < nv * no3; t += blockDim.x) A[t] = qo[(t / no3) * total_old + oo + t % no3];
  __syncthreads();
  // along xi_1: X[v][c][b][I] = sum_a T[I][a] A[v][c][b][a]
  const int s1 = no * no * nn;
  for (int t = threadIdx.x; t < nv * s1; t += blockDim.x) {
    const int v = t / s1, r = t % s1, I = r % nn, cb = r / nn;
    double s = 0.0;
    for (int a = 0; a < no; ++a) s += T[I * NP + a] * A[v * no3 + cb * no + a];
    X[v * s1 + cb * nn + I] = s;
  }
  __syncthreads();
  // along xi_2: A[v][c][J][I] = sum_b T[J][b] X[v][c][b][I]
  const int s2 = no * nn * nn;
  for (int t = threadIdx.x; t < nv * s2; t += blockDim.x) {
    const int v = t / s2, r = t % s2, I = r % nn, J = (r / nn) % nn, c = r / (nn * nn);
    double s = 0.0;
    for (int b = 0; b < no; ++b) s += T[J * NP + b] * X[v * s1 + (c * no + b) * nn + I];
    A[v * s2 + (c * nn + J) * nn + I] = s;
  }
  __syncthreads();
  // along xi_3: qn[v][K][J][I] = sum_c T[K][c] A[v][c][J][I]
  const int nn3 = nn * nn * nn;
  for (int t = threadIdx.x; t < nv * nn3; t += blockDim.x) {
    const int v = t / nn3, r = t % nn3, IJ = r % (nn * nn), K = r / (nn * nn);
    double s = 0.0;
    for (int c = 0; c < no; ++c) s += T[K * NP + c] * A[v * s2 + c * nn * nn + IJ];
    qn[v * M.total + on + r] = s;
  }
}

// ---------------------------------------------------------------------------------------
// node coordinates and conservation sums (not on the hot path)
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void k_node_coords(DevMesh M, const int32_t* __restrict__ list, int count, const double* gn,
                              int gdeg, double* xyz) {
  constexpr int n = N + 1, n3 = n * n * n;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)count * n3) return;
  const int e = list[gid / n3], p = (int)(gid % n3);
  const int i = p % n, j = (p / n) % n, k = p / (n * n);
  const int ng = gdeg + 1, ng3 = ng * ng * ng;
  const double* I = (M.nodes == 1 ? M.interp_gl : M.interp) + (gdeg * NP + N) * NP * NP;
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int cc = 0; cc < ng; ++cc)
      for (int bb = 0; bb < ng; ++bb)
        for (int aa = 0; aa < ng; ++aa)
          s += I[i * NP + aa] * I[j * NP + bb] * I[k * NP + cc] * gn[((int64_t)e * ng3 + aa + ng * (bb + ng * cc)) * 3 + c];
    xyz[c * M.total + M.elem_off[e] + p] = s;
  }
}

template <int N>
__global__ void k_conservation(DevMesh M, const int32_t* __restrict__ list, int count, const double* R, int nvar,
                               double* partial) {
  constexpr int n = N + 1, n3 = n * n * n;
  int le = blockIdx.x * blockDim.x + threadIdx.x;
  if (le >= count) return;
  const int e = list[le];
  const int64_t off = M.elem_off[e];
  const bool curved = M.ec[e].curved != 0.0;
  for (int v = 0; v < nvar; ++v) {
    double s = 0.0;
    for (int p = 0; p < n3; ++p) {
      const double(*wt)[NP] = M.nodes == 1 ? c_ops.wg : c_ops.w;
      const double w = wt[N][p % n] * wt[N][(p / n) % n] * wt[N][p / (n * n)];
      const double J = curved ? M.geo[9 * M.total + off + p] : M.ec[e].J;
      s += w * J * R[v * M.total + off + p];
    }
    partial[v * M.n_elem + e] = s;
  }
}

// ---------------------------------------------------------------------------------------
// host <-> device copy by the SMs (page-locked host memory is directly addressable)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16,
                                                const double* __restrict__ src_tail, double* __restrict__ dst_tail,
                                                int64_t n_tail) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {  // four independent 16-byte loads in flight
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x < n_tail) dst_tail[threadIdx.x] = src_tail[threadIdx.x];
}

cudaError_t launch_copy_sm(void* dst, const void* src, size_t bytes, int sms, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  const bool aligned = ((uintptr_t)dst % 16 == 0) && ((uintptr_t)src % 16 == 0) && bytes % 8 == 0;
  if (!aligned) return cudaErrorInvalidValue;
  const int64_t n16 = (int64_t)(bytes / 16), tail = (int64_t)((bytes % 16) / 8);
  const unsigned grid = (unsigned)std::max(1, sms * 4);
  k_copy16<<<grid, 256, 0, s>>>(reinterpret_cast<const uint4*>(src), reinterpret_cast<uint4*>(dst), n16,
                                reinterpret_cast<const double*>(src) + 2 * n16, reinterpret_cast<double*>(dst) + 2 * n16,
                                tail);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------------------
cudaError_t upload_ops(const Ops1D& ops) {
  cudaError_t r = cudaMemcpyToSymbol(c_ops, &ops, sizeof(Ops1D));
  if (r == cudaSuccess) r = upload_ops_cns(ops);
  if (r == cudaSuccess) r = upload_ops_gl(ops);
  if (r == cudaSuccess) r = upload_ops_cns_gl(ops);
  return r == cudaSuccess ? upload_ops32(ops) : r;
}

template <int N, bool C>
static size_t visc_smem() {
  return sizeof(double) * (NP * NP + Shape<N>::EPB * (3 + (C ? 9 : 0) + 9) * Shape<N>::n3);
}
template <int N>
static size_t inv_smem(bool kep = false) {
  return sizeof(double) * (NP * NP + Shape<N>::EPB * (kep ? 13 : 12) * Shape<N>::n3);
}

template <int N>
static cudaError_t prep_n() {
  cudaError_t r;
  if ((r = cudaFuncSetAttribute(k_viscous<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem<N, false>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem<N, true>())) != cudaSuccess) return r;
  const int is = (int)inv_smem<N>(), ks = (int)inv_smem<N>(true);
  if ((r = cudaFuncSetAttribute(k_inviscid<N, false, MODE_RESIDUAL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, true, MODE_RESIDUAL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, false, MODE_RK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, true, MODE_RK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, false, MODE_RESIDUAL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, true, MODE_RESIDUAL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, false, MODE_RK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid<N, true, MODE_RK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks)) != cudaSuccess) return r;
  return cudaSuccess;
}

template <int MO>
static cudaError_t prep_mortar() {
  cudaError_t r = cudaFuncSetAttribute(k_mortar_lift_w<MO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)mortar_smem<MO>(false));
  if (r != cudaSuccess) return r;
  return cudaFuncSetAttribute(k_mortar_flux_w<MO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)mortar_smem<MO>(true));
}

cudaError_t prepare_kernels() {
  cudaError_t r;
  if ((r = prep_mortar<1>()) != cudaSuccess) return r;
  if ((r = prep_mortar<2>()) != cudaSuccess) return r;
  if ((r = prep_mortar<3>()) != cudaSuccess) return r;
  if ((r = prep_mortar<4>()) != cudaSuccess) return r;
  if ((r = prep_mortar<5>()) != cudaSuccess) return r;
  if ((r = prep_mortar<6>()) != cudaSuccess) return r;
  if ((r = prep_mortar<7>()) != cudaSuccess) return r;
  if ((r = prep_n<1>()) != cudaSuccess) return r;
  if ((r = prep_n<2>()) != cudaSuccess) return r;
  if ((r = prep_n<3>()) != cudaSuccess) return r;
  if ((r = prep_n<4>()) != cudaSuccess) return r;
  if ((r = prep_n<5>()) != cudaSuccess) return r;
  if ((r = prep_n<6>()) != cudaSuccess) return r;
  if ((r = prep_n<7>()) != cudaSuccess) return r;
  if ((r = prepare_kernels_cns()) != cudaSuccess) return r;
  if ((r = prepare_kernels_gl()) != cudaSuccess) return r;
  if ((r = prepare_kernels_cns_gl()) != cudaSuccess) return r;
  return prepare_kernels32();
}


cudaError_t launch_traces(const DevMesh& M, const Bucket& b, const double* q, int precision, cudaStream_t s) {
  if (precision == 1) return launch_traces32(M, b, q, s);
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * 6 * (NN + 1) * (NN + 1);
    const int thr = 256;
    k_traces<NN><<<(unsigned)((tot + thr - 1) / thr), thr, 0, s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

cudaError_t launch_viscous(const DevMesh& M, const Bucket& b, const double* q, int precision, cudaStream_t s) {
  if (precision == 1) return launch_viscous32(M, b, q, s);
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (b.curved)
      k_viscous<NN, true><<<grid, SH::threads, visc_smem<NN, true>(), s>>>(M, b.list, b.count, q);
    else
      k_viscous<NN, false><<<grid, SH::threads, visc_smem<NN, false>(), s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

template <int N, bool CURVED, int MODE, bool KEP>
static cudaError_t launch_inv64(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                                int stage, double dt, int write_tr, cudaStream_t s) {
  using SH = Shape<N>;
  const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
  k_inviscid<N, CURVED, MODE, KEP><<<grid, SH::threads, inv_smem<N>(KEP), s>>>(M, b.list, b.count, q, out, g, stage,
                                                                                dt, write_tr);
  return cudaGetLastError();
}

cudaError_t launch_inviscid(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                            int mode, int stage, double dt, int write_tr, int precision, cudaStream_t s) {
  if (precision == 1) return launch_inviscid32(M, b, q, out, g, mode, stage, write_tr, s);
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    if (M.split == 1) {
      if (mode == MODE_RESIDUAL)
        return b.curved ? launch_inv64<NN, true, MODE_RESIDUAL, true>(M, b, q, out, g, stage, dt, write_tr, s)
                        : launch_inv64<NN, false, MODE_RESIDUAL, true>(M, b, q, out, g, stage, dt, write_tr, s);
      return b.curved ? launch_inv64<NN, true, MODE_RK, true>(M, b, q, out, g, stage, dt, write_tr, s)
                      : launch_inv64<NN, false, MODE_RK, true>(M, b, q, out, g, stage, dt, write_tr, s);
    }
    if (mode == MODE_RESIDUAL)
      return b.curved ? launch_inv64<NN, true, MODE_RESIDUAL, false>(M, b, q, out, g, stage, dt, write_tr, s)
                      : launch_inv64<NN, false, MODE_RESIDUAL, false>(M, b, q, out, g, stage, dt, write_tr, s);
    return b.curved ? launch_inv64<NN, true, MODE_RK, false>(M, b, q, out, g, stage, dt, write_tr, s)
                    : launch_inv64<NN, false, MODE_RK, false>(M, b, q, out, g, stage, dt, write_tr, s);
  });
  return cudaGetLastError();
}

cudaError_t launch_project_state(const DevMesh& M, const int8_t* old_order, const int64_t* old_off, int64_t total_old,
                                 const double* qo, double* qn, cudaStream_t s) {
  if (M.n_elem == 0) return cudaSuccess;
  k_project_state<<<(unsigned)M.n_elem, 256, 0, s>>>(M, old_order, old_off, total_old, qo, qn);
  return cudaGetLastError();
}

// slots sorted by mortar order, mo_start[MO] .. mo_start[MO + 1] the slots of order MO
static cudaError_t launch_mortar(bool flux, const DevMesh& M, const int32_t* slots, const int* mo_start, int* nlaunch,
                                 cudaStream_t s) {
  for (int mo = 1; mo <= MAXN; ++mo) {
    const int count = mo_start[mo + 1] - mo_start[mo];
    if (count <= 0) continue;
    const int32_t* sl = slots + mo_start[mo];
    const unsigned grid = (unsigned)((count + kMortarWarps - 1) / kMortarWarps);
    DG_SWITCH_N(mo, {
      const size_t sm = mortar_smem<NN>(flux);
      if (flux)
        k_mortar_flux_w<NN><<<grid, 32 * kMortarWarps, sm, s>>>(M, sl, count);
      else
        k_mortar_lift_w<NN><<<grid, 32 * kMortarWarps, sm, s>>>(M, sl, count);
    });
    if (nlaunch) ++*nlaunch;
  }
  return cudaGetLastError();
}

cudaError_t launch_mortar_lift(const DevMesh& M, const int32_t* slots, const int* mo_start, int* nlaunch,
                               cudaStream_t s) {
  return launch_mortar(false, M, slots, mo_start, nlaunch, s);
}

cudaError_t launch_mortar_flux(const DevMesh& M, const int32_t* slots, const int* mo_start, int* nlaunch,
                               cudaStream_t s) {
  return launch_mortar(true, M, slots, mo_start, nlaunch, s);
}

cudaError_t launch_node_coords(const DevMesh& M, const double* gn, int gdeg, const Bucket& b, double* xyz,
                               cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * (NN + 1) * (NN + 1) * (NN + 1);
    k_node_coords<NN><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, b.list, b.count, gn, gdeg, xyz);
  });
  return cudaGetLastError();
}

cudaError_t launch_conservation(const DevMesh& M, const Bucket& b, const double* R, int nvar, double* partial,
                                cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    k_conservation<NN><<<(unsigned)((b.count + 127) / 128), 128, 0, s>>>(M, b.list, b.count, R, nvar, partial);
  });
  return cudaGetLastError();
}

}  // namespace dgk
