// dg_cns.cu -- sm_103a kernels of the compressible form (arXiv 2403.05463, App. A), FP64.
//
// State u = (rho, rho v1, rho v2, rho v3, rho e), ideal gas with unit gas constant:
// p = (gamma - 1)(rho e - rho |v|^2 / 2), T = p / rho, H = (rho e + p) / rho. Flag 0 elements
// solve the Euler equations, flag 1 the Navier-Stokes equations with the eddy viscosity
// mu_t = rho nu_t of the selected closure and the heat flux kappa grad T,
// kappa = c_p (mu / Pr + mu_t / Pr_t), c_p = gamma / (gamma - 1). Conforming faces between
// elements of one order (interior or periodic) node by node; p-nonconforming faces (Sec. 3.2)
// on the mortar of the larger order (five-variable mortar kernels below: interpolated states
// and viscous traces, L2 projection back); boundary faces: far-field inflow and pressure
// outflow (ghost states, interior viscous flux), adiabatic walls (no-slip, free-slip: mirror
// ghost states, no viscous energy flux).
//
// Per residual evaluation / Runge-Kutta stage (the passes of the incompressible FP64 path with
// five variables):
//   traces   : the 5 conservative face values of every element into the trace buffer;
//   viscous  (NS elements): BR1 gradient of phi = (v1, v2, v3, T) with the average {{phi}} on
//              faces, eddy viscosity, stress, heat flux, contravariant viscous flux of momentum
//              and energy, its divergence (J r_v) and the outward traces Fv . S;
//   inviscid (all elements): contravariant Euler flux and its divergence from shared memory,
//              Roe (or LLF) fluctuation and the BR1 viscous face average, + J r_v, then
//              R = (1/J)(...) or the in-place low-storage RK3 update (next-stage traces too).
// Strong form on Gauss-Lobatto nodes, equal to the weak form of App. B, Eq. NS4 by summation
// by parts:
//   J R = -sum_d D_d (Ftil_e^d - Ftil_v^d) - sum_faces (1/w_end) [(F_e* - F_v*) . S - (Ftil_e - Ftil_v)_out]
#include "dg_device.cuh"
#include "dg_cns_phys.cuh"

namespace dgk {

__constant__ double c_Dc[NP][NP * NP];  // Gauss-Lobatto derivative matrices D[N][i*n+m]
__constant__ double c_w0c[NP];          // end weights w[N][0]
// Williamson 2N-storage RK3 (the paper's low-storage third-order scheme, Sec. 2.3)
__constant__ double c_rkAc[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
__constant__ double c_rkBc[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

cudaError_t upload_ops_cns(const Ops1D& ops) {
  cudaError_t r = cudaMemcpyToSymbol(c_Dc, ops.D, sizeof(ops.D));
  if (r != cudaSuccess) return r;
  double w0[NP];
  for (int N = 0; N < NP; ++N) w0[N] = ops.w[N][0];
  return cudaMemcpyToSymbol(c_w0c, w0, sizeof(w0));
}

// ---------------------------------------------------------------------------------------
// mortars (p-nonconforming faces): one block of 64 threads per (element, face) slot
// ---------------------------------------------------------------------------------------
// sum_{aa, bb} T[a][aa] T[b][bb] src[aa + ns bb]: a 1D operator T (rows of NP) on both face
// directions
__device__ __forceinline__ double face_op(const double* T, int ns, int a, int b, const double* src) {
  double s = 0.0;
  for (int bb = 0; bb < ns; ++bb) {
    double t = 0.0;
    for (int aa = 0; aa < ns; ++aa) t += T[a * NP + aa] * src[aa + ns * bb];
    s += T[b * NP + bb] * t;
  }
  return s;
}

struct CnsMortarSmem {
  double mine[9][NP * NP];  // my face states (5) and outward viscous traces (4), my order
  double nbr[9][NP * NP];   // the neighbour's, its order
  double mM[9][NP * NP];    // mine on the mortar
  double nM[9][NP * NP];    // the neighbour's on the mortar, in my face coordinates
  double Sm[3][NP * NP];    // my outward face metric S, my order
  double SM[3][NP * NP];    // S on the mortar
  double H[12][NP * NP];    // mortar result
};

// my outward S at face node t and my (and the neighbour's) face planes [0, nv) (+5 viscous)
__device__ __forceinline__ void cns_mortar_load(const DevMesh& M, int e, int f, const FaceLink& L, int nm, int nn,
                                                bool visc_m, bool visc_n, int nplanes, CnsMortarSmem& sm) {
  const int t = threadIdx.x, d = f >> 1;
  const double sg = (f & 1) ? 1.0 : -1.0;
  if (t < nm * nm) {
    const bool cur = M.ec[e].curved != 0.0;
    if (M.nodes == 1 && cur) {  // Gauss-Legendre: the interpolant of Ja^d along the normal line
      const double* l = M.lb_g + ((nm - 1) * 2 + (f & 1)) * NP;
      double Sk[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < nm; ++i) {
        const int64_t node = M.elem_off[e] + line_node(f, nm, t % nm, t / nm, i);
        for (int k = 0; k < 3; ++k) Sk[k] += l[i] * M.geo[(d * 3 + k) * M.total + node];
      }
      for (int k = 0; k < 3; ++k) sm.Sm[k][t] = sg * Sk[k];
    } else {
      const int64_t node = M.elem_off[e] + face_node(f, nm, t % nm, t / nm);
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.Sm[k][t] = sg * (cur ? M.geo[(d * 3 + k) * M.total + node] : M.ec[e].Ja[d * 3 + k]);
    }
    const int64_t s0 = M.tr_off[e] + f * nm * nm + t;
    for (int v = 0; v < 5; ++v) sm.mine[v][t] = M.Tq[v * M.tr_total + s0];
    for (int v = 5; v < nplanes; ++v) sm.mine[v][t] = visc_m ? M.Tv[(v - 5) * M.tr_total + s0] : 0.0;
  }
  if (t < nn * nn) {
    const int64_t s1 = M.tr_off[L.nbr] + L.nface * nn * nn + t;
    for (int v = 0; v < 5; ++v) sm.nbr[v][t] = M.Tq[v * M.tr_total + s1];
    for (int v = 5; v < nplanes; ++v) sm.nbr[v][t] = visc_n ? M.Tv[(v - 5) * M.tr_total + s1] : 0.0;
  }
}

// both sides' planes and my S interpolated to the mortar of order Mo
__device__ __forceinline__ void cns_to_mortar(const DevMesh& M, const FaceLink& L, int Nm, int Nn, int Mo, int nplanes,
                                              CnsMortarSmem& sm) {
  const int t = threadIdx.x, nm = Nm + 1, nn = Nn + 1, nM = Mo + 1;
  if (t < nM * nM) {
    const int a = t % nM, b = t / nM;
    const double* I = M.nodes == 1 ? M.interp_g : M.interp;  // the node set's tables
    const double* Im = I + (Nm * NP + Mo) * NP * NP;
    const double* In = I + (Nn * NP + Mo) * NP * NP;
    for (int v = 0; v < nplanes; ++v) sm.mM[v][t] = face_op(Im, nm, a, b, sm.mine[v]);
    for (int k = 0; k < 3; ++k) sm.SM[k][t] = face_op(Im, nm, a, b, sm.Sm[k]);
    int a0, b0;
    fwd_orient(L.orient, Mo, a, b, a0, b0);  // (a, b) are the neighbour's mortar coordinates here
    for (int v = 0; v < nplanes; ++v) sm.nM[v][a0 + nM * b0] = face_op(In, nn, a, b, sm.nbr[v]);
  }
}

// BR1 lifting data of the NS elements' mortar faces: LU[c*3+k] = P(phi*_c S_k), phi = (v, T)
__global__ void __launch_bounds__(64) k_mortar_lift_cns(DevMesh M, const int32_t* __restrict__ slots, int count) {
  __shared__ CnsMortarSmem sm;
  if (blockIdx.x >= count) return;
  const int es = slots[blockIdx.x], e = es / 6, f = es % 6;
  const FaceLink L = M.link[es];
  const int Nm = M.order[e], Nn = M.order[L.nbr], Mo = Nm > Nn ? Nm : Nn;
  const int nm = Nm + 1, nM = Mo + 1, t = threadIdx.x;
  cns_mortar_load(M, e, f, L, nm, Nn + 1, false, false, 5, sm);
  __syncthreads();
  cns_to_mortar(M, L, Nm, Nn, Mo, 5, sm);
  __syncthreads();
  if (t < nM * nM) {
    double um[5], up[5];
    for (int v = 0; v < 5; ++v) {
      um[v] = sm.mM[v][t];
      up[v] = sm.nM[v][t];
    }
    const Prim A = prim(um, M.gamma), B = prim(up, M.gamma);
    const double ps[4] = {0.5 * (A.v[0] + B.v[0]), 0.5 * (A.v[1] + B.v[1]), 0.5 * (A.v[2] + B.v[2]),
                          0.5 * (A.p / A.rho + B.p / B.rho)};
    for (int c = 0; c < 4; ++c)
      for (int k = 0; k < 3; ++k) sm.H[c * 3 + k][t] = ps[c] * sm.SM[k][t];
  }
  __syncthreads();
  if (t < nm * nm) {
    const double* P = (M.nodes == 1 ? M.proj_g : M.proj) + (Mo * NP + Nm) * NP * NP;
    const int a = t % nm, b = t / nm;
    for (int ck = 0; ck < 12; ++ck)
      M.LU[ck * M.tr_total + M.tr_off[e] + f * nm * nm + t] = face_op(P, nM, a, b, sm.H[ck]);
  }
}

// total flux of every mortar face: LH[v] = P((F_e*(u-, u+) - F_v*) . S), my outward S
__global__ void __launch_bounds__(64) k_mortar_flux_cns(DevMesh M, const int32_t* __restrict__ slots, int count) {
  __shared__ CnsMortarSmem sm;
  if (blockIdx.x >= count) return;
  const int es = slots[blockIdx.x], e = es / 6, f = es % 6;
  const FaceLink L = M.link[es];
  const int Nm = M.order[e], Nn = M.order[L.nbr], Mo = Nm > Nn ? Nm : Nn;
  const int nm = Nm + 1, nM = Mo + 1, t = threadIdx.x;
  const bool vm = M.flag[e] != 0, vn = L.nflag != 0;
  cns_mortar_load(M, e, f, L, nm, Nn + 1, vm, vn, 9, sm);
  __syncthreads();
  cns_to_mortar(M, L, Nm, Nn, Mo, 9, sm);
  __syncthreads();
  if (t < nM * nM) {
    const double Sv[3] = {sm.SM[0][t], sm.SM[1][t], sm.SM[2][t]};
    const double s = sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
    const double nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
    double um[5], up[5], Fn[5], fx[5];
    for (int v = 0; v < 5; ++v) {
      um[v] = sm.mM[v][t];
      up[v] = sm.nM[v][t];
    }
    cns_normal_flux(um, nh, M.gamma, Fn);
    cns_fluct(um, up, nh, M.gamma, M.riemann, fx);
    // F_v* . S = wm (mine) - wp (the neighbour's outward): the average, or the NS side alone
    const bool one = M.mixed_face == 1 && vm != vn;
    const double wm = one ? (vm ? 1.0 : 0.0) : 0.5, wp = one ? (vm ? 0.0 : 1.0) : 0.5;
    sm.H[0][t] = s * (Fn[0] + fx[0]);
    for (int v = 0; v < 4; ++v) sm.H[1 + v][t] = s * (Fn[1 + v] + fx[1 + v]) - (wm * sm.mM[5 + v][t] - wp * sm.nM[5 + v][t]);
  }
  __syncthreads();
  if (t < nm * nm) {
    const double* P = (M.nodes == 1 ? M.proj_g : M.proj) + (Mo * NP + Nm) * NP * NP;
    const int a = t % nm, b = t / nm;
    for (int v = 0; v < 5; ++v)
      M.LH[v * M.tr_total + M.tr_off[e] + f * nm * nm + t] = face_op(P, nM, a, b, sm.H[v]);
  }
}

// ---------------------------------------------------------------------------------------
// traces
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void k_traces_cns(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ u) {
  constexpr int n = N + 1, n2 = n * n, per = 6 * n2;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)count * per) return;
  const int le = (int)(gid / per), r = (int)(gid % per);
  const int f = r / n2, ab = r % n2;
  const int e = list[le];
  const int64_t src = M.elem_off[e] + face_node(f, n, ab % n, ab / n);
  const int64_t dst = M.tr_off[e] + f * n2 + ab;
#pragma unroll
  for (int v = 0; v < 5; ++v) M.Tq[v * M.tr_total + dst] = __ldg(&u[v * M.total + src]);
}

// ---------------------------------------------------------------------------------------
// viscous pass (NS elements)
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_viscous_cns(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ u) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;                                 // n*n
  double* sP = sD + NP * NP;                       // EPB * 4 * n3: phi = (v1, v2, v3, T)
  double* sJa = sP + EPB * 4 * n3;                 // EPB * 9 * n3 (curved only)
  double* sF = sJa + (CURVED ? EPB * 9 * n3 : 0);  // EPB * 12 * n3: Ftil_v[d][4]
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_Dc[N][t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* P = sP + le * 4 * n3;
  double* JA = sJa + le * 9 * n3;
  double* F = sF + le * 12 * n3;
  const double gamma = M.gamma;
  double Ja[9], invJ = 0.0, uu[5] = {1.0, 0.0, 0.0, 0.0, 1.0}, ph[4] = {0.0, 0.0, 0.0, 0.0};
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) uu[v] = __ldg(&u[v * M.total + off + p]);
    const Prim Q = prim(uu, gamma);
    ph[0] = Q.v[0], ph[1] = Q.v[1], ph[2] = Q.v[2], ph[3] = Q.p / Q.rho;
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
  if (active) {
    double G[4][3];  // G[c][k] = d phi_c / d x_k
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[c][k] = 0.0;
    // volume part: J G_ck = sum_d D_d (Ja^d_k phi_c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
      if (!CURVED) {
        double dp[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const double dm = sD[ii[d] * n + m];
          const int pm = base + m * str[d];
#pragma unroll
          for (int c = 0; c < 4; ++c) dp[c] += dm * P[c * n3 + pm];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += Ja[d * 3 + k] * dp[c];
      } else {
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const double dm = sD[ii[d] * n + m];
          const int pm = base + m * str[d];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double dj = dm * JA[(d * 3 + k) * n3 + pm];
#pragma unroll
            for (int c = 0; c < 4; ++c) G[c][k] += dj * P[c * n3 + pm];
          }
        }
      }
    }
    // BR1 lifting on the faces this node lies on: (1/w_end) ({{phi}} - phi) S
    const double invw = 1.0 / c_w0c[N];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
      const double sg = side ? 1.0 : -1.0;
      const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
      const FaceLink L = M.link[e * 6 + f];
      const double Sv[3] = {sg * Ja[d * 3], sg * Ja[d * 3 + 1], sg * Ja[d * 3 + 2]};
      if (L.kind == FK_MORTAR) {  // the projected phi* S from the mortar
        const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += invw * (M.LU[(c * 3 + k) * M.tr_total + ms] - ph[c] * Sv[k]);
        continue;
      }
      double jump[4];
      if (L.kind == FK_CONF) {
        int a1, b1;
        inv_orient(L.orient, N, a, b, a1, b1);
        const int64_t ns = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
        double un[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) un[v] = M.Tq[v * M.tr_total + ns];
        const Prim Q = prim(un, gamma);
        jump[0] = Q.v[0] - ph[0], jump[1] = Q.v[1] - ph[1], jump[2] = Q.v[2] - ph[2], jump[3] = Q.p / Q.rho - ph[3];
      } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {  // mirror ghost: T kept, velocity reflected
        const double vo[3] = {ph[0], ph[1], ph[2]};
        double jw[3];
        wall_jump<double>(L.kind, vo, Sv, jw);
        jump[0] = jw[0], jump[1] = jw[1], jump[2] = jw[2], jump[3] = 0.0;
      } else if (L.kind == FK_INFLOW) {  // the far field: v_inf, T = p_inf / rho_inf
#pragma unroll
        for (int c = 0; c < 3; ++c) jump[c] = M.inflow[1 + c] - ph[c];
        jump[3] = M.p_inf / M.inflow[0] - ph[3];
      } else if (L.kind == FK_OUTFLOW) {  // interior velocity, T = p_inf / rho
        jump[0] = jump[1] = jump[2] = 0.0;
        jump[3] = M.p_inf / uu[0] - ph[3];
      } else {  // no other face kind exists
        atomicCAS(&M.err[0], 0, 5);
        atomicCAS(&M.err[1], 0, 10);
        continue;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[c][k] += invw * 0.5 * jump[c] * Sv[k];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[c][k] *= invJ;
    // eddy viscosity, stress, heat flux
    const double Gv[3][3] = {{G[0][0], G[0][1], G[0][2]}, {G[1][0], G[1][1], G[1][2]}, {G[2][0], G[2][1], G[2][2]}};
    const double mut = uu[0] * eddy_visc(Gv, M.ec[e].delta, M.closure, M.cs, M.cv);
    const double mu = M.nu + mut;
    const double kappa = gamma / (gamma - 1.0) * (M.nu / M.prandtl + mut / M.prandtl_t);
    const double tr = Gv[0][0] + Gv[1][1] + Gv[2][2];
    double fv[4][3];  // physical viscous flux rows: momentum 1..3, energy
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) fv[c][k] = mu * (Gv[c][k] + Gv[k][c]) - (c == k ? (2.0 / 3.0) * mu * tr : 0.0);
#pragma unroll
    for (int k = 0; k < 3; ++k) fv[3][k] = ph[0] * fv[0][k] + ph[1] * fv[1][k] + ph[2] * fv[2][k] + kappa * G[3][k];
    // contravariant viscous flux Ftil_v^d = sum_k Ja^d_k fv_k
    double Fc[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Fc[d][v] = Ja[d * 3] * fv[v][0] + Ja[d * 3 + 1] * fv[v][1] + Ja[d * 3 + 2] * fv[v][2];
        F[(d * 4 + v) * n3 + p] = Fc[d][v];
      }
    // outward viscous flux traces Fv . S = sigma Ftil_v^d
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
      const double sg = side ? 1.0 : -1.0;
      const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
      const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
#pragma unroll
      for (int v = 0; v < 4; ++v) M.Tv[v * M.tr_total + ms] = sg * Fc[d][v];
    }
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
  }
}

// ---------------------------------------------------------------------------------------
// inviscid pass + assembly + (optional) RK update
// ---------------------------------------------------------------------------------------
template <int N, bool CURVED, int MODE>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_inviscid_cns(DevMesh M, const int32_t* __restrict__ list, int count, const double* uin, double* out,
                   double* g, int stage, double dt, int write_tr) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ double sm[];
  double* sD = sm;
  double* sF = sD + NP * NP;  // EPB * 15 * n3: Ftil_e[d][v]
  const int tid = threadIdx.x;
  for (int t = tid; t < n2; t += blockDim.x) sD[t] = c_Dc[N][t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* F = sF + le * 15 * n3;
  const double gamma = M.gamma;
  double uu[5] = {1.0, 0.0, 0.0, 0.0, 1.0}, Ja[9], invJ = 0.0;
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) uu[v] = uin[v * M.total + off + p];
    if (CURVED) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = __ldg(&M.geo[k * M.total + off + p]);
      invJ = 1.0 / __ldg(&M.geo[9 * M.total + off + p]);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = M.ec[e].Ja[k];
      invJ = M.ec[e].invJ;
    }
    // physical Euler flux fl[v][k] and its contravariant form
    const Prim Q = prim(uu, gamma);
    double fl[5][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      fl[0][k] = uu[1 + k];
#pragma unroll
      for (int c = 0; c < 3; ++c) fl[1 + c][k] = uu[1 + c] * Q.v[k] + (c == k ? Q.p : 0.0);
      fl[4][k] = (uu[4] + Q.p) * Q.v[k];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v)
        F[(d * 5 + v) * n3 + p] = Ja[d * 3] * fl[v][0] + Ja[d * 3 + 1] * fl[v][1] + Ja[d * 3 + 2] * fl[v][2];
  }
  __syncthreads();
  if (!active) return;
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  double JR[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
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
  const bool ns = M.flag[e] != 0;
  if (ns) {
#pragma unroll
    for (int v = 0; v < 4; ++v) JR[1 + v] += M.rv[v * M.total + off + p];
  }
  const double invw = 1.0 / c_w0c[N];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (ii[d] != 0 && ii[d] != N) continue;
    const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
    const double sg = side ? 1.0 : -1.0;
    const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
    const FaceLink L = M.link[e * 6 + f];
    const double Sv[3] = {sg * Ja[d * 3], sg * Ja[d * 3 + 1], sg * Ja[d * 3 + 2]};
    const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
    const double s = sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
    const double nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
    if (L.kind == FK_MORTAR) {
      // the projected (F_e* - F_v*) . S from the mortar minus the own outward flux (Euler, and
      // viscous for NS elements)
      double Fo[5];
      cns_normal_flux(uu, nh, gamma, Fo);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double own = s * Fo[v];
        if (v > 0 && ns) own -= M.Tv[(v - 1) * M.tr_total + ms];
        JR[v] -= invw * (M.LH[v * M.tr_total + ms] - own);
      }
      continue;
    }
    double up[5];  // the neighbour's face state, or the mirror ghost behind a wall
    int64_t nsl = 0;
    if (L.kind == FK_CONF) {
      int a1, b1;
      inv_orient(L.orient, N, a, b, a1, b1);
      nsl = M.tr_off[L.nbr] + L.nface * n2 + a1 + n * b1;
#pragma unroll
      for (int v = 0; v < 5; ++v) up[v] = M.Tq[v * M.tr_total + nsl];
    } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {  // density and energy kept, momentum reflected
      const double mo[3] = {uu[1], uu[2], uu[3]};
      double jw[3];
      wall_jump<double>(L.kind, mo, Sv, jw);
      up[0] = uu[0];
      up[4] = uu[4];
#pragma unroll
      for (int c = 0; c < 3; ++c) up[1 + c] = uu[1 + c] + jw[c];
    } else if (L.kind == FK_INFLOW) {  // the far-field state
      const double r = M.inflow[0];
      up[0] = r;
#pragma unroll
      for (int c = 0; c < 3; ++c) up[1 + c] = r * M.inflow[1 + c];
      up[4] = M.p_inf / (gamma - 1.0) +
              0.5 * r * (M.inflow[1] * M.inflow[1] + M.inflow[2] * M.inflow[2] + M.inflow[3] * M.inflow[3]);
    } else if (L.kind == FK_OUTFLOW) {  // interior density and momentum, the far-field pressure
      up[0] = uu[0];
#pragma unroll
      for (int c = 0; c < 3; ++c) up[1 + c] = uu[1 + c];
      up[4] = M.p_inf / (gamma - 1.0) + 0.5 * (uu[1] * uu[1] + uu[2] * uu[2] + uu[3] * uu[3]) / uu[0];
    } else {  // no other face kind exists
      atomicCAS(&M.err[0], 0, 5);
      atomicCAS(&M.err[1], 0, 11);
      continue;
    }
    double fx[5];
    cns_fluct(uu, up, nh, gamma, M.riemann, fx);
#pragma unroll
    for (int v = 0; v < 5; ++v) JR[v] -= invw * s * fx[v];
    if (L.kind != FK_CONF) {
      // inflow, outflow: F_v* . S is the own flux, nothing is left. Adiabatic wall, NS element:
      // F_v* . S is the own traction (no-slip) or its normal part (free-slip) and carries no
      // energy, so the own outward flux minus F_v* . S leaves nothing (no-slip) or the
      // tangential traction (free-slip) in momentum, and the own energy flux
      if (ns && (L.kind == FK_WALL || L.kind == FK_SLIP)) {
        const double tw[3] = {M.Tv[ms], M.Tv[M.tr_total + ms], M.Tv[2 * M.tr_total + ms]};
        if (L.kind == FK_SLIP) {
          double tt[3];
          slip_visc_term<double>(tw, Sv, tt);
#pragma unroll
          for (int c = 0; c < 3; ++c) JR[1 + c] -= invw * tt[c];
        }
        JR[4] -= invw * M.Tv[3 * M.tr_total + ms];
      }
      continue;
    }
    if (ns || L.nflag) {
      // BR1: Ftil_v,out - F_v* . S = wo Fv_own . S_own + wn Fv_nbr . S_nbr
      float wo, wn;
      visc_face_weights(M.mixed_face, ns, L.nflag != 0, wo, wn);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double t = 0.0;
        if (ns) t += (double)wo * M.Tv[v * M.tr_total + ms];
        if (L.nflag) t += (double)wn * M.Tv[v * M.tr_total + nsl];
        JR[1 + v] -= invw * t;
      }
    }
  }
  if (MODE == MODE_RESIDUAL) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * M.total + off + p] = JR[v] * invJ;
  } else {
    const double A = c_rkAc[stage], B = c_rkBc[stage];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int64_t ix = v * M.total + off + p;
      double gi = dt * (JR[v] * invJ);
      if (stage > 0) gi = fma(A, g[ix], gi);  // explicit FMAs: one rounding order in every code path
      g[ix] = gi;
      const double qn = fma(B, gi, uu[v]);
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
// dispatch
// ---------------------------------------------------------------------------------------
template <int N, bool C>
static size_t visc_smem_cns() {
  return sizeof(double) * (NP * NP + Shape<N>::EPB * (4 + (C ? 9 : 0) + 12) * Shape<N>::n3);
}
template <int N>
static size_t inv_smem_cns() {
  return sizeof(double) * (NP * NP + Shape<N>::EPB * 15 * Shape<N>::n3);
}

template <int N>
static cudaError_t prep_cns() {
  cudaError_t r;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((r = cudaFuncSetAttribute(k_viscous_cns<N, false>, attr, (int)visc_smem_cns<N, false>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous_cns<N, true>, attr, (int)visc_smem_cns<N, true>())) != cudaSuccess) return r;
  const int is = (int)inv_smem_cns<N>();
  if ((r = cudaFuncSetAttribute(k_inviscid_cns<N, false, MODE_RESIDUAL>, attr, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_cns<N, true, MODE_RESIDUAL>, attr, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_cns<N, false, MODE_RK>, attr, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid_cns<N, true, MODE_RK>, attr, is)) != cudaSuccess) return r;
  return cudaSuccess;
}

cudaError_t prepare_kernels_cns() {
  cudaError_t r;
  if ((r = prep_cns<1>()) != cudaSuccess) return r;
  if ((r = prep_cns<2>()) != cudaSuccess) return r;
  if ((r = prep_cns<3>()) != cudaSuccess) return r;
  if ((r = prep_cns<4>()) != cudaSuccess) return r;
  if ((r = prep_cns<5>()) != cudaSuccess) return r;
  if ((r = prep_cns<6>()) != cudaSuccess) return r;
  return prep_cns<7>();
}


cudaError_t launch_mortar_lift_cns(const DevMesh& M, const int32_t* slots, int count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_mortar_lift_cns<<<count, 64, 0, s>>>(M, slots, count);
  return cudaGetLastError();
}

cudaError_t launch_mortar_flux_cns(const DevMesh& M, const int32_t* slots, int count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_mortar_flux_cns<<<count, 64, 0, s>>>(M, slots, count);
  return cudaGetLastError();
}

cudaError_t launch_traces_cns(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * 6 * (NN + 1) * (NN + 1);
    k_traces_cns<NN><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, b.list, b.count, u);
  });
  return cudaGetLastError();
}

cudaError_t launch_viscous_cns(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (b.curved)
      k_viscous_cns<NN, true><<<grid, SH::threads, visc_smem_cns<NN, true>(), s>>>(M, b.list, b.count, u);
    else
      k_viscous_cns<NN, false><<<grid, SH::threads, visc_smem_cns<NN, false>(), s>>>(M, b.list, b.count, u);
  });
  return cudaGetLastError();
}

cudaError_t launch_inviscid_cns(const DevMesh& M, const Bucket& b, const double* u, double* out, double* g,
                                int mode, int stage, double dt, int write_tr, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    const size_t sm = inv_smem_cns<NN>();
    if (mode == MODE_RESIDUAL) {
      if (b.curved)
        k_inviscid_cns<NN, true, MODE_RESIDUAL><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, u, out, g, stage, dt, write_tr);
      else
        k_inviscid_cns<NN, false, MODE_RESIDUAL><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, u, out, g, stage, dt, write_tr);
    } else {
      if (b.curved)
        k_inviscid_cns<NN, true, MODE_RK><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, u, out, g, stage, dt, write_tr);
      else
        k_inviscid_cns<NN, false, MODE_RK><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, u, out, g, stage, dt, write_tr);
    }
  });
  return cudaGetLastError();
}

}  // namespace dgk
