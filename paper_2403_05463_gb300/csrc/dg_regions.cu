// dg_regions.cu -- viscous/inviscid region detection on the device (arXiv 2403.05463, Sec. 2.1).
//
// One thread per node, Shape<N>::EPB elements per block (the tiling of the FP64 passes):
//   1. the element's velocity planes are staged in shared memory and differentiated along the
//      three reference directions with the Gauss-Lobatto derivative matrix D; the chain rule
//      with the element's metric terms (constant for affine elements, per node for curved
//      ones) gives J_ck = du_c/dx_k = (1/J) sum_d (J dxi_d/dx_k) du_c/dxi_d;
//   2. Q_S = (tr(S)^2 - tr(S^2))/2 and R_S = -det(S)/3 of S = (J + J^T)/2, and
//      Q_Omega = -tr(Omega^2)/2 of Omega = (J - J^T)/2, written out with the symmetry of S
//      and the skew-symmetry of Omega;
//   3. the two components' log-weights a_k = log w_k - log det(C_k)/2 - (x - mu_k)^T C_k^-1
//      (x - mu_k)/2 (common constant dropped) and the posteriors as logistic functions of
//      their difference: with E = exp(a_i - a_v), p_v = 1/(1 + E) and p_i = 1/(1 + 1/E)
//      (one exponential; E = 0 or inf give the limits 1, 0 and 0, 1);
//   4. per element, the plain means of p_v and p_i over its (N+1)^3 nodes, summed by one warp
//      in a fixed order (lane-strided partial sums, then a shuffle tree), and the flag
//      (mean p_v >= mean p_i: viscous/NS).
// FP64 throughout, so the flag is decided in the precision of the solver's state.
#include "dg_device.cuh"

namespace dgk {

// GEO: 0 axis-aligned box (diagonal metric), 1 affine, 2 curved (per-node metric terms)
template <int N, int GEO>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_detect_regions(DevMesh M, const int32_t* __restrict__ list, int count, GmmDev g, DMatArg Dm,
                     const double* __restrict__ q, uint8_t* __restrict__ flags, double* __restrict__ pbar,
                     double* __restrict__ feat) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  __shared__ double sD[n * n];
  __shared__ double sU[EPB * 3 * n3];
  __shared__ double sPv[EPB * n3];
  __shared__ double sPi[EPB * n3];
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += blockDim.x) sD[t] = Dm.D[t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  double* U = sU + le * 3 * n3;
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c * n3 + p] = __ldg(&q[(1 + c) * M.total + off + p]);
  }
  __syncthreads();
  if (active) {
    const int ii[3] = {p % n, (p / n) % n, p / n2};
    const int str[3] = {1, n, n2};
    double du[3][3];  // du[c][d] = d u_c / d xi_d
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double dm = sD[ii[d] * n + m];
        const int pm = base + m * str[d];
        s0 += dm * U[pm];
        s1 += dm * U[n3 + pm];
        s2 += dm * U[2 * n3 + pm];
      }
      du[0][d] = s0;
      du[1][d] = s1;
      du[2][d] = s2;
    }
    double G[3][3];
    if (GEO == 0) {
      const double invJ = M.ec[e].invJ;
      const double a0 = M.ec[e].Ja[0], a1 = M.ec[e].Ja[4], a2 = M.ec[e].Ja[8];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        G[c][0] = invJ * (a0 * du[c][0]);
        G[c][1] = invJ * (a1 * du[c][1]);
        G[c][2] = invJ * (a2 * du[c][2]);
      }
    } else {
      double Ja[9], invJ;
      if (GEO == 2) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Ja[k] = __ldg(&M.geo[k * M.total + off + p]);
        invJ = 1.0 / __ldg(&M.geo[9 * M.total + off + p]);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Ja[k] = M.ec[e].Ja[k];
        invJ = M.ec[e].invJ;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[c][k] = invJ * (Ja[k] * du[c][0] + Ja[3 + k] * du[c][1] + Ja[6 + k] * du[c][2]);
    }
    // strain rate (symmetric) and rotation rate (skew) parts
    const double s00 = G[0][0], s11 = G[1][1], s22 = G[2][2];
    const double s01 = 0.5 * (G[0][1] + G[1][0]), s02 = 0.5 * (G[0][2] + G[2][0]), s12 = 0.5 * (G[1][2] + G[2][1]);
    const double o01 = 0.5 * (G[0][1] - G[1][0]), o02 = 0.5 * (G[0][2] - G[2][0]), o12 = 0.5 * (G[1][2] - G[2][1]);
    const double trS = s00 + s11 + s22;
    const double trS2 = s00 * s00 + s11 * s11 + s22 * s22 + 2.0 * (s01 * s01 + s02 * s02 + s12 * s12);
    const double detS = s00 * (s11 * s22 - s12 * s12) - s01 * (s01 * s22 - s12 * s02) + s02 * (s01 * s12 - s11 * s02);
    const double x[3] = {0.5 * (trS * trS - trS2), -detS / 3.0, o01 * o01 + o02 * o02 + o12 * o12};
    double a[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double d0 = x[0] - g.mu[k][0], d1 = x[1] - g.mu[k][1], d2 = x[2] - g.mu[k][2];
      const double* P = g.P[k];
      const double m = P[0] * d0 * d0 + P[3] * d1 * d1 + P[5] * d2 * d2 +
                       2.0 * (P[1] * d0 * d1 + P[2] * d0 * d2 + P[4] * d1 * d2);
      a[k] = g.c[k] - 0.5 * m;
    }
    const double av = g.viscous ? a[1] : a[0], ai = g.viscous ? a[0] : a[1];
    const double E = exp(ai - av);
    const double pv = 1.0 / (1.0 + E);
    const double pi = 1.0 / (1.0 + 1.0 / E);
    sPv[le * n3 + p] = pv;
    sPi[le * n3 + p] = pi;
    if (feat) {
      const int64_t i = off + p;
      feat[i] = x[0];
      feat[M.total + i] = x[1];
      feat[2 * M.total + i] = x[2];
      feat[3 * M.total + i] = pv;
    }
  }
  __syncthreads();
  // element means: one warp per element, fixed summation order
  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  for (int el = warp; el < EPB; el += nwarps) {
    const int sl = blockIdx.x * EPB + el;
    if (sl >= count) break;
    double sv = 0.0, si = 0.0;
    for (int j = lane; j < n3; j += 32) {
      sv += sPv[el * n3 + j];
      si += sPi[el * n3 + j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const int ee = list[sl];
      const double mv = sv / n3, mi = si / n3;
      if (pbar) {
        pbar[ee] = mv;
        pbar[M.n_elem + ee] = mi;
      }
      if (flags) flags[ee] = mv >= mi ? 1 : 0;
    }
  }
}

#define DG_DETECT_N(NVAR, ...)                                   \
  switch (NVAR) {                                                \
    case 1: { constexpr int NN = 1; __VA_ARGS__; } break;        \
    case 2: { constexpr int NN = 2; __VA_ARGS__; } break;        \
    case 3: { constexpr int NN = 3; __VA_ARGS__; } break;        \
    case 4: { constexpr int NN = 4; __VA_ARGS__; } break;        \
    case 5: { constexpr int NN = 5; __VA_ARGS__; } break;        \
    case 6: { constexpr int NN = 6; __VA_ARGS__; } break;        \
    case 7: { constexpr int NN = 7; __VA_ARGS__; } break;        \
    default: return cudaErrorInvalidValue;                       \
  }

cudaError_t launch_detect_regions(const DevMesh& M, const Bucket& b, const GmmDev& g, const DMatArg& D,
                                  const double* q, uint8_t* flags, double* pbar, double* feat, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_DETECT_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (b.geo == 2)
      k_detect_regions<NN, 2><<<grid, SH::threads, 0, s>>>(M, b.list, b.count, g, D, q, flags, pbar, feat);
    else if (b.geo == 1)
      k_detect_regions<NN, 1><<<grid, SH::threads, 0, s>>>(M, b.list, b.count, g, D, q, flags, pbar, feat);
    else
      k_detect_regions<NN, 0><<<grid, SH::threads, 0, s>>>(M, b.list, b.count, g, D, q, flags, pbar, feat);
  });
  return cudaGetLastError();
}

}  // namespace dgk
