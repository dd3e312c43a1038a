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
// FP64 by default, so that the flag is decided in the precision of the solver's state; the FP32
// variant (gmm.precision 1) runs the same steps in FP32 and is bound by HBM instead of the FP64
// pipe.
#include "dg_device.cuh"

namespace dgk {

// GEO: 0 axis-aligned box (diagonal metric), 1 affine, 2 curved (per-node metric terms).
// T: double (FP64 pass) or float (FP32 pass: the velocity rounded to FP32 with integer
// instructions, FP32 metric copies, FP32 arithmetic, outputs widened to FP64).
template <typename T>
__device__ __forceinline__ T to_t(double x);
template <>
__device__ __forceinline__ double to_t<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_t<float>(double x) {
  float h, l;
  split_hilo(x, h, l);
  return h + l;
}
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return widen_f32(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }

template <int N, int GEO, typename T>
__global__ void __launch_bounds__(Shape<N>::threads)
    k_detect_regions(DevMesh M, const int32_t* __restrict__ list, int count, GmmDev g, DMatArg Dm,
                     const double* __restrict__ q, uint8_t* __restrict__ flags, double* __restrict__ pbar,
                     double* __restrict__ feat) {
  using S = Shape<N>;
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  __shared__ T sD[n * n];
  __shared__ T sU[EPB * 3 * n3];
  __shared__ T sPv[EPB * n3];
  __shared__ T sPi[EPB * n3];
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += blockDim.x) sD[t] = (T)Dm.D[t];
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  T* U = sU + le * 3 * n3;
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c * n3 + p] = to_t<T>(__ldg(&q[(1 + c) * M.total + off + p]));
  }
  __syncthreads();
  if (active) {
    const int ii[3] = {p % n, (p / n) % n, p / n2};
    const int str[3] = {1, n, n2};
    T du[3][3];  // du[c][d] = d u_c / d xi_d
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int base = p - ii[d] * str[d];
      T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const T dm = sD[ii[d] * n + m];
        const int pm = base + m * str[d];
        s0 += dm * U[pm];
        s1 += dm * U[n3 + pm];
        s2 += dm * U[2 * n3 + pm];
      }
      du[0][d] = s0;
      du[1][d] = s1;
      du[2][d] = s2;
    }
    T G[3][3];
    if (GEO == 0) {
      const T invJ = F32 ? (T)M.ec32[e].invJ : (T)M.ec[e].invJ;
      const T a0 = F32 ? (T)M.ec32[e].Ja[0] : (T)M.ec[e].Ja[0];
      const T a1 = F32 ? (T)M.ec32[e].Ja[4] : (T)M.ec[e].Ja[4];
      const T a2 = F32 ? (T)M.ec32[e].Ja[8] : (T)M.ec[e].Ja[8];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        G[c][0] = invJ * (a0 * du[c][0]);
        G[c][1] = invJ * (a1 * du[c][1]);
        G[c][2] = invJ * (a2 * du[c][2]);
      }
    } else {
      T Ja[9], invJ;
      if (GEO == 2) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          Ja[k] = F32 ? (T)__ldg(&M.geo32[k * M.total + off + p]) : (T)__ldg(&M.geo[k * M.total + off + p]);
        invJ = F32 ? (T)__ldg(&M.geo32[9 * M.total + off + p]) : (T)(1.0 / __ldg(&M.geo[9 * M.total + off + p]));
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Ja[k] = F32 ? (T)M.ec32[e].Ja[k] : (T)M.ec[e].Ja[k];
        invJ = F32 ? (T)M.ec32[e].invJ : (T)M.ec[e].invJ;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[c][k] = invJ * (Ja[k] * du[c][0] + Ja[3 + k] * du[c][1] + Ja[6 + k] * du[c][2]);
    }
    // strain rate (symmetric) and rotation rate (skew) parts
    const T h = (T)0.5;
    const T s00 = G[0][0], s11 = G[1][1], s22 = G[2][2];
    const T s01 = h * (G[0][1] + G[1][0]), s02 = h * (G[0][2] + G[2][0]), s12 = h * (G[1][2] + G[2][1]);
    const T o01 = h * (G[0][1] - G[1][0]), o02 = h * (G[0][2] - G[2][0]), o12 = h * (G[1][2] - G[2][1]);
    const T trS = s00 + s11 + s22;
    const T trS2 = s00 * s00 + s11 * s11 + s22 * s22 + (T)2 * (s01 * s01 + s02 * s02 + s12 * s12);
    const T detS = s00 * (s11 * s22 - s12 * s12) - s01 * (s01 * s22 - s12 * s02) + s02 * (s01 * s12 - s11 * s02);
    const T x[3] = {h * (trS * trS - trS2), -detS / (T)3, o01 * o01 + o02 * o02 + o12 * o12};
    T a[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const T d0 = x[0] - (F32 ? (T)g.mu32[k][0] : (T)g.mu[k][0]);
      const T d1 = x[1] - (F32 ? (T)g.mu32[k][1] : (T)g.mu[k][1]);
      const T d2 = x[2] - (F32 ? (T)g.mu32[k][2] : (T)g.mu[k][2]);
      T P[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) P[i] = F32 ? (T)g.P32[k][i] : (T)g.P[k][i];
      const T m = P[0] * d0 * d0 + P[3] * d1 * d1 + P[5] * d2 * d2 + (T)2 * (P[1] * d0 * d1 + P[2] * d0 * d2 + P[4] * d1 * d2);
      a[k] = (F32 ? (T)g.c32[k] : (T)g.c[k]) - h * m;
    }
    const T av = g.viscous ? a[1] : a[0], ai = g.viscous ? a[0] : a[1];
    const T E = t_exp(ai - av);
    const T pv = (T)1 / ((T)1 + E);
    const T pi = (T)1 / ((T)1 + (T)1 / E);
    sPv[le * n3 + p] = pv;
    sPi[le * n3 + p] = pi;
    if (feat) {
      const int64_t i = off + p;
      feat[i] = to_f64(x[0]);
      feat[M.total + i] = to_f64(x[1]);
      feat[2 * M.total + i] = to_f64(x[2]);
      feat[3 * M.total + i] = to_f64(pv);
    }
  }
  __syncthreads();
  // element means: one warp per element, fixed summation order
  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  for (int el = warp; el < EPB; el += nwarps) {
    const int sl = blockIdx.x * EPB + el;
    if (sl >= count) break;
    T sv = 0, si = 0;
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
      const T mv = sv / (T)n3, mi = si / (T)n3;
      if (pbar) {
        pbar[ee] = to_f64(mv);
        pbar[M.n_elem + ee] = to_f64(mi);
      }
      if (flags) flags[ee] = mv >= mi ? 1 : 0;
    }
  }
}


template <int N, typename T>
static void launch_detect_t(const DevMesh& M, const Bucket& b, const GmmDev& g, const DMatArg& D, const double* q,
                            uint8_t* flags, double* pbar, double* feat, cudaStream_t s) {
  using SH = Shape<N>;
  const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
  if (b.geo == 2)
    k_detect_regions<N, 2, T><<<grid, SH::threads, 0, s>>>(M, b.list, b.count, g, D, q, flags, pbar, feat);
  else if (b.geo == 1)
    k_detect_regions<N, 1, T><<<grid, SH::threads, 0, s>>>(M, b.list, b.count, g, D, q, flags, pbar, feat);
  else
    k_detect_regions<N, 0, T><<<grid, SH::threads, 0, s>>>(M, b.list, b.count, g, D, q, flags, pbar, feat);
}

cudaError_t launch_detect_regions(const DevMesh& M, const Bucket& b, const GmmDev& g, const DMatArg& D, int fp32,
                                  const double* q, uint8_t* flags, double* pbar, double* feat, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    if (fp32)
      launch_detect_t<NN, float>(M, b, g, D, q, flags, pbar, feat, s);
    else
      launch_detect_t<NN, double>(M, b, g, D, q, flags, pbar, feat, s);
  });
  return cudaGetLastError();
}

}  // namespace dgk
