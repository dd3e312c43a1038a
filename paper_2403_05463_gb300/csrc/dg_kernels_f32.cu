// dg_kernels_f32.cu -- reduced-precision (FP32 arithmetic) viscous and inviscid passes.
//
// The state and the Runge-Kutta accumulation stay FP64. Every FP64 value is split into an FP32
// pair hi + lo (split_hilo: integer and FP32 instructions only, since GB300 runs FP64 and
// FP64<->FP32 conversions at 1/64 of the FP32 rate), and FP32 only ever sees small
// quantities, so its rounding is relative to those and not to the O(c0^2 |u|) fluxes:
//   * volume: fluxes in deviation form f(q) - f(q_r), q_r = the element's first node, with
//     q - q_r = (hi - hi_r) + (lo - lo_r). sum_m D_im f(q_r) Ja = f(q_r) . sum_d D_d Ja^d = 0
//     by the discrete metric identities, so the deviation form is the same discretisation;
//   * faces: traces are stored as (hi, lo) pairs; the Roe/LLF fluctuation A^-(qbar) (q+ - q-)
//     takes the jump (hi+ - hi-) + (lo+ - lo-);
//   * BR1: the same jumps for u* - u, gradients of u - u_r;
//   * mortar faces (rare): the projected flux minus the own flux in FP64.
// The derivative matrix D is held in FP32 in shared memory; contractions accumulate in FP32.
// The only FP64 arithmetic per node is the RK update g <- A g + dt R, q <- q + B g.
#include "dg_device.cuh"

namespace dgk {

struct Ops1D32 {
  float D[NP][NP * NP];
  float w0inv[NP];  // 1 / w_end
};
__constant__ Ops1D32 c_ops32;
__constant__ double c32_rkA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
__constant__ double c32_rkB[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
__constant__ float c32_rkA32[3] = {0.0f, -5.0f / 9.0f, -153.0f / 128.0f};

__device__ __forceinline__ void jac_apply32(const float ub[3], float un, const float nh[3], float c0sq,
                                            const float x[4], float y[4]) {
  float nx = nh[0] * x[1] + nh[1] * x[2] + nh[2] * x[3];
  y[0] = c0sq * nx;
#pragma unroll
  for (int c = 0; c < 3; ++c) y[1 + c] = nh[c] * x[0] + ub[c] * nx + un * x[1 + c];
}

// A^-(qbar) dq (Roe) or 1/2 (A dq - lambda_max dq) (LLF); dq, ub and the side velocities
// normal components given in FP32.
__device__ __forceinline__ void flux_fluct32(const float dq[4], const float ub[3], const float nh[3], float c0sq,
                                             int riemann, float unm, float unp, float out[4]) {
  float un = ub[0] * nh[0] + ub[1] * nh[1] + ub[2] * nh[2];
  float y1[4];
  jac_apply32(ub, un, nh, c0sq, dq, y1);
  if (riemann == 0) {
    float y2[4];
    jac_apply32(ub, un, nh, c0sq, y1, y2);
    float a = sqrtf(un * un + c0sq);
    float ia = 1.0f / a;
    float aun = fabsf(un);
    float lm = un - a;
    float d1 = (aun + un - a) * ia;
    float d2 = (a - aun) * ia * ia;
    float k0 = -lm - d1 * lm + d2 * lm * un;
    float k1 = d1 - d2 * (lm + un);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.5f * (y1[v] - (k0 * dq[v] + k1 * y1[v] + d2 * y2[v]));
  } else {
    float lam = fmaxf(fabsf(unm) + sqrtf(unm * unm + c0sq), fabsf(unp) + sqrtf(unp * unp + c0sq));
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.5f * (y1[v] - lam * dq[v]);
  }
}

// The same fluctuation for the axis-aligned unit normal n = sg e_d (boxes).
__device__ __forceinline__ float pick3(const float v[3], int d) { return d == 0 ? v[0] : (d == 1 ? v[1] : v[2]); }

__device__ __forceinline__ void flux_fluct32_axis(const float dq[4], const float ub[3], const float um[3], int d,
                                                  float sg, float c0sq, int riemann, float out[4]) {
  // register arrays are only indexed with compile-time indices (pick3 selects)
  const float un = sg * pick3(ub, d);
  const float dqu[3] = {dq[1], dq[2], dq[3]};
  const float nx1 = sg * pick3(dqu, d);
  float y1[4];
  y1[0] = c0sq * nx1;
#pragma unroll
  for (int c = 0; c < 3; ++c) y1[1 + c] = ub[c] * nx1 + un * dq[1 + c] + (c == d ? sg * dq[0] : 0.f);
  if (riemann == 0) {
    const float y1u[3] = {y1[1], y1[2], y1[3]};
    const float nx2 = sg * pick3(y1u, d);
    float y2[4];
    y2[0] = c0sq * nx2;
#pragma unroll
    for (int c = 0; c < 3; ++c) y2[1 + c] = ub[c] * nx2 + un * y1[1 + c] + (c == d ? sg * y1[0] : 0.f);
    const float a = sqrtf(un * un + c0sq);
    const float ia = 1.0f / a;
    const float aun = fabsf(un);
    const float lm = un - a;
    const float d1 = (aun + un - a) * ia;
    const float d2 = (a - aun) * ia * ia;
    const float k0 = -lm - d1 * lm + d2 * lm * un;
    const float k1 = d1 - d2 * (lm + un);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.5f * (y1[v] - (k0 * dq[v] + k1 * y1[v] + d2 * y2[v]));
  } else {
    const float unm = sg * pick3(um, d), unp = unm + nx1;
    const float lam = fmaxf(fabsf(unm) + sqrtf(unm * unm + c0sq), fabsf(unp) + sqrtf(unp * unp + c0sq));
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.5f * (y1[v] - lam * dq[v]);
  }
}

__device__ __forceinline__ float eddy_visc32(const float G[3][3], float delta, int closure, float cs, float cv) {
  if (closure == 0) {
    float s2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float s = 0.5f * (G[c][k] + G[k][c]);
        s2 += s * s;
      }
    float l = cs * delta;
    return l * l * sqrtf(2.f * s2);
  }
  float aa = 0.f, b[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      aa += G[j][i] * G[j][i];
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < 3; ++m) s += G[i][m] * G[j][m];
      b[i][j] = delta * delta * s;
    }
  float B = b[0][0] * b[1][1] - b[0][1] * b[0][1] + b[0][0] * b[2][2] - b[0][2] * b[0][2] + b[1][1] * b[2][2] -
            b[1][2] * b[1][2];
  if (aa < 1e-30f || B <= 0.f) return 0.f;
  return cv * sqrtf(B / aa);
}

__device__ __forceinline__ float2 tq2(const DevMesh& M, int64_t i) {
  return reinterpret_cast<const float2*>(M.Tq)[i];
}

// FP32 geometry of element e at node p (affine: element constants; curved: per node)
template <bool CURVED>
__device__ __forceinline__ void metric32(const DevMesh& M, int e, int64_t node, float Ja[9], float& invJ) {
  if (CURVED) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Ja[k] = __ldg(&M.geo32[k * M.total + node]);
    invJ = __ldg(&M.geo32[9 * M.total + node]);
  } else {
    const ElemConst32& c = M.ec32[e];
#pragma unroll
    for (int k = 0; k < 9; ++k) Ja[k] = c.Ja[k];
    invJ = c.invJ;
  }
}

// ---------------------------------------------------------------------------------------
// traces as (hi, lo) FP32 pairs
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void k_traces32(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ q) {
  constexpr int n = N + 1, n2 = n * n, per = 6 * n2;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)count * per) return;
  const int le = (int)(gid / per), r = (int)(gid % per);
  const int f = r / n2, ab = r % n2;
  const int e = list[le];
  const int64_t src = M.elem_off[e] + face_node(f, n, ab % n, ab / n);
  const int64_t dst = M.tr_off[e] + f * n2 + ab;
  float2* T = reinterpret_cast<float2*>(M.Tq);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float2 t;
    split_hilo(__ldg(&q[v * M.total + src]), t.x, t.y);
    T[v * M.tr_total + dst] = t;
  }
}

// Minimum resident blocks per SM for the register cap (four 256-thread blocks: 64 registers).
template <int N>
struct MinBlocks32 {
  static constexpr int value = Shape<N>::threads <= 256 ? 4 : (Shape<N>::threads <= 352 ? 2 : 1);
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// hi part of x (x truncated to 24 significant bits), integer operations only; 0 for |x| < 2^-126
__device__ __forceinline__ float hi_part(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e < 897 || e > 1150) return 0.f;
  return __uint_as_float(((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                         (unsigned)((b >> 29) & 0x7fffffu));
}

// ---------------------------------------------------------------------------------------
// viscous pass, FP32 arithmetic
// ---------------------------------------------------------------------------------------
// shared-memory layout of k_viscous32 (floats), per element of the block:
//   U [3 n3] velocity deviations | JA [9 n3] metric (curved only) | F [9 n3] viscous fluxes |
//   NU [6][3][n2] neighbours' velocity traces (hi, lo) | EC [16] constants + reference velocity
template <int N, int GEO>
struct ViscSmem32 {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = Shape<N>::EPB;
  static constexpr int oU = 0, oJA = 3 * n3, oF = oJA + (GEO == 2 ? 9 * n3 : 0);
  static constexpr int oNU = ((oF + 9 * n3) + 1) / 2 * 2;  // float2-aligned
  static constexpr int oEC = oNU + 36 * n2, per_elem = oEC + 16;
  static constexpr size_t bytes = sizeof(float) * (NP * NP + EPB * per_elem) + sizeof(FaceLink) * EPB * 6;
};

template <int N, int GEO>
__global__ void __launch_bounds__(Shape<N>::threads, MinBlocks32<N>::value)
    k_viscous32(DevMesh M, const int32_t* __restrict__ list, int count, const double* __restrict__ q) {
  using S = Shape<N>;
  using LV = ViscSmem32<N, GEO>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB, PE = LV::per_elem;
  extern __shared__ float smf[];
  float* sD = smf;
  float* sE = sD + NP * NP;
  FaceLink* sL = reinterpret_cast<FaceLink*>(sE + EPB * PE);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ebase = blockIdx.x * EPB;
  float* Tvf = reinterpret_cast<float*>(M.Tv);
  float* rvf = reinterpret_cast<float*>(M.rv);
  const float2* Tq2 = reinterpret_cast<const float2*>(M.Tq);
  for (int t = tid; t < n2; t += nthr) sD[t] = c_ops32.D[N][t];
  // stage the neighbours' velocity traces of every conforming face asynchronously
  for (int t = tid; t < EPB * 6 * n2; t += nthr) {
    const int le2 = t / (6 * n2), r = t % (6 * n2), f = r / n2, ab = r % n2;
    if (ebase + le2 >= count) continue;
    const FaceLink L = M.link[list[ebase + le2] * 6 + f];
    if (ab == 0) sL[le2 * 6 + f] = L;
    if (L.kind != FK_CONF) continue;
    const int64_t src = L.nslot + ab;
    float2* nu = reinterpret_cast<float2*>(sE + le2 * PE + LV::oNU);
#pragma unroll
    for (int c = 0; c < 3; ++c) cp_async8(&nu[(f * 3 + c) * n2 + ab], &Tq2[(1 + c) * M.tr_total + src]);
  }
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = ebase + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  float* base = sE + le * PE;
  float* U = base + LV::oU;
  float* JA = base + LV::oJA;
  float* F = base + LV::oF;
  float Ja[9], invJ = 0.f, delta = 0.f;
  float uh[3] = {0.f, 0.f, 0.f}, ul[3] = {0.f, 0.f, 0.f};
  if (active) {
    const ElemConst32& ec = M.ec32[e];
    delta = ec.delta;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      split_hilo(__ldg(&q[(1 + c) * M.total + off + p]), uh[c], ul[c]);
      const float ur = hi_part(__ldg(&q[(1 + c) * M.total + off]));  // reference velocity
      U[c * n3 + p] = (uh[c] - ur) + ul[c];
    }
    if (GEO == 2) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        Ja[k] = __ldg(&M.geo32[k * M.total + off + p]);
        JA[k * n3 + p] = Ja[k];
      }
      invJ = __ldg(&M.geo32[9 * M.total + off + p]);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = ec.Ja[k];
      invJ = ec.invJ;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const int str[3] = {1, n, n2};
  if (active) {
    float G[3][3];
    if (GEO != 2) {
      float du[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int bs = p - ii[d] * str[d];
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const float dm = sD[ii[d] * n + m];
          const int pm = bs + m * str[d];
          s0 += dm * U[pm];
          s1 += dm * U[n3 + pm];
          s2 += dm * U[2 * n3 + pm];
        }
        du[0][d] = s0;
        du[1][d] = s1;
        du[2][d] = s2;
      }
      if (GEO == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] = Ja[k * 4] * du[c][k];
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] = Ja[k] * du[c][0] + Ja[3 + k] * du[c][1] + Ja[6 + k] * du[c][2];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[c][k] = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int bs = p - ii[d] * str[d];
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const float dm = sD[ii[d] * n + m];
          const int pm = bs + m * str[d];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float dj = dm * JA[(d * 3 + k) * n3 + pm];
#pragma unroll
            for (int c = 0; c < 3; ++c) G[c][k] += dj * U[c * n3 + pm];
          }
        }
      }
    }
    // BR1 lifting on the faces of this node: (1/w_end) (u* - u) S
    const float invw = c_ops32.w0inv[N];
    const float2* NU = reinterpret_cast<const float2*>(base + LV::oNU);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
      const float sg = side ? 1.f : -1.f;
      const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
      const FaceLink L = sL[le * 6 + f];
      const float Sv[3] = {sg * Ja[d * 3], sg * Ja[d * 3 + 1], sg * Ja[d * 3 + 2]};
      if (L.kind == FK_MORTAR) {
        const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
        double Sd[3];
        if (GEO == 2) {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sd[k] = sg * M.geo[(d * 3 + k) * M.total + off + p];
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sd[k] = sg * M.ec[e].Ja[d * 3 + k];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double uc = q[(1 + c) * M.total + off + p];
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += invw * (float)(M.LU[(c * 3 + k) * M.tr_total + ms] - uc * Sd[k]);
        }
      } else {
        float jump[3] = {0.f, 0.f, 0.f};
        if (L.kind == FK_CONF) {
          int a1, b1;
          inv_orient(L.orient, N, a, b, a1, b1);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 t = NU[(f * 3 + c) * n2 + a1 + n * b1];
            jump[c] = (t.x - uh[c]) + (t.y - ul[c]);
          }
        } else if (L.kind == FK_INFLOW) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float ih, il;
            split_hilo(M.inflow[1 + c], ih, il);
            jump[c] = (ih - uh[c]) + (il - ul[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] += invw * 0.5f * jump[c] * Sv[k];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[c][k] *= invJ;
    const float mu = M.nu32 + eddy_visc32(G, delta, M.closure, M.cs32, M.cv32);
    const float tr = G[0][0] + G[1][1] + G[2][2];
    float tau[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) tau[c][k] = mu * (G[c][k] + G[k][c]) - (c == k ? (2.f / 3.f) * mu * tr : 0.f);
    float Fv[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Fv[d][c] = GEO == 0 ? Ja[d * 4] * tau[c][d]
                            : Ja[d * 3] * tau[c][0] + Ja[d * 3 + 1] * tau[c][1] + Ja[d * 3 + 2] * tau[c][2];
        F[(d * 3 + c) * n3 + p] = Fv[d][c];
      }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
      const float sg = side ? 1.f : -1.f;
      const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
      const int64_t ms = M.tr_off[e] + f * n2 + a + n * b;
#pragma unroll
      for (int c = 0; c < 3; ++c) Tvf[c * M.tr_total + ms] = sg * Fv[d][c];
    }
  }
  __syncthreads();
  if (active) {
    float V[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int bs = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const float dm = sD[ii[d] * n + m];
        const int pm = bs + m * str[d];
#pragma unroll
        for (int c = 0; c < 3; ++c) V[c] += dm * F[(d * 3 + c) * n3 + pm];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) rvf[c * M.total + off + p] = V[c];
  }
}

// shared-memory layout of k_inviscid32 (floats), per element of the block:
//   F  [3][n3] float4   contravariant flux deviations (4 variables packed); after the
//                       contraction: face terms [6][n2] float4
//   Q  [2][n3] float4   hi, lo of q; after the face phase: hi, lo of the updated q
//   NT [48 n2]  neighbours' q traces (hi, lo)[6][4][n2] (neighbour face coordinates)
//   NV [18 n2]  neighbours' viscous traces [6][3][n2];  OV [18 n2] own viscous traces
//   EC [16]     element constants (Ja, 1/J, delta, kind)
//   QD [4 n3]   the exact FP64 state (doubles) for the update
// then the block's face links.
template <int N>
struct InvSmem32 {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = Shape<N>::EPB;
  static constexpr int oF = 0, oQ = 12 * n3, oNT = oQ + 8 * n3, oNV = oNT + 48 * n2, oOV = oNV + 18 * n2,
                       oEC = oOV + 18 * n2, oQD = oEC + 16, per_elem = oQD + 8 * n3;
  static constexpr size_t bytes = sizeof(float) * (NP * NP + EPB * per_elem) + sizeof(FaceLink) * EPB * 6;
};

// Geometry kinds of a bucket: 0 axis-aligned box (diagonal constant metric), 1 affine
// (constant metric), 2 curved (metric per node).
template <int N, int GEO, int MODE>
__global__ void __launch_bounds__(Shape<N>::threads, MinBlocks32<N>::value)
    k_inviscid32(DevMesh M, const int32_t* __restrict__ list, int count, const double* qin, double* out, double* g,
                 int stage, int write_tr) {
  using S = Shape<N>;
  using L32 = InvSmem32<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB, PE = L32::per_elem;
  extern __shared__ float smf[];
  float* sD = smf;
  float* sE = sD + NP * NP;
  FaceLink* sL = reinterpret_cast<FaceLink*>(sE + EPB * PE);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ebase = blockIdx.x * EPB;
  const float* Tvf = reinterpret_cast<const float*>(M.Tv);
  const float* rvf = reinterpret_cast<const float*>(M.rv);
  float* g32 = reinterpret_cast<float*>(g);
  const float2* Tq2 = reinterpret_cast<const float2*>(M.Tq);
  const float c0sq = M.c0sq32;
  const float invw = c_ops32.w0inv[N];
  for (int t = tid; t < n2; t += nthr) sD[t] = c_ops32.D[N][t];
  // stage the neighbours' traces (and the viscous traces) of every conforming face
  for (int t = tid; t < EPB * 6 * n2; t += nthr) {
    const int le2 = t / (6 * n2), r = t % (6 * n2), f = r / n2, ab = r % n2;
    if (ebase + le2 >= count) continue;
    const int e2 = list[ebase + le2];
    const FaceLink L = M.link[e2 * 6 + f];
    if (ab == 0) sL[le2 * 6 + f] = L;
    float* base = sE + le2 * PE;
    if (L.kind == FK_CONF) {
      const int64_t src = L.nslot + ab;
      float2* nt = reinterpret_cast<float2*>(base + L32::oNT);
#pragma unroll
      for (int v = 0; v < 4; ++v) cp_async8(&nt[(f * 4 + v) * n2 + ab], &Tq2[v * M.tr_total + src]);
      if (L.nflag) {
#pragma unroll
        for (int c = 0; c < 3; ++c) cp_async4(&base[L32::oNV + (f * 3 + c) * n2 + ab], &Tvf[c * M.tr_total + src]);
      }
    }
    if (M.flag[e2]) {
      const int64_t own = M.tr_off[e2] + f * n2 + ab;
#pragma unroll
      for (int c = 0; c < 3; ++c) cp_async4(&base[L32::oOV + (f * 3 + c) * n2 + ab], &Tvf[c * M.tr_total + own]);
    }
  }
  // ---- node phase: state, flux deviations --------------------------------------------
  int le = tid / n3;
  const int p = tid % n3;
  const int slot = ebase + le;
  const bool active = (le < EPB) && (slot < count);
  if (le >= EPB) le = EPB - 1;
  const int e = active ? list[slot] : 0;
  const int64_t off = active ? M.elem_off[e] : 0;
  const bool ns = active && M.flag[e] != 0;
  float* base = sE + le * PE;
  float* F = base + L32::oF;
  float4* F4 = reinterpret_cast<float4*>(F);
  float4* QH4 = reinterpret_cast<float4*>(base + L32::oQ);
  float4* QL4 = QH4 + n3;
  float* EC = base + L32::oEC;
  double* QD = reinterpret_cast<double*>(base + L32::oQD);
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  float invJ = 0.f;
  float gold[4] = {0.f, 0.f, 0.f, 0.f}, rvp[3] = {0.f, 0.f, 0.f};
  if (active) {
    if (MODE == MODE_RK && stage > 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) gold[v] = g32[v * M.total + off + p];
    }
    if (ns) {
#pragma unroll
      for (int c = 0; c < 3; ++c) rvp[c] = rvf[c * M.total + off + p];
    }
    const ElemConst32& ec = M.ec32[e];
    for (int k = p; k < 12; k += n3) EC[k] = k < 9 ? ec.Ja[k] : (k == 9 ? ec.invJ : (k == 10 ? ec.delta : ec.curved));
    float dq[4], qr32[4], h[4], l[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double qv = qin[v * M.total + off + p];
      QD[v * n3 + p] = qv;
      split_hilo(qv, h[v], l[v]);
      qr32[v] = hi_part(qin[v * M.total + off]);  // any per-element constant serves as reference
      dq[v] = (h[v] - qr32[v]) + l[v];
    }
    QH4[p] = make_float4(h[0], h[1], h[2], h[3]);
    QL4[p] = make_float4(l[0], l[1], l[2], l[3]);
    float fl[4][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      fl[0][k] = c0sq * dq[1 + k];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        fl[1 + c][k] = qr32[1 + c] * dq[1 + k] + dq[1 + c] * (qr32[1 + k] + dq[1 + k]) + (c == k ? dq[0] : 0.f);
    }
    if (GEO == 0) {
      invJ = ec.invJ;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float j = ec.Ja[d * 4];
        F4[d * n3 + p] = make_float4(j * fl[0][d], j * fl[1][d], j * fl[2][d], j * fl[3][d]);
      }
    } else {
      float Ja[9];
      if (GEO == 2) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Ja[k] = __ldg(&M.geo32[k * M.total + off + p]);
        invJ = __ldg(&M.geo32[9 * M.total + off + p]);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Ja[k] = ec.Ja[k];
        invJ = ec.invJ;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float c4[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) c4[v] = Ja[d * 3] * fl[v][0] + Ja[d * 3 + 1] * fl[v][1] + Ja[d * 3 + 2] * fl[v][2];
        F4[d * n3 + p] = make_float4(c4[0], c4[1], c4[2], c4[3]);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // ---- volume: J R = -sum_d D_d Ftil^d ------------------------------------------------
  float JR[4] = {0.f, 0.f, 0.f, 0.f};
  if (active) {
    const int str[3] = {1, n, n2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int bs = p - ii[d] * str[d];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const float dm = sD[ii[d] * n + m];
        const float4 f4 = F4[d * n3 + bs + m * str[d]];
        JR[0] -= dm * f4.x;
        JR[1] -= dm * f4.y;
        JR[2] -= dm * f4.z;
        JR[3] -= dm * f4.w;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) JR[1 + c] += rvp[c];
  }
  __syncthreads();  // F is reused for the face terms below
  // ---- faces, one thread per (element, face, face node) -------------------------------
  for (int t = tid; t < EPB * 6 * n2; t += nthr) {
    const int le2 = t / (6 * n2), r = t % (6 * n2), f = r / n2, ab = r % n2;
    if (ebase + le2 >= count) continue;
    const int e2 = list[ebase + le2];
    const FaceLink L = sL[le2 * 6 + f];
    float* b2 = sE + le2 * PE;
    const float* E2 = b2 + L32::oEC;
    const int d = f >> 1;
    const float sg = (f & 1) ? 1.f : -1.f;
    const int a = ab % n, bb = ab / n;
    const int pv = face_node(f, n, a, bb);
    const bool ns2 = M.flag[e2] != 0;
    float term[4];
    if (L.kind == FK_MORTAR) {
      const int64_t node = M.elem_off[e2] + pv;
      const int64_t ms = M.tr_off[e2] + f * n2 + ab;
      double Sd[3], qq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) qq[v] = qin[v * M.total + node];
      if (GEO == 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) Sd[k] = sg * M.geo[(d * 3 + k) * M.total + node];
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) Sd[k] = sg * M.ec[e2].Ja[d * 3 + k];
      }
      const double un = qq[1] * Sd[0] + qq[2] * Sd[1] + qq[3] * Sd[2];
      term[0] = (float)(M.LH[ms] - M.c0sq * un);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double own = qq[1 + c] * un + qq[0] * Sd[c];
        term[1 + c] = (float)(M.LH[(1 + c) * M.tr_total + ms] - own) + (ns2 ? b2[L32::oOV + (f * 3 + c) * n2 + ab] : 0.f);
      }
    } else {
      float Sv[3];
      if (GEO == 2) {
        const int64_t node = M.elem_off[e2] + pv;
#pragma unroll
        for (int k = 0; k < 3; ++k) Sv[k] = sg * __ldg(&M.geo32[(d * 3 + k) * M.total + node]);
      } else if (GEO == 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) Sv[k] = sg * E2[d * 3 + k];
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) Sv[k] = (k == d) ? sg * E2[d * 4] : 0.f;
      }
      const float s = GEO == 0 ? fabsf(E2[d * 4]) : sqrtf(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
      const float is = 1.f / s;
      const float nh[3] = {Sv[0] * is, Sv[1] * is, Sv[2] * is};
      const float4 h4 = reinterpret_cast<const float4*>(b2 + L32::oQ)[pv];
      const float4 l4 = reinterpret_cast<const float4*>(b2 + L32::oQ)[n3 + pv];
      const float qh[4] = {h4.x, h4.y, h4.z, h4.w}, ql[4] = {l4.x, l4.y, l4.z, l4.w};
      float dqf[4];
      int nab = 0;
      if (L.kind == FK_CONF) {
        int a1, b1;
        inv_orient(L.orient, N, a, bb, a1, b1);
        nab = a1 + n * b1;
        const float2* nt = reinterpret_cast<const float2*>(b2 + L32::oNT);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float2 tq = nt[(f * 4 + v) * n2 + nab];
          dqf[v] = (tq.x - qh[v]) + (tq.y - ql[v]);
        }
      } else if (L.kind == FK_INFLOW) {
        dqf[0] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float ih, il;
          split_hilo(M.inflow[1 + c], ih, il);
          dqf[1 + c] = (ih - qh[1 + c]) + (il - ql[1 + c]);
        }
      } else {
        dqf[0] = -(qh[0] + ql[0]);
        dqf[1] = dqf[2] = dqf[3] = 0.f;
      }
      float ub[3], um[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        um[c] = qh[1 + c] + ql[1 + c];
        ub[c] = um[c] + 0.5f * dqf[1 + c];
      }
      float fx[4];
      if (GEO == 0) {
        flux_fluct32_axis(dqf, ub, um, d, sg, c0sq, M.riemann, fx);
      } else {
        const float unm = um[0] * nh[0] + um[1] * nh[1] + um[2] * nh[2];
        const float unp = unm + dqf[1] * nh[0] + dqf[2] * nh[1] + dqf[3] * nh[2];
        flux_fluct32(dqf, ub, nh, c0sq, M.riemann, unm, unp, fx);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) term[v] = s * fx[v];
      if (L.kind == FK_CONF && (ns2 || L.nflag)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float tv = 0.f;
          if (ns2) tv += b2[L32::oOV + (f * 3 + c) * n2 + ab];
          if (L.nflag) tv += b2[L32::oNV + (f * 3 + c) * n2 + nab];
          term[1 + c] += 0.5f * tv;
        }
      }
    }
    reinterpret_cast<float4*>(b2 + L32::oF)[f * n2 + ab] = make_float4(term[0], term[1], term[2], term[3]);
  }
  __syncthreads();
  // ---- assembly and update (node phase) -------------------------------------------------
  const bool on_face = ii[0] == 0 || ii[0] == N || ii[1] == 0 || ii[1] == N || ii[2] == 0 || ii[2] == N;
  if (active) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (ii[d] != 0 && ii[d] != N) continue;
      const int f = 2 * d + (ii[d] == N ? 1 : 0);
      const int a = d == 0 ? ii[1] : ii[0], bb = d == 2 ? ii[1] : ii[2];
      const float4 sc = F4[f * n2 + a + n * bb];
      JR[0] -= invw * sc.x;
      JR[1] -= invw * sc.y;
      JR[2] -= invw * sc.z;
      JR[3] -= invw * sc.w;
    }
    if (MODE == MODE_RESIDUAL) {
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v * M.total + off + p] = (double)(JR[v] * invJ);
    } else {
      // g <- A g + dt R in FP32 (the RK register of this path); q <- q + B g in FP64
      const float A = c32_rkA32[stage];
      const double B = c32_rkB[stage];
      const float dtf = M.dt32;
      float h[4], l[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int64_t ix = v * M.total + off + p;
        const float gi = fmaf(A, gold[v], JR[v] * invJ * dtf);
        g32[ix] = gi;
        const double qn = fma(B, (double)gi, QD[v * n3 + p]);
        out[ix] = qn;
        if (write_tr && on_face) split_hilo(qn, h[v], l[v]);
      }
      if (write_tr && on_face) {
        QH4[p] = make_float4(h[0], h[1], h[2], h[3]);
        QL4[p] = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
  }
  if (MODE == MODE_RK && write_tr) {
    __syncthreads();
    // traces of the new state for the next stage, one thread per face slot (coalesced)
    float2* Tn = reinterpret_cast<float2*>(M.Tq_next);
    for (int t = tid; t < EPB * 6 * n2; t += nthr) {
      const int le2 = t / (6 * n2), r = t % (6 * n2), f = r / n2, ab = r % n2;
      if (ebase + le2 >= count) continue;
      const int e2 = list[ebase + le2];
      const float4* Q2 = reinterpret_cast<const float4*>(sE + le2 * PE + L32::oQ);
      const int pv = face_node(f, n, ab % n, ab / n);
      const int64_t dst = M.tr_off[e2] + f * n2 + ab;
      const float4 h4 = Q2[pv], l4 = Q2[n3 + pv];
      Tn[dst] = make_float2(h4.x, l4.x);
      Tn[M.tr_total + dst] = make_float2(h4.y, l4.y);
      Tn[2 * M.tr_total + dst] = make_float2(h4.z, l4.z);
      Tn[3 * M.tr_total + dst] = make_float2(h4.w, l4.w);
    }
  }
}

// ---------------------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------------------
cudaError_t upload_ops32(const Ops1D& ops) {
  Ops1D32 o{};
  for (int N = 1; N <= MAXN; ++N) {
    for (int i = 0; i < NP * NP; ++i) o.D[N][i] = (float)ops.D[N][i];
    o.w0inv[N] = (float)(1.0 / ops.w[N][0]);
  }
  return cudaMemcpyToSymbol(c_ops32, &o, sizeof o);
}

template <int N, int GEO>
static size_t visc_smem32() {
  return ViscSmem32<N, GEO>::bytes;
}
template <int N>
static size_t inv_smem32() {
  return InvSmem32<N>::bytes;
}

template <int N>
static cudaError_t prep32_n() {
  cudaError_t r;
  if ((r = cudaFuncSetAttribute(k_viscous32<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem32<N, 0>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem32<N, 1>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem32<N, 2>())) != cudaSuccess) return r;
  const int is = (int)inv_smem32<N>();
  if ((r = cudaFuncSetAttribute(k_inviscid32<N, 0, MODE_RESIDUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32<N, 1, MODE_RESIDUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32<N, 2, MODE_RESIDUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32<N, 0, MODE_RK>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32<N, 1, MODE_RK>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32<N, 2, MODE_RK>, cudaFuncAttributeMaxDynamicSharedMemorySize, is)) != cudaSuccess) return r;
  return cudaSuccess;
}

cudaError_t prepare_kernels32() {
  cudaError_t r;
  if ((r = prep32_n<1>()) != cudaSuccess) return r;
  if ((r = prep32_n<2>()) != cudaSuccess) return r;
  if ((r = prep32_n<3>()) != cudaSuccess) return r;
  if ((r = prep32_n<4>()) != cudaSuccess) return r;
  if ((r = prep32_n<5>()) != cudaSuccess) return r;
  if ((r = prep32_n<6>()) != cudaSuccess) return r;
  if ((r = prep32_n<7>()) != cudaSuccess) return r;
  return cudaSuccess;
}

#define DG32_DISPATCH_N(NVAR, ...)                         \
  switch (NVAR) {                                          \
    case 1: { constexpr int NN = 1; __VA_ARGS__; } break;  \
    case 2: { constexpr int NN = 2; __VA_ARGS__; } break;  \
    case 3: { constexpr int NN = 3; __VA_ARGS__; } break;  \
    case 4: { constexpr int NN = 4; __VA_ARGS__; } break;  \
    case 5: { constexpr int NN = 5; __VA_ARGS__; } break;  \
    case 6: { constexpr int NN = 6; __VA_ARGS__; } break;  \
    case 7: { constexpr int NN = 7; __VA_ARGS__; } break;  \
    default: return cudaErrorInvalidValue;                 \
  }

cudaError_t launch_traces32(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG32_DISPATCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * 6 * (NN + 1) * (NN + 1);
    k_traces32<NN><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

cudaError_t launch_viscous32(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG32_DISPATCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    if (b.geo == 0)
      k_viscous32<NN, 0><<<grid, SH::threads, visc_smem32<NN, 0>(), s>>>(M, b.list, b.count, q);
    else if (b.geo == 1)
      k_viscous32<NN, 1><<<grid, SH::threads, visc_smem32<NN, 1>(), s>>>(M, b.list, b.count, q);
    else
      k_viscous32<NN, 2><<<grid, SH::threads, visc_smem32<NN, 2>(), s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

cudaError_t launch_inviscid32(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g, int mode,
                              int stage, int write_tr, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG32_DISPATCH_N(b.N, {
    using SH = Shape<NN>;
    const unsigned grid = (unsigned)((b.count + SH::EPB - 1) / SH::EPB);
    const size_t sm = inv_smem32<NN>();
    const int geo = b.geo;
    if (mode == MODE_RESIDUAL) {
      if (geo == 0)
        k_inviscid32<NN, 0, MODE_RESIDUAL><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, q, out, g, stage, write_tr);
      else if (geo == 1)
        k_inviscid32<NN, 1, MODE_RESIDUAL><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, q, out, g, stage, write_tr);
      else
        k_inviscid32<NN, 2, MODE_RESIDUAL><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, q, out, g, stage, write_tr);
    } else {
      if (geo == 0)
        k_inviscid32<NN, 0, MODE_RK><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, q, out, g, stage, write_tr);
      else if (geo == 1)
        k_inviscid32<NN, 1, MODE_RK><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, q, out, g, stage, write_tr);
      else
        k_inviscid32<NN, 2, MODE_RK><<<grid, SH::threads, sm, s>>>(M, b.list, b.count, q, out, g, stage, write_tr);
    }
  });
  return cudaGetLastError();
}

}  // namespace dgk
