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
#include <climits>

#include "dg_device.cuh"

namespace dgk {

struct Ops1D32 {
  float D[NP][NP * NP];
  float w0inv[NP];  // 1 / w_end
};
__constant__ Ops1D32 c_ops32;
// FP64 D[N][i*n+m] for the FP64 divergence of the box-element inviscid pass (read through L1:
// the lanes of a warp read up to n different rows, which constant memory would serialise)
__device__ double g_D64[NP][NP * NP];
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
    const float ia = rsqrtf(un * un + c0sq);  // 1/a, a^2 = un^2 + c0^2 >= c0^2 > 0
    const float a = (un * un + c0sq) * ia;
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
    const float ia = rsqrtf(un * un + c0sq);
    const float a = (un * un + c0sq) * ia;
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
// traces as (hi, lo) FP32 pairs, one 32-byte record (p, u, v, w) per face node
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
  float h[4], l[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) split_hilo(__ldg(&q[v * M.total + src]), h[v], l[v]);
  float4* T = reinterpret_cast<float4*>(M.Tq) + 2 * dst;
  T[0] = make_float4(h[0], l[0], h[1], l[1]);
  T[1] = make_float4(h[2], l[2], h[3], l[3]);
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
    for (int c = 0; c < 3; ++c) cp_async8(&nu[(f * 3 + c) * n2 + ab], &Tq2[src * 4 + 1 + c]);
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
        } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {
          const float uo[3] = {uh[0] + ul[0], uh[1] + ul[1], uh[2] + ul[2]};
          wall_jump<float>(L.kind, uo, Sv, jump);
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
      for (int c = 0; c < 3; ++c) Tvf[ms * 3 + c] = sg * Fv[d][c];
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

// ---------------------------------------------------------------------------------------
// inviscid pass, persistent, TMA-staged
// ---------------------------------------------------------------------------------------
// Each block loops over tiles of EPB elements. While its consumer warps compute tile i from one
// shared input buffer, the producer warp fetches tile i+1 into the other buffer with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier): per element the four planes
// of its FP64 state, every conforming face's neighbour traces (one 32-byte record per face
// node), the neighbours' and its own viscous traces (12 bytes per face node) and its
// constants — at most 18 copies instead of ~2000 thread-level copies. A bulk copy needs
// 16-byte-aligned ends, so each copy covers the 16-byte-aligned superset of its range and the
// offset of the first wanted byte is kept in a small table. Per element (bytes):
//   QD [4] slots of a16(8 n3 + 8) | NT [6] slots of a16(32 n2 + 16) |
//   NV [6] slots of a16(12 n2 + 16) | OV a16(72 n2 + 16) | LK 96 | EC 48 |
//   MT 32 (EntryMeta) | SH 32 (byte offsets of the slots' first wanted byte)
// Tile shape of the pipelined passes: E elements per tile, one consumer thread per node
// (rounded up to whole warps). The default E packs about 256 nodes; the alternative halves it
// (orders 1..4) or doubles it (orders 5, 6); the autotuner picks per (order, geometry).
template <int N, int E>
struct Tile {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = E;
  static constexpr int threads = ((E * n3 + 31) / 32) * 32;
};
template <int N>
struct AltEPB {
  static constexpr int value = N <= 4 ? Shape<N>::EPB / 2 : (N <= 6 ? 2 : Shape<N>::EPB);
};

// LAST0: buffer 0 after the work area (the one-launch stage kernel with tile queues stages its
// first inviscid tile there while the viscous phase still uses the space before it)
template <int N, int E = Shape<N>::EPB, bool KEPC = false, bool TCX = false, bool LAST0 = false>
struct TmaSmem32 {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = E;
  static constexpr int a16(int x) { return (x + 15) / 16 * 16; }
  // QD: q is 8-byte aligned, so its copies start at most 8 bytes early
  static constexpr int SQD = a16(8 * n3 + 8), SNT = a16(32 * n2 + 16), SNV = a16(12 * n2 + 16),
                       SOV = a16(72 * n2 + 16);
  static constexpr int iQD = 0, iNT = 4 * SQD, iNV = iNT + 6 * SNT, iOV = iNV + 6 * SNV, iLK = iOV + SOV,
                       iEC = iLK + 96, iMT = iEC + 48, iSH = iMT + 32, in_elem = a16(iSH + 32);
  static constexpr int ITEMS = 18;  // copies per element: 4 QD, 6 NT, 6 NV, OV, EC
  // work per element: F [3 n3] flux deviations, QH/QL [n3] hi/lo state, T [6 n2] face terms
  // (split form on curved elements: F holds the state deviations and the three metric vectors,
  // 4 n3 float4, so everything after it moves by 16 n3)
  // (tensor-core contraction: each item writes its D contraction over the flux rows it read, so
  // F holds the three directions' results afterwards and no extra tile is needed)
  static constexpr int FB = KEPC ? 64 * n3 : 48 * n3;
  static constexpr int wF = 0, wQ = FB, wT = FB + 32 * n3, work_elem = FB + 32 * n3 + 96 * n2;
  static constexpr int oBAR = 0, oD = 128;
  static constexpr int oIN0 = LAST0 ? 384 + EPB * (in_elem + work_elem) : 384;
  static constexpr int oIN1 = LAST0 ? 384 : oIN0 + EPB * in_elem;
  static constexpr int oW = oIN1 + EPB * in_elem;
  static constexpr size_t bytes = (size_t)384 + (size_t)EPB * (2 * in_elem + work_elem);
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// global load whose issue point the compiler keeps (used to prefetch values needed much later)
__device__ __forceinline__ float ld_early(const float* p) {
  float v;
  asm volatile("ld.global.f32 %0, [%1];\n" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void mbar_init(void* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(void* bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(void* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, void* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One bulk copy of a tile element, item k (see TmaSmem32), described from the element's record
// and links already in shared memory: returns false if the item does not apply. src/len give
// the wanted bytes, slot the element-relative destination, sh_index the shift-table entry.
template <int N>
__device__ __forceinline__ bool tma_item(const DevMesh& M, const double* qin, const EntryMeta& mt,
                                         const FaceLink* lk, int k, const char*& src, int& len, int& slot,
                                         int& sh_index) {
  using P = TmaSmem32<N>;
  constexpr int n2 = P::n2, n3 = P::n3;
  if (k < 4) {
    src = reinterpret_cast<const char*>(qin + (int64_t)k * M.total + mt.off);
    len = 8 * n3;
    slot = P::iQD + k * P::SQD;
    sh_index = k;
    return true;
  }
  if (k < 10) {
    const FaceLink& L = lk[k - 4];
    if (L.kind != FK_CONF) return false;
    src = reinterpret_cast<const char*>(M.Tq + L.nslot * 4);  // 4 (hi, lo) pairs = 4 doubles
    len = 32 * n2;
    slot = P::iNT + (k - 4) * P::SNT;
    sh_index = k;
    return true;
  }
  if (k < 16) {
    const FaceLink& L = lk[k - 10];
    if (L.kind != FK_CONF || !L.nflag) return false;
    src = reinterpret_cast<const char*>(reinterpret_cast<const float*>(M.Tv) + L.nslot * 3);
    len = 12 * n2;
    slot = P::iNV + (k - 10) * P::SNV;
    sh_index = k;
    return true;
  }
  if (k == 16) {
    if (!mt.flag) return false;
    src = reinterpret_cast<const char*>(reinterpret_cast<const float*>(M.Tv) + mt.troff * 3);
    len = 72 * n2;
    slot = P::iOV;
    sh_index = k;
    return true;
  }
  src = reinterpret_cast<const char*>(&M.ec32[mt.elem]);
  len = 48;
  slot = P::iEC;
  sh_index = -1;
  return true;
}

// Shared-memory layout of the pipelined viscous pass (box and affine elements), per element
// (bytes): QV [3] slots of a16(8 n3 + 16) (velocity planes) | NT [6] slots of a16(32 n2 + 16)
// (neighbours' trace records) | LK 96 | EC 48 | MT 32 | SH 32; work: U [3 n3] velocity
// deviations and F [9 n3] contravariant viscous fluxes (floats).
template <int N, int E = Shape<N>::EPB>
struct ViscTmaSmem32 {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n, EPB = E;
  static constexpr int a16(int x) { return (x + 15) / 16 * 16; }
  static constexpr int SQV = a16(8 * n3 + 16), SNT = a16(32 * n2 + 16);
  static constexpr int iQV = 0, iNT = 3 * SQV, iLK = iNT + 6 * SNT, iEC = iLK + 96, iMT = iEC + 48,
                       iSH = iMT + 32, in_elem = a16(iSH + 32);
  static constexpr int ITEMS = 10;  // copies per element: 3 QV, 6 NT, EC
  // work area per element: U (3 x n3 FP32), F (9 x n3 FP32); the velocity's (hi, lo) pairs
  // overwrite its staged FP64 values in the input buffer (each node's own slot)
  static constexpr int wU = 0, wF = 12 * n3, work_elem = a16(48 * n3);
  static constexpr int oBAR = 0, oD = 128, oIN0 = 384, oIN1 = oIN0 + EPB * in_elem, oW = oIN1 + EPB * in_elem;
  static constexpr size_t bytes = (size_t)oW + (size_t)EPB * work_elem;
};

template <int N>
__device__ __forceinline__ bool vtma_item(const DevMesh& M, const double* q, const EntryMeta& mt, const FaceLink* lk,
                                          int k, const char*& src, int& len, int& slot, int& sh_index) {
  using P = ViscTmaSmem32<N>;
  if (k < 3) {
    src = reinterpret_cast<const char*>(q + (int64_t)(1 + k) * M.total + mt.off);
    len = 8 * P::n3;
    slot = P::iQV + k * P::SQV;
    sh_index = k;
    return true;
  }
  if (k < 9) {
    const FaceLink& L = lk[k - 3];
    if (L.kind != FK_CONF) return false;
    src = reinterpret_cast<const char*>(M.Tq + L.nslot * 4);
    len = 32 * P::n2;
    slot = P::iNT + (k - 3) * P::SNT;
    sh_index = k;
    return true;
  }
  src = reinterpret_cast<const char*>(&M.ec32[mt.elem]);
  len = 48;
  slot = P::iEC;
  sh_index = -1;
  return true;
}

// TF32 (tensor-core input) split of an FP32 value with integer instructions (conversions to
// TF32 run on a slow pipe): big = x rounded to 10 mantissa bits (half away from zero, by adding
// half a TF32 unit to the bit pattern and clearing the 13 low bits), small = x - big (exact in
// FP32) truncated to TF32, so big + small = x to 2^-21 relative.
__device__ __forceinline__ void tf32_split(float x, unsigned& big, unsigned& small) {
  big = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  small = __float_as_uint(x - __uint_as_float(big)) & 0xffffe000u;
}

// D += A B for one 16x8x8 TF32 tile (A row-major 16x8, B column-major 8x8, FP32 accumulators);
// fragment ownership as the PTX ISA defines it for m16n8k8 with .tf32 operands.
__device__ __forceinline__ void mma_tf32(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The records of one tile, held in the producer warp's registers between the time they are
// loaded and the time the tile's input buffer is free: record r = lane + 32 j of the tile's
// EPB x 7 records (k = r % 7 = 0: the element's 32-byte EntryMeta, 1..6: its face links).
template <int E>
struct TileRecs {
  static constexpr int R = (E * 7 + 31) / 32;
  uint4 a[R], b[R];
};

template <int E>
__device__ __forceinline__ void load_recs(const Bucket& B, int tile, TileRecs<E>& T) {
  constexpr int EPB = E;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < TileRecs<E>::R; ++j) {
    const int r = lane + 32 * j, le = r / 7, k = r % 7, i = tile * EPB + le;
    if (r < EPB * 7 && i < B.count) {
      if (k == 0) {
        const uint4* m = reinterpret_cast<const uint4*>(&B.bmeta[i]);
        T.a[j] = m[0];
        T.b[j] = m[1];
      } else {
        T.a[j] = *reinterpret_cast<const uint4*>(&B.blink[(int64_t)i * 6 + (k - 1)]);
      }
    }
  }
}

template <class P>
__device__ __forceinline__ void store_recs(const Bucket& B, int tile, const TileRecs<P::EPB>& T, char* IN) {
  constexpr int EPB = P::EPB;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < TileRecs<EPB>::R; ++j) {
    const int r = lane + 32 * j, le = r / 7, k = r % 7, i = tile * EPB + le;
    if (r < EPB * 7 && i < B.count) {
      char* base = IN + le * P::in_elem;
      if (k == 0) {
        reinterpret_cast<uint4*>(base + P::iMT)[0] = T.a[j];
        reinterpret_cast<uint4*>(base + P::iMT)[1] = T.b[j];
      } else {
        reinterpret_cast<uint4*>(base + P::iLK)[k - 1] = T.a[j];
      }
    }
  }
}

// The producer warp fills buffer IN with tile `tile`, completion on `bar` (32 arrivals), from
// the records already in the buffer's MT/LK slots: the copy plan, the shift table and the
// expected byte count, then the bulk copies. P is the shared-memory layout, VISC selects the
// viscous pass's copies (velocity planes, neighbour trace records, constants).
template <int N, class P, bool VISC>
__device__ __forceinline__ bool stage_item(const DevMesh& M, const double* qin, const EntryMeta& mt,
                                           const FaceLink* lk, int k, const char*& src, int& len, int& slot,
                                           int& sh) {
  if constexpr (VISC)
    return vtma_item<N>(M, qin, mt, lk, k, src, len, slot, sh);
  else
    return tma_item<N>(M, qin, mt, lk, k, src, len, slot, sh);
}

template <int N, class P, bool VISC>
__device__ __forceinline__ void tma_stage(const DevMesh& M, const Bucket& B, const double* qin, int tile, char* IN,
                                          void* bar) {
  constexpr int EPB = P::EPB;
  const int lane = threadIdx.x & 31;
  unsigned total = 0;
  for (int it = lane; it < EPB * P::ITEMS; it += 32) {
    const int le = it / P::ITEMS, k = it % P::ITEMS;
    if (tile * EPB + le >= B.count) continue;
    char* base = IN + le * P::in_elem;
    const char* src;
    int len, slot, sh;
    if (!stage_item<N, P, VISC>(M, qin, *reinterpret_cast<const EntryMeta*>(base + P::iMT),
                                reinterpret_cast<const FaceLink*>(base + P::iLK), k, src, len, slot, sh))
      continue;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    const uintptr_t s0 = a & ~(uintptr_t)15, e0 = (a + len + 15) & ~(uintptr_t)15;
    total += (unsigned)(e0 - s0);
    if (sh >= 0) reinterpret_cast<unsigned char*>(base + P::iSH)[sh] = (unsigned char)(a - s0);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_arrive_expect_tx(bar, total);
  for (int it = lane; it < EPB * P::ITEMS; it += 32) {
    const int le = it / P::ITEMS, k = it % P::ITEMS;
    if (tile * EPB + le >= B.count) continue;
    char* base = IN + le * P::in_elem;
    const char* src;
    int len, slot, sh;
    if (!stage_item<N, P, VISC>(M, qin, *reinterpret_cast<const EntryMeta*>(base + P::iMT),
                                reinterpret_cast<const FaceLink*>(base + P::iLK), k, src, len, slot, sh))
      continue;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    const uintptr_t s0 = a & ~(uintptr_t)15, e0 = (a + len + 15) & ~(uintptr_t)15;
    bulk_copy_g2s(base + slot, reinterpret_cast<const void*>(s0), (unsigned)(e0 - s0), bar);
  }
}

// Overlapped launches (PTX griddepcontrol, programmatic dependent launch): a kernel launched
// with programmatic stream serialisation may be scheduled before the previous kernel in the
// stream has completed. pdl_wait() blocks the calling thread until that kernel has completed
// and its memory operations are visible; pdl_launch_dependents() allows the next such launch to
// be scheduled once every block of this grid has issued it or exited. In a kernel launched
// without the attribute both return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Launch of a pipelined pass; with M.overlap it carries programmatic stream serialisation, so
// its blocks may be scheduled while the previous kernel in the stream drains (the kernel waits
// for that kernel with griddepcontrol.wait before it touches memory the kernel may write).
template <typename... KArgs, typename... Args>
static cudaError_t launch_overlapped(const DevMesh& M, void (*kern)(KArgs...), int grid, int block, size_t smem,
                                     cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = M.overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Tile queue of a persistent pass (one launch per RK stage): the producer warp claims the next
// tile index from a global counter (lane 0's atomic, broadcast to the warp) and passes it to the
// consumers in shared memory, its last tile flagged with kLastTile (-1: the block got no tile).
constexpr int kLastTile = 1 << 30;
__device__ __forceinline__ int claim_tile(unsigned* counter) {
  unsigned v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(counter, 1u);
  return (int)__shfl_sync(0xffffffffu, v, 0);
}

// bounded wait on an mbarrier phase: false if it did not complete within the limit
__device__ __forceinline__ bool mbar_wait_bounded(void* bar, unsigned parity, int polls) {
  bool ok = false;
  for (int spin = 0; spin < polls && !ok; ++spin) ok = mbar_try_wait(bar, parity);
  return ok;
}
// The producer's wait for a free input buffer (it-th tile, buffer it & 1, empty barrier ebar):
// tiles 0 and 1 find their buffers free. With shift1 (the stage kernel with tile queues) buffer
// 1 overlaps the viscous phase's shared memory, and its empty barrier's first phase is the
// consumers' release of that space, so tile 1 waits for phase 0 and tile it for phase it / 2.
__device__ __forceinline__ bool buffer_free(void* ebar, int it, bool shift1, int polls) {
  if (shift1 && (it & 1)) return mbar_wait_bounded(ebar, (unsigned)((it >> 1) & 1), polls);
  return it < 2 || mbar_wait_bounded(ebar, (unsigned)(((it >> 1) - 1) & 1), polls);
}
__device__ __forceinline__ void mbar_arrive(void* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}
// barrier 1 among the consumer threads only (the producer warp never joins it)
__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}
// OR of `pred` over the consumer threads (barrier 2)
__device__ __forceinline__ bool consumer_any(bool pred, int nthreads) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 2, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(nthreads)
      : "memory");
  return r != 0;
}

template <int N>
struct TmaMinBlocks {
  static constexpr int value = N == 4 ? 3 : (N == 5 ? 4 : (N == 1 || N == 7 ? 1 : 2));
};
// register cap of a tile shape: the default shapes as above; 128-thread tiles 5 blocks, larger
// ones none
template <int N, int E>
struct InvMinBlocks {
  static constexpr int value = E == Shape<N>::EPB ? TmaMinBlocks<N>::value : (Tile<N, E>::threads <= 128 ? 5 : 1);
};

// Warp-specialised: threads [0, Shape<N>::threads) compute (one per node, as elsewhere), the
// last warp only fetches tiles. Input buffer b is handed over through full[b] (the copies'
// bytes) and returned through empty[b] (one arrival per consumer warp).
// KEP: the split form's volume term sum_m 2 D_im F#(q_i, q_m), in deviation form like the
// standard one: F#(q_i, q_m) - F#(q_r, q_r) with the averages {{q}} = q_r + {{dq}} has only terms
// of the size of the deviations, and sum_d sum_m 2 D_im F#(q_r, q_r) = f(q_r) . sum_d (D_d Ja^d)
// vanishes by the discrete metric identities. Shared memory then holds the deviations dq (and,
// on curved elements, the metric vectors Ja^d) instead of the contravariant fluxes.
//
// VOL = 2: the standard volume term with the D contractions on the tensor cores in 3xTF32.
// Along direction d, C[(line, v), i] = sum_m F[(line, v), m] D[i][m] is a 16x8x8 TF32 tile
// product per 16 (line, variable) rows (m and i padded from n to 8 with zeros); each FP32
// operand is split into big + small TF32 parts and C accumulates big*big + big*small +
// small*big in FP32. Consumer warps take the (element, direction, row tile) items in turn and
// store C per direction; after the face phase each node sums its three directions.
// dep_tile: tiles from this index on touch memory that the viscous pass (or, in a plain
// overlapped launch, the previous launch in the stream) may still write or read; the tiles
// before it are independent of it. Static order (QU false): block b takes tiles b, b + grid,
// ...; each thread waits for the previous launch (griddepcontrol) before its first dependent
// tile. Queue order (QU true, one launch per stage after the viscous tiles): the producer warp
// claims tiles from *qc and passes each index to the consumers in shared memory (the last one
// flagged, see claim_tile); before staging a dependent tile it waits until *vdone (viscous tiles
// finished, each block's count added after its results) reaches vneed. Its buffer 0 lies after
// the work area and buffer 1's first release is the end of the stage kernel's viscous phase.
template <int N, int GEO, int MODE, int E, int VOL, bool QU = false>
__device__ __forceinline__ void inviscid_tiles(const DevMesh& M, const Bucket& B, const double* qin, double* out,
                                               double* g, int stage, int write_tr, char* smc, int bar_base,
                                               int dep_tile, unsigned* qc = nullptr, const unsigned* vdone = nullptr,
                                               unsigned vneed = 0) {
  // VOL 3 / 4: VOL 0 / 2 on box elements with the divergence S = sum_d Ja_dd D_d u_d taken in FP64
  // from the staged FP64 state. It gives the pressure row (-c0^2 S) and the U_c du_d part of the
  // momentum fluxes (U_c S); the FP32 (or tensor-core) contractions carry only the rest of the
  // momentum fluxes.
  constexpr bool KEP = VOL == 1, TC = VOL == 2 || VOL == 4;
  constexpr bool div64 = GEO == 0 && (VOL == 3 || VOL == 4);
  using S = Tile<N, E>;
  using P = TmaSmem32<N, E, KEP && GEO == 2, TC, QU>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  void* bar0 = smc + P::oBAR + bar_base;        // full[0]
  void* bar1 = smc + P::oBAR + bar_base + 8;    // full[1]
  void* ebar0 = smc + P::oBAR + bar_base + 16;  // empty[0]
  void* ebar1 = smc + P::oBAR + bar_base + 24;  // empty[1]
  int* tslot = reinterpret_cast<int*>(smc + P::oBAR + bar_base + 64);  // queue order: tile per buffer
  constexpr int NC = S::threads;  // consumer threads
  float* sD = reinterpret_cast<float*>(smc + P::oD);
  char* const IN0 = smc + P::oIN0;
  char* const IN1 = smc + P::oIN1;
  char* W = smc + P::oW;
  const int tid = threadIdx.x, nthr = NC;
  const int ntiles = (B.count + EPB - 1) / EPB;
  const float* rvf = reinterpret_cast<const float*>(M.rv);
  float* g32 = reinterpret_cast<float*>(g);
  const float c0sq = M.c0sq32;
  const float invw = c_ops32.w0inv[N];
  if (!QU) {  // queue order: the stage kernel set these up before its viscous phase
    for (int t = tid; t < n2; t += nthr) sD[t] = c_ops32.D[N][t];
    if (tid == 0) {
      mbar_init(bar0, 32);
      mbar_init(bar1, 32);
      mbar_init(ebar0, NC / 32);
      mbar_init(ebar1, NC / 32);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
  }
  if (tid >= NC) {
    // ---- producer warp ----------------------------------------------------------------
    // the records of the next tile are loaded one tile ahead, so their latency is hidden
    // behind the wait for a free buffer and the copies of the current tile
    TileRecs<E> recs;
    int tile = QU ? claim_tile(qc) : (int)blockIdx.x;
    int next = QU ? claim_tile(qc) : tile + (int)gridDim.x;  // one tile ahead
    if (tile < ntiles) load_recs<E>(B, tile, recs);
    bool dep_ok = false;
    int it = 0;
    for (; tile < ntiles; tile = next, next = QU ? claim_tile(qc) : next + (int)gridDim.x, ++it) {
      const int b = it & 1;
      if (!buffer_free(b ? ebar1 : ebar0, it, QU, M.wait_polls)) {
        if (tid == NC) {
          atomicCAS(&M.err[0], 0, kErrTimeout);
          atomicCAS(&M.err[1], 0, 2);
        }
        return;
      }
      // test hook: stage nothing more, so the consumers' bounded wait for this tile runs out
      // (every copy staged before was waited for by the consumers; none is left in flight)
      if (blockIdx.x == 0 && it == M.stop_tile) return;
      char* IN = b ? IN1 : IN0;
      if (QU && tid == NC) tslot[b] = tile | (next < ntiles ? 0 : kLastTile);
      store_recs<P>(B, tile, recs, IN);
      if (next < ntiles) load_recs<E>(B, next, recs);
      if (!QU && tile >= dep_tile && tile - (int)gridDim.x < dep_tile) pdl_wait();  // this block's first such tile
      if (QU && tile >= dep_tile && !dep_ok) {
        // every viscous tile finished (bounded, site 6); then the bulk copies may read its results
        bool ok = ld_acquire_u32(vdone) >= vneed;
        for (int spin = 0; !ok && spin < M.wait_polls; ++spin) {
          __nanosleep(128);
          ok = ld_acquire_u32(vdone) >= vneed;
        }
        if (!ok) {
          if (tid == NC) {
            atomicCAS(&M.err[0], 0, kErrTimeout);
            atomicCAS(&M.err[1], 0, 6);
          }
          return;
        }
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        dep_ok = true;
      }
      __syncwarp();
      tma_stage<N, P, false>(M, B, qin, tile, IN, b ? bar1 : bar0);
    }
    if (QU && it == 0) {  // no tile for this block: an empty one with index -1 (buffer 0 is free)
      if (tid == NC) tslot[0] = -1;
      __syncwarp();
      mbar_arrive(bar0);
    }
    return;
  }
  int le = tid / n3;
  const int p = tid % n3;
  const bool lane_ok = le < EPB;
  if (!lane_ok) le = EPB - 1;
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  const bool on_face = ii[0] == 0 || ii[0] == N || ii[1] == 0 || ii[1] == N || ii[2] == 0 || ii[2] == N;
  float4* F4 = reinterpret_cast<float4*>(W + le * P::work_elem + P::wF);
  float4* QH4 = reinterpret_cast<float4*>(W + le * P::work_elem + P::wQ);
  float4* QL4 = QH4 + n3;
  // This thread's (element, face, face node) items of the face and trace-write phases, the
  // same in every tile: le2 | f << 5 | a << 8 | b << 11 | pv << 14, or -1.
  constexpr int NFI = EPB * 6 * n2, FR = (NFI + NC - 1) / NC;
  int fdesc[FR];
#pragma unroll
  for (int r = 0; r < FR; ++r) {
    const int t = tid + r * NC;
    const int le2 = t / (6 * n2), rr = t % (6 * n2), f = rr / n2, ab = rr % n2;
    fdesc[r] = t < NFI ? (le2 | f << 5 | (ab % n) << 8 | (ab / n) << 11 | face_node(f, n, ab % n, ab / n) << 14) : -1;
  }
  // ---- consumer threads ----------------------------------------------------------------
  bool more = true;
  int tile = QU ? 0 : (int)blockIdx.x;
  for (int it = 0; QU ? more : tile < ntiles; ++it, tile += QU ? 0 : (int)gridDim.x) {
    // at this block's first dependent tile, before the bounded wait for the tile's data (the
    // wait for the previous launch is not part of the poll budget)
    if (!QU && tile >= dep_tile && tile - (int)gridDim.x < dep_tile) pdl_wait();
    const int cur = it & 1;
    const bool ok = mbar_wait_bounded(cur ? bar1 : bar0, (unsigned)((it >> 1) & 1), M.wait_polls);
    if (consumer_any(!ok, NC)) {
      if (tid == 0) {
        atomicCAS(&M.err[0], 0, kErrTimeout);
        atomicCAS(&M.err[1], 0, 1);
      }
      return;
    }
    if (QU) {
      tile = tslot[cur];
      if (tile < 0) break;
      // (a dependent tile's data, and the viscous results its threads load themselves, are
      // ordered before this point: the producer's acquire of the finished-tile counter, then
      // its arrival on the tile's mbarrier, which this wait acquires)
      more = !(tile & kLastTile);
      tile &= ~kLastTile;
    }
    const int i = tile * EPB + le;
    const bool active = lane_ok && i < B.count;
    char* IN = cur ? IN1 : IN0;
    const char* INe = IN + le * P::in_elem;
    const EntryMeta* MT = reinterpret_cast<const EntryMeta*>(INe + P::iMT);
    // prefetch what this node needs only at the end of the tile
    int64_t off = 0;
    float gold[4] = {0.f, 0.f, 0.f, 0.f}, rvp[3] = {0.f, 0.f, 0.f};
    if (active) {
      off = MT->off;
      if (MODE == MODE_RK && stage > 0) {
#pragma unroll
        for (int v = 0; v < 4; ++v) gold[v] = ld_early(&g32[v * M.total + off + p]);
      }
      if (MT->flag) {
#pragma unroll
        for (int c = 0; c < 3; ++c) rvp[c] = ld_early(&rvf[c * M.total + off + p]);
      }
    }
    const unsigned char* SH = reinterpret_cast<const unsigned char*>(INe + P::iSH);
    const ElemConst32* EC = reinterpret_cast<const ElemConst32*>(INe + P::iEC);
    float invJ = 0.f;
    // ---- node phase: split state, flux deviations --------------------------------------
    // the element's reference state (hi parts of node 0; any per-element constant serves):
    // computed once per element and passed through the element's T area, which the face
    // phase writes only after the node phase's barrier
    float4* QR = reinterpret_cast<float4*>(W + le * P::work_elem + P::wT);
    if (active && p == 0) {
      float r[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        r[v] = hi_part(reinterpret_cast<const double*>(INe + P::iQD + v * P::SQD + SH[v])[0]);
      *QR = make_float4(r[0], r[1], r[2], r[3]);
    }
    consumer_sync(NC);
    float qr32[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
      const float4 r4 = *QR;
      qr32[0] = r4.x, qr32[1] = r4.y, qr32[2] = r4.z, qr32[3] = r4.w;
      float dq[4], h[4], l[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double* QDv = reinterpret_cast<const double*>(INe + P::iQD + v * P::SQD + SH[v]);
        split_hilo(QDv[p], h[v], l[v]);
        dq[v] = (h[v] - qr32[v]) + l[v];
      }
      QH4[p] = make_float4(h[0], h[1], h[2], h[3]);
      QL4[p] = make_float4(l[0], l[1], l[2], l[3]);
      float fl[4][3];
      if (div64) {  // the U_c du_k part goes through the FP64 divergence
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          fl[0][k] = c0sq * dq[1 + k];
#pragma unroll
          for (int c = 0; c < 3; ++c) fl[1 + c][k] = dq[1 + c] * (qr32[1 + k] + dq[1 + k]) + (c == k ? dq[0] : 0.f);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          fl[0][k] = c0sq * dq[1 + k];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            fl[1 + c][k] = qr32[1 + c] * dq[1 + k] + dq[1 + c] * (qr32[1 + k] + dq[1 + k]) + (c == k ? dq[0] : 0.f);
        }
      }
      if (KEP) F4[p] = make_float4(dq[0], dq[1], dq[2], dq[3]);
      if (GEO == 0) {
        invJ = EC->invJ;
        if (!KEP) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float j = EC->Ja[d * 4];
            F4[d * n3 + p] = make_float4(j * fl[0][d], j * fl[1][d], j * fl[2][d], j * fl[3][d]);
          }
        }
      } else {
        float Ja[9];
        if (GEO == 2) {
#pragma unroll
          for (int k = 0; k < 9; ++k) Ja[k] = __ldg(&M.geo32[k * M.total + off + p]);
          invJ = __ldg(&M.geo32[9 * M.total + off + p]);
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) Ja[k] = EC->Ja[k];
          invJ = EC->invJ;
        }
        if (!KEP) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float c4[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) c4[v] = Ja[d * 3] * fl[v][0] + Ja[d * 3 + 1] * fl[v][1] + Ja[d * 3 + 2] * fl[v][2];
            F4[d * n3 + p] = make_float4(c4[0], c4[1], c4[2], c4[3]);
          }
        } else if (GEO == 2) {
#pragma unroll
          for (int d = 0; d < 3; ++d) F4[(1 + d) * n3 + p] = make_float4(Ja[d * 3], Ja[d * 3 + 1], Ja[d * 3 + 2], 0.f);
        }
      }
    }
    consumer_sync(NC);
    // ---- volume: J R = -sum_d D_d Ftil^d ----------------------------------------------
    float JR[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
      const int str[3] = {1, n, n2};
      if (TC) {
        // done below by the tensor-core items; the node sums follow the face phase
      } else if (!KEP) {
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
      } else {
        const float4 di = F4[p];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int bs = p - ii[d] * str[d];
          float jai[3];
          if (GEO == 2) {
            const float4 j4 = F4[(1 + d) * n3 + p];
            jai[0] = j4.x, jai[1] = j4.y, jai[2] = j4.z;
          } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) jai[k] = GEO == 0 ? (k == d ? EC->Ja[d * 4] : 0.f) : EC->Ja[d * 3 + k];
          }
#pragma unroll
          for (int m = 0; m < n; ++m) {
            const int pm = bs + m * str[d];
            const float d2 = 2.f * sD[ii[d] * n + m];
            const float4 dmv = F4[pm];
            // averaged deviations and metric of the pair (i, m)
            const float bp = 0.5f * (di.x + dmv.x), bu[3] = {0.5f * (di.y + dmv.y), 0.5f * (di.z + dmv.z),
                                                               0.5f * (di.w + dmv.w)};
            float ja[3];
            if (GEO == 2) {
              const float4 j4 = F4[(1 + d) * n3 + pm];
              ja[0] = 0.5f * (jai[0] + j4.x), ja[1] = 0.5f * (jai[1] + j4.y), ja[2] = 0.5f * (jai[2] + j4.z);
            } else {
              ja[0] = jai[0], ja[1] = jai[1], ja[2] = jai[2];
            }
            const float Ur = ja[0] * qr32[1] + ja[1] * qr32[2] + ja[2] * qr32[3];
            const float Ud = ja[0] * bu[0] + ja[1] * bu[1] + ja[2] * bu[2];
            JR[0] -= d2 * (c0sq * Ud);
#pragma unroll
            for (int c = 0; c < 3; ++c) JR[1 + c] -= d2 * (qr32[1 + c] * Ud + bu[c] * (Ur + Ud) + bp * ja[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) JR[1 + c] += rvp[c];
      if (div64) {
        // S = sum_d Ja_dd (D u_d)_i in FP64 (the pressure row is a small difference of the three
        // directional derivatives, so FP32 rounding of each would be amplified by c0^2 / |R_p|)
        const int str[3] = {1, n, n2};
        const ElemConst* ec64 = M.ec + MT->elem;
        double S64 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int bs = p - ii[d] * str[d];
          const double* ud = reinterpret_cast<const double*>(INe + P::iQD + (1 + d) * P::SQD + SH[1 + d]);
          const double* Dr = &g_D64[N][ii[d] * n];
          double sd = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) sd = fma(__ldg(Dr + m), ud[bs + m * str[d]], sd);
          S64 = fma(__ldg(&ec64->Ja[d * 4]), sd, S64);
        }
        const float s32 = (float)S64;
        JR[0] = -c0sq * s32;  // replaces the FP32 contraction of the pressure row
#pragma unroll
        for (int c = 0; c < 3; ++c) JR[1 + c] -= qr32[1 + c] * s32;
      }
    }
    if (TC) {
      // tensor-core items: (element, direction, 16-row tile), rows r = 4 line + v
      constexpr int R = 4 * n2, TR = (R + 15) / 16, ITEMS = EPB * 3 * TR;
      const int lane = tid & 31, gq = lane >> 2, tq = lane & 3;
      for (int item = tid >> 5; item < ITEMS; item += NC / 32) {
        const int le2 = item / (3 * TR), rem = item % (3 * TR), d = rem / TR, rt = rem % TR;
        if (tile * EPB + le2 >= B.count) continue;
        // C overwrites the F rows of this item in place: the item's A operands (all of its rows
        // and positions m) are in registers before its mma, and no other item reads these rows
        float* Fs = reinterpret_cast<float*>(W + le2 * P::work_elem + P::wF) + d * n3 * 4;
        float4* Cd = reinterpret_cast<float4*>(Fs);
        // node of (line, position m) along direction d: base(line) + m * stride, line = a + n b
        // over the other two indices; this lane's rows are r0 = 16 rt + gq and r0 + 8, i.e.
        // lines l0 = r0 / 4 and l0 + 2 with variable v = gq % 4
        const int stride = d == 0 ? 1 : (d == 1 ? n : n2);
        auto base_of = [&](int line) {
          const int a = line % n, b = line / n;
          return d == 0 ? n * (a + n * b) : (d == 1 ? a + n2 * b : a + n * b);
        };
        const int r0 = rt * 16 + gq, v = gq & 3;
        const bool ok0 = r0 < R, ok1 = r0 + 8 < R;
        const int b0 = ok0 ? base_of(r0 >> 2) : 0, b1 = ok1 ? base_of((r0 + 8) >> 2) : 0;
        unsigned ab[4], as[4], bb[2], bs[2];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int m = tq + ((k & 2) ? 4 : 0);
          const bool ok = ((k & 1) ? ok1 : ok0) && m < n;
          const float x = ok ? Fs[((k & 1) ? b1 : b0) * 4 + m * stride * 4 + v] : 0.f;
          tf32_split(x, ab[k], as[k]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int m = tq + 4 * k;  // B[k = m][column = i = gq] = D[i][m]
          tf32_split((m < n && gq < n) ? sD[gq * n + m] : 0.f, bb[k], bs[k]);
        }
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        if (M.tc == 1) {  // 3xTF32: the two correction products first; plain TF32 (tc 2) skips them
          mma_tf32(c, as, bb);
          mma_tf32(c, ab, bs);
        }
        mma_tf32(c, ab, bb);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = 2 * tq + (k & 1);
          const bool ok = ((k & 2) ? ok1 : ok0) && i < n;
          if (ok) reinterpret_cast<float*>(Cd)[(((k & 2) ? b1 : b0) + i * stride) * 4 + v] = c[k];
        }
      }
    }
    // no barrier: the face phase reads QH/QL and the input buffer and writes T, none of which
    // the contraction touches
    // ---- faces, one thread per (element, face, face node) -----------------------------
#pragma unroll
    for (int r = 0; r < FR; ++r) {
      const int fd = fdesc[r];
      if (fd < 0) break;
      const int le2 = fd & 31, f = (fd >> 5) & 7, a = (fd >> 8) & 7, bb = (fd >> 11) & 7, pv = fd >> 14;
      const int ab = a + n * bb;
      if (tile * EPB + le2 >= B.count) continue;
      const char* I2 = IN + le2 * P::in_elem;
      const unsigned char* SH2 = reinterpret_cast<const unsigned char*>(I2 + P::iSH);
      const FaceLink L = reinterpret_cast<const FaceLink*>(I2 + P::iLK)[f];
      const ElemConst32* E2 = reinterpret_cast<const ElemConst32*>(I2 + P::iEC);
      const EntryMeta* MT2 = reinterpret_cast<const EntryMeta*>(I2 + P::iMT);
      char* W2 = W + le2 * P::work_elem;
      const int d = f >> 1;
      const float sg = (f & 1) ? 1.f : -1.f;
      const bool ns2 = MT2->flag != 0;
      float term[4];
      if (L.kind == FK_MORTAR) {
        const int64_t node = MT2->off + pv;
        const int64_t ms = MT2->troff + f * n2 + ab;
        const int e2 = MT2->elem;
        double Sd[3], qq[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) qq[v] = reinterpret_cast<const double*>(I2 + P::iQD + v * P::SQD + SH2[v])[pv];
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
          float t2 = (float)(M.LH[(1 + c) * M.tr_total + ms] - own);
          if (ns2) t2 += reinterpret_cast<const float*>(I2 + P::iOV + SH2[16])[(f * n2 + ab) * 3 + c];
          term[1 + c] = t2;
        }
      } else {
        float Sv[3];
        if (GEO == 2) {
          const int64_t node = MT2->off + pv;
#pragma unroll
          for (int k = 0; k < 3; ++k) Sv[k] = sg * __ldg(&M.geo32[(d * 3 + k) * M.total + node]);
        } else if (GEO == 1) {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sv[k] = sg * E2->Ja[d * 3 + k];
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) Sv[k] = (k == d) ? sg * E2->Ja[d * 4] : 0.f;
        }
        const float ss = Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2];
        const float is = GEO == 0 ? 0.f : rsqrtf(ss);  // face area element S = |Sv| > 0
        const float s = GEO == 0 ? fabsf(E2->Ja[d * 4]) : ss * is;
        const float nh[3] = {Sv[0] * is, Sv[1] * is, Sv[2] * is};
        const float4 h4 = reinterpret_cast<const float4*>(W2 + P::wQ)[pv];
        const float4 l4 = reinterpret_cast<const float4*>(W2 + P::wQ)[n3 + pv];
        const float qh[4] = {h4.x, h4.y, h4.z, h4.w}, ql[4] = {l4.x, l4.y, l4.z, l4.w};
        float dqf[4];
        int nab = 0;
        if (L.kind == FK_CONF) {
          int a1, b1;
          inv_orient(L.orient, N, a, bb, a1, b1);
          nab = a1 + n * b1;
          // the neighbour's 32-byte record (p, u, v, w as hi, lo); 16-byte aligned, no shift
          const float4* tr = reinterpret_cast<const float4*>(I2 + P::iNT + f * P::SNT) + 2 * nab;
          const float4 t01 = tr[0], t23 = tr[1];
          dqf[0] = (t01.x - qh[0]) + (t01.y - ql[0]);
          dqf[1] = (t01.z - qh[1]) + (t01.w - ql[1]);
          dqf[2] = (t23.x - qh[2]) + (t23.y - ql[2]);
          dqf[3] = (t23.z - qh[3]) + (t23.w - ql[3]);
        } else if (L.kind == FK_INFLOW) {
          dqf[0] = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float ih, il;
            split_hilo(M.inflow[1 + c], ih, il);
            dqf[1 + c] = (ih - qh[1 + c]) + (il - ql[1 + c]);
          }
        } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {
          // mirror ghost: -2u (no-slip) or -2 (u.n)n (free-slip; n the unit normal, the axis on
          // a box), written with n rather than S so that S need not stay live
          const float uo[3] = {qh[1] + ql[1], qh[2] + ql[2], qh[3] + ql[3]};
          dqf[0] = 0.f;
          if (L.kind == FK_WALL) {
#pragma unroll
            for (int c = 0; c < 3; ++c) dqf[1 + c] = -2.f * uo[c];
          } else if (GEO == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) dqf[1 + c] = c == d ? -2.f * uo[c] : 0.f;
          } else {
            const float un = uo[0] * nh[0] + uo[1] * nh[1] + uo[2] * nh[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) dqf[1 + c] = -2.f * un * nh[c];
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
          float wo, wn;
          visc_face_weights(M.mixed_face, ns2, L.nflag != 0, wo, wn);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float tv = 0.f;
            if (ns2) tv += wo * reinterpret_cast<const float*>(I2 + P::iOV + SH2[16])[(f * n2 + ab) * 3 + c];
            if (L.nflag) tv += wn * reinterpret_cast<const float*>(I2 + P::iNV + f * P::SNV + SH2[10 + f])[nab * 3 + c];
            term[1 + c] += tv;
          }
        } else if (L.kind == FK_SLIP && ns2) {
          // free-slip wall: the tangential part of the own outward trace t = tau . S
          const float* ov = reinterpret_cast<const float*>(I2 + P::iOV + SH2[16]) + (f * n2 + ab) * 3;
          const float tv[3] = {ov[0], ov[1], ov[2]};
          if (GEO == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) term[1 + c] += c == d ? 0.f : tv[c];
          } else {
            const float tn = tv[0] * nh[0] + tv[1] * nh[1] + tv[2] * nh[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) term[1 + c] += tv[c] - tn * nh[c];
          }
        }
      }
      reinterpret_cast<float4*>(W2 + P::wT)[f * n2 + ab] = make_float4(term[0], term[1], term[2], term[3]);
    }
    consumer_sync(NC);
    // ---- assembly and update ------------------------------------------------------------
    if (TC && active) {
      const float4* Cp = reinterpret_cast<const float4*>(W + le * P::work_elem + P::wF);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float4 c4 = Cp[d * n3 + p];
        if (!div64) JR[0] -= c4.x;  // with div64 the pressure row is -c0^2 S, set above
        JR[1] -= c4.y;
        JR[2] -= c4.z;
        JR[3] -= c4.w;
      }
    }
    if (active) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (ii[d] != 0 && ii[d] != N) continue;
        const int f = 2 * d + (ii[d] == N ? 1 : 0);
        const int a = d == 0 ? ii[1] : ii[0], bb = d == 2 ? ii[1] : ii[2];
        const float4 sc = reinterpret_cast<const float4*>(W + le * P::work_elem + P::wT)[f * n2 + a + n * bb];
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
        const double Bc = c32_rkB[stage];
        const float dtf = M.dt32;
        float h[4], l[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int64_t ix = v * M.total + off + p;
          const float gi = fmaf(A, gold[v], JR[v] * invJ * dtf);
          g32[ix] = gi;
          const double qo = reinterpret_cast<const double*>(INe + P::iQD + v * P::SQD + SH[v])[p];
          const double qn = fma(Bc, widen_f32(gi), qo);
          out[ix] = qn;
          if (write_tr && on_face) split_hilo(qn, h[v], l[v]);
        }
        if (write_tr && on_face) {
          // the next stage's trace records of this node's faces (32 bytes each, one sector)
          float4* Tn = reinterpret_cast<float4*>(M.Tq_next) + 2 * MT->troff;  // record still staged
          const float4 r01 = make_float4(h[0], l[0], h[1], l[1]), r23 = make_float4(h[2], l[2], h[3], l[3]);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            if (ii[d] != 0 && ii[d] != N) continue;
            const int f = 2 * d + (ii[d] == N ? 1 : 0);
            const int a = d == 0 ? ii[1] : ii[0], bb = d == 2 ? ii[1] : ii[2];
            const int dst = f * n2 + a + n * bb;
            Tn[2 * dst] = r01;
            Tn[2 * dst + 1] = r23;
          }
        }
      }
    }
    // No barrier here: the next tile writes F and QH/QL only after its node phase, which no
    // thread starts before every consumer has passed the next tile's vote (bar.red), i.e.
    // finished this assembly; T is rewritten only after the next tile's first barrier.
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(cur ? ebar1 : ebar0);  // this warp no longer reads the buffer
  }
}

template <int N, int GEO, int MODE, int E, int VOL>
__global__ void __launch_bounds__(Tile<N, E>::threads + 32, (InvMinBlocks<N, E>::value))
    k_inviscid32t(DevMesh M, Bucket B, const double* qin, double* out, double* g, int stage, int write_tr) {
  extern __shared__ __align__(128) char smc[];
  // An overlapped launch: the next launch (which waits for this one before it touches memory)
  // may be scheduled as soon as every block runs. After the viscous pass of the same stage
  // (M.after_visc) the bucket's first B.n_indep entries (Euler elements without an NS or
  // mortar neighbour) read and write nothing that pass touches, and run without waiting for it.
  pdl_launch_dependents();
  const int dep_tile = M.after_visc ? B.n_indep / Tile<N, E>::EPB : 0;
  inviscid_tiles<N, GEO, MODE, E, VOL>(M, B, qin, out, g, stage, write_tr, smc, 0, dep_tile);
  // every thread waits for the previous launch before it exits, so this launch completes after
  // it: a later launch that waits for this one has waited for that one too
  pdl_wait();
}

// ---------------------------------------------------------------------------------------
// viscous pass, persistent, TMA-staged (box and affine elements)
// ---------------------------------------------------------------------------------------
// Line contractions in shared memory, one thread per (element, direction, line): along the
// line of direction d with index l (the other two node indices a = l % n, b = l / n), the
// thread loads the n values of each of three node arrays once and forms all n outputs
// out[i] = sum_m D[i][m] in[m], summed in order m = 0 .. N, with D read from the constant bank
// (compile-time indices: no load, no register). in(c) = src + c * src_stride, out(c) = dst +
// c * dst_stride; dst may equal src (each line's values are read before they are written, and
// no other line touches them). With `ends`, ends[0][c] is added to out(c) at i = 0 and
// ends[1][c] at i = N.
template <int N>
__device__ __forceinline__ void line_contract3(const float* src, int src_stride, float* dst, int dst_stride, int d,
                                               int l, const float (*ends)[3] = nullptr) {
  constexpr int n = N + 1, n2 = n * n;
  const int a = l % n, b = l / n;
  const int base = d == 0 ? a * n + b * n2 : (d == 1 ? a + b * n2 : a + b * n);
  const int st = d == 0 ? 1 : (d == 1 ? n : n2);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float u[n];
#pragma unroll
    for (int m = 0; m < n; ++m) u[m] = src[c * src_stride + base + m * st];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < n; ++m) acc = fmaf(c_ops32.D[N][i * n + m], u[m], acc);
      if (ends && i == 0) acc += ends[0][c];
      if (ends && i == N) acc += ends[1][c];
      dst[c * dst_stride + base + i * st] = acc;
    }
  }
}

// BR1 lifting (1/w_end) (u* - u) S at the two end nodes of the line (d, l) of one element
// (the face nodes (a, b) = (l % n, l / n) of faces 2d and 2d + 1), for box and affine
// elements: it equals adding sg (u* - u)_c / (2 w_end) to du_c/dxi_d there (the metric terms
// multiply both alike). Conforming, inflow and wall faces; mortar faces give 0 here. INe: the
// element's staged input, its velocity planes already overwritten by (hi, lo) pairs per node.
template <int N, typename P>
__device__ __forceinline__ void face_lift(const char* INe, const DevMesh& M, float invw, int d, int l,
                                          float lift[2][3]) {
  constexpr int n = N + 1, n2 = n * n;
  const int a = l % n, b = l / n;
  const FaceLink* LK = reinterpret_cast<const FaceLink*>(INe + P::iLK);
  const unsigned char* SH = reinterpret_cast<const unsigned char*>(INe + P::iSH);
  const float2* H0 = reinterpret_cast<const float2*>(INe + P::iQV + SH[0]);
  const float2* H1 = reinterpret_cast<const float2*>(INe + P::iQV + P::SQV + SH[1]);
  const float2* H2 = reinterpret_cast<const float2*>(INe + P::iQV + 2 * P::SQV + SH[2]);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int f = 2 * d + side, e0 = side ? N : 0;
    const int node = d == 0 ? e0 + a * n + b * n2 : (d == 1 ? a + e0 * n + b * n2 : a + b * n + e0 * n2);
    const FaceLink L = LK[f];
    const float2 h0 = H0[node], h1 = H1[node], h2 = H2[node];
    float jump[3] = {0.f, 0.f, 0.f};
    if (L.kind == FK_CONF) {
      int a1, b1;
      inv_orient(L.orient, N, a, b, a1, b1);
      // the neighbour's record (p, u, v, w as hi, lo); 16-byte aligned, no shift
      const float4* tr = reinterpret_cast<const float4*>(INe + P::iNT + f * P::SNT) + 2 * (a1 + n * b1);
      const float4 t01 = tr[0], t23 = tr[1];
      jump[0] = (t01.z - h0.x) + (t01.w - h0.y);
      jump[1] = (t23.x - h1.x) + (t23.y - h1.y);
      jump[2] = (t23.z - h2.x) + (t23.w - h2.y);
    } else if (L.kind == FK_INFLOW) {
      const float2 hh[3] = {h0, h1, h2};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float ih, il;
        split_hilo(M.inflow[1 + c], ih, il);
        jump[c] = (ih - hh[c].x) + (il - hh[c].y);
      }
    } else if (L.kind == FK_WALL || L.kind == FK_SLIP) {
      const ElemConst32* EC = reinterpret_cast<const ElemConst32*>(INe + P::iEC);
      const float sg = side ? 1.f : -1.f;
      const float Sv[3] = {sg * EC->Ja[d * 3], sg * EC->Ja[d * 3 + 1], sg * EC->Ja[d * 3 + 2]};
      const float uo[3] = {h0.x + h0.y, h1.x + h1.y, h2.x + h2.y};
      wall_jump<float>(L.kind, uo, Sv, jump);
    }
    const float sl = (side ? 0.5f : -0.5f) * invw;
#pragma unroll
    for (int c = 0; c < 3; ++c) lift[side][c] = sl * jump[c];
  }
}

// Static or queue order of the tiles as in inviscid_tiles (qc: the claim counter). Returns the
// number of tiles this block's consumers finished (thread 0's count).
template <int N, int GEO, int E = Shape<N>::EPB, bool QU = false>
__device__ __forceinline__ int viscous_tiles(const DevMesh& M, const Bucket& B, const double* q, char* smc,
                                             int bar_base, unsigned* qc = nullptr) {
  using S = Tile<N, E>;
  using P = ViscTmaSmem32<N, E>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  constexpr int NC = S::threads;  // consumer threads
  void* bar0 = smc + P::oBAR + bar_base;
  void* bar1 = smc + P::oBAR + bar_base + 8;
  void* ebar0 = smc + P::oBAR + bar_base + 16;
  void* ebar1 = smc + P::oBAR + bar_base + 24;
  int* tslot = reinterpret_cast<int*>(smc + P::oBAR + bar_base + 64);  // queue order: tile per buffer
  char* const IN0 = smc + P::oIN0;
  char* const IN1 = smc + P::oIN1;
  char* W = smc + P::oW;
  const int tid = threadIdx.x;
  const int ntiles = (B.count + EPB - 1) / EPB;
  float* Tvf = reinterpret_cast<float*>(M.Tv);
  float* rvf = reinterpret_cast<float*>(M.rv);
  if (tid == 0) {
    mbar_init(bar0, 32);
    mbar_init(bar1, 32);
    mbar_init(ebar0, NC / 32);
    mbar_init(ebar1, NC / 32);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid >= NC) {
    // ---- producer warp ----------------------------------------------------------------
    TileRecs<EPB> recs;
    int tile = QU ? claim_tile(qc) : (int)blockIdx.x;
    int next = QU ? claim_tile(qc) : tile + (int)gridDim.x;  // one tile ahead
    if (tile < ntiles) load_recs<EPB>(B, tile, recs);
    int it = 0;
    for (; tile < ntiles; tile = next, next = QU ? claim_tile(qc) : next + (int)gridDim.x, ++it) {
      const int b = it & 1;
      if (it >= 2 && !mbar_wait_bounded(b ? ebar1 : ebar0, (unsigned)(((it >> 1) - 1) & 1), M.wait_polls)) {
        if (tid == NC) {
          atomicCAS(&M.err[0], 0, kErrTimeout);
          atomicCAS(&M.err[1], 0, 4);
        }
        return 0;
      }
      if (blockIdx.x == 0 && it == M.stop_tile) return 0;  // test hook, as in the inviscid pass
      char* IN = b ? IN1 : IN0;
      if (QU && tid == NC) tslot[b] = tile | (next < ntiles ? 0 : kLastTile);
      store_recs<P>(B, tile, recs, IN);
      if (next < ntiles) load_recs<EPB>(B, next, recs);
      __syncwarp();
      tma_stage<N, P, true>(M, B, q, tile, IN, b ? bar1 : bar0);
    }
    if (QU && it == 0) {  // no tile for this block: an empty one with index -1 (buffer 0 is free)
      if (tid == NC) tslot[0] = -1;
      __syncwarp();
      mbar_arrive(bar0);
    }
    return 0;
  }
  int le = tid / n3;
  const int p = tid % n3;
  const bool lane_ok = le < EPB;
  if (!lane_ok) le = EPB - 1;
  const int ii[3] = {p % n, (p / n) % n, p / n2};
  float* U = reinterpret_cast<float*>(W + le * P::work_elem + P::wU);
  float* F = reinterpret_cast<float*>(W + le * P::work_elem + P::wF);
  const float invw = c_ops32.w0inv[N];
  int done = 0;
  bool more = true;
  int tile = QU ? 0 : (int)blockIdx.x;
  for (int it = 0; QU ? more : tile < ntiles; ++it, tile += QU ? 0 : (int)gridDim.x) {
    const int cur = it & 1;
    const bool ok = mbar_wait_bounded(cur ? bar1 : bar0, (unsigned)((it >> 1) & 1), M.wait_polls);
    if (consumer_any(!ok, NC)) {
      if (tid == 0) {
        atomicCAS(&M.err[0], 0, kErrTimeout);
        atomicCAS(&M.err[1], 0, 3);
      }
      return done;
    }
    if (QU) {
      tile = tslot[cur];
      if (tile < 0) break;
      more = !(tile & kLastTile);
      tile &= ~kLastTile;
    }
    const bool active = lane_ok && tile * EPB + le < B.count;
    const char* INe = (cur ? IN1 : IN0) + le * P::in_elem;
    const EntryMeta* MT = reinterpret_cast<const EntryMeta*>(INe + P::iMT);
    const ElemConst32* EC = reinterpret_cast<const ElemConst32*>(INe + P::iEC);
    const unsigned char* SH = reinterpret_cast<const unsigned char*>(INe + P::iSH);
    int64_t off = 0, troff = 0;
    int e = 0;
    float Ja[9], invJ = 0.f, delta = 0.f;
    // the element's reference velocity (hi parts of node 0), once per element, through the
    // element's F area (the previous tile's divergence read it before this tile's vote; this
    // tile writes F only after its first barrier)
    if (active && p == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] = hi_part(reinterpret_cast<const double*>(INe + P::iQV + c * P::SQV + SH[c])[0]);
    }
    consumer_sync(NC);
    if (active) {
      float uh[3], ul[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double* QV = reinterpret_cast<const double*>(INe + P::iQV + c * P::SQV + SH[c]);
        split_hilo(QV[p], uh[c], ul[c]);
        U[c * n3 + p] = (uh[c] - F[c]) + ul[c];  // deviation from the element's first node
        reinterpret_cast<float2*>(const_cast<double*>(QV))[p] = make_float2(uh[c], ul[c]);
      }
    }
    consumer_sync(NC);
    // gradient: du_c / dxi_d along every line of direction d, into the F area as
    // [(c * 3 + d) * n3 + node] (the reference velocity there was read before the last
    // barrier), with the BR1 lifting of the line's two end faces (the faces of direction d;
    // mortar faces are lifted per node below)
    for (int t = tid; t < EPB * 3 * n2; t += NC) {
      const int lt = t / (3 * n2), r = t - lt * (3 * n2), d = r / n2, l = r - d * n2;
      if (tile * EPB + lt >= B.count) continue;
      char* We = W + lt * P::work_elem;
      float lift[2][3];
      face_lift<N, P>((cur ? IN1 : IN0) + lt * P::in_elem, M, invw, d, l, lift);
      line_contract3<N>(reinterpret_cast<const float*>(We + P::wU), n3, reinterpret_cast<float*>(We + P::wF) + d * n3,
                        3 * n3, d, l, lift);
    }
    consumer_sync(NC);
    if (active) {
      off = MT->off;
      troff = MT->troff;
      e = MT->elem;
      delta = EC->delta;
      invJ = EC->invJ;
#pragma unroll
      for (int k = 0; k < 9; ++k) Ja[k] = EC->Ja[k];
      float G[3][3];
      {
        // this node's nine derivatives (its own thread overwrites them with F below)
        float du[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) du[c][d] = F[(c * 3 + d) * n3 + p];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k)
            G[c][k] = GEO == 0 ? Ja[k * 4] * du[c][k] : Ja[k] * du[c][0] + Ja[3 + k] * du[c][1] + Ja[6 + k] * du[c][2];
      }
      // BR1 lifting on this node's mortar faces (projected u*_c S_k from the mortar pass)
      if (MT->has_mortar) {
        const FaceLink* LK = reinterpret_cast<const FaceLink*>(INe + P::iLK);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (ii[d] != 0 && ii[d] != N) continue;
          const int side = ii[d] == N ? 1 : 0, f = 2 * d + side;
          if (LK[f].kind != FK_MORTAR) continue;
          const double sg = side ? 1.0 : -1.0;
          const int a = d == 0 ? ii[1] : ii[0], b = d == 2 ? ii[1] : ii[2];
          const int64_t ms = troff + f * n2 + a + n * b;
          double Sd[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) Sd[k] = sg * M.ec[e].Ja[d * 3 + k];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double uc = q[(1 + c) * M.total + off + p];
#pragma unroll
            for (int k = 0; k < 3; ++k) G[c][k] += invw * (float)(M.LU[(c * 3 + k) * M.tr_total + ms] - uc * Sd[k]);
          }
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
        const int64_t ms = troff + f * n2 + a + n * b;
#pragma unroll
        for (int c = 0; c < 3; ++c) Tvf[ms * 3 + c] = sg * Fv[d][c];
      }
    }
    // the input buffer is no longer read; its velocity slots were written here, and the next
    // bulk copies into it are async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    consumer_sync(NC);
    if ((tid & 31) == 0) mbar_arrive(cur ? ebar1 : ebar0);
    // divergence: D_d applied along every line of direction d to the three fluxes F[d][c],
    // in place
    for (int t = tid; t < EPB * 3 * n2; t += NC) {
      const int lt = t / (3 * n2), r = t - lt * (3 * n2);
      if (tile * EPB + lt >= B.count) continue;
      float* Fe = reinterpret_cast<float*>(W + lt * P::work_elem + P::wF) + r / n2 * 3 * n3;
      line_contract3<N>(Fe, n3, Fe, n3, r / n2, r % n2);
    }
    consumer_sync(NC);
    if (active) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        rvf[c * M.total + off + p] = (F[c * n3 + p] + F[(3 + c) * n3 + p]) + F[(6 + c) * n3 + p];
    }
    ++done;
  }
  return done;
}

// E: elements per tile, the default shape (Shape<N>::EPB) or the alternative (AltEPB<N>)
template <int N, int GEO, int E>
__global__ void __launch_bounds__(Tile<N, E>::threads + 32, (InvMinBlocks<N, E>::value))
    k_viscous32t(DevMesh M, Bucket B, const double* q) {
  extern __shared__ __align__(128) char smc[];
  // an overlapped launch: every input comes from the previous launches, and the inviscid pass
  // before it reads the viscous buffers this pass writes. The next launch is allowed only
  // after the wait, so it may rely on everything before this launch having completed.
  pdl_wait();
  pdl_launch_dependents();
  viscous_tiles<N, GEO, E>(M, B, q, smc, 0);
}

// ---------------------------------------------------------------------------------------
// one persistent kernel per Runge-Kutta stage (viscous tiles, grid barrier, inviscid tiles)
// ---------------------------------------------------------------------------------------
// Grid-wide barrier of a launch whose blocks are all resident (a cooperative launch). Bounded:
// gbar[0] counts the arrivals, the last one resets it and advances the generation gbar[1];
// a block that sees no new generation within M.wait_polls polls records DG_ERR_TIMEOUT (site 5).
// Test hook: with M.stop_tile == -2 block 0 does not arrive, so every block's wait runs out.
__device__ __forceinline__ bool grid_barrier(const DevMesh& M) {
  unsigned* gbar = reinterpret_cast<unsigned*>(M.err + 4);
  bool ok = true;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(gbar + 1);  // cannot advance before this block arrives
    if (!(M.stop_tile == -2 && blockIdx.x == 0)) {
      __threadfence();  // this block's results (ordered before by the __syncthreads) first
      if (atomicAdd(gbar, 1u) == gridDim.x - 1) {
        atomicExch(gbar, 0u);
        __threadfence();
        atomicAdd(gbar + 1, 1u);
      }
    }
    ok = ld_acquire_u32(gbar + 1) != gen;
    for (int spin = 0; !ok && spin < M.wait_polls; ++spin) {
      __nanosleep(128);
      ok = ld_acquire_u32(gbar + 1) != gen;
    }
    if (!ok) {
      atomicCAS(&M.err[0], 0, kErrTimeout);
      atomicCAS(&M.err[1], 0, 5);
    }
  }
  // thread 0's verdict to the block (no static shared memory: the dynamic layouts use it all)
  ok = __syncthreads_and(ok) != 0;
  // the second phase's bulk copies (async proxy) read what other blocks stored before the
  // barrier and overwrite shared memory that this block's first phase read and wrote
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  return ok;
}

// A whole RK stage of one (order, geometry) bucket after its traces: the viscous pass over the
// bucket's NS elements (Bv), a grid barrier (the inviscid pass reads the neighbours' viscous
// traces), the inviscid pass with the RK update over all its elements (Bi). The same device code
// as k_viscous32t and k_inviscid32t (default tile shape, FP32 contractions); the second phase's
// mbarriers sit 32 bytes after the first's.
template <int N, int GEO>
__global__ void __launch_bounds__(Shape<N>::threads + 32, TmaMinBlocks<N>::value)
    k_stage32t(DevMesh M, Bucket Bv, Bucket Bi, const double* q, double* out, double* g, int stage, int write_tr) {
  extern __shared__ __align__(128) char smc[];
  if (Bv.count > 0) {  // no NS element: nothing to wait for
    viscous_tiles<N, GEO>(M, Bv, q, smc, 0);
    if (!grid_barrier(M)) return;
  }
  inviscid_tiles<N, GEO, MODE_RK, Shape<N>::EPB, 0>(M, Bi, q, out, g, stage, write_tr, smc, 32, INT_MAX);
}

template <int N>
constexpr size_t stage_smem_bound() {
  return ViscTmaSmem32<N>::bytes > TmaSmem32<N>::bytes ? ViscTmaSmem32<N>::bytes : TmaSmem32<N>::bytes;
}

// A whole RK stage in one ordinary launch, the tiles taken from queues: every block claims
// viscous tiles (Bv's NS elements) until that queue is empty and adds the number it finished to
// a counter; then it claims inviscid tiles (Bi, independent entries first). A block stages a
// tile that reads the viscous results only once that counter covers every viscous tile, and
// such tiles are claimed only after every viscous tile was claimed by a running block, so the
// wait needs no co-resident grid. Until then the blocks run the independent tiles, so the
// viscous pass drains into inviscid work. Overlapped launch: everything waits for the previous
// launch first. Queue counters: err[8] viscous claims, err[9] inviscid claims, err[10] viscous
// tiles finished, err[11] blocks finished; the last block resets them for the next launch.
// VOL: the inviscid pass's volume variant, 0 (FP32 contractions) or 3 (with the FP64 velocity
// divergence, box elements).
template <int N, int GEO, int VOL>
__global__ void __launch_bounds__(Shape<N>::threads + 32, TmaMinBlocks<N>::value)
    k_stage32q(DevMesh M, Bucket Bv, Bucket Bi, const double* q, double* out, double* g, int stage, int write_tr) {
  extern __shared__ __align__(128) char smc[];
  constexpr int EPB = Shape<N>::EPB, NC = Shape<N>::threads, n = N + 1;
  // the inviscid phase's layout keeps its buffer 0 clear of the viscous phase's shared memory, so
  // its producer stages the first inviscid tile while the consumers finish the viscous tiles
  using PI = TmaSmem32<N, EPB, false, false, true>;
  static_assert(PI::oIN0 >= (int)ViscTmaSmem32<N>::bytes, "inviscid buffer 0 overlaps the viscous phase");
  static_assert(PI::bytes <= stage_smem_bound<N>(), "stage kernel shared memory");
  unsigned* qc = reinterpret_cast<unsigned*>(M.err + 8);
  const int tid = threadIdx.x;
  pdl_wait();
  pdl_launch_dependents();
  // the inviscid phase's operator table and barriers (its mbarriers sit 32 bytes after the
  // viscous phase's; the viscous phase uses no operator table)
  float* sD = reinterpret_cast<float*>(smc + PI::oD);
  for (int t = tid; t < n * n; t += blockDim.x) sD[t] = c_ops32.D[N][t];
  if (tid == 0) {
    mbar_init(smc + PI::oBAR + 32, 32);
    mbar_init(smc + PI::oBAR + 40, 32);
    mbar_init(smc + PI::oBAR + 48, NC / 32);
    mbar_init(smc + PI::oBAR + 56, NC / 32);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const unsigned nv = (unsigned)((Bv.count + EPB - 1) / EPB);
  // the blocks that start with the viscous queue: all, or a share that follows the flags (the
  // others begin with independent inviscid tiles, so that both kinds of tiles share the SMs
  // while the viscous pass runs; without independent tiles every block starts with it)
  int nvb = (int)gridDim.x;
  if (Bi.vsplit > 0 && Bi.n_indep >= EPB) {
    const float share = (float)Bi.vsplit * (float)nv / (float)(nv + (unsigned)(Bi.n_indep / EPB));
    if (share < 1.f) nvb = max(1, (int)(share * (float)gridDim.x));
  }
  if (Bv.count > 0 && (int)blockIdx.x < nvb) {
    // the producer warp returns from here when the viscous queue is empty and goes on to stage
    // inviscid tiles; the consumers return when they have finished their viscous tiles
    const int done = viscous_tiles<N, GEO, EPB, true>(M, Bv, q, smc, 0, qc);
    if (tid < NC) {
      consumer_sync(NC);  // the block's viscous results are written
      if (tid == 0) {
        __threadfence();
        atomicAdd(qc + 2, (unsigned)done);
      }
    }
  }
  if (tid < NC) {
    // release the viscous phase's shared memory to the inviscid buffer 1 (first phase of its
    // empty barrier); the bulk copies that follow are async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(smc + PI::oBAR + 56);
  }
  inviscid_tiles<N, GEO, MODE_RK, EPB, VOL, true>(M, Bi, q, out, g, stage, write_tr, smc, 32, Bi.n_indep / EPB,
                                                  qc + 1, qc + 2, nv);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(qc + 3, 1u) == gridDim.x - 1) {
      atomicExch(qc, 0u);
      atomicExch(qc + 1, 0u);
      atomicExch(qc + 2, 0u);
      atomicExch(qc + 3, 0u);
    }
  }
}

template <int N>
constexpr size_t stage_smem32() {
  return ViscTmaSmem32<N>::bytes > TmaSmem32<N>::bytes ? ViscTmaSmem32<N>::bytes : TmaSmem32<N>::bytes;
}

template <int N, int GEO>
static cudaError_t launch_stage_n(const DevMesh& M, const Bucket& bv, const Bucket& bi, const double* q, double* out,
                                  double* g, int stage, int write_tr, cudaStream_t s) {
  static int per_sm = -1, sms = 0;
  const size_t sm = stage_smem32<N>();
  if (per_sm < 0) {
    cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage32t<N, GEO>, Shape<N>::threads + 32, sm);
    if (r != cudaSuccess) return r;
    int dev = 0;
    if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  // every block resident: the grid barrier needs it, the cooperative launch guarantees it
  const int bps = bi.bps > 0 && bi.bps < per_sm ? bi.bps : per_sm;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(bps * sms));
  cfg.blockDim = dim3(Shape<N>::threads + 32);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_stage32t<N, GEO>, M, bv, bi, q, out, g, stage, write_tr);
}

template <int N, int GEO, int VOL>
static cudaError_t launch_stage_q(const DevMesh& M, const Bucket& bv, const Bucket& bi, const double* q, double* out,
                                  double* g, int stage, int write_tr, cudaStream_t s) {
  static int per_sm = -1, sms = 0;
  const size_t sm = stage_smem32<N>();
  if (per_sm < 0) {
    cudaError_t r =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage32q<N, GEO, VOL>, Shape<N>::threads + 32, sm);
    if (r != cudaSuccess) return r;
    int dev = 0;
    if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  const int bps = bi.bps > 0 && bi.bps < per_sm ? bi.bps : per_sm;
  return launch_overlapped(M, k_stage32q<N, GEO, VOL>, bps * sms, Shape<N>::threads + 32, sm, s, M, bv, bi, q, out,
                           g, stage, write_tr);
}

cudaError_t launch_stage32(const DevMesh& M, const Bucket& bv, const Bucket& bi, const double* q, double* out,
                           double* g, int stage, int write_tr, int queue, cudaStream_t s) {
  if (bi.geo > 1 || (bv.count > 0 && (bv.N != bi.N || bv.geo != bi.geo))) return cudaErrorInvalidValue;
  if (!bi.blink || !bi.bmeta || (bv.count > 0 && (!bv.blink || !bv.bmeta))) return cudaErrorInvalidValue;
  DG_SWITCH_N(bi.N, {
    if (queue) {
      if (bi.geo == 0)
        return M.div64 ? launch_stage_q<NN, 0, 3>(M, bv, bi, q, out, g, stage, write_tr, s)
                       : launch_stage_q<NN, 0, 0>(M, bv, bi, q, out, g, stage, write_tr, s);
      return launch_stage_q<NN, 1, 0>(M, bv, bi, q, out, g, stage, write_tr, s);
    }
    if (M.div64) return cudaErrorInvalidValue;  // the grid-barrier kernel has no FP64 divergence
    return bi.geo == 0 ? launch_stage_n<NN, 0>(M, bv, bi, q, out, g, stage, write_tr, s)
                       : launch_stage_n<NN, 1>(M, bv, bi, q, out, g, stage, write_tr, s);
  });
  return cudaSuccess;
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
  cudaError_t r = cudaMemcpyToSymbol(c_ops32, &o, sizeof o);
  if (r != cudaSuccess) return r;
  return cudaMemcpyToSymbol(g_D64, ops.D, sizeof ops.D);
}

template <int N, int GEO>
static size_t visc_smem32() {
  return ViscSmem32<N, GEO>::bytes;
}

// the FP64-divergence variants (VOL 3, 4) exist for box elements only
template <int N, int E, int VOL>
static cudaError_t prep_inv_div() {
  const int ps = (int)TmaSmem32<N, E, false, VOL == 4>::bytes;
  cudaError_t r;
  if ((r = cudaFuncSetAttribute(k_inviscid32t<N, 0, MODE_RESIDUAL, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps)) != cudaSuccess) return r;
  return cudaFuncSetAttribute(k_inviscid32t<N, 0, MODE_RK, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps);
}

template <int N, int E, int VOL>
static cudaError_t prep_inv() {
  const int ps = (int)TmaSmem32<N, E, false, VOL == 2>::bytes, pc = (int)TmaSmem32<N, E, VOL == 1, VOL == 2>::bytes;
  cudaError_t r;
  if ((r = cudaFuncSetAttribute(k_inviscid32t<N, 0, MODE_RESIDUAL, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32t<N, 1, MODE_RESIDUAL, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32t<N, 2, MODE_RESIDUAL, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, pc)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32t<N, 0, MODE_RK, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_inviscid32t<N, 1, MODE_RK, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps)) != cudaSuccess) return r;
  return cudaFuncSetAttribute(k_inviscid32t<N, 2, MODE_RK, E, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, pc);
}

template <int N>
static cudaError_t prep32_n() {
  cudaError_t r;
  if ((r = cudaFuncSetAttribute(k_stage32t<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem32<N>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_stage32t<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem32<N>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_stage32q<N, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem32<N>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_stage32q<N, 0, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem32<N>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_stage32q<N, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem32<N>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem32<N, 0>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem32<N, 1>())) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)visc_smem32<N, 2>())) != cudaSuccess) return r;
  constexpr int EA = AltEPB<N>::value;
  const int vs = (int)ViscTmaSmem32<N>::bytes, va = (int)ViscTmaSmem32<N, EA>::bytes;
  if ((r = cudaFuncSetAttribute(k_viscous32t<N, 0, Shape<N>::EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, vs)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32t<N, 1, Shape<N>::EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, vs)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32t<N, 0, EA>, cudaFuncAttributeMaxDynamicSharedMemorySize, va)) != cudaSuccess) return r;
  if ((r = cudaFuncSetAttribute(k_viscous32t<N, 1, EA>, cudaFuncAttributeMaxDynamicSharedMemorySize, va)) != cudaSuccess) return r;
  if ((r = prep_inv<N, Shape<N>::EPB, 0>()) != cudaSuccess) return r;
  if ((r = prep_inv<N, Shape<N>::EPB, 1>()) != cudaSuccess) return r;
  if ((r = prep_inv<N, Shape<N>::EPB, 2>()) != cudaSuccess) return r;
  if ((r = prep_inv_div<N, Shape<N>::EPB, 3>()) != cudaSuccess) return r;
  if ((r = prep_inv_div<N, Shape<N>::EPB, 4>()) != cudaSuccess) return r;
  if ((r = prep_inv_div<N, AltEPB<N>::value, 3>()) != cudaSuccess) return r;
  return prep_inv<N, AltEPB<N>::value, 0>();
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

cudaError_t launch_traces32(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  DG_SWITCH_N(b.N, {
    const int64_t tot = (int64_t)b.count * 6 * (NN + 1) * (NN + 1);
    k_traces32<NN><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, b.list, b.count, q);
  });
  return cudaGetLastError();
}

// grid of the persistent viscous kernel: every resident block slot of the GPU (or b.bps blocks
// per SM when the autotuner chose fewer), at most one per tile
template <int N, int GEO, int E>
static cudaError_t launch_vpipe(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  static int per_sm = -1, sms = 0;
  const size_t sm = ViscTmaSmem32<N, E>::bytes;
  if (per_sm < 0) {
    cudaError_t r =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_viscous32t<N, GEO, E>, Tile<N, E>::threads + 32, sm);
    if (r != cudaSuccess) return r;
    int dev = 0;
    if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    if (per_sm < 1) per_sm = 1;
  }
  const int ntiles = (b.count + E - 1) / E;
  const int bps = b.bps > 0 && b.bps < per_sm ? b.bps : per_sm;
  const int grid = ntiles < bps * sms ? ntiles : bps * sms;
  return launch_overlapped(M, k_viscous32t<N, GEO, E>, grid, Tile<N, E>::threads + 32, sm, s, M, b, q);
}

cudaError_t launch_viscous32(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  if (b.geo != 2 && b.visc_alt == 0) {  // box and affine: the pipelined kernel unless tuned away
    if (!b.blink || !b.bmeta) return cudaErrorInvalidValue;
    DG_SWITCH_N(b.N, {
      constexpr int EA = AltEPB<NN>::value, ED = Shape<NN>::EPB;
      if (b.tile_alt && EA != ED)
        return b.geo == 0 ? launch_vpipe<NN, 0, EA>(M, b, q, s) : launch_vpipe<NN, 1, EA>(M, b, q, s);
      return b.geo == 0 ? launch_vpipe<NN, 0, ED>(M, b, q, s) : launch_vpipe<NN, 1, ED>(M, b, q, s);
    });
    return cudaSuccess;
  }
  DG_SWITCH_N(b.N, {
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

// grid of the persistent kernel: every resident block slot of the GPU (or b.bps blocks per SM
// when the autotuner chose fewer), at most one per tile
template <int N, int GEO, int MODE, int E, int VOL>
static cudaError_t launch_pipe(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                               int stage, int write_tr, cudaStream_t s) {
  static int per_sm = -1, sms = 0;
  const size_t sm = TmaSmem32<N, E, VOL == 1 && GEO == 2, VOL == 2 || VOL == 4>::bytes;
  if (per_sm < 0) {
    cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inviscid32t<N, GEO, MODE, E, VOL>,
                                                                  Tile<N, E>::threads + 32, sm);
    if (r != cudaSuccess) return r;
    int dev = 0;
    if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    if (per_sm < 1) per_sm = 1;
  }
  const int ntiles = (b.count + E - 1) / E;
  const int bps = b.bps > 0 && b.bps < per_sm ? b.bps : per_sm;
  const int grid = ntiles < bps * sms ? ntiles : bps * sms;
  return launch_overlapped(M, k_inviscid32t<N, GEO, MODE, E, VOL>, grid, Tile<N, E>::threads + 32, sm, s, M, b, q,
                           out, g, stage, write_tr);
}

template <int N, int E, int VOL>
static cudaError_t launch_inv_shape(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                                   int mode, int stage, int write_tr, cudaStream_t s) {
  if (mode == MODE_RESIDUAL) {
    if (b.geo == 0) return launch_pipe<N, 0, MODE_RESIDUAL, E, VOL>(M, b, q, out, g, stage, write_tr, s);
    if (b.geo == 1) return launch_pipe<N, 1, MODE_RESIDUAL, E, VOL>(M, b, q, out, g, stage, write_tr, s);
    return launch_pipe<N, 2, MODE_RESIDUAL, E, VOL>(M, b, q, out, g, stage, write_tr, s);
  }
  if (b.geo == 0) return launch_pipe<N, 0, MODE_RK, E, VOL>(M, b, q, out, g, stage, write_tr, s);
  if (b.geo == 1) return launch_pipe<N, 1, MODE_RK, E, VOL>(M, b, q, out, g, stage, write_tr, s);
  return launch_pipe<N, 2, MODE_RK, E, VOL>(M, b, q, out, g, stage, write_tr, s);
}

// box buckets with the FP64 divergence (VOL 3 from 0, 4 from 2); other buckets run VOL 0 or 2
template <int N, int E, int VOL>
static cudaError_t launch_inv_div(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                                  int mode, int stage, int write_tr, cudaStream_t s) {
  if (b.geo != 0) return launch_inv_shape<N, E, VOL == 3 ? 0 : 2>(M, b, q, out, g, mode, stage, write_tr, s);
  if (mode == MODE_RESIDUAL) return launch_pipe<N, 0, MODE_RESIDUAL, E, VOL>(M, b, q, out, g, stage, write_tr, s);
  return launch_pipe<N, 0, MODE_RK, E, VOL>(M, b, q, out, g, stage, write_tr, s);
}

int tile_epb32(int N, int alt) {
  switch (N) {
    case 1: return alt ? AltEPB<1>::value : Shape<1>::EPB;
    case 2: return alt ? AltEPB<2>::value : Shape<2>::EPB;
    case 3: return alt ? AltEPB<3>::value : Shape<3>::EPB;
    case 4: return alt ? AltEPB<4>::value : Shape<4>::EPB;
    case 5: return alt ? AltEPB<5>::value : Shape<5>::EPB;
    case 6: return alt ? AltEPB<6>::value : Shape<6>::EPB;
    case 7: return alt ? AltEPB<7>::value : Shape<7>::EPB;
    default: return 0;
  }
}

cudaError_t launch_inviscid32(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g, int mode,
                              int stage, int write_tr, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  if (!b.boff || !b.btr || !b.blink || !b.bflag || !b.bmeta) return cudaErrorInvalidValue;
  DG_SWITCH_N(b.N, {
    // the split form and the tensor-core contraction are built for the default tile shape; the
    // split form's two-point sums are no plain contraction and stay on the FP32 pipe
    if (M.split == 1) return launch_inv_shape<NN, Shape<NN>::EPB, 1>(M, b, q, out, g, mode, stage, write_tr, s);
    if (M.tc) {
      if (M.div64) return launch_inv_div<NN, Shape<NN>::EPB, 4>(M, b, q, out, g, mode, stage, write_tr, s);
      return launch_inv_shape<NN, Shape<NN>::EPB, 2>(M, b, q, out, g, mode, stage, write_tr, s);
    }
    if (b.tile_alt) {
      if (M.div64) return launch_inv_div<NN, AltEPB<NN>::value, 3>(M, b, q, out, g, mode, stage, write_tr, s);
      return launch_inv_shape<NN, AltEPB<NN>::value, 0>(M, b, q, out, g, mode, stage, write_tr, s);
    }
    if (M.div64) return launch_inv_div<NN, Shape<NN>::EPB, 3>(M, b, q, out, g, mode, stage, write_tr, s);
    return launch_inv_shape<NN, Shape<NN>::EPB, 0>(M, b, q, out, g, mode, stage, write_tr, s);
  });
  return cudaSuccess;
}

}  // namespace dgk
