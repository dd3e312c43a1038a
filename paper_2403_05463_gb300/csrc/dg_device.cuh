// dg_device.cuh -- device helpers shared by the FP64 and FP32 kernel files.
#pragma once
#include "dg_internal.h"

namespace dgk {

// Runs the statements with the compile-time order NN = NVAR (1..MAXN); other values return
// cudaErrorInvalidValue from the enclosing launcher.
#define DG_SWITCH_N(NVAR, ...)                                  \
  switch (NVAR) {                                               \
    case 1: { constexpr int NN = 1; __VA_ARGS__; } break;       \
    case 2: { constexpr int NN = 2; __VA_ARGS__; } break;       \
    case 3: { constexpr int NN = 3; __VA_ARGS__; } break;       \
    case 4: { constexpr int NN = 4; __VA_ARGS__; } break;       \
    case 5: { constexpr int NN = 5; __VA_ARGS__; } break;       \
    case 6: { constexpr int NN = 6; __VA_ARGS__; } break;       \
    case 7: { constexpr int NN = 7; __VA_ARGS__; } break;       \
    default: return cudaErrorInvalidValue;                      \
  }

template <int N>
struct Shape {
  static constexpr int n = N + 1, n2 = n * n, n3 = n * n * n;
  static constexpr int EPB = (256 / n3) > 0 ? (256 / n3) : 1;   // elements per block
  static constexpr int threads = ((EPB * n3 + 31) / 32) * 32;
};

// Weights of the own and the neighbour's outward viscous traces (tau . S) in the face term
// F_v,own . S - F_v* . S. BR1 averages: (1/2, 1/2). With the one-sided choice on a face between
// an NS and an Euler element, F_v* is the NS side's flux: the NS side's term vanishes (0, 0)
// and the Euler side takes the whole neighbour flux (1, 1; its own trace is zero).
__host__ __device__ __forceinline__ void visc_face_weights(int mixed_face, bool own_ns, bool nbr_ns, float& wo,
                                                           float& wn) {
  const bool one = mixed_face == 1 && own_ns != nbr_ns;
  wo = one ? (own_ns ? 0.f : 1.f) : 0.5f;
  wn = one ? (own_ns ? 0.f : 1.f) : 0.5f;
}

// Velocity jump u_ghost - u behind a wall face with area-weighted outward normal S: -2u at a
// no-slip wall, -2 (u.n) n at a free-slip one.
template <typename T>
__device__ __forceinline__ void wall_jump(int kind, const T u[3], const T S[3], T jump[3]) {
  if (kind == FK_WALL) {
#pragma unroll
    for (int c = 0; c < 3; ++c) jump[c] = T(-2) * u[c];
  } else {
    const T us = (u[0] * S[0] + u[1] * S[1] + u[2] * S[2]) / (S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) jump[c] = T(-2) * us * S[c];
  }
}

// The viscous face term F_v,own . S - F_v* . S behind a free-slip wall (F_v* keeps only the
// normal part of the traction): the tangential part of the own outward trace t = tau . S.
template <typename T>
__device__ __forceinline__ void slip_visc_term(const T t[3], const T S[3], T out[3]) {
  const T ts = (t[0] * S[0] + t[1] * S[1] + t[2] * S[2]) / (S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = t[c] - ts * S[c];
}

// y = A(ub) x for the artificial-compressibility flux Jacobian in direction nh
__device__ __forceinline__ void ac_jac_apply(const double ub[3], double un, const double nh[3],
                                             double c0sq, const double x[4], double y[4]) {
  double nx = nh[0] * x[1] + nh[1] * x[2] + nh[2] * x[3];
  y[0] = c0sq * nx;
#pragma unroll
  for (int c = 0; c < 3; ++c) y[1 + c] = nh[c] * x[0] + ub[c] * nx + un * x[1 + c];
}

// Fluctuation A^-(qbar) dq = (F* - F_n(q-)) for Roe (riemann == 0): the flux is quadratic,
// so F(q+) - F(q-) = A(qbar) dq exactly with qbar the arithmetic mean, and |A| is the
// quadratic polynomial in A that matches |lambda| on the three distinct eigenvalues
// u_n - a, u_n, u_n + a (a = sqrt(u_n^2 + c0^2)). For LLF: 1/2 (A dq - lambda_max dq).
__device__ __forceinline__ void flux_fluct(const double qm[4], const double qp[4], const double nh[3],
                                           double c0sq, int riemann, double out[4]) {
  double dq[4], ub[3];
#pragma unroll
  for (int v = 0; v < 4; ++v) dq[v] = qp[v] - qm[v];
#pragma unroll
  for (int c = 0; c < 3; ++c) ub[c] = 0.5 * (qm[1 + c] + qp[1 + c]);
  double un = ub[0] * nh[0] + ub[1] * nh[1] + ub[2] * nh[2];
  double y1[4];
  ac_jac_apply(ub, un, nh, c0sq, dq, y1);
  if (riemann == 0) {
    double y2[4];
    ac_jac_apply(ub, un, nh, c0sq, y1, y2);
    double a = sqrt(un * un + c0sq);
    double aun = fabs(un);
    double lm = un - a, l0 = un;
    double d1 = (aun + un - a) / a;        // divided difference of |.| on (lm, l0)
    double d2 = (a - aun) / (a * a);       // second divided difference on (lm, l0, lp)
    double k0 = -lm - d1 * lm + d2 * lm * l0;
    double k1 = d1 - d2 * (lm + l0);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.5 * (y1[v] - (k0 * dq[v] + k1 * y1[v] + d2 * y2[v]));
  } else {
    double unm = qm[1] * nh[0] + qm[2] * nh[1] + qm[3] * nh[2];
    double unp = qp[1] * nh[0] + qp[2] * nh[1] + qp[3] * nh[2];
    double lam = fmax(fabs(unm) + sqrt(unm * unm + c0sq), fabs(unp) + sqrt(unp * unp + c0sq));
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.5 * (y1[v] - lam * dq[v]);
  }
}

// LES eddy viscosity from G[c][k] = d u_c / d x_k (App. A: Vreman; Smagorinsky alternative).
__device__ __forceinline__ double eddy_visc(const double G[3][3], double delta, int closure, double cs,
                                            double cv) {
  if (closure == 0) {
    double s2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double s = 0.5 * (G[c][k] + G[k][c]);
        s2 += s * s;
      }
    double l = cs * delta;
    return l * l * sqrt(2.0 * s2);
  }
  // Vreman: alpha_ij = d u_j / d x_i = G[j][i]; beta = delta^2 alpha^T alpha
  double aa = 0.0, b[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      aa += G[j][i] * G[j][i];
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < 3; ++m) s += G[i][m] * G[j][m];  // alpha_mi alpha_mj = G[i][m] G[j][m]
      b[i][j] = delta * delta * s;
    }
  double B = b[0][0] * b[1][1] - b[0][1] * b[0][1] + b[0][0] * b[2][2] - b[0][2] * b[0][2] +
             b[1][1] * b[2][2] - b[1][2] * b[1][2];
  if (aa < 1e-300 || B <= 0.0) return 0.0;
  return cv * sqrt(B / aa);
}

// volume node of face f = 2d+s at face coordinates (a, b)
__host__ __device__ __forceinline__ int face_node(int f, int n, int a, int b) {
  int d = f >> 1, fix = (f & 1) ? n - 1 : 0;
  if (d == 0) return fix + n * (a + n * b);
  if (d == 1) return a + n * (fix + n * b);
  return a + n * (b + n * fix);
}

// volume node at position i along the normal line of face f through face coordinates (a, b)
// (face_node is the node of that line on the face)
__host__ __device__ __forceinline__ int line_node(int f, int n, int a, int b, int i) {
  const int d = f >> 1;
  if (d == 0) return i + n * (a + n * b);
  if (d == 1) return a + n * (i + n * b);
  return a + n * (b + n * i);
}

// my face coordinates (a, b) at order N -> neighbour's (a1, b1)
__device__ __forceinline__ void inv_orient(int o, int N, int a, int b, int& a1, int& b1) {
  int x = (o & 2) ? N - a : a;
  int y = (o & 4) ? N - b : b;
  if (o & 1) { a1 = y; b1 = x; } else { a1 = x; b1 = y; }
}

// neighbour face coordinates (a1, b1) at order M -> mine
__device__ __forceinline__ void fwd_orient(int o, int M, int a1, int b1, int& a0, int& b0) {
  int x = (o & 1) ? b1 : a1, y = (o & 1) ? a1 : b1;
  a0 = (o & 2) ? M - x : x;
  b0 = (o & 4) ? M - y : y;
}

// Splits x into FP32 hi + lo: hi is x truncated to 24 significant bits, lo the remainder
// rounded to 24 bits, so |x - hi - lo| <= 2^-48 |x| for 2^-74 <= |x| < 2^128. Uses integer
// and FP32 instructions only (no FP64 pipe), without branches: the 29 mantissa bits below hi
// are converted to FP32 with one rounding (integer-to-float conversion) and scaled by a power
// of two. |x| < 2^-126 gives 0; |x| >= 2^128, inf or NaN give a NaN hi.
__device__ __forceinline__ void split_hilo(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned top = (unsigned)(b >> 32);
  const unsigned sign = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7ffu);
  const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  hi = e < 897 ? 0.f : (e > 1150 ? __int_as_float(0x7fc00000) : h);
  const unsigned m = (unsigned)(b & 0x1fffffffu);
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075), for e >= 949
  const float l = __uint_as_float(__float_as_uint(__uint2float_rn(m) * scale) | sign);
  lo = (e < 949 || e > 1150) ? 0.f : l;
}

// Exact FP32 -> FP64 widening with integer instructions only (GB300 runs FP32<->FP64
// conversions on the FP64 pipe, 1/64 of the FP32 rate): the exponent is re-biased from 127 to
// 1023 and the 23-bit mantissa moved to the top of the 52-bit field. FP32 subnormals
// (|x| < 2^-126) become a signed zero; infinities and NaNs stay infinities and NaNs.
__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned ew = e == 0xffu ? 0x7ffu : e + 896u;
  const unsigned hi = e == 0u ? sign : (sign | (ew << 20) | (m >> 3));
  const unsigned lo = e == 0u ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

}  // namespace dgk
