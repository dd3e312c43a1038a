// dg_cns_phys.cuh -- pointwise physics of the compressible form (arXiv 2403.05463, App. A)
// shared by its Gauss-Lobatto and Gauss-Legendre kernels: primitive variables, the Euler
// flux along a normal, and the Roe (or LLF) fluctuation.
#pragma once
#include "dg_device.cuh"

namespace dgk {

struct Prim {
  double rho, v[3], p;
};

__device__ __forceinline__ Prim prim(const double u[5], double gamma) {
  Prim P;
  P.rho = u[0];
  const double ir = 1.0 / u[0];
#pragma unroll
  for (int c = 0; c < 3; ++c) P.v[c] = u[1 + c] * ir;
  P.p = (gamma - 1.0) * (u[4] - 0.5 * (u[1] * P.v[0] + u[2] * P.v[1] + u[3] * P.v[2]));
  return P;
}

// Fluctuation F*(uL, uR) . n - F(uL) . n. Roe (riemann == 0) in wave-strength form with the
// Roe averages (sqrt(rho)-weighted v and H, a^2 = (gamma - 1)(H - |v|^2/2)): the jump uR - uL
// is split into two acoustic waves (vn -+ a), an entropy wave and the shear part (vn), each
// weighted by |lambda|. LLF: the largest |vn| + a of the two sides.
__device__ __forceinline__ void cns_fluct(const double uL[5], const double uR[5], const double nh[3], double gamma,
                                          int riemann, double fx[5]) {
  const Prim L = prim(uL, gamma), R = prim(uR, gamma);
  const double vnL = L.v[0] * nh[0] + L.v[1] * nh[1] + L.v[2] * nh[2];
  const double vnR = R.v[0] * nh[0] + R.v[1] * nh[1] + R.v[2] * nh[2];
  double dF[5];  // F(uR).n - F(uL).n
  dF[0] = uR[0] * vnR - uL[0] * vnL;
#pragma unroll
  for (int c = 0; c < 3; ++c) dF[1 + c] = (uR[1 + c] * vnR + R.p * nh[c]) - (uL[1 + c] * vnL + L.p * nh[c]);
  dF[4] = (uR[4] + R.p) * vnR - (uL[4] + L.p) * vnL;
  if (riemann == 0) {
    const double sL = sqrt(L.rho), sR = sqrt(R.rho), inv = 1.0 / (sL + sR);
    const double HL = (uL[4] + L.p) / L.rho, HR = (uR[4] + R.p) / R.rho;
    double v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = (sL * L.v[c] + sR * R.v[c]) * inv;
    const double H = (sL * HL + sR * HR) * inv;
    const double q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double a2 = (gamma - 1.0) * (H - 0.5 * q2), a = sqrt(a2);
    const double vn = v[0] * nh[0] + v[1] * nh[1] + v[2] * nh[2];
    const double rho = sL * sR;
    const double dr = R.rho - L.rho, dp = R.p - L.p;
    double dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dv[c] = R.v[c] - L.v[c];
    const double dvn = dv[0] * nh[0] + dv[1] * nh[1] + dv[2] * nh[2];
    const double al1 = (dp - rho * a * dvn) / (2.0 * a2);  // acoustic, vn - a
    const double al5 = (dp + rho * a * dvn) / (2.0 * a2);  // acoustic, vn + a
    const double al2 = dr - dp / a2;                       // entropy, vn
    const double l1 = fabs(vn - a), l2 = fabs(vn), l5 = fabs(vn + a);
    const double w1 = l1 * al1, w5 = l5 * al5;
    double d[5];
    d[0] = w1 + l2 * al2 + w5;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      d[1 + c] = w1 * (v[c] - a * nh[c]) + l2 * (al2 * v[c] + rho * (dv[c] - dvn * nh[c])) + w5 * (v[c] + a * nh[c]);
    const double vdv = v[0] * dv[0] + v[1] * dv[1] + v[2] * dv[2];
    d[4] = w1 * (H - a * vn) + l2 * (al2 * 0.5 * q2 + rho * (vdv - vn * dvn)) + w5 * (H + a * vn);
#pragma unroll
    for (int k = 0; k < 5; ++k) fx[k] = 0.5 * (dF[k] - d[k]);
  } else {
    const double lam = fmax(fabs(vnL) + sqrt(gamma * L.p / L.rho), fabs(vnR) + sqrt(gamma * R.p / R.rho));
#pragma unroll
    for (int k = 0; k < 5; ++k) fx[k] = 0.5 * (dF[k] - lam * (uR[k] - uL[k]));
  }
}

// F(u) . n of the Euler flux
__device__ __forceinline__ void cns_normal_flux(const double u[5], const double nh[3], double gamma, double F[5]) {
  const Prim P = prim(u, gamma);
  const double vn = P.v[0] * nh[0] + P.v[1] * nh[1] + P.v[2] * nh[2];
  F[0] = u[0] * vn;
#pragma unroll
  for (int c = 0; c < 3; ++c) F[1 + c] = u[1 + c] * vn + P.p * nh[c];
  F[4] = (u[4] + P.p) * vn;
}

}  // namespace dgk
