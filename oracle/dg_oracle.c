/*
 * dg_oracle.c -- plain FP64 CPU oracle for the flagged Euler / NS-LES DGSEM residual.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
 * CPU-baseline leg. The CUDA library never links, includes or calls it, and it shares no
 * code with that library. Everything here is deliberately direct: no blocking, no fusion,
 * no reordering beyond what the discretisation states.
 *
 * Discretisation (arXiv 2403.05463, App. B, Eqs. NS2-NS5) on Gauss-Lobatto nodes:
 *   weak form per element, integrated with the tensor-product quadrature,
 *     w J dq/dt = sum_d (1/w_{i_d}) sum_m w_m D_{m i_d} Ftil^d_m  -  sum_faces (1/w_end) H*
 *   with Ftil^d the contravariant (Ja^d-weighted) total flux F_e - F_v,turb and H* the
 *   area-weighted outward numerical flux F_e* - F_v* on each face (projected from the
 *   mortar when the two sides have different orders).
 * Sec. 2.3: Euler elements omit every viscous/turbulent term; convective terms everywhere;
 * faces couple with Roe (convective) and BR1 (viscous). Reading for an Euler/NS face: the
 * single-valued BR1 flux is the average of the NS side's viscous flux and zero.
 */
#include "dg_oracle.h"
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(OR_EXTENDED) && OR_EXTENDED
#define SQRT sqrtl
#define FABS fabsl
#define COS cosl
#define CBRT cbrtl
#define PI_R 3.141592653589793238462643383279502884L
#else
#define SQRT sqrt
#define FABS fabs
#define COS cos
#define CBRT cbrt
#define PI_R M_PI
#endif

#define OR_MAXN 15
#define OR_MAXG 4

static __thread char g_err[512];
static void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
const char* or_error(void) { return g_err; }

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------------------
 * 1D: Gauss-Lobatto-Legendre nodes and weights, differentiation, interpolation,
 * L2 projection. (Quadrature of App. B, last paragraph; Gauss-Lobatto variant.)
 * ---------------------------------------------------------------------------------- */

/* Legendre polynomials L_{N-1}, L_N, L_{N+1} at x by the three-term recurrence
 * (k+1) L_{k+1} = (2k+1) x L_k - k L_{k-1}, L_0 = 1, L_1 = x. */
static void legendre3(int N, or_real x, or_real* Lm1, or_real* L0, or_real* Lp1) {
  or_real lkm1 = 0.0, lk = 1.0; /* L_{-1} (unused), L_0 */
  or_real lkp1 = x;             /* L_1 */
  for (int k = 1; k <= N; ++k) {
    lkm1 = lk;
    lk = lkp1;
    lkp1 = ((2.0 * k + 1.0) * x * lk - k * lkm1) / (k + 1.0);
  }
  /* after the loop: lkm1 = L_{N-1}, lk = L_N, lkp1 = L_{N+1} */
  *Lm1 = lkm1;
  *L0 = lk;
  *Lp1 = lkp1;
}

int or_lgl(int N, or_real* x, or_real* w) {
  if (N < 1 || N > OR_MAXN) {
    set_err("order %d outside 1..%d", N, OR_MAXN);
    return -1;
  }
  x[0] = -1.0;
  x[N] = 1.0;
  /* interior nodes: roots of L_{N+1} - L_{N-1} (proportional to (1-x^2) L'_N);
   * Newton from Chebyshev-Gauss-Lobatto guesses, d/dx (L_{N+1}-L_{N-1}) = (2N+1) L_N. */
  for (int j = 1; j < N; ++j) {
    or_real xj = -COS(PI_R * j / N);
    for (int it = 0; it < 200; ++it) {
      or_real lm1, l0, lp1;
      legendre3(N, xj, &lm1, &l0, &lp1);
      or_real dx = (lp1 - lm1) / ((2.0 * N + 1.0) * l0);
      xj -= dx;
      if (FABS(dx) <= 1e-17) break;
    }
    x[j] = xj;
  }
  /* enforce the exact symmetry of the node set */
  for (int j = 0; j < (N + 1) / 2; ++j) {
    or_real s = 0.5 * (x[N - j] - x[j]);
    x[j] = -s;
    x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    or_real lm1, l0, lp1;
    legendre3(N, x[j], &lm1, &l0, &lp1);
    w[j] = 2.0 / (N * (N + 1.0) * l0 * l0);
  }
  return 0;
}

/* Gauss-Legendre nodes (the N+1 roots of L_{N+1}) and weights 2 / ((1 - x^2) L'_{N+1}(x)^2),
 * Newton from the guesses -cos(pi (j + 3/4) / (N + 3/2)); L'_{N+1} = (N+1)(x L_{N+1} - L_N)/(x^2 - 1). */
int or_gl(int N, or_real* x, or_real* w) {
  if (N < 1 || N > OR_MAXN) {
    set_err("order %d outside 1..%d", N, OR_MAXN);
    return -1;
  }
  for (int j = 0; j <= N; ++j) {
    or_real xj = -COS(PI_R * (j + 0.75) / (N + 1.5));
    for (int it = 0; it < 200; ++it) {
      or_real lm1, l0, lp1;
      legendre3(N, xj, &lm1, &l0, &lp1);
      const or_real dl = (N + 1.0) * (xj * lp1 - l0) / (xj * xj - 1.0);
      const or_real dx = lp1 / dl;
      xj -= dx;
      if (FABS(dx) <= 1e-17) break;
    }
    x[j] = xj;
  }
  for (int j = 0; j < (N + 1) / 2; ++j) {
    or_real s = 0.5 * (x[N - j] - x[j]);
    x[j] = -s;
    x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    or_real lm1, l0, lp1;
    legendre3(N, x[j], &lm1, &l0, &lp1);
    const or_real dl = (N + 1.0) * (x[j] * lp1 - l0) / (x[j] * x[j] - 1.0);
    w[j] = 2.0 / ((1.0 - x[j] * x[j]) * dl * dl);
  }
  return 0;
}

/* Lagrange basis l_j(y) on nodes xs[0..n-1] by the product formula. */
static or_real lagrange(int n, const or_real* xs, int j, or_real y) {
  or_real v = 1.0;
  for (int k = 0; k < n; ++k)
    if (k != j) v *= (y - xs[k]) / (xs[j] - xs[k]);
  return v;
}

/* D_ij = l_j'(x_i) on the nodes x[0..n-1], barycentric form */
static void dmat_nodes(int n, const or_real* x, or_real* D) {
  or_real lam[OR_MAXN + 1];
  /* barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k) */
  for (int j = 0; j < n; ++j) {
    or_real p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (x[j] - x[k]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < n; ++i) {
    or_real s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * n + j];
    }
    D[i * n + i] = -s;
  }
}

int or_dmat(int N, or_real* D) {
  or_real x[OR_MAXN + 1], w[OR_MAXN + 1];
  if (or_lgl(N, x, w)) return -1;
  dmat_nodes(N + 1, x, D);
  return 0;
}

int or_dmat_gl(int N, or_real* D) {
  or_real x[OR_MAXN + 1], w[OR_MAXN + 1];
  if (or_gl(N, x, w)) return -1;
  dmat_nodes(N + 1, x, D);
  return 0;
}

/* the rule of a node set: 0 Gauss-Lobatto, 1 Gauss-Legendre */
static int node_set(int gl, int N, or_real* x, or_real* w) { return gl ? or_gl(N, x, w) : or_lgl(N, x, w); }

/* I[i][j] = l_j(x_i): the degree-Ns interpolant through the source nodes, evaluated at the
 * destination nodes (both of the same node set) */
static int interp_nodes(int gl, int Ns, int Nd, or_real* I) {
  or_real xs[OR_MAXN + 1], ws[OR_MAXN + 1], xd[OR_MAXN + 1], wd[OR_MAXN + 1];
  if (node_set(gl, Ns, xs, ws) || node_set(gl, Nd, xd, wd)) return -1;
  for (int i = 0; i <= Nd; ++i)
    for (int j = 0; j <= Ns; ++j) I[i * (Ns + 1) + j] = lagrange(Ns + 1, xs, j, xd[i]);
  return 0;
}

int or_interp_lgl(int Ns, int Nd, or_real* I) { return interp_nodes(0, Ns, Nd, I); }
int or_interp_gl(int Ns, int Nd, or_real* I) { return interp_nodes(1, Ns, Nd, I); }

/* Solve A X = B in place (A n x n, B n x m, row-major) by Gauss-Jordan with partial
 * pivoting. Returns -1 if A is singular. */
static int gauss_jordan(int n, or_real* A, int m, or_real* B) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (FABS(A[r * n + c]) > FABS(A[piv * n + c])) piv = r;
    if (FABS(A[piv * n + c]) < 1e-300) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        or_real t = A[c * n + k];
        A[c * n + k] = A[piv * n + k];
        A[piv * n + k] = t;
      }
      for (int k = 0; k < m; ++k) {
        or_real t = B[c * m + k];
        B[c * m + k] = B[piv * m + k];
        B[piv * m + k] = t;
      }
    }
    or_real d = A[c * n + c];
    for (int k = 0; k < n; ++k) A[c * n + k] /= d;
    for (int k = 0; k < m; ++k) B[c * m + k] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      or_real f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
    }
  }
  return 0;
}

/* L2 projection from the degree-Nh polynomial given at its Gauss-Lobatto nodes onto
 * degree Nl <= Nh: P = M_l^{-1} I^T W_h, where I interpolates Nl -> Nh nodes and
 * M_l = I^T W_h I is the exact mass matrix (Nh-point Lobatto quadrature is exact for
 * degree 2 Nl <= 2 Nh - 1 when Nh > Nl). For Nh == Nl, P is the identity. */
/* L2 projection of a degree-Nh nodal polynomial onto degree Nl, both on the same node set:
 * P = M^-1 B with the mass matrix M_ab = (l_a, l_b) and B_aj = (l_a, L_j) of the low (l) and
 * high (L) Lagrange bases, both integrated exactly by the high rule (degree <= 2 Nh - 1 for
 * Lobatto, 2 Nh + 1 for Legendre, and the integrands have degree <= Nl + Nh) */
static int project_nodes(int gl, int Nh, int Nl, or_real* P) {
  int nh = Nh + 1, nl = Nl + 1;
  if (Nl > Nh) {
    set_err("projection needs Nl <= Nh");
    return -1;
  }
  if (Nh == Nl) {
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < nh; ++j) P[i * nh + j] = (i == j) ? 1.0 : 0.0;
    return 0;
  }
  or_real xh[OR_MAXN + 1], wh[OR_MAXN + 1];
  or_real I[(OR_MAXN + 1) * (OR_MAXN + 1)];
  or_real M[(OR_MAXN + 1) * (OR_MAXN + 1)];
  if (node_set(gl, Nh, xh, wh) || interp_nodes(gl, Nl, Nh, I)) return -1;
  for (int a = 0; a < nl; ++a)
    for (int b = 0; b < nl; ++b) {
      or_real s = 0.0;
      for (int j = 0; j < nh; ++j) s += I[j * nl + a] * wh[j] * I[j * nl + b];
      M[a * nl + b] = s;
    }
  for (int a = 0; a < nl; ++a)
    for (int j = 0; j < nh; ++j) P[a * nh + j] = I[j * nl + a] * wh[j];
  if (gauss_jordan(nl, M, nh, P)) {
    set_err("singular mass matrix");
    return -1;
  }
  return 0;
}

int or_project_lgl(int Nh, int Nl, or_real* P) { return project_nodes(0, Nh, Nl, P); }
int or_project_gl(int Nh, int Nl, or_real* P) { return project_nodes(1, Nh, Nl, P); }

/* ------------------------------------------------------------------------------------
 * Pointwise physics (App. A in artificial-compressibility form, rho = 1).
 *   F_e in direction x_k: (c0^2 u_k, u u_k + p e_1k, v u_k + p e_2k, w u_k + p e_3k)
 *   tau = (nu + nu_t)(G + G^T) - 2/3 (nu + nu_t) tr(G) I,  G_ck = d u_c / d x_k
 * ---------------------------------------------------------------------------------- */

void or_normal_flux(const or_real q[4], const or_real nh[3], or_real c0sq, or_real out[4]) {
  or_real un = q[1] * nh[0] + q[2] * nh[1] + q[3] * nh[2];
  out[0] = c0sq * un;
  for (int c = 0; c < 3; ++c) out[1 + c] = q[1 + c] * un + q[0] * nh[c];
}

/* A = d F_n / d q, rows/cols ordered (p, u, v, w). */
void or_flux_jacobian(const or_real q[4], const or_real nh[3], or_real c0sq, or_real A[16]) {
  or_real un = q[1] * nh[0] + q[2] * nh[1] + q[3] * nh[2];
  memset(A, 0, 16 * sizeof(or_real));
  for (int c = 0; c < 3; ++c) A[0 * 4 + 1 + c] = c0sq * nh[c];
  for (int r = 0; r < 3; ++r) {
    A[(1 + r) * 4 + 0] = nh[r];
    for (int c = 0; c < 3; ++c) A[(1 + r) * 4 + 1 + c] = q[1 + r] * nh[c] + (r == c ? un : 0.0);
  }
}

/* |A| = R |Lambda| R^{-1} from the explicit eigen-decomposition of A:
 *   lambda = u_n (twice, eigenvectors (0, t) with t tangent to the face),
 *   lambda = u_n +- SQRT(u_n^2 + c0^2), eigenvectors with n . u_hat = 1,
 *     p_hat = lambda - 2 u_n, u_hat = (n p_hat + u) / (lambda - u_n).
 * R^{-1} is formed numerically (Gauss-Jordan), not from a closed form. */
int or_abs_jacobian(const or_real q[4], const or_real nh[3], or_real c0sq, or_real absA[16]) {
  or_real un = q[1] * nh[0] + q[2] * nh[1] + q[3] * nh[2];
  or_real a = SQRT(un * un + c0sq);
  or_real lam[4] = {un, un, un + a, un - a};
  /* tangent vectors: t1 = normalize(e x n) with e the axis least aligned with n */
  int ax = 0;
  if (FABS(nh[1]) < FABS(nh[ax])) ax = 1;
  if (FABS(nh[2]) < FABS(nh[ax])) ax = 2;
  or_real e[3] = {0, 0, 0};
  e[ax] = 1.0;
  or_real t1[3] = {e[1] * nh[2] - e[2] * nh[1], e[2] * nh[0] - e[0] * nh[2], e[0] * nh[1] - e[1] * nh[0]};
  or_real l1 = SQRT(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int c = 0; c < 3; ++c) t1[c] /= l1;
  or_real t2[3] = {nh[1] * t1[2] - nh[2] * t1[1], nh[2] * t1[0] - nh[0] * t1[2], nh[0] * t1[1] - nh[1] * t1[0]};
  or_real R[16], Rinv[16], Rw[16];
  /* column k of R = eigenvector k */
  for (int r = 0; r < 4; ++r) R[r * 4 + 0] = (r == 0) ? 0.0 : t1[r - 1];
  for (int r = 0; r < 4; ++r) R[r * 4 + 1] = (r == 0) ? 0.0 : t2[r - 1];
  for (int k = 2; k < 4; ++k) {
    or_real ph = lam[k] - 2.0 * un;
    R[0 * 4 + k] = ph;
    for (int c = 0; c < 3; ++c) R[(1 + c) * 4 + k] = (nh[c] * ph + q[1 + c]) / (lam[k] - un);
  }
  memcpy(Rw, R, sizeof R);
  for (int i = 0; i < 16; ++i) Rinv[i] = (i % 5 == 0) ? 1.0 : 0.0;
  if (gauss_jordan(4, Rw, 4, Rinv)) {
    set_err("singular eigenvector matrix");
    return -1;
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      or_real s = 0.0;
      for (int k = 0; k < 4; ++k) s += R[i * 4 + k] * FABS(lam[k]) * Rinv[k * 4 + j];
      absA[i * 4 + j] = s;
    }
  return 0;
}

/* Convective numerical flux through a face with unit normal nh pointing from the
 * qm side to the qp side (Sec. 2.3: Roe; LLF as the alternative flux). */
void or_kep_flux(const or_real qi[4], const or_real qm[4], const or_real Ja_i[3], const or_real Ja_m[3],
                 or_real c0sq, or_real out[4]) {
  or_real ja[3], u[3];
  for (int k = 0; k < 3; ++k) {
    ja[k] = 0.5 * (Ja_i[k] + Ja_m[k]);
    u[k] = 0.5 * (qi[1 + k] + qm[1 + k]);
  }
  const or_real p = 0.5 * (qi[0] + qm[0]);
  const or_real U = ja[0] * u[0] + ja[1] * u[1] + ja[2] * u[2];
  out[0] = c0sq * U;
  for (int c = 0; c < 3; ++c) out[1 + c] = u[c] * U + p * ja[c];
}

int or_riemann(const or_real qm[4], const or_real qp[4], const or_real nh[3], const or_params* prm,
               or_real out[4]) {
  or_real fm[4], fp[4];
  or_normal_flux(qm, nh, prm->c0sq, fm);
  or_normal_flux(qp, nh, prm->c0sq, fp);
  if (prm->riemann == 0) {
    or_real qb[4], absA[16];
    for (int v = 0; v < 4; ++v) qb[v] = 0.5 * (qm[v] + qp[v]);
    if (or_abs_jacobian(qb, nh, prm->c0sq, absA)) return -1;
    for (int v = 0; v < 4; ++v) {
      or_real d = 0.0;
      for (int k = 0; k < 4; ++k) d += absA[v * 4 + k] * (qp[k] - qm[k]);
      out[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * d;
    }
  } else {
    or_real unm = qm[1] * nh[0] + qm[2] * nh[1] + qm[3] * nh[2];
    or_real unp = qp[1] * nh[0] + qp[2] * nh[1] + qp[3] * nh[2];
    or_real sm = FABS(unm) + SQRT(unm * unm + prm->c0sq);
    or_real sp = FABS(unp) + SQRT(unp * unp + prm->c0sq);
    or_real s = sm > sp ? sm : sp;
    for (int v = 0; v < 4; ++v) out[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * s * (qp[v] - qm[v]);
  }
  return 0;
}

/* LES eddy viscosity (App. A, Eq. for the Vreman model; Smagorinsky as the alternative
 * closure): G[c*3+k] = d u_c / d x_k, delta the filter width. */
or_real or_eddy_viscosity(const or_real G[9], or_real delta, const or_params* prm) {
  if (prm->closure == 0) {
    or_real ss = 0.0;
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 3; ++k) {
        or_real s = 0.5 * (G[c * 3 + k] + G[k * 3 + c]);
        ss += s * s;
      }
    or_real cd = prm->cs * delta;
    return cd * cd * SQRT(2.0 * ss);
  }
  /* Vreman: alpha_ij = d u_j / d x_i, beta_ij = delta^2 alpha_mi alpha_mj */
  or_real al[3][3], aa = 0.0, be[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      al[i][j] = G[j * 3 + i];
      aa += al[i][j] * al[i][j];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      or_real s = 0.0;
      for (int m = 0; m < 3; ++m) s += al[m][i] * al[m][j];
      be[i][j] = delta * delta * s;
    }
  or_real B = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] - be[0][2] * be[0][2] +
             be[1][1] * be[2][2] - be[1][2] * be[1][2];
  if (aa < 1e-300 || B <= 0.0) return 0.0;
  return prm->cv * SQRT(B / aa);
}

/* Low-storage third-order Runge-Kutta (Sec. 2.3 cites a low-storage explicit RK3; the
 * Williamson 2N-storage coefficients are used):  g <- A_s g + dt R(q),  q <- q + B_s g. */
static const or_real RK_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const or_real RK_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

or_real or_rk3_linear(or_real z) {
  or_real y = 1.0, g = 0.0;
  for (int s = 0; s < 3; ++s) {
    g = (s == 0 ? 0.0 : RK_A[s] * g) + z * y;
    y = y + RK_B[s] * g;
  }
  return y;
}

/* ------------------------------------------------------------------------------------
 * Mesh
 * ---------------------------------------------------------------------------------- */

typedef struct {
  or_real x[OR_MAXN + 1], w[OR_MAXN + 1], D[(OR_MAXN + 1) * (OR_MAXN + 1)];
  or_real lb[2][OR_MAXN + 1]; /* l_i(-1), l_i(+1): face interpolation (unit vectors on Lobatto nodes) */
} op1d;

struct or_mesh {
  int64_t ne, total;
  int g;
  int8_t* N;
  uint8_t* flag;
  int64_t* off;
  or_real* gx;     /* [ne][(g+1)^3][3] */
  int64_t* nb_e;  /* [ne][6]: neighbour element, -1 at a boundary */
  int8_t* nb_f;   /* [ne][6]: neighbour local face */
  int8_t* nb_o;   /* [ne][6]: orientation code mapping neighbour face coords to mine */
  int8_t* bc;     /* [ne][6]: boundary tag (-1 interior) */
  or_real* vscale; /* [ne] */
  or_params p;
  op1d op[OR_MAXN + 1];
};

int64_t or_total_nodes(const or_mesh* m) { return m->total; }
const int64_t* or_offsets(const or_mesh* m) { return m->off; }

/* Local faces: f = 2 d + s on the plane xi_d = (s ? +1 : -1). Face coordinates (a, b) run
 * along the two remaining directions in increasing order. */
static void face_dirs(int d, int* t0, int* t1) {
  *t0 = (d == 0) ? 1 : 0;
  *t1 = (d == 2) ? 1 : 2;
}
static int64_t face_node(int f, int N, int a, int b) {
  int d = f >> 1, s = f & 1, t0, t1, ijk[3];
  face_dirs(d, &t0, &t1);
  ijk[d] = s ? N : 0;
  ijk[t0] = a;
  ijk[t1] = b;
  int n = N + 1;
  return ijk[0] + (int64_t)n * (ijk[1] + (int64_t)n * ijk[2]);
}
static int face_corner(int f, int ca, int cb) {
  int d = f >> 1, s = f & 1, t0, t1, c[3];
  face_dirs(d, &t0, &t1);
  c[d] = s;
  c[t0] = ca;
  c[t1] = cb;
  return c[0] + 2 * c[1] + 4 * c[2];
}
/* Orientation code o = swap | flip_a << 1 | flip_b << 2 maps neighbour face coords
 * (a1, b1) at order M to mine: (x, y) = swap ? (b1, a1) : (a1, b1); a0 = flip_a ? M - x : x;
 * b0 = flip_b ? M - y : y. */
static void orient_map(int o, int M, int a1, int b1, int* a0, int* b0) {
  int x = (o & 1) ? b1 : a1, y = (o & 1) ? a1 : b1;
  *a0 = (o & 2) ? M - x : x;
  *b0 = (o & 4) ? M - y : y;
}

typedef struct {
  int64_t k[4];
  int64_t e;
  int f;
} face_rec;

static int cmp_face(const void* A, const void* B) {
  const face_rec* a = (const face_rec*)A;
  const face_rec* b = (const face_rec*)B;
  for (int i = 0; i < 4; ++i)
    if (a->k[i] != b->k[i]) return a->k[i] < b->k[i] ? -1 : 1;
  if (a->e != b->e) return a->e < b->e ? -1 : 1;
  return a->f - b->f;
}

void or_destroy(or_mesh* m) {
  if (!m) return;
  free(m->N);
  free(m->flag);
  free(m->off);
  free(m->gx);
  free(m->nb_e);
  free(m->nb_f);
  free(m->nb_o);
  free(m->bc);
  free(m->vscale);
  free(m);
}

or_mesh* or_create(int64_t ne, const int64_t* hex, int g, const or_real* gxyz, const int8_t* bc_tag,
                   const int8_t* order, const uint8_t* flag, const or_params* prm) {
  if (ne <= 0 || !hex || !gxyz || !order || !flag || !prm) {
    set_err("bad arguments");
    return NULL;
  }
  if (g < 1 || g > OR_MAXG) {
    set_err("geometry degree %d unsupported", g);
    return NULL;
  }
  if (prm->split != 0 && prm->split != 1) {
    set_err("split %d invalid", prm->split);
    return NULL;
  }
  if (prm->mixed_face != 0 && prm->mixed_face != 1) {
    set_err("mixed_face %d invalid", prm->mixed_face);
    return NULL;
  }
  or_mesh* m = (or_mesh*)calloc(1, sizeof(or_mesh));
  m->ne = ne;
  m->g = g;
  m->p = *prm;
  if (prm->nodes != 0 && prm->nodes != 1) {
    set_err("nodes %d invalid", prm->nodes);
    free(m);
    return NULL;
  }
  if (prm->nodes == 1 && prm->split == 1) {
    set_err("the split form needs Gauss-Lobatto nodes");
    free(m);
    return NULL;
  }
  for (int N = 1; N <= OR_MAXN; ++N) {
    if (prm->nodes == 1) {
      or_gl(N, m->op[N].x, m->op[N].w);
      dmat_nodes(N + 1, m->op[N].x, m->op[N].D);
    } else {
      or_lgl(N, m->op[N].x, m->op[N].w);
      or_dmat(N, m->op[N].D);
    }
    for (int i = 0; i <= N; ++i) {
      m->op[N].lb[0][i] = lagrange(N + 1, m->op[N].x, i, -1.0);
      m->op[N].lb[1][i] = lagrange(N + 1, m->op[N].x, i, 1.0);
    }
  }
  int ng = g + 1, ng3 = ng * ng * ng;
  m->N = (int8_t*)malloc(ne);
  m->flag = (uint8_t*)malloc(ne);
  m->off = (int64_t*)malloc(sizeof(int64_t) * (ne + 1));
  m->gx = (or_real*)malloc(sizeof(or_real) * ne * ng3 * 3);
  m->nb_e = (int64_t*)malloc(sizeof(int64_t) * ne * 6);
  m->nb_f = (int8_t*)malloc(ne * 6);
  m->nb_o = (int8_t*)malloc(ne * 6);
  m->bc = (int8_t*)malloc(ne * 6);
  m->vscale = (or_real*)malloc(sizeof(or_real) * ne);
  memcpy(m->gx, gxyz, sizeof(or_real) * ne * ng3 * 3);
  m->off[0] = 0;
  for (int64_t e = 0; e < ne; ++e) {
    if (order[e] < 1 || order[e] > OR_MAXN || order[e] < g) {
      set_err("element %lld: order %d invalid (geometry degree %d)", (long long)e, order[e], g);
      or_destroy(m);
      return NULL;
    }
    if (flag[e] > 1) {
      set_err("element %lld: flag %d invalid", (long long)e, flag[e]);
      or_destroy(m);
      return NULL;
    }
    m->N[e] = order[e];
    m->flag[e] = flag[e];
    m->vscale[e] = 1.0;
    int n = order[e] + 1;
    m->off[e + 1] = m->off[e] + (int64_t)n * n * n;
    for (int f = 0; f < 6; ++f) {
      m->nb_e[e * 6 + f] = -1;
      m->nb_f[e * 6 + f] = -1;
      m->nb_o[e * 6 + f] = 0;
      m->bc[e * 6 + f] = bc_tag ? bc_tag[e * 6 + f] : -1;
      if (m->bc[e * 6 + f] == 0 || m->bc[e * 6 + f] < -1 || m->bc[e * 6 + f] > 4) {
        set_err("element %lld face %d: boundary tag %d invalid", (long long)e, f, m->bc[e * 6 + f]);
        or_destroy(m);
        return NULL;
      }
    }
  }
  m->total = m->off[ne];

  /* face matching by the sorted corner vertex ids */
  face_rec* rec = (face_rec*)malloc(sizeof(face_rec) * ne * 6);
  for (int64_t e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f) {
      face_rec* r = &rec[e * 6 + f];
      for (int c = 0; c < 4; ++c) r->k[c] = hex[e * 8 + face_corner(f, c & 1, c >> 1)];
      for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) {
          if (r->k[i] == r->k[j]) {
            set_err("element %lld face %d has repeated vertex ids", (long long)e, f);
            free(rec);
            or_destroy(m);
            return NULL;
          }
          if (r->k[j] < r->k[i]) {
            int64_t t = r->k[i];
            r->k[i] = r->k[j];
            r->k[j] = t;
          }
        }
      r->e = e;
      r->f = f;
    }
  qsort(rec, (size_t)ne * 6, sizeof(face_rec), cmp_face);
  int64_t i = 0;
  while (i < ne * 6) {
    int64_t j = i + 1;
    while (j < ne * 6 && memcmp(rec[j].k, rec[i].k, sizeof rec[i].k) == 0) ++j;
    if (j - i > 2) {
      set_err("a face is shared by more than two elements");
      free(rec);
      or_destroy(m);
      return NULL;
    }
    if (j - i == 1) {
      if (m->bc[rec[i].e * 6 + rec[i].f] < 1) {
        set_err("element %lld face %d is unmatched and has no boundary tag", (long long)rec[i].e, rec[i].f);
        free(rec);
        or_destroy(m);
        return NULL;
      }
    } else {
      for (int s = 0; s < 2; ++s) {
        int64_t e0 = rec[i + s].e, e1 = rec[i + 1 - s].e;
        int f0 = rec[i + s].f, f1 = rec[i + 1 - s].f;
        if (m->bc[e0 * 6 + f0] >= 1) {
          set_err("element %lld face %d is interior but carries a boundary tag", (long long)e0, f0);
          free(rec);
          or_destroy(m);
          return NULL;
        }
        int found = -1;
        for (int o = 0; o < 8 && found < 0; ++o) {
          int ok = 1;
          for (int cb = 0; cb < 2 && ok; ++cb)
            for (int ca = 0; ca < 2 && ok; ++ca) {
              int a0, b0;
              orient_map(o, 1, ca, cb, &a0, &b0);
              if (hex[e1 * 8 + face_corner(f1, ca, cb)] != hex[e0 * 8 + face_corner(f0, a0, b0)]) ok = 0;
            }
          if (ok) found = o;
        }
        if (found < 0) {
          set_err("no orientation matches element %lld face %d", (long long)e0, f0);
          free(rec);
          or_destroy(m);
          return NULL;
        }
        m->nb_e[e0 * 6 + f0] = e1;
        m->nb_f[e0 * 6 + f0] = (int8_t)f1;
        m->nb_o[e0 * 6 + f0] = (int8_t)found;
      }
    }
    i = j;
  }
  free(rec);
  return m;
}

int or_set_visc_scale(or_mesh* m, const or_real* scale) {
  for (int64_t e = 0; e < m->ne; ++e) m->vscale[e] = scale ? scale[e] : 1.0;
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Geometry (App. B: transfinite polynomial map x(xi), Jacobian J, contravariant metric).
 * Metric terms in the curl (conservative) form, computed at the geometry degree g and
 * interpolated to the element's nodes (exact because N >= g):
 *   Ja^i_n = - e_i . curl_xi ( I^g( X_l grad_xi X_m ) ),  (n, m, l) cyclic.
 * J = det(dX/dxi) of the degree-g map at the element's nodes.
 * ---------------------------------------------------------------------------------- */

/* derivative along direction k of a field on an n^3 tensor grid with matrix D (n x n) */
static void deriv3(int n, const or_real* D, int k, const or_real* u, or_real* du) {
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        int ijk[3] = {a, b, c};
        or_real s = 0.0;
        for (int mm = 0; mm < n; ++mm) {
          int src[3] = {a, b, c};
          src[k] = mm;
          s += D[ijk[k] * n + mm] * u[src[0] + n * (src[1] + n * src[2])];
        }
        du[a + n * (b + n * c)] = s;
      }
}

/* tensor interpolation from an ns^3 grid to an nd^3 grid with I (nd x ns) */
static void interp3(int ns, int nd, const or_real* I, const or_real* u, or_real* out) {
  for (int k = 0; k < nd; ++k)
    for (int j = 0; j < nd; ++j)
      for (int i = 0; i < nd; ++i) {
        or_real s = 0.0;
        for (int c = 0; c < ns; ++c)
          for (int b = 0; b < ns; ++b)
            for (int a = 0; a < ns; ++a)
              s += I[i * ns + a] * I[j * ns + b] * I[k * ns + c] * u[a + ns * (b + ns * c)];
        out[i + nd * (j + nd * k)] = s;
      }
}

/* Interpolation from the geometry nodes (Gauss-Lobatto points of degree g) to the element's
 * nodes of order N (Gauss-Lobatto or Gauss-Legendre): I[(N+1)][(g+1)] */
static void geom_interp(const or_mesh* m, int N, or_real* I) {
  or_real xg[OR_MAXG + 1], wg[OR_MAXG + 1];
  or_lgl(m->g, xg, wg);
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= m->g; ++j) I[i * (m->g + 1) + j] = lagrange(m->g + 1, xg, j, m->op[N].x[i]);
}

int or_element_geometry(const or_mesh* m, int64_t e, or_real* J, or_real* Ja) {
  int g = m->g, ng = g + 1, ng3 = ng * ng * ng;
  int N = m->N[e], n = N + 1, n3 = n * n * n;
  /* the geometry nodes are Gauss-Lobatto points of degree g whatever the element's node set */
  or_real Dg[(OR_MAXG + 1) * (OR_MAXG + 1)];
  or_dmat(g, Dg);
  or_real I[(OR_MAXN + 1) * (OR_MAXG + 1)];
  geom_interp(m, N, I);
  or_real X[3][(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
  or_real dX[3][3][(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
  for (int p = 0; p < ng3; ++p)
    for (int c = 0; c < 3; ++c) X[c][p] = m->gx[(e * ng3 + p) * 3 + c];
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) deriv3(ng, Dg, k, X[c], dX[c][k]);
  /* J at the element nodes */
  or_real* dXn = (or_real*)malloc(sizeof(or_real) * 9 * n3);
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) interp3(ng, n, I, dX[c][k], dXn + (c * 3 + k) * n3);
  for (int p = 0; p < n3; ++p) {
    or_real a[3][3];
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 3; ++k) a[c][k] = dXn[(c * 3 + k) * n3 + p];
    J[p] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  }
  free(dXn);
  /* curl form at degree g */
  for (int nn = 0; nn < 3; ++nn) {
    int mm = (nn + 1) % 3, ll = (nn + 2) % 3;
    or_real v[3][(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
    or_real dv[3][3][(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
    for (int k = 0; k < 3; ++k)
      for (int p = 0; p < ng3; ++p) v[k][p] = X[ll][p] * dX[mm][k][p];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) deriv3(ng, Dg, d, v[k], dv[k][d]); /* dv[k][d] = d v_k / d xi_d */
    or_real curl[3][(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
    for (int p = 0; p < ng3; ++p) {
      curl[0][p] = dv[2][1][p] - dv[1][2][p];
      curl[1][p] = dv[0][2][p] - dv[2][0][p];
      curl[2][p] = dv[1][0][p] - dv[0][1][p];
    }
    for (int i = 0; i < 3; ++i) {
      or_real neg[(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
      for (int p = 0; p < ng3; ++p) neg[p] = -curl[i][p];
      interp3(ng, n, I, neg, Ja + (i * 3 + nn) * n3);
    }
  }
  return 0;
}

int or_node_coords(const or_mesh* m, or_real* xyz) {
  int g = m->g, ng = g + 1, ng3 = ng * ng * ng;
  for (int64_t e = 0; e < m->ne; ++e) {
    int N = m->N[e], n = N + 1, n3 = n * n * n;
    or_real I[(OR_MAXN + 1) * (OR_MAXG + 1)];
    geom_interp(m, N, I);
    or_real X[(OR_MAXG + 1) * (OR_MAXG + 1) * (OR_MAXG + 1)];
    or_real* out = (or_real*)malloc(sizeof(or_real) * n3);
    for (int c = 0; c < 3; ++c) {
      for (int p = 0; p < ng3; ++p) X[p] = m->gx[(e * ng3 + p) * 3 + c];
      interp3(ng, n, I, X, out);
      for (int p = 0; p < n3; ++p) xyz[c * m->total + m->off[e] + p] = out[p];
    }
    free(out);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Residual machinery
 * ---------------------------------------------------------------------------------- */

typedef struct {
  or_real* J;   /* [n3] */
  or_real* Ja;  /* [3][3][n3] */
  or_real delta;
} geo_t;

typedef struct {
  const or_mesh* m;
  const or_real* q;
  geo_t* geo;    /* per element, J == NULL if not computed */
  or_real** G;    /* per element gradient [3][3][n3], NULL if not computed */
} work_t;

static void compute_geo(const or_mesh* m, int64_t e, geo_t* gt) {
  int n = m->N[e] + 1, n3 = n * n * n;
  gt->J = (or_real*)malloc(sizeof(or_real) * n3);
  gt->Ja = (or_real*)malloc(sizeof(or_real) * 9 * n3);
  or_element_geometry(m, e, gt->J, gt->Ja);
  const or_real* w = m->op[m->N[e]].w;
  or_real V = 0.0;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) V += w[i] * w[j] * w[k] * gt->J[i + n * (j + n * k)];
  /* filter width: cube root of the element volume over the nodes per direction */
  gt->delta = CBRT(V) / n;
}

/* 2D tensor interpolation on a face: ns^2 -> nd^2 with I (nd x ns) */
static void interp2(int ns, int nd, const or_real* I, const or_real* u, or_real* out) {
  for (int b = 0; b < nd; ++b)
    for (int a = 0; a < nd; ++a) {
      or_real s = 0.0;
      for (int bb = 0; bb < ns; ++bb)
        for (int aa = 0; aa < ns; ++aa) s += I[a * ns + aa] * I[b * ns + bb] * u[aa + ns * bb];
      out[a + nd * b] = s;
    }
}

/* outward area-weighted normal S = sigma Ja^d at the face nodes of element e, face f */
/* volume node i along the normal line of face f through the face coordinates (a, b) */
static int64_t line_node(int f, int N, int a, int b, int i) {
  int d = f >> 1, t0, t1, ijk[3];
  face_dirs(d, &t0, &t1);
  ijk[d] = i;
  ijk[t0] = a;
  ijk[t1] = b;
  int n = N + 1;
  return ijk[0] + (int64_t)n * (ijk[1] + (int64_t)n * ijk[2]);
}

/* the value at face f of a nodal field u[n3] at face coordinates (a, b): the face node's value
 * on Gauss-Lobatto nodes, the interpolation sum_i l_i(+-1) u_i along the normal line on
 * Gauss-Legendre nodes */
static or_real face_value(const or_mesh* m, int N, int f, int a, int b, const or_real* u) {
  if (m->p.nodes == 0) return u[face_node(f, N, a, b)];
  const or_real* l = m->op[N].lb[f & 1];
  or_real s = 0.0;
  for (int i = 0; i <= N; ++i) s += l[i] * u[line_node(f, N, a, b, i)];
  return s;
}

/* adds v * (lifting of face f at (a, b)) to the nodal field u[n3]: v / w_end at the face node
 * on Gauss-Lobatto nodes, v l_i(+-1) / w_i along the normal line on Gauss-Legendre nodes
 * (the surface integral of the weak form divided by the node's quadrature weight) */
static void face_lift(const or_mesh* m, int N, int f, int a, int b, or_real v, or_real* u) {
  const or_real* w = m->op[N].w;
  if (m->p.nodes == 0) {
    u[face_node(f, N, a, b)] += v / w[0];
    return;
  }
  const or_real* l = m->op[N].lb[f & 1];
  for (int i = 0; i <= N; ++i) u[line_node(f, N, a, b, i)] += v * l[i] / w[i];
}

static void face_S(const or_mesh* m, const geo_t* gt, int64_t e, int f, or_real* S /*[3][n2]*/) {
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  int d = f >> 1;
  or_real sg = (f & 1) ? 1.0 : -1.0;
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < 3; ++c) S[c * n2 + a + n * b] = sg * face_value(m, N, f, a, b, gt->Ja + (d * 3 + c) * n3);
}

static void face_q(const or_mesh* m, const or_real* q, int64_t e, int f, or_real* T /*[4][n2]*/) {
  int N = m->N[e], n = N + 1, n2 = n * n;
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a)
      for (int v = 0; v < 4; ++v) T[v * n2 + a + n * b] = face_value(m, N, f, a, b, q + v * m->total + m->off[e]);
}

/* viscous stress at one node of an NS element */
static void stress(const or_mesh* m, const geo_t* gt, const or_real* G, int64_t e, int n3, int64_t p,
                   or_real tau[3][3]) {
  or_real Gp[9];
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) Gp[c * 3 + k] = G[(c * 3 + k) * n3 + p];
  or_real nut = or_eddy_viscosity(Gp, gt->delta, &m->p);
  or_real mu = (m->p.nu + nut) * m->vscale[e];
  or_real tr = Gp[0] + Gp[4] + Gp[8];
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) tau[c][k] = mu * (Gp[c * 3 + k] + Gp[k * 3 + c]) - (c == k ? 2.0 / 3.0 * mu * tr : 0.0);
}

/* area-weighted outward viscous flux trace tau . S of element e on face f (zero for Euler) */
static void face_fv(const work_t* W, int64_t e, int f, or_real* Fv /*[3][n2]*/) {
  const or_mesh* m = W->m;
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  if (!m->flag[e]) {
    memset(Fv, 0, sizeof(or_real) * 3 * n2);
    return;
  }
  const geo_t* gt = &W->geo[e];
  if (m->p.nodes == 1) {
    /* Gauss-Legendre: the outward contravariant viscous flux sigma Ja^d . tau at every node,
     * interpolated to the face */
    const int d = f >> 1;
    const or_real sg = (f & 1) ? 1.0 : -1.0;
    or_real* Ft = (or_real*)malloc(sizeof(or_real) * 3 * n3);
    for (int p = 0; p < n3; ++p) {
      or_real tau[3][3];
      stress(m, gt, W->G[e], e, n3, p, tau);
      for (int c = 0; c < 3; ++c) {
        or_real s = 0.0;
        for (int k = 0; k < 3; ++k) s += tau[c][k] * gt->Ja[(d * 3 + k) * n3 + p];
        Ft[c * n3 + p] = sg * s;
      }
    }
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < 3; ++c) Fv[c * n2 + a + n * b] = face_value(m, N, f, a, b, Ft + c * n3);
    free(Ft);
    return;
  }
  or_real* S = (or_real*)malloc(sizeof(or_real) * 3 * n2);
  face_S(m, gt, e, f, S);
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      int64_t p = face_node(f, N, a, b);
      or_real tau[3][3];
      stress(m, gt, W->G[e], e, n3, p, tau);
      for (int c = 0; c < 3; ++c) {
        or_real s = 0.0;
        for (int k = 0; k < 3; ++k) s += tau[c][k] * S[k * n2 + a + n * b];
        Fv[c * n2 + a + n * b] = s;
      }
    }
  free(S);
}

/* ghost state behind a boundary face with area-weighted outward normal S */
static void ghost_state(const or_mesh* m, int tag, const or_real* qin, const or_real S[3], or_real* qg) {
  qg[0] = qin[0];
  if (tag == 1) { /* inflow: prescribed velocity, interior pressure */
    for (int c = 0; c < 3; ++c) qg[1 + c] = m->p.inflow[1 + c];
  } else if (tag == 2) { /* outflow: interior velocity, zero pressure */
    qg[0] = 0.0;
    for (int c = 0; c < 3; ++c) qg[1 + c] = qin[1 + c];
  } else if (tag == 3) { /* no-slip wall: the mirror state with every velocity component reversed */
    for (int c = 0; c < 3; ++c) qg[1 + c] = -qin[1 + c];
  } else { /* free-slip wall: the mirror state, normal velocity reversed */
    const or_real s = SQRT(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    const or_real un = (qin[1] * S[0] + qin[2] * S[1] + qin[3] * S[2]) / s;
    for (int c = 0; c < 3; ++c) qg[1 + c] = qin[1 + c] - 2.0 * un * S[c] / s;
  }
}

/* Mortar data of face (e, f) in e's face coordinates at order M = max(N_e, N_nbr):
 * my trace, the neighbour trace (or ghost), my S interpolated. */
typedef struct {
  int M, nm;          /* mortar order, my order */
  or_real* qm;         /* [4][(M+1)^2] */
  or_real* qp;         /* [4][(M+1)^2] */
  or_real* S;          /* [3][(M+1)^2] */
  int64_t nbr;        /* -1 at a boundary */
  int nf, no, tag;
} mortar_t;

static void mortar_free(mortar_t* mt) {
  free(mt->qm);
  free(mt->qp);
  free(mt->S);
}

/* interpolate a neighbour face field (order Nn) to the mortar order M and rotate it into
 * my face coordinates */
static void nbr_to_mortar(int gl, int Nn, int M, int o, int nvar, const or_real* src, or_real* dst) {
  int nn = Nn + 1, nM = M + 1, nM2 = nM * nM;
  or_real I[(OR_MAXN + 1) * (OR_MAXN + 1)];
  interp_nodes(gl, Nn, M, I);
  or_real* tmp = (or_real*)malloc(sizeof(or_real) * nM2);
  for (int v = 0; v < nvar; ++v) {
    interp2(nn, nM, I, src + v * nn * nn, tmp);
    for (int b1 = 0; b1 < nM; ++b1)
      for (int a1 = 0; a1 < nM; ++a1) {
        int a0, b0;
        orient_map(o, M, a1, b1, &a0, &b0);
        dst[v * nM2 + a0 + nM * b0] = tmp[a1 + nM * b1];
      }
  }
  free(tmp);
}

static void mine_to_mortar(int gl, int Nm, int M, int nvar, const or_real* src, or_real* dst) {
  int nm = Nm + 1, nM = M + 1;
  or_real I[(OR_MAXN + 1) * (OR_MAXN + 1)];
  interp_nodes(gl, Nm, M, I);
  for (int v = 0; v < nvar; ++v) interp2(nm, nM, I, src + v * nm * nm, dst + v * nM * nM);
}

/* project a mortar field (order M, my coordinates) to my order */
static void mortar_to_mine(int gl, int M, int Nm, int nvar, const or_real* src, or_real* dst) {
  int nm = Nm + 1, nM = M + 1;
  or_real P[(OR_MAXN + 1) * (OR_MAXN + 1)];
  project_nodes(gl, M, Nm, P);
  for (int v = 0; v < nvar; ++v) interp2(nM, nm, P, src + v * nM * nM, dst + v * nm * nm);
}

static void mortar_build(const work_t* W, int64_t e, int f, mortar_t* mt) {
  const or_mesh* m = W->m;
  int Nm = m->N[e], nm = Nm + 1;
  int64_t nb = m->nb_e[e * 6 + f];
  int Nn = nb >= 0 ? m->N[nb] : Nm;
  int M = Nm > Nn ? Nm : Nn, nM = M + 1, nM2 = nM * nM;
  mt->M = M;
  mt->nm = Nm;
  mt->nbr = nb;
  mt->nf = m->nb_f[e * 6 + f];
  mt->no = m->nb_o[e * 6 + f];
  mt->tag = m->bc[e * 6 + f];
  mt->qm = (or_real*)malloc(sizeof(or_real) * 4 * nM2);
  mt->qp = (or_real*)malloc(sizeof(or_real) * 4 * nM2);
  mt->S = (or_real*)malloc(sizeof(or_real) * 3 * nM2);
  or_real* tq = (or_real*)malloc(sizeof(or_real) * 4 * nm * nm);
  or_real* tS = (or_real*)malloc(sizeof(or_real) * 3 * nm * nm);
  face_q(m, W->q, e, f, tq);
  face_S(m, &W->geo[e], e, f, tS);
  mine_to_mortar(m->p.nodes, Nm, M, 4, tq, mt->qm);
  mine_to_mortar(m->p.nodes, Nm, M, 3, tS, mt->S);
  if (nb >= 0) {
    int nn = Nn + 1;
    or_real* tn = (or_real*)malloc(sizeof(or_real) * 4 * nn * nn);
    face_q(m, W->q, nb, mt->nf, tn);
    nbr_to_mortar(m->p.nodes, Nn, M, mt->no, 4, tn, mt->qp);
    free(tn);
  } else {
    for (int p = 0; p < nM2; ++p) {
      or_real qi[4], qg[4];
      for (int v = 0; v < 4; ++v) qi[v] = mt->qm[v * nM2 + p];
      const or_real Sp[3] = {mt->S[p], mt->S[nM2 + p], mt->S[2 * nM2 + p]};
      ghost_state(m, mt->tag, qi, Sp, qg);
      for (int v = 0; v < 4; ++v) mt->qp[v * nM2 + p] = qg[v];
    }
  }
  free(tq);
  free(tS);
}

/* BR1 lifting data on face (e, f): projected u*_c S_k, shape [3][3][n2] */
static void face_ustar(const work_t* W, int64_t e, int f, or_real* LU) {
  mortar_t mt;
  mortar_build(W, e, f, &mt);
  int nM = mt.M + 1, nM2 = nM * nM;
  or_real* U = (or_real*)malloc(sizeof(or_real) * 9 * nM2);
  for (int p = 0; p < nM2; ++p)
    for (int c = 0; c < 3; ++c) {
      or_real us = 0.5 * (mt.qm[(1 + c) * nM2 + p] + mt.qp[(1 + c) * nM2 + p]);
      for (int k = 0; k < 3; ++k) U[(c * 3 + k) * nM2 + p] = us * mt.S[k * nM2 + p];
    }
  mortar_to_mine(W->m->p.nodes, mt.M, mt.nm, 9, U, LU);
  free(U);
  mortar_free(&mt);
}

/* Total numerical flux on face (e, f): projected (F_e* - F_v*) . S (my outward), [4][n2] */
static int face_hstar(const work_t* W, int64_t e, int f, or_real* LH) {
  const or_mesh* m = W->m;
  mortar_t mt;
  mortar_build(W, e, f, &mt);
  int nM = mt.M + 1, nM2 = nM * nM, nm = mt.nm + 1, nm2 = nm * nm;
  or_real* H = (or_real*)malloc(sizeof(or_real) * 4 * nM2);
  or_real* Fvm = (or_real*)calloc(3 * nM2, sizeof(or_real));
  or_real* Fvp = (or_real*)calloc(3 * nM2, sizeof(or_real));
  int any_visc = m->flag[e] || (mt.nbr >= 0 && m->flag[mt.nbr]);
  if (any_visc) {
    or_real* t = (or_real*)malloc(sizeof(or_real) * 3 * nm2);
    face_fv(W, e, f, t);
    mine_to_mortar(m->p.nodes, mt.nm, mt.M, 3, t, Fvm);
    free(t);
    if (mt.nbr >= 0) {
      int nn = m->N[mt.nbr] + 1;
      or_real* tn = (or_real*)malloc(sizeof(or_real) * 3 * nn * nn);
      face_fv(W, mt.nbr, mt.nf, tn);
      nbr_to_mortar(m->p.nodes, m->N[mt.nbr], mt.M, mt.no, 3, tn, Fvp);
      free(tn);
    } else if (mt.tag == 4) {
      /* free-slip wall: the mirror ghost's outward viscous flux is R Fvm, R = I - 2 n n^T the
       * reflection, so the BR1 average keeps only the normal part of the traction */
      for (int p = 0; p < nM2; ++p) {
        const or_real S[3] = {mt.S[p], mt.S[nM2 + p], mt.S[2 * nM2 + p]};
        const or_real ss = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
        const or_real fn = (Fvm[p] * S[0] + Fvm[nM2 + p] * S[1] + Fvm[2 * nM2 + p] * S[2]) / ss;
        for (int c = 0; c < 3; ++c) Fvp[c * nM2 + p] = Fvm[c * nM2 + p] - 2.0 * fn * S[c];
      }
    } else {
      /* inflow, outflow and no-slip wall: the interior viscous flux (at a no-slip wall the
       * interior traction) -- the ghost carries it, pointing the other way */
      for (int i = 0; i < 3 * nM2; ++i) Fvp[i] = -Fvm[i];
    }
  }
  /* F_v* . S = wm Fvm - wp Fvp: the BR1 average, except on a face between an NS and an Euler
   * element with the one-sided choice, where the NS side's flux alone is taken */
  or_real wm = 0.5, wp = 0.5;
  if (m->p.mixed_face == 1 && mt.nbr >= 0 && m->flag[e] != m->flag[mt.nbr]) {
    wm = m->flag[e] ? 1.0 : 0.0;
    wp = m->flag[e] ? 0.0 : 1.0;
  }
  int rc = 0;
  for (int p = 0; p < nM2; ++p) {
    or_real S[3] = {mt.S[p], mt.S[nM2 + p], mt.S[2 * nM2 + p]};
    or_real s = SQRT(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    or_real nh[3] = {S[0] / s, S[1] / s, S[2] / s};
    or_real qm[4], qp[4], Fs[4];
    for (int v = 0; v < 4; ++v) {
      qm[v] = mt.qm[v * nM2 + p];
      qp[v] = mt.qp[v * nM2 + p];
    }
    if (or_riemann(qm, qp, nh, &m->p, Fs)) rc = -1;
    H[p] = Fs[0] * s;
    for (int c = 0; c < 3; ++c) {
      or_real fv = wm * Fvm[c * nM2 + p] - wp * Fvp[c * nM2 + p];
      H[(1 + c) * nM2 + p] = Fs[1 + c] * s - fv;
    }
  }
  mortar_to_mine(m->p.nodes, mt.M, mt.nm, 4, H, LH);
  free(H);
  free(Fvm);
  free(Fvp);
  mortar_free(&mt);
  return rc;
}

/* BR1 gradient, weak form (integrated by parts, Bassi-Rebay 1):
 *   w J G_ck = -sum_d (w/w_{i_d}) sum_m w_m D_{m i_d} (u_c Ja^d_k)_m + face terms u*_c S_k */
static void element_gradient(const work_t* W, int64_t e, or_real* G) {
  const or_mesh* m = W->m;
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  const or_real* w = m->op[N].w;
  const or_real* D = m->op[N].D;
  const geo_t* gt = &W->geo[e];
  const or_real* q = W->q;
  int64_t o = m->off[e];
  memset(G, 0, sizeof(or_real) * 9 * n3);
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) {
      or_real* Gck = G + (c * 3 + k) * n3;
      for (int kk = 0; kk < n; ++kk)
        for (int jj = 0; jj < n; ++jj)
          for (int ii = 0; ii < n; ++ii) {
            int ijk[3] = {ii, jj, kk};
            or_real s = 0.0;
            for (int d = 0; d < 3; ++d) {
              or_real sd = 0.0;
              for (int mm = 0; mm < n; ++mm) {
                int src[3] = {ii, jj, kk};
                src[d] = mm;
                int64_t ps = src[0] + n * (src[1] + n * src[2]);
                sd += w[mm] * D[mm * n + ijk[d]] * q[(1 + c) * m->total + o + ps] * gt->Ja[(d * 3 + k) * n3 + ps];
              }
              s -= sd / w[ijk[d]];
            }
            Gck[ii + n * (jj + n * kk)] = s;
          }
    }
  or_real* LU = (or_real*)malloc(sizeof(or_real) * 9 * n2);
  for (int f = 0; f < 6; ++f) {
    face_ustar(W, e, f, LU);
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a)
        for (int ck = 0; ck < 9; ++ck) face_lift(m, N, f, a, b, LU[ck * n2 + a + n * b], G + ck * n3);
  }
  free(LU);
  for (int ck = 0; ck < 9; ++ck)
    for (int p = 0; p < n3; ++p) G[ck * n3 + p] /= gt->J[p];
}

int or_element_gradient(const or_mesh* m, const or_real* q, int64_t e, or_real* G) {
  if (e < 0 || e >= m->ne) return -1;
  work_t W;
  W.m = m;
  W.q = q;
  W.geo = (geo_t*)calloc(m->ne, sizeof(geo_t));
  W.G = NULL;
  compute_geo(m, e, &W.geo[e]);
  element_gradient(&W, e, G);
  free(W.geo[e].J);
  free(W.geo[e].Ja);
  free(W.geo);
  return 0;
}

/* Residual of one element, weak form (App. B, Eq. NS4 with the viscous terms integrated
 * by parts under BR1):
 *   w J R = sum_d (w / w_{i_d}) sum_m w_m D_{m i_d} Ftil^d_m - w_face H*  */
static int element_residual(const work_t* W, int64_t e, or_real* R) {
  const or_mesh* m = W->m;
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  const or_real* w = m->op[N].w;
  const or_real* D = m->op[N].D;
  const geo_t* gt = &W->geo[e];
  const or_real* q = W->q;
  int64_t o = m->off[e], T = m->total;
  or_real c0sq = m->p.c0sq;
  /* contravariant total flux Ftil[d][v][p] = sum_k Ja^d_k (F_e - F_v)_{v,k}, and its convective
   * part Fc (kept for the split form) */
  or_real* Ft = (or_real*)malloc(sizeof(or_real) * 12 * n3);
  or_real* Fc = (or_real*)malloc(sizeof(or_real) * 12 * n3);
  for (int p = 0; p < n3; ++p) {
    or_real qq[4];
    for (int v = 0; v < 4; ++v) qq[v] = q[v * T + o + p];
    or_real F[4][3];
    for (int k = 0; k < 3; ++k) {
      F[0][k] = c0sq * qq[1 + k];
      for (int c = 0; c < 3; ++c) F[1 + c][k] = qq[1 + c] * qq[1 + k] + (c == k ? qq[0] : 0.0);
    }
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 4; ++v) {
        or_real sc = 0.0;
        for (int k = 0; k < 3; ++k) sc += gt->Ja[(d * 3 + k) * n3 + p] * F[v][k];
        Fc[(d * 4 + v) * n3 + p] = sc;
      }
    if (m->flag[e]) {
      or_real tau[3][3];
      stress(m, gt, W->G[e], e, n3, p, tau);
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 3; ++k) F[1 + c][k] -= tau[c][k];
    }
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 4; ++v) {
        or_real s = 0.0;
        for (int k = 0; k < 3; ++k) s += gt->Ja[(d * 3 + k) * n3 + p] * F[v][k];
        Ft[(d * 4 + v) * n3 + p] = s;
      }
  }
  or_real* JR = (or_real*)calloc(4 * n3, sizeof(or_real));
  for (int v = 0; v < 4; ++v)
    for (int kk = 0; kk < n; ++kk)
      for (int jj = 0; jj < n; ++jj)
        for (int ii = 0; ii < n; ++ii) {
          int ijk[3] = {ii, jj, kk};
          or_real s = 0.0;
          for (int d = 0; d < 3; ++d) {
            or_real sd = 0.0;
            for (int mm = 0; mm < n; ++mm) {
              int src[3] = {ii, jj, kk};
              src[d] = mm;
              sd += w[mm] * D[mm * n + ijk[d]] * Ft[(d * 4 + v) * n3 + src[0] + n * (src[1] + n * src[2])];
            }
            s += sd / w[ijk[d]];
          }
          JR[v * n3 + ii + n * (jj + n * kk)] = s;
        }
  if (m->p.split == 1) {
    /* By summation by parts the weak convective volume term above equals -sum_m D_im Fc_m plus
     * the end-node terms; the split form replaces -sum_m D_im Fc_m along each direction by
     * -sum_m 2 D_im F#(q_i, q_m). Both sums are taken directly here. */
    for (int kk = 0; kk < n; ++kk)
      for (int jj = 0; jj < n; ++jj)
        for (int ii = 0; ii < n; ++ii) {
          int ijk[3] = {ii, jj, kk};
          const int pi = ii + n * (jj + n * kk);
          or_real qi[4];
          for (int v = 0; v < 4; ++v) qi[v] = q[v * T + o + pi];
          for (int d = 0; d < 3; ++d) {
            or_real jai[3] = {gt->Ja[(d * 3) * n3 + pi], gt->Ja[(d * 3 + 1) * n3 + pi], gt->Ja[(d * 3 + 2) * n3 + pi]};
            for (int mm = 0; mm < n; ++mm) {
              int src[3] = {ii, jj, kk};
              src[d] = mm;
              const int pm = src[0] + n * (src[1] + n * src[2]);
              or_real qm2[4], fs[4];
              for (int v = 0; v < 4; ++v) qm2[v] = q[v * T + o + pm];
              or_real jam[3] = {gt->Ja[(d * 3) * n3 + pm], gt->Ja[(d * 3 + 1) * n3 + pm], gt->Ja[(d * 3 + 2) * n3 + pm]};
              or_kep_flux(qi, qm2, jai, jam, c0sq, fs);
              const or_real Dim = D[ijk[d] * n + mm];
              for (int v = 0; v < 4; ++v)
                JR[v * n3 + pi] += Dim * Fc[(d * 4 + v) * n3 + pm] - 2.0 * Dim * fs[v];
            }
          }
        }
  }
  or_real* LH = (or_real*)malloc(sizeof(or_real) * 4 * n2);
  int rc = 0;
  for (int f = 0; f < 6; ++f) {
    if (face_hstar(W, e, f, LH)) rc = -1;
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a)
        for (int v = 0; v < 4; ++v) face_lift(m, N, f, a, b, -LH[v * n2 + a + n * b], JR + v * n3);
  }
  for (int v = 0; v < 4; ++v)
    for (int p = 0; p < n3; ++p) R[v * T + o + p] = JR[v * n3 + p] / gt->J[p];
  free(LH);
  free(JR);
  free(Ft);
  free(Fc);
  return rc;
}

static void free_work(work_t* W) {
  for (int64_t e = 0; e < W->m->ne; ++e) {
    free(W->geo[e].J);
    free(W->geo[e].Ja);
    if (W->G) free(W->G[e]);
  }
  free(W->geo);
  free(W->G);
}

int or_residual(const or_mesh* m, const or_real* q, or_real* R, int64_t n_sel, const int64_t* sel) {
  int64_t ne = m->ne;
  /* elements whose residual is wanted */
  uint8_t* want = (uint8_t*)calloc(ne, 1);
  if (sel) {
    for (int64_t i = 0; i < n_sel; ++i) {
      if (sel[i] < 0 || sel[i] >= ne) {
        free(want);
        set_err("selected element out of range");
        return -1;
      }
      want[sel[i]] = 1;
    }
  } else {
    memset(want, 1, ne);
  }
  /* geometry is needed on the wanted elements and their face neighbours; gradients on
   * the NS elements among them */
  uint8_t* need = (uint8_t*)calloc(ne, 1);
  for (int64_t e = 0; e < ne; ++e)
    if (want[e]) {
      need[e] = 1;
      for (int f = 0; f < 6; ++f)
        if (m->nb_e[e * 6 + f] >= 0) need[m->nb_e[e * 6 + f]] = 1;
    }
  work_t W;
  W.m = m;
  W.q = q;
  W.geo = (geo_t*)calloc(ne, sizeof(geo_t));
  W.G = (or_real**)calloc(ne, sizeof(or_real*));
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * ne);
  int64_t nl = 0;
  for (int64_t e = 0; e < ne; ++e)
    if (need[e]) list[nl++] = e;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nl; ++i) compute_geo(m, list[i], &W.geo[list[i]]);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nl; ++i) {
    int64_t e = list[i];
    if (!m->flag[e]) continue;
    int n = m->N[e] + 1;
    W.G[e] = (or_real*)malloc(sizeof(or_real) * 9 * n * n * n);
    element_gradient(&W, e, W.G[e]);
  }
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : rc)
  for (int64_t e = 0; e < ne; ++e)
    if (want[e]) rc |= element_residual(&W, e, R) ? 1 : 0;
  free(list);
  free_work(&W);
  free(need);
  free(want);
  if (rc) {
    set_err("Riemann solver failed");
    return -1;
  }
  return 0;
}

int or_rk_step(const or_mesh* m, or_real* q, or_real* g, or_real dt, int nsteps) {
  int64_t T4 = 4 * m->total;
  or_real* R = (or_real*)malloc(sizeof(or_real) * T4);
  for (int st = 0; st < nsteps; ++st)
    for (int s = 0; s < 3; ++s) {
      if (or_residual(m, q, R, 0, NULL)) {
        free(R);
        return -1;
      }
      for (int64_t i = 0; i < T4; ++i) {
        g[i] = (s == 0 ? 0.0 : RK_A[s] * g[i]) + dt * R[i];
        q[i] = q[i] + RK_B[s] * g[i];
      }
    }
  free(R);
  return 0;
}

int or_conservation(const or_mesh* m, const or_real* R, or_real out[4]) {
  int64_t ne = m->ne;
  or_real* part = (or_real*)calloc(4 * ne, sizeof(or_real));
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t e = 0; e < ne; ++e) {
    geo_t gt;
    compute_geo(m, e, &gt);
    int N = m->N[e], n = N + 1;
    const or_real* w = m->op[N].w;
    for (int v = 0; v < 4; ++v) {
      or_real s = 0.0;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            int64_t p = i + n * (j + n * k);
            s += w[i] * w[j] * w[k] * gt.J[p] * R[v * m->total + m->off[e] + p];
          }
      part[v * ne + e] = s;
    }
    free(gt.J);
    free(gt.Ja);
  }
  for (int v = 0; v < 4; ++v) {
    or_real s = 0.0;
    for (int64_t e = 0; e < ne; ++e) s += part[v * ne + e];
    out[v] = s;
  }
  free(part);
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Compressible Navier-Stokes (App. A): state u = (rho, rho v, rho e), ideal gas with unit
 * gas constant (p = (gamma - 1)(rho e - rho |v|^2 / 2), T = p / rho, H = (rho e + p) / rho).
 * The same weak form as above (App. B, Eq. NS4, viscous terms under BR1), five variables.
 * ---------------------------------------------------------------------------------- */

static void cns_prim(const or_real u[5], or_real gamma, or_real v[3], or_real* p) {
  for (int c = 0; c < 3; ++c) v[c] = u[1 + c] / u[0];
  *p = (gamma - 1.0) * (u[4] - 0.5 * u[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
}

/* Euler flux along n_hat: (rho v.n, rho v v.n + p n, (rho e + p) v.n) */
void or_cns_flux(const or_real u[5], const or_real nh[3], or_real gamma, or_real out[5]) {
  or_real v[3], p;
  cns_prim(u, gamma, v, &p);
  const or_real vn = v[0] * nh[0] + v[1] * nh[1] + v[2] * nh[2];
  out[0] = u[0] * vn;
  for (int c = 0; c < 3; ++c) out[1 + c] = u[1 + c] * vn + p * nh[c];
  out[4] = (u[4] + p) * vn;
}

/* d(F.n)/du written in (v, H): for an ideal gas the Jacobian depends on the state only
 * through the velocity and the total enthalpy. Rows/columns (rho, m1, m2, m3, E). */
static void cns_jacobian_vH(const or_real v[3], or_real H, const or_real nh[3], or_real gamma, or_real A[25]) {
  const or_real g1 = gamma - 1.0;
  const or_real vn = v[0] * nh[0] + v[1] * nh[1] + v[2] * nh[2];
  const or_real k = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int i = 0; i < 25; ++i) A[i] = 0.0;
  /* mass: d(m.n)/du */
  for (int c = 0; c < 3; ++c) A[0 * 5 + 1 + c] = nh[c];
  /* momentum: m_i vn + p n_i, with dp/du = g1 (k, -v, 1) */
  for (int i = 0; i < 3; ++i) {
    A[(1 + i) * 5 + 0] = -v[i] * vn + g1 * k * nh[i];
    for (int c = 0; c < 3; ++c) A[(1 + i) * 5 + 1 + c] = v[i] * nh[c] - g1 * v[c] * nh[i] + (i == c ? vn : 0.0);
    A[(1 + i) * 5 + 4] = g1 * nh[i];
  }
  /* energy: H m.n, with d(rho H)/du = (g1 k, -g1 v, gamma) */
  A[4 * 5 + 0] = vn * (g1 * k - H);
  for (int c = 0; c < 3; ++c) A[4 * 5 + 1 + c] = H * nh[c] - g1 * v[c] * vn;
  A[4 * 5 + 4] = gamma * vn;
}

void or_cns_jacobian(const or_real u[5], const or_real nh[3], or_real gamma, or_real A[25]) {
  or_real v[3], p;
  cns_prim(u, gamma, v, &p);
  cns_jacobian_vH(v, (u[4] + p) / u[0], nh, gamma, A);
}

/* |A| at the Roe average (sqrt(rho)-weighted v and H) by its eigen-decomposition
 * R |Lambda| R^-1, R^-1 by Gauss-Jordan. Eigenvectors: acoustic (1, v -+ a n, H -+ a vn),
 * entropy (1, v, |v|^2/2), shear (0, t, v.t) for two unit tangents t. */
int or_cns_roe_abs_jacobian(const or_real uL[5], const or_real uR[5], const or_real nh[3], or_real gamma,
                            or_real absA[25]) {
  or_real vL[3], vR[3], pL, pR;
  cns_prim(uL, gamma, vL, &pL);
  cns_prim(uR, gamma, vR, &pR);
  if (!(uL[0] > 0.0) || !(uR[0] > 0.0)) return -1;
  const or_real sL = SQRT(uL[0]), sR = SQRT(uR[0]);
  const or_real HL = (uL[4] + pL) / uL[0], HR = (uR[4] + pR) / uR[0];
  or_real v[3];
  for (int c = 0; c < 3; ++c) v[c] = (sL * vL[c] + sR * vR[c]) / (sL + sR);
  const or_real H = (sL * HL + sR * HR) / (sL + sR);
  const or_real k = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const or_real a2 = (gamma - 1.0) * (H - k);
  if (!(a2 > 0.0)) return -1;
  const or_real a = SQRT(a2);
  const or_real vn = v[0] * nh[0] + v[1] * nh[1] + v[2] * nh[2];
  /* two unit tangents: t1 from the coordinate axis least aligned with n */
  int ax = 0;
  for (int c = 1; c < 3; ++c)
    if (FABS(nh[c]) < FABS(nh[ax])) ax = c;
  or_real e[3] = {0.0, 0.0, 0.0};
  e[ax] = 1.0;
  or_real t1[3] = {nh[1] * e[2] - nh[2] * e[1], nh[2] * e[0] - nh[0] * e[2], nh[0] * e[1] - nh[1] * e[0]};
  const or_real l1 = SQRT(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int c = 0; c < 3; ++c) t1[c] /= l1;
  const or_real t2[3] = {nh[1] * t1[2] - nh[2] * t1[1], nh[2] * t1[0] - nh[0] * t1[2], nh[0] * t1[1] - nh[1] * t1[0]};
  or_real R[25], lam[5];
  /* columns: 0 acoustic -, 1 entropy, 2 shear t1, 3 shear t2, 4 acoustic + */
  R[0 * 5 + 0] = 1.0;
  R[0 * 5 + 1] = 1.0;
  R[0 * 5 + 2] = 0.0;
  R[0 * 5 + 3] = 0.0;
  R[0 * 5 + 4] = 1.0;
  for (int c = 0; c < 3; ++c) {
    R[(1 + c) * 5 + 0] = v[c] - a * nh[c];
    R[(1 + c) * 5 + 1] = v[c];
    R[(1 + c) * 5 + 2] = t1[c];
    R[(1 + c) * 5 + 3] = t2[c];
    R[(1 + c) * 5 + 4] = v[c] + a * nh[c];
  }
  R[4 * 5 + 0] = H - a * vn;
  R[4 * 5 + 1] = k;
  R[4 * 5 + 2] = v[0] * t1[0] + v[1] * t1[1] + v[2] * t1[2];
  R[4 * 5 + 3] = v[0] * t2[0] + v[1] * t2[1] + v[2] * t2[2];
  R[4 * 5 + 4] = H + a * vn;
  lam[0] = vn - a;
  lam[1] = lam[2] = lam[3] = vn;
  lam[4] = vn + a;
  or_real Rc[25], Ri[25];
  for (int i = 0; i < 25; ++i) {
    Rc[i] = R[i];
    Ri[i] = (i % 6 == 0) ? 1.0 : 0.0;
  }
  if (gauss_jordan(5, Rc, 5, Ri)) return -1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      or_real s = 0.0;
      for (int w = 0; w < 5; ++w) s += R[i * 5 + w] * FABS(lam[w]) * Ri[w * 5 + j];
      absA[i * 5 + j] = s;
    }
  return 0;
}

/* Roe: (F(uL) + F(uR))/2 - |A_roe| (uR - uL)/2; LLF: the largest |vn| + a of the two sides */
int or_cns_riemann(const or_real uL[5], const or_real uR[5], const or_real nh[3], const or_params* prm,
                   or_real out[5]) {
  or_real fL[5], fR[5];
  or_cns_flux(uL, nh, prm->gamma, fL);
  or_cns_flux(uR, nh, prm->gamma, fR);
  if (prm->riemann == 0) {
    or_real absA[25];
    if (or_cns_roe_abs_jacobian(uL, uR, nh, prm->gamma, absA)) return -1;
    for (int i = 0; i < 5; ++i) {
      or_real d = 0.0;
      for (int j = 0; j < 5; ++j) d += absA[i * 5 + j] * (uR[j] - uL[j]);
      out[i] = 0.5 * (fL[i] + fR[i]) - 0.5 * d;
    }
  } else {
    or_real s = 0.0;
    const or_real* us[2] = {uL, uR};
    for (int k = 0; k < 2; ++k) {
      or_real v[3], p;
      cns_prim(us[k], prm->gamma, v, &p);
      if (!(us[k][0] > 0.0) || !(p > 0.0)) return -1;
      const or_real sp = FABS(v[0] * nh[0] + v[1] * nh[1] + v[2] * nh[2]) + SQRT(prm->gamma * p / us[k][0]);
      if (sp > s) s = sp;
    }
    for (int i = 0; i < 5; ++i) out[i] = 0.5 * (fL[i] + fR[i]) - 0.5 * s * (uR[i] - uL[i]);
  }
  return 0;
}

/* primitive quantities lifted by BR1: phi = (v1, v2, v3, T) */
static void cns_phi(const or_real u[5], or_real gamma, or_real phi[4]) {
  or_real v[3], p;
  cns_prim(u, gamma, v, &p);
  for (int c = 0; c < 3; ++c) phi[c] = v[c];
  phi[3] = p / u[0];
}

/* the conservative state at the face points: the face nodes (Gauss-Lobatto) or the
 * interpolation along the normal lines (Gauss-Legendre) */
static void face_u5(const or_mesh* m, const or_real* u, int64_t e, int f, or_real* T /*[5][n2]*/) {
  int N = m->N[e], n = N + 1, n2 = n * n;
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a)
      for (int v = 0; v < 5; ++v) T[v * n2 + a + n * b] = face_value(m, N, f, a, b, u + v * m->total + m->off[e]);
}

/* the neighbour's face state in my face coordinates (conforming faces: same order), or the ghost
 * behind a boundary face: the far-field state at an inflow (tag 1); interior density and
 * momentum with the far-field pressure at an outflow (tag 2); the mirror state (rho, -rho v,
 * rho e) at a no-slip wall (tag 3), the normal momentum reversed at a free-slip wall (tag 4),
 * density and energy, hence p and T, kept */
static void cns_nbr_face(const or_mesh* m, const or_real* u, const geo_t* gt, int64_t e, int f, or_real* T /*[5][n2]*/) {
  int N = m->N[e], n = N + 1, n2 = n * n;
  int64_t nb = m->nb_e[e * 6 + f];
  if (nb < 0) {
    const int tag = m->bc[e * 6 + f];
    const or_real g1 = m->p.gamma - 1.0;
    face_u5(m, u, e, f, T);
    if (tag == 1) { /* far-field inflow: (rho_inf, rho_inf v_inf, p_inf/(gamma-1) + rho_inf |v_inf|^2/2) */
      const or_real r = m->p.inflow[0], v[3] = {m->p.inflow[1], m->p.inflow[2], m->p.inflow[3]};
      for (int p = 0; p < n2; ++p) {
        T[p] = r;
        for (int c = 0; c < 3; ++c) T[(1 + c) * n2 + p] = r * v[c];
        T[4 * n2 + p] = m->p.p_inf / g1 + 0.5 * r * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      }
      return;
    }
    if (tag == 2) { /* pressure outflow: interior density and momentum, the far-field pressure */
      for (int p = 0; p < n2; ++p) {
        const or_real mm = T[n2 + p] * T[n2 + p] + T[2 * n2 + p] * T[2 * n2 + p] + T[3 * n2 + p] * T[3 * n2 + p];
        T[4 * n2 + p] = m->p.p_inf / g1 + 0.5 * mm / T[p];
      }
      return;
    }
    or_real* S = (or_real*)malloc(sizeof(or_real) * 3 * n2);
    face_S(m, gt, e, f, S);
    for (int p = 0; p < n2; ++p) {
      const or_real Sv[3] = {S[p], S[n2 + p], S[2 * n2 + p]};
      const or_real ss = Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2];
      const or_real mn = (T[n2 + p] * Sv[0] + T[2 * n2 + p] * Sv[1] + T[3 * n2 + p] * Sv[2]) / ss;
      for (int c = 0; c < 3; ++c)
        T[(1 + c) * n2 + p] = tag == 3 ? -T[(1 + c) * n2 + p] : T[(1 + c) * n2 + p] - 2.0 * mn * Sv[c];
    }
    free(S);
    return;
  }
  or_real* tn = (or_real*)malloc(sizeof(or_real) * 5 * n * n);
  face_u5(m, u, nb, m->nb_f[e * 6 + f], tn);
  nbr_to_mortar(m->p.nodes, N, N, m->nb_o[e * 6 + f], 5, tn, T);
  free(tn);
}

typedef struct {
  const or_mesh* m;
  const or_real* u;
  geo_t* geo;
  or_real** G;  /* per NS element [4][3][n3] */
} cwork_t;

static int cns_face_mortar(const cwork_t* W, int64_t e, int f, or_real* LU, or_real* LH);

/* BR1 gradient of phi, weak form: w J G_ck = -sum_d (w/w_{i_d}) sum_m w_m D_{m i_d} (phi_c Ja^d_k)_m
 * + face terms phi*_c S_k with phi* = (phi^- + phi^+)/2 */
static void cns_gradient(const cwork_t* W, int64_t e, or_real* G) {
  const or_mesh* m = W->m;
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  const or_real* w = m->op[N].w;
  const or_real* D = m->op[N].D;
  const geo_t* gt = &W->geo[e];
  or_real* phi = (or_real*)malloc(sizeof(or_real) * 4 * n3);
  for (int p = 0; p < n3; ++p) {
    or_real uu[5], ph[4];
    for (int v = 0; v < 5; ++v) uu[v] = W->u[v * m->total + m->off[e] + p];
    cns_phi(uu, m->p.gamma, ph);
    for (int c = 0; c < 4; ++c) phi[c * n3 + p] = ph[c];
  }
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < 3; ++k)
      for (int kk = 0; kk < n; ++kk)
        for (int jj = 0; jj < n; ++jj)
          for (int ii = 0; ii < n; ++ii) {
            int ijk[3] = {ii, jj, kk};
            or_real s = 0.0;
            for (int d = 0; d < 3; ++d) {
              or_real sd = 0.0;
              for (int mm = 0; mm < n; ++mm) {
                int src[3] = {ii, jj, kk};
                src[d] = mm;
                int64_t ps = src[0] + n * (src[1] + n * src[2]);
                sd += w[mm] * D[mm * n + ijk[d]] * phi[c * n3 + ps] * gt->Ja[(d * 3 + k) * n3 + ps];
              }
              s -= sd / w[ijk[d]];
            }
            G[(c * 3 + k) * n3 + ii + n * (jj + n * kk)] = s;
          }
  or_real* LU = (or_real*)malloc(sizeof(or_real) * 12 * n2);
  for (int f = 0; f < 6; ++f) {
    cns_face_mortar(W, e, f, LU, NULL); /* projected phi* S at my face points */
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a)
        for (int ck = 0; ck < 12; ++ck) face_lift(m, N, f, a, b, LU[ck * n2 + a + n * b], G + ck * n3);
  }
  free(LU);
  free(phi);
  for (int ck = 0; ck < 12; ++ck)
    for (int p = 0; p < n3; ++p) G[ck * n3 + p] /= gt->J[p];
}

/* viscous flux rows at one node of an NS element: Fv[v][k], v = momentum 1..3 then energy */
static void cns_visc_flux(const cwork_t* W, int64_t e, int n3, int64_t p, const or_real u[5], or_real Fv[4][3]) {
  const or_mesh* m = W->m;
  const or_real* G = W->G[e];
  or_real Gv[9], gT[3];
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) Gv[c * 3 + k] = G[(c * 3 + k) * n3 + p];
  for (int k = 0; k < 3; ++k) gT[k] = G[(9 + k) * n3 + p];
  const or_real mut = u[0] * or_eddy_viscosity(Gv, W->geo[e].delta, &m->p);
  const or_real mu = m->p.nu * m->vscale[e], mt = mut * m->vscale[e];
  const or_real mue = mu + mt;
  const or_real cp = m->p.gamma / (m->p.gamma - 1.0);
  const or_real kappa = cp * (mu / m->p.prandtl + mt / m->p.prandtl_t);
  const or_real tr = Gv[0] + Gv[4] + Gv[8];
  or_real tau[3][3];
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 3; ++k) tau[c][k] = mue * (Gv[c * 3 + k] + Gv[k * 3 + c]) - (c == k ? 2.0 / 3.0 * mue * tr : 0.0);
  or_real v[3];
  for (int c = 0; c < 3; ++c) v[c] = u[1 + c] / u[0];
  for (int k = 0; k < 3; ++k) {
    for (int c = 0; c < 3; ++c) Fv[c][k] = tau[c][k];
    Fv[3][k] = v[0] * tau[0][k] + v[1] * tau[1][k] + v[2] * tau[2][k] + kappa * gT[k];
  }
}

/* outward area-weighted viscous flux trace Fv . S of element e on face f, [4][n2] (zero for Euler) */
static void cns_face_fv(const cwork_t* W, int64_t e, int f, or_real* out) {
  const or_mesh* m = W->m;
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  if (!m->flag[e]) {
    memset(out, 0, sizeof(or_real) * 4 * n2);
    return;
  }
  if (m->p.nodes == 1) {
    /* Gauss-Legendre: the outward contravariant viscous flux sigma Ja^d . Fv at every node,
     * interpolated to the face */
    const geo_t* gt = &W->geo[e];
    const int d = f >> 1;
    const or_real sg = (f & 1) ? 1.0 : -1.0;
    or_real* Ft = (or_real*)malloc(sizeof(or_real) * 4 * n3);
    for (int p = 0; p < n3; ++p) {
      or_real uu[5], Fv[4][3];
      for (int v = 0; v < 5; ++v) uu[v] = W->u[v * m->total + m->off[e] + p];
      cns_visc_flux(W, e, n3, p, uu, Fv);
      for (int v = 0; v < 4; ++v) {
        or_real s = 0.0;
        for (int k = 0; k < 3; ++k) s += Fv[v][k] * gt->Ja[(d * 3 + k) * n3 + p];
        Ft[v * n3 + p] = sg * s;
      }
    }
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a)
        for (int v = 0; v < 4; ++v) out[v * n2 + a + n * b] = face_value(m, N, f, a, b, Ft + v * n3);
    free(Ft);
    return;
  }
  or_real* S = (or_real*)malloc(sizeof(or_real) * 3 * n2);
  face_S(m, &W->geo[e], e, f, S);
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      const int fp = a + n * b;
      const int64_t p = face_node(f, N, a, b);
      or_real uu[5], Fv[4][3];
      for (int v = 0; v < 5; ++v) uu[v] = W->u[v * m->total + m->off[e] + p];
      cns_visc_flux(W, e, n3, p, uu, Fv);
      for (int v = 0; v < 4; ++v) out[v * n2 + fp] = Fv[v][0] * S[fp] + Fv[v][1] * S[n2 + fp] + Fv[v][2] * S[2 * n2 + fp];
    }
  free(S);
}

/* Face (e, f) of the compressible form on the mortar of the larger order (reading 10 with
 * five variables): both sides' conservative face states (and, for LH, their outward viscous
 * traces) interpolated to the mortar, combined point by point, L2-projected back to my order.
 * A conforming face is its own mortar (identity operators); a boundary face takes the ghost
 * state and the boundary's viscous rule on my own face.
 *   LU [12][n2] (NULL to skip): projected phi*_c S_k, phi* = ({{phi(u)}}) for phi = (v, T);
 *   LH [5][n2]  (NULL to skip): projected F_e*(u-, u+) . S - F_v* . S, my outward S.
 * Returns -1 if a Riemann flux failed. */
static int cns_face_mortar(const cwork_t* W, int64_t e, int f, or_real* LU, or_real* LH) {
  const or_mesh* m = W->m;
  const geo_t* gt = &W->geo[e];
  const int N = m->N[e], n = N + 1, n2 = n * n;
  const int64_t nb = m->nb_e[e * 6 + f];
  const int Nn = nb >= 0 ? m->N[nb] : N, nn = Nn + 1, nn2 = nn * nn;
  const int Mo = N > Nn ? N : Nn, nM = Mo + 1, nM2 = nM * nM;
  const int nf = m->nb_f[e * 6 + f], o = m->nb_o[e * 6 + f], gl = m->p.nodes;
  or_real* buf = (or_real*)calloc((size_t)(5 * n2 + 3 * n2 + 4 * n2 + 5 * nn2 + 4 * nn2) + (size_t)nM2 * (5 + 5 + 3 + 4 + 4 + 12),
                                  sizeof(or_real));
  or_real *um = buf, *S = um + 5 * n2, *fvm = S + 3 * n2, *tn = fvm + 4 * n2, *fvn = tn + 5 * nn2;
  or_real *uM = fvn + 4 * nn2, *uP = uM + 5 * nM2, *SM = uP + 5 * nM2, *FvM = SM + 3 * nM2, *FvP = FvM + 4 * nM2;
  or_real* H = FvP + 4 * nM2; /* [12][nM2] */
  face_u5(m, W->u, e, f, um);
  face_S(m, gt, e, f, S);
  mine_to_mortar(gl, N, Mo, 5, um, uM);
  mine_to_mortar(gl, N, Mo, 3, S, SM);
  if (nb >= 0) {
    face_u5(m, W->u, nb, nf, tn);
    nbr_to_mortar(gl, Nn, Mo, o, 5, tn, uP);
  } else {
    cns_nbr_face(m, W->u, gt, e, f, uP); /* the ghost on my own face (Mo = N) */
  }
  if (LU) {
    for (int p = 0; p < nM2; ++p) {
      or_real qm[5], qp[5], pm[4], pp[4];
      for (int v = 0; v < 5; ++v) {
        qm[v] = uM[v * nM2 + p];
        qp[v] = uP[v * nM2 + p];
      }
      cns_phi(qm, m->p.gamma, pm);
      cns_phi(qp, m->p.gamma, pp);
      for (int c = 0; c < 4; ++c)
        for (int k = 0; k < 3; ++k) H[(c * 3 + k) * nM2 + p] = 0.5 * (pm[c] + pp[c]) * SM[k * nM2 + p];
    }
    mortar_to_mine(gl, Mo, N, 12, H, LU);
  }
  int rc = 0;
  if (LH) {
    const int any_visc = m->flag[e] || (nb >= 0 && m->flag[nb]);
    if (any_visc) {
      cns_face_fv(W, e, f, fvm);
      mine_to_mortar(gl, N, Mo, 4, fvm, FvM);
      if (nb >= 0) {
        cns_face_fv(W, nb, nf, fvn);
        nbr_to_mortar(gl, Nn, Mo, o, 4, fvn, FvP);
      } else {
        /* inflow, outflow: the interior viscous flux. Adiabatic walls: the ghost's outward flux
         * makes the BR1 average the interior traction (no-slip) or its normal part (free-slip,
         * the reflection R = I - 2 n n^T of the traction), and a zero energy flux (no heat flux,
         * no work by a traction on a resting or tangentially moving wall) */
        const int tag = m->bc[e * 6 + f];
        for (int p = 0; p < nM2; ++p) {
          if (tag == 1 || tag == 2) {
            for (int v = 0; v < 4; ++v) FvP[v * nM2 + p] = -FvM[v * nM2 + p];
            continue;
          }
          const or_real Sv[3] = {SM[p], SM[nM2 + p], SM[2 * nM2 + p]};
          const or_real ss = Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2];
          const or_real fn = (FvM[p] * Sv[0] + FvM[nM2 + p] * Sv[1] + FvM[2 * nM2 + p] * Sv[2]) / ss;
          for (int c = 0; c < 3; ++c)
            FvP[c * nM2 + p] = tag == 3 ? -FvM[c * nM2 + p] : FvM[c * nM2 + p] - 2.0 * fn * Sv[c];
          FvP[3 * nM2 + p] = FvM[3 * nM2 + p];
        }
      }
    }
    /* F_v* . S = wm Fv^- . S - wp Fv^+ . S^+: the BR1 average, or the NS side alone on an
     * Euler-NS face with the one-sided choice */
    or_real wm = 0.5, wp = 0.5;
    if (m->p.mixed_face == 1 && nb >= 0 && m->flag[e] != m->flag[nb]) {
      wm = m->flag[e] ? 1.0 : 0.0;
      wp = m->flag[e] ? 0.0 : 1.0;
    }
    for (int p = 0; p < nM2; ++p) {
      const or_real Sv[3] = {SM[p], SM[nM2 + p], SM[2 * nM2 + p]};
      const or_real s = SQRT(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
      const or_real nh[3] = {Sv[0] / s, Sv[1] / s, Sv[2] / s};
      or_real qm[5], qp[5], Fs[5];
      for (int v = 0; v < 5; ++v) {
        qm[v] = uM[v * nM2 + p];
        qp[v] = uP[v * nM2 + p];
      }
      if (or_cns_riemann(qm, qp, nh, &m->p, Fs)) rc = -1;
      H[p] = Fs[0] * s;
      for (int v = 0; v < 4; ++v) H[(1 + v) * nM2 + p] = Fs[1 + v] * s - (wm * FvM[v * nM2 + p] - wp * FvP[v * nM2 + p]);
    }
    mortar_to_mine(gl, Mo, N, 5, H, LH);
  }
  free(buf);
  return rc;
}

/* w J R = sum_d (w / w_{i_d}) sum_m w_m D_{m i_d} Ftil^d_m - w_face H*, five variables */
static int cns_element_residual(const cwork_t* W, int64_t e, or_real* R) {
  const or_mesh* m = W->m;
  int N = m->N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
  const or_real* w = m->op[N].w;
  const or_real* D = m->op[N].D;
  const geo_t* gt = &W->geo[e];
  int64_t o = m->off[e], T = m->total;
  or_real* Ft = (or_real*)malloc(sizeof(or_real) * 15 * n3);
  for (int p = 0; p < n3; ++p) {
    or_real uu[5], F[5][3];
    for (int v = 0; v < 5; ++v) uu[v] = W->u[v * T + o + p];
    for (int k = 0; k < 3; ++k) {
      const or_real ek[3] = {k == 0 ? 1.0 : 0.0, k == 1 ? 1.0 : 0.0, k == 2 ? 1.0 : 0.0};
      or_real fk[5];
      or_cns_flux(uu, ek, m->p.gamma, fk);
      for (int v = 0; v < 5; ++v) F[v][k] = fk[v];
    }
    if (m->flag[e]) {
      or_real Fv[4][3];
      cns_visc_flux(W, e, n3, p, uu, Fv);
      for (int v = 0; v < 4; ++v)
        for (int k = 0; k < 3; ++k) F[1 + v][k] -= Fv[v][k];
    }
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 5; ++v) {
        or_real s = 0.0;
        for (int k = 0; k < 3; ++k) s += gt->Ja[(d * 3 + k) * n3 + p] * F[v][k];
        Ft[(d * 5 + v) * n3 + p] = s;
      }
  }
  or_real* JR = (or_real*)calloc(5 * n3, sizeof(or_real));
  for (int v = 0; v < 5; ++v)
    for (int kk = 0; kk < n; ++kk)
      for (int jj = 0; jj < n; ++jj)
        for (int ii = 0; ii < n; ++ii) {
          int ijk[3] = {ii, jj, kk};
          or_real s = 0.0;
          for (int d = 0; d < 3; ++d) {
            or_real sd = 0.0;
            for (int mm = 0; mm < n; ++mm) {
              int src[3] = {ii, jj, kk};
              src[d] = mm;
              sd += w[mm] * D[mm * n + ijk[d]] * Ft[(d * 5 + v) * n3 + src[0] + n * (src[1] + n * src[2])];
            }
            s += sd / w[ijk[d]];
          }
          JR[v * n3 + ii + n * (jj + n * kk)] = s;
        }
  /* faces: the projected H* = F_e* . S - F_v* . S from each face's mortar */
  or_real* LH = (or_real*)malloc(sizeof(or_real) * 5 * n2);
  int rc = 0;
  for (int f = 0; f < 6; ++f) {
    if (cns_face_mortar(W, e, f, NULL, LH)) rc = -1;
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a)
        for (int v = 0; v < 5; ++v) face_lift(m, N, f, a, b, -LH[v * n2 + a + n * b], JR + v * n3);
  }
  for (int v = 0; v < 5; ++v)
    for (int p = 0; p < n3; ++p) R[v * T + o + p] = JR[v * n3 + p] / gt->J[p];
  free(LH);
  free(JR);
  free(Ft);
  return rc;
}

static int cns_check(const or_mesh* m) {
  if (!(m->p.gamma > 1.0) || !(m->p.prandtl > 0.0) || !(m->p.prandtl_t > 0.0)) {
    set_err("compressible form: need gamma > 1 and positive Prandtl numbers");
    return -1;
  }
  for (int64_t e = 0; e < m->ne; ++e)
    for (int f = 0; f < 6; ++f) {
      const int64_t nb = m->nb_e[e * 6 + f];
      if (nb < 0) {
        const int tag = m->bc[e * 6 + f];
        if ((tag == 1 || tag == 2) && !(m->p.inflow[0] > 0.0 && m->p.p_inf > 0.0)) {
          set_err("compressible form: inflow/outflow faces need a positive far-field density and pressure");
          return -1;
        }
        continue;
      }
    }
  return 0;
}

static void cns_free(cwork_t* W) {
  for (int64_t e = 0; e < W->m->ne; ++e) {
    free(W->geo[e].J);
    free(W->geo[e].Ja);
    free(W->G[e]);
  }
  free(W->geo);
  free(W->G);
}

int or_cns_element_gradient(const or_mesh* m, const or_real* u, int64_t e, or_real* G) {
  if (e < 0 || e >= m->ne || cns_check(m)) return -1;
  uint8_t* need = (uint8_t*)calloc(m->ne, 1);
  need[e] = 1;
  for (int f = 0; f < 6; ++f)
        if (m->nb_e[e * 6 + f] >= 0) need[m->nb_e[e * 6 + f]] = 1;
  cwork_t W;
  W.m = m;
  W.u = u;
  W.geo = (geo_t*)calloc(m->ne, sizeof(geo_t));
  W.G = (or_real**)calloc(m->ne, sizeof(or_real*));
  for (int64_t i = 0; i < m->ne; ++i)
    if (need[i]) compute_geo(m, i, &W.geo[i]);
  cns_gradient(&W, e, G);
  cns_free(&W);
  free(need);
  return 0;
}

int or_cns_residual(const or_mesh* m, const or_real* u, or_real* R, int64_t n_sel, const int64_t* sel) {
  if (cns_check(m)) return -1;
  int64_t ne = m->ne;
  uint8_t* want = (uint8_t*)calloc(ne, 1);
  if (sel) {
    for (int64_t i = 0; i < n_sel; ++i) {
      if (sel[i] < 0 || sel[i] >= ne) {
        free(want);
        set_err("selected element out of range");
        return -1;
      }
      want[sel[i]] = 1;
    }
  } else {
    memset(want, 1, ne);
  }
  uint8_t* need = (uint8_t*)calloc(ne, 1);
  for (int64_t e = 0; e < ne; ++e)
    if (want[e]) {
      need[e] = 1;
      for (int f = 0; f < 6; ++f)
        if (m->nb_e[e * 6 + f] >= 0) need[m->nb_e[e * 6 + f]] = 1;
    }
  /* a neighbour's gradient needs its own neighbours' geometry */
  uint8_t* need2 = (uint8_t*)calloc(ne, 1);
  for (int64_t e = 0; e < ne; ++e)
    if (need[e]) {
      need2[e] = 1;
      for (int f = 0; f < 6; ++f)
        if (m->nb_e[e * 6 + f] >= 0) need2[m->nb_e[e * 6 + f]] = 1;
    }
  cwork_t W;
  W.m = m;
  W.u = u;
  W.geo = (geo_t*)calloc(ne, sizeof(geo_t));
  W.G = (or_real**)calloc(ne, sizeof(or_real*));
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t e = 0; e < ne; ++e)
    if (need2[e]) compute_geo(m, e, &W.geo[e]);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t e = 0; e < ne; ++e) {
    if (!need[e] || !m->flag[e]) continue;
    int n = m->N[e] + 1;
    W.G[e] = (or_real*)malloc(sizeof(or_real) * 12 * n * n * n);
    cns_gradient(&W, e, W.G[e]);
  }
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : rc)
  for (int64_t e = 0; e < ne; ++e)
    if (want[e]) rc |= cns_element_residual(&W, e, R) ? 1 : 0;
  cns_free(&W);
  free(need);
  free(need2);
  free(want);
  if (rc) {
    set_err("Riemann solver failed (non-positive density or pressure)");
    return -1;
  }
  return 0;
}

int or_cns_rk_step(const or_mesh* m, or_real* u, or_real* g, or_real dt, int nsteps) {
  int64_t T5 = 5 * m->total;
  or_real* R = (or_real*)malloc(sizeof(or_real) * T5);
  for (int st = 0; st < nsteps; ++st)
    for (int s = 0; s < 3; ++s) {
      if (or_cns_residual(m, u, R, 0, NULL)) {
        free(R);
        return -1;
      }
      for (int64_t i = 0; i < T5; ++i) {
        g[i] = (s == 0 ? 0.0 : RK_A[s] * g[i]) + dt * R[i];
        u[i] = u[i] + RK_B[s] * g[i];
      }
    }
  free(R);
  return 0;
}

int or_cns_conservation(const or_mesh* m, const or_real* R, or_real out[5]) {
  int64_t ne = m->ne;
  or_real* part = (or_real*)calloc(5 * ne, sizeof(or_real));
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t e = 0; e < ne; ++e) {
    geo_t gt;
    compute_geo(m, e, &gt);
    int N = m->N[e], n = N + 1;
    const or_real* w = m->op[N].w;
    for (int v = 0; v < 5; ++v) {
      or_real s = 0.0;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            int64_t p = i + n * (j + n * k);
            s += w[i] * w[j] * w[k] * gt.J[p] * R[v * m->total + m->off[e] + p];
          }
      part[v * ne + e] = s;
    }
    free(gt.J);
    free(gt.Ja);
  }
  for (int v = 0; v < 5; ++v) {
    or_real s = 0.0;
    for (int64_t e = 0; e < ne; ++e) s += part[v * ne + e];
    out[v] = s;
  }
  free(part);
  return 0;
}
