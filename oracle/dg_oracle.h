/*
 * dg_oracle.h -- plain FP64 CPU oracle for the flagged Euler / NS-LES DGSEM residual.
 *
 * TEST INFRASTRUCTURE ONLY. This library exists so that tests, the smoke check and the
 * CPU-baseline leg of the benchmark can compare the CUDA path against an independent,
 * slow, obviously correct evaluation of the method. Nothing in the product links it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Method (Otmani et al., arXiv 2403.05463):
 *   - Sec. 2.3: each hexahedral element is flagged inviscid (Euler: convective terms only)
 *     or viscous/turbulent (full Navier-Stokes + LES eddy viscosity); elements couple only
 *     through interface numerical fluxes (Roe for convection, BR1 for viscous terms).
 *   - App. A: governing equations u_t + div F_e = div F_v,turb with the stress tensor
 *     tau = (mu+mu_t)(grad v + grad v^T) - 2/3 (mu+mu_t) I div v and the Vreman model.
 *     Read here in artificial-compressibility form with rho = 1, state q = (p, u, v, w).
 *   - App. B, Eqs. NS2-NS5: DGSEM on curvilinear hexahedra, weak form with the
 *     convective numerical flux on element faces, tensor-product Gauss quadrature
 *     (Gauss-Lobatto nodes, or the paper's Gauss-Legendre nodes with params.nodes = 1).
 *   - Sec. 2.3 (last paragraph): low-storage explicit third-order Runge-Kutta.
 *
 * Layout: q and R are SoA [4][total_nodes]; element e occupies nodes
 * [offset[e], offset[e] + (N_e+1)^3) with xi_1 fastest, then xi_2, then xi_3.
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

/* Floating-point type of the oracle: FP64 by default. Built with -DOR_EXTENDED=1 it computes
 * in long double (x87 80-bit on x86-64, IEEE binary128 on AArch64); that build only serves
 * parity checks whose FP64 conditioning is too poor to verify an FP64 tolerance. */
#if defined(OR_EXTENDED) && OR_EXTENDED
typedef long double or_real;
#else
typedef double or_real;
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  or_real nu;        /* kinematic viscosity 1/Re                                  */
  or_real c0sq;      /* artificial-compressibility wave speed squared             */
  or_real cs;        /* Smagorinsky constant                                      */
  or_real cv;        /* Vreman constant (paper: 0.07)                             */
  int closure;      /* 0 Smagorinsky, 1 Vreman                                   */
  int riemann;      /* 0 Roe, 1 local Lax-Friedrichs                             */
  int mixed_face;   /* viscous flux on a face between an NS and an Euler element
                       (Sec. 2.3 asks only that it be single-valued): 0 the average
                       of the NS side's flux and zero, 1 the NS side's flux alone    */
  int split;        /* convective volume term: 0 the standard form (App. B, Eq. NS4),
                       1 the kinetic-energy-preserving split form: along each direction
                       sum_m 2 D_im F#(q_i, q_m) with the two-point flux of or_kep_flux */
  or_real inflow[4]; /* ghost state used at inflow faces (velocity part)          */
  /* compressible form only (the or_cns_* entry points): ideal gas with unit gas constant,
     so T = p / rho and c_p = gamma / (gamma - 1); nu is then the dynamic viscosity mu   */
  or_real gamma;     /* ratio of specific heats                                   */
  or_real prandtl;   /* laminar Prandtl number                                    */
  or_real prandtl_t; /* turbulent Prandtl number                                  */
  int nodes;        /* element nodes and quadrature: 0 Gauss-Lobatto, 1 Gauss-Legendre
                       (the paper's choice, App. B): face values, face metric terms and
                       face fluxes are interpolated from the element's nodes and face terms
                       are lifted with l_i(+-1) / w_i; the split form needs
                       Gauss-Lobatto                                               */
  or_real p_inf;     /* compressible form: far-field pressure at inflow (with the far-field
                       (rho, u, v, w) in inflow[]) and static pressure at outflow     */
} or_params;

typedef struct or_mesh or_mesh;

/* 1D building blocks (Gauss-Lobatto-Legendre nodes on [-1,1]). */
int or_lgl(int N, or_real* x, or_real* w);                  /* x[N+1], w[N+1]          */
int or_gl(int N, or_real* x, or_real* w);                   /* Gauss-Legendre, N+1 nodes */
int or_dmat(int N, or_real* D);                            /* D[(N+1)*(N+1)] row-major */
int or_dmat_gl(int N, or_real* D);                         /* the same on Gauss-Legendre nodes */
int or_interp_lgl(int Ns, int Nd, or_real* I);             /* I[(Nd+1)][(Ns+1)]        */
int or_project_lgl(int Nh, int Nl, or_real* P);            /* P[(Nl+1)][(Nh+1)]        */
int or_interp_gl(int Ns, int Nd, or_real* I);              /* the same two on Gauss-Legendre */
int or_project_gl(int Nh, int Nl, or_real* P);             /* nodes                     */

/* Pointwise building blocks. n_hat must be a unit vector. */
void or_normal_flux(const or_real q[4], const or_real n_hat[3], or_real c0sq, or_real out[4]);
void or_flux_jacobian(const or_real q[4], const or_real n_hat[3], or_real c0sq, or_real A[16]);
int or_abs_jacobian(const or_real q[4], const or_real n_hat[3], or_real c0sq, or_real absA[16]);
/* Kinetic-energy-preserving two-point flux along one direction between nodes i and m, with
 * their contravariant metric vectors Ja_i, Ja_m (J dxi/dx for that direction): averages
 * {{.}} = (a_i + a_m)/2, U = {{Ja}}.{{u}}; out = (c0^2 U, {{u}} U + {{p}} {{Ja}}). */
void or_kep_flux(const or_real qi[4], const or_real qm[4], const or_real Ja_i[3], const or_real Ja_m[3],
                 or_real c0sq, or_real out[4]);
int or_riemann(const or_real qm[4], const or_real qp[4], const or_real n_hat[3],
               const or_params* prm, or_real out[4]);
or_real or_eddy_viscosity(const or_real G[9], or_real delta, const or_params* prm);
or_real or_rk3_linear(or_real z);   /* amplification of one RK3 step on y' = lambda y, z = lambda dt */

/* Mesh + discretisation. Returns NULL on error (see or_error()). */
or_mesh* or_create(int64_t n_elem, const int64_t* hex, int geom_degree, const or_real* geom_xyz,
                   const int8_t* bc_tag, const int8_t* order, const uint8_t* flag,
                   const or_params* prm);
void or_destroy(or_mesh* m);
const char* or_error(void);
int64_t or_total_nodes(const or_mesh* m);
const int64_t* or_offsets(const or_mesh* m);
int or_node_coords(const or_mesh* m, or_real* xyz);   /* [3][total_nodes] */
/* Per-element multiplier on (nu + nu_t) in NS elements (test hook; default 1). */
int or_set_visc_scale(or_mesh* m, const or_real* scale);
/* Element geometry: J[n^3], Ja[3][3][n^3] (Ja[i][c] = J dxi_i/dx_c). */
int or_element_geometry(const or_mesh* m, int64_t e, or_real* J, or_real* Ja);
/* BR1 velocity gradient of one NS element: G[3][3][n^3], G[c][k] = d u_c / d x_k. */
int or_element_gradient(const or_mesh* m, const or_real* q, int64_t e, or_real* G);
/* Residual R = dq/dt. sel == NULL: every element; otherwise only the listed ones are
 * written (the other entries of R are left untouched). */
int or_residual(const or_mesh* m, const or_real* q, or_real* R, int64_t n_sel, const int64_t* sel);
/* nsteps low-storage RK3 steps in place on q, g. */
int or_rk_step(const or_mesh* m, or_real* q, or_real* g, or_real dt, int nsteps);
/* out[v] = sum_e sum_nodes w_i w_j w_k J R_v. */
int or_conservation(const or_mesh* m, const or_real* R, or_real out[4]);

/* ---- Compressible Navier-Stokes (App. A) --------------------------------------------------
 * Conservative state u = (rho, rho v1, rho v2, rho v3, rho e), SoA [5][total_nodes], on the
 * same mesh, orders, flags and parameters (nu = mu, gamma, prandtl, prandtl_t, closure,
 * riemann, mixed_face). Flag 0 elements solve the Euler equations, flag 1 the Navier-Stokes
 * equations with the eddy viscosity mu_t = rho nu_t of the selected closure; heat flux
 * kappa grad T with kappa = c_p (mu / Pr + mu_t / Pr_t). BR1 lifts the primitive
 * (v1, v2, v3, T). p-nonconforming faces through five-variable mortars; boundary faces:
 * far-field inflow (tag 1) and pressure outflow (tag 2), which need inflow[0] > 0 and
 * p_inf > 0, and adiabatic no-slip (3) and free-slip (4) walls. Either node set. */
void or_cns_flux(const or_real u[5], const or_real n_hat[3], or_real gamma, or_real out[5]);
void or_cns_jacobian(const or_real u[5], const or_real n_hat[3], or_real gamma, or_real A[25]);
/* Roe matrix |A(u_roe)| = R |Lambda| R^-1 at the Roe average of uL, uR */
int or_cns_roe_abs_jacobian(const or_real uL[5], const or_real uR[5], const or_real n_hat[3], or_real gamma,
                            or_real absA[25]);
int or_cns_riemann(const or_real uL[5], const or_real uR[5], const or_real n_hat[3], const or_params* prm,
                   or_real out[5]);
/* BR1 gradient of (v1, v2, v3, T) of one NS element: G[4][3][n^3], G[c][k] = d phi_c / d x_k. */
int or_cns_element_gradient(const or_mesh* m, const or_real* u, int64_t e, or_real* G);
int or_cns_residual(const or_mesh* m, const or_real* u, or_real* R, int64_t n_sel, const int64_t* sel);
int or_cns_rk_step(const or_mesh* m, or_real* u, or_real* g, or_real dt, int nsteps);
int or_cns_conservation(const or_mesh* m, const or_real* R, or_real out[5]);
/* Number of OpenMP threads the oracle uses. */
int or_num_threads(void);
void or_set_num_threads(int n);  /* OpenMP threads of the element loops (n > 0) */

#ifdef __cplusplus
}
#endif
#endif
