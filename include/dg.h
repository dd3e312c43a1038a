/*
 * dg.h -- C ABI of the GB300 (sm_103a) flagged Euler / NS-LES DGSEM residual library.
 *
 * The library evaluates the explicit-time-step spatial residual of a nodal
 * Gauss-Lobatto DGSEM discretisation of incompressible flow in artificial-compressibility
 * form and advances it with a low-storage third-order Runge-Kutta scheme, after
 *   Otmani, Mateo-Gabin, Rubio, Ferrer, arXiv 2403.05463:
 *   - Sec. 2.3 (viscous/turbulent-inviscid interactions): every hexahedral element carries a
 *     flag; flag 0 solves the Euler equations (convective terms only), flag 1 the full
 *     Navier-Stokes equations with an LES eddy viscosity. Neighbours couple only through
 *     interface numerical fluxes: Roe for the convective part, BR1 for the viscous part.
 *   - App. A: u_t + div F_e = div F_v,turb with tau = (nu + nu_t)(grad v + grad v^T)
 *     - 2/3 (nu + nu_t) I div v, the Vreman closure (Smagorinsky selectable).
 *   - App. B, Eqs. NS2-NS5: DGSEM on curvilinear hexahedra (transfinite map, Jacobian J,
 *     contravariant fluxes), numerical flux on faces, tensor-product quadrature.
 *   - Sec. 2.3 (last paragraph): low-storage explicit third-order Runge-Kutta.
 *   - Sec. 3.2: local p-adaptation, one polynomial order per element, p-nonconforming faces.
 *
 * State: q = (p, u, v, w), rho = 1 (dg_params.model 0), or the compressible conservative
 * state u = (rho, rho v, rho e) of App. A (model 1). All state arrays are FP64, structure-of-
 * arrays [4][total_nodes] (model 0) or [5][total_nodes] (model 1; wherever this header says
 * [4][...] for q, g or R, read [5][...] under model 1): variable v of global node i lives at
 * q[v * total_nodes + i]. Element e
 * owns nodes [elem_offset[e], elem_offset[e] + (N_e + 1)^3), lexicographic with xi_1
 * fastest, then xi_2, then xi_3 (see dg_get_layout).
 *
 * Errors: every entry point returns a dg_status; none aborts. dg_last_error() gives a
 * thread-local message for the last failing call on that thread. Calls that take a stream
 * are asynchronous with respect to the host; device-side faults found by a kernel (a
 * non-positive Jacobian, a bounded wait that timed out) land in a device error word that
 * dg_check_device() and dg_conservation() read.
 *
 * Streams: one context is one solver; its calls must be ordered (one stream, or streams the
 * caller orders with events). Its library-owned buffers -- face traces, viscous results, the
 * tile queues of the one-launch stage kernel, the error word -- are shared by its launches, so
 * two of its calls running concurrently on unordered streams race. Separate contexts are
 * independent.
 *
 * Ownership: descriptors and host arrays passed in are copied; the caller keeps them.
 * Device arrays (q, g, R, xyz) are caller-owned, FP64, contiguous; the library never frees
 * them. Library-owned buffers (traces, geometry, tables) are freed by dg_destroy. The
 * reduced-precision path reads q with bulk copies of whole 16-byte blocks, so the 16-byte
 * blocks containing q's first and last bytes must be readable (true for any cudaMalloc or
 * PyTorch CUDA allocation).
 */
#ifndef DG_H
#define DG_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,         /* invalid argument (null pointer, out-of-range value)      */
  DG_ERR_MESH = 2,        /* inconsistent mesh (unmatched face, bad orientation, J<=0) */
  DG_ERR_CUDA = 3,        /* a CUDA runtime call failed                                */
  DG_ERR_OOM = 4,         /* device allocation failed                                  */
  DG_ERR_UNSUPPORTED = 5, /* valid input outside what this build implements            */
  DG_ERR_STATE = 6,       /* call out of order                                         */
  DG_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up                        */
  DG_ERR_DEVICE = 8       /* a kernel reported a fault in the device error word        */
} dg_status;

/* Mesh description (App. B: curvilinear hexahedra given by a polynomial map). */
typedef struct {
  int64_t n_elem;
  /* [n_elem][8] vertex ids, corner c = c1 + 2 c2 + 4 c3 sits at xi = (2c1-1, 2c2-1, 2c3-1).
   * Faces match by their four corner ids; periodic faces are those whose corners share ids.
   * The orientation of a shared face is derived from the corner ids (all 8 are supported). */
  const int64_t* hex;
  /* Geometry degree g (1 trilinear, 2 quadratic) and [n_elem][(g+1)^3][3] node coordinates at
   * the Gauss-Lobatto points of degree g (i.e. {-1,1} or {-1,0,1}), xi_1 fastest. Orders must
   * satisfy N_e >= g. */
  int geom_degree;
  const double* geom_xyz;
  /* [n_elem][6] boundary tag per local face f = 2 d + s (plane xi_{d+1} = s ? +1 : -1):
   * -1 interior or periodic, 1 inflow (velocity from dg_params.inflow, interior pressure),
   * 2 outflow (interior velocity, zero pressure), 3 no-slip wall (mirror ghost with the velocity
   * reversed; the interior viscous traction), 4 free-slip wall (mirror ghost with the normal
   * velocity reversed; the BR1 average with the mirror ghost keeps the normal traction).
   * NULL means every face is interior; any other value is DG_ERR_ARG. */
  const int8_t* bc_tag;
} dg_mesh_desc;

/* Physical and numerical parameters (App. A, Sec. 2.3). */
typedef struct {
  double nu;        /* kinematic viscosity 1/Re                                        */
  double c0sq;      /* artificial-compressibility wave speed squared                   */
  double cs;        /* Smagorinsky constant                                            */
  double cv;        /* Vreman constant (the paper uses 0.07)                           */
  int closure;      /* 0 Smagorinsky, 1 Vreman                                         */
  int riemann;      /* 0 Roe, 1 local Lax-Friedrichs                                   */
  int precision;    /* 0 FP64 throughout; 1 FP32 element/face arithmetic with FP64 state,
                       traces and Runge-Kutta accumulation; 2 as 1, with the inviscid
                       volume term's D contractions on the tensor cores in 3xTF32 (each
                       FP32 operand split into two TF32 parts, big*big + big*small +
                       small*big accumulated in FP32; the split form keeps FP32 FMAs);
                       3 as 2 with plain TF32 (only big*big: operands rounded to 10
                       mantissa bits; an accuracy contrast, not a production setting)    */
  int mixed_face;   /* viscous flux on a face between an NS and an Euler element (Sec. 2.3
                       asks only that it be single-valued): 0 the average of the NS side's
                       flux and zero (BR1 with an inviscid side), 1 the NS side's flux
                       alone; faces between two NS elements always take the average      */
  int split;        /* convective volume term: 0 the standard form (App. B, Eq. NS4), 1 the
                       kinetic-energy-preserving split form: along each direction
                       sum_m 2 D_im F#(q_i, q_m) with F# = (c0^2 U, {{u}} U + {{p}} {{Ja}}),
                       U = {{Ja}}.{{u}}, {{.}} the two-node average                       */
  int model;        /* governing equations: 0 incompressible flow in artificial-
                       compressibility form, state q = (p, u, v, w), rho = 1; 1 the
                       compressible Navier-Stokes equations of App. A, conservative state
                       u = (rho, rho v1, rho v2, rho v3, rho e), ideal gas with unit gas
                       constant (p = (gamma - 1)(rho e - rho |v|^2 / 2), T = p / rho), nu the
                       dynamic viscosity mu, eddy viscosity mu_t = rho nu_t of the closure,
                       heat flux kappa grad T with kappa = c_p (mu / Pr + mu_t / Pr_t),
                       c_p = gamma / (gamma - 1), BR1 on (v, T). Model 1 runs in FP64
                       (precision 0) with the standard volume term (split 0), p-nonconforming
                       faces through five-variable mortars, and boundary faces that
                       are far-field inflow (tag 1, the ghost is the state of inflow[] and
                       p_inf), pressure outflow (tag 2, interior density and velocity with
                       p_inf), both with the interior viscous flux, or adiabatic walls:
                       no-slip (tag 3, the mirror ghost (rho, -rho v, rho e), the interior
                       traction) or free-slip (tag 4, the normal momentum reversed, the normal
                       traction), with no viscous energy flux at walls; other settings give
                       DG_ERR_UNSUPPORTED. Its state, RK register
                       and residual arrays have 5 planes, [5][total_nodes].               */
  double inflow[4]; /* ghost state at inflow faces: model 0 uses the velocity part;
                       model 1 reads (rho, u, v, w) of the far field                    */
  double gamma;     /* model 1: ratio of specific heats (> 1)                           */
  double prandtl;   /* model 1: laminar Prandtl number (> 0)                            */
  double prandtl_t; /* model 1: turbulent Prandtl number (> 0)                          */
  int nodes;        /* element nodes and quadrature (App. B): 0 Gauss-Lobatto, 1 Gauss-
                       Legendre (the paper's choice): the element's (N+1)^3 nodes are the
                       tensor Gauss points, face values, face metric terms and viscous
                       traces are interpolated along the normal lines and face terms lifted
                       with l_i(+-1) / w_i. Nodes 1 runs either form (model 0 or 1) in FP64
                       (precision 0) with the standard volume term (split 0), with
                       p-nonconforming faces (mortars interpolating and projecting between
                       the Gauss point sets) and the boundary faces' ghost states of the
                       Gauss-Lobatto path; other settings give
                       DG_ERR_UNSUPPORTED. dg_node_coords returns the Gauss points;
                       dg_detect_regions, dg_project_state and the conservation sums work
                       on them.                                                          */
  int fp64_divergence; /* precision 1..3, standard volume term (split 0), axis-aligned box
                       elements: 0 every volume contraction in FP32 (fast; the pressure row
                       R_p = -c0^2 div u of a nearly divergence-free field is a small difference
                       of three directional derivatives, so their FP32 rounding is amplified
                       by about c0^2 |grad u| / |R_p|); 1 the divergence
                       S = sum_d Ja_dd (D_d u_d) in FP64 from the FP64 state, used for the
                       pressure row and for the U_c du_d part of the momentum fluxes (the
                       deviation form's linear term), the rest of the momentum fluxes in FP32
                       (more accurate, but runs on the FP64 pipe: slower). Affine and curved
                       elements and the split form ignore it. Other values: DG_ERR_ARG      */
  double p_inf;     /* model 1: far-field pressure of the inflow ghost (with inflow[]) and
                       the static pressure of the outflow ghost (interior density and
                       velocity); both need rho_inf = inflow[0] > 0 and p_inf > 0          */
} dg_params;

/* Build the mesh topology (face matching, orientations, periodic pairs), the geometry
 * (curl-form metric terms at the geometry degree, Kopriva 2006) and upload everything to
 * `device`. Orders default to 3 (or the geometry degree if larger) and flags to 1 (NS).
 * Returns DG_ERR_MESH for an unmatched face without a boundary tag, a face shared by more
 * than two elements, repeated corner ids on one face or a non-positive Jacobian. */
dg_status dg_create_mesh(const dg_mesh_desc* mesh, const dg_params* params, int device, dg_ctx** out);

/* Per-element polynomial order N_e in 1..7 (host array, length n_elem; Sec. 3.2 local
 * p-adaptation). Faces between different orders become mortars (interpolation to the
 * larger order, exact L2 projection back). Re-lays out the state: previous q/g/R arrays
 * no longer match the layout. */
dg_status dg_set_orders(dg_ctx* ctx, const int8_t* orders);

/* Re-lay out a state for the orders set by the last successful dg_set_orders (Sec. 3.2:
 * restarting after the orders are re-assigned). q_old ([nvar][total before that call], device;
 * nvar = 4, or 5 under model 1) is read in the previous layout, q_new ([nvar][current
 * total_nodes], device, caller-allocated,
 * not overlapping q_old) is written in the current one: per element, Lagrange interpolation
 * onto the new nodes (Gauss-Lobatto, or Gauss points with nodes 1) where the order grew or
 * stayed (exact for the old
 * polynomial), the L2 projection in reference coordinates where it dropped (keeps each
 * element's reference-space integral), applied along each direction. Asynchronous on
 * `stream`. DG_ERR_STATE before any dg_set_orders. */
dg_status dg_project_state(dg_ctx* ctx, const double* q_old_dev, double* q_new_dev, void* stream);

/* Per-element flag (host array, length n_elem): 0 Euler, 1 Navier-Stokes + LES (Sec. 2.3).
 * Does not change the layout. */
dg_status dg_set_element_flags(dg_ctx* ctx, const uint8_t* flags);

/* Replace the parameters (same validation as dg_create_mesh). */
dg_status dg_set_params(dg_ctx* ctx, const dg_params* params);

/* total_nodes = sum_e (N_e + 1)^3; *elem_offset points to a library-owned host array of
 * n_elem + 1 offsets, valid until the next dg_set_orders or dg_destroy. */
dg_status dg_get_layout(const dg_ctx* ctx, int64_t* total_nodes, const int64_t** elem_offset);

/* Physical coordinates of every node, device array [3][total_nodes]. */
dg_status dg_node_coords(dg_ctx* ctx, double* xyz_dev, void* stream);

/* R = dq/dt (App. B, Eq. NS4 with the BR1 viscous terms) for device arrays q, R of shape
 * [4][total_nodes] (they must not overlap). Asynchronous on `stream` (a cudaStream_t,
 * NULL = default stream). */
dg_status dg_residual(dg_ctx* ctx, const double* q_dev, double* R_dev, void* stream);

/* nsteps steps of the Williamson 2N-storage RK3 in place on device arrays q and g
 * ([4][total_nodes] FP64 each): per stage s, g <- A_s g + dt R(q), q <- q + B_s g, with
 * A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15) (g need not be initialised: A_1 = 0
 * overwrites it). q is always accumulated in FP64. g is the scheme's register: FP64 with
 * precision 0; with precision 1 it holds FP32 values (the first half of its bytes, laid out
 * [4][total_nodes]), like the residual it accumulates. One step is captured once as a CUDA
 * graph per (q, g, dt) and replayed. With nsteps > 1 the steps are chained: every stage's
 * update also writes the face traces of the next stage (the last stage those of the next step),
 * so only the first step runs the separate trace kernel; the results are bitwise those of
 * nsteps calls with nsteps = 1. t is the time at the start (the residual has no explicit time
 * dependence). */
dg_status dg_rk_step(dg_ctx* ctx, double* q_dev, double* g_dev, double t, double dt, int nsteps,
                     void* stream);

/* Host-buffer variants: copy the host arrays to library-owned device buffers, compute on
 * `stream`, copy the result back and synchronise the stream before returning. Each transfer is
 * split over several library-owned streams so that copy engines can work in parallel; the
 * host arrays should be pinned (page-locked) for full speed. g_host may be NULL: the first
 * stage of every step overwrites the RK register without reading it, so it then stays in a
 * library-owned device buffer and only q is copied in and out. */
dg_status dg_residual_host(dg_ctx* ctx, const double* q_host, double* R_host, void* stream);
dg_status dg_rk_step_host(dg_ctx* ctx, double* q_host, double* g_host, double t, double dt, int nsteps,
                          void* stream);

/* out_host[v] = sum_e sum_nodes w_i w_j w_k J R_v (FP64, deterministic order) for every
 * variable of the model: out_host holds 4 values (model 0) or 5 (model 1). Synchronises the
 * stream and also reports a pending device error. On a periodic mesh the exact
 * discretisation conserves every variable, so these sums vanish to rounding. */
dg_status dg_conservation(dg_ctx* ctx, const double* R_dev, double* out_host, void* stream);

/* Launch-shape autotuner of the reduced-precision passes (precision 1). For every bucket of
 * the current mesh -- one per (polynomial order, geometry kind) -- it times the candidate
 * launch shapes on this GPU and keeps the fastest: for the inviscid pass the elements per
 * tile (the default ~256-node tile or the alternative: half of it for orders 1..4, two
 * elements for orders 5, 6) and the resident blocks per SM (all that fit, 1 or 2); for the
 * viscous pass on box/affine elements the pipelined (bulk-copy) kernel with either tile shape at
 * those block counts or the cp.async-staged kernel; and, when the mesh is one (order, box or affine) bucket without
 * p-nonconforming faces run with FP32 contractions, whether each Runge-Kutta stage after its
 * traces runs as one launch (the default tile shapes) instead of separate viscous and inviscid
 * launches (chosen only when at least 1% faster): either one persistent cooperative kernel
 * (the viscous pass, a bounded grid barrier, the inviscid pass and update), or one kernel whose
 * blocks take tiles from queues (viscous tiles first, then the inviscid tiles of the Euler
 * elements with no NS neighbour, which run while the viscous pass drains, then the rest, which
 * wait on a bounded counter of finished viscous tiles).
 * Timing uses a library-owned scratch state, so q, g and R are
 * untouched; the choices then apply to every later call (they are kept per order and
 * geometry kind across dg_set_orders / dg_set_element_flags) and the captured step graph
 * is rebuilt. cache_path (NULL: none) names a text file of choices keyed by the device
 * name: choices found there are used without timing, and the file is rewritten with this
 * device's choices. report (NULL allowed) receives a human-readable summary, truncated to
 * report_len bytes. Precision 0 has nothing to tune and returns DG_OK. Synchronises. Errors:
 * DG_ERR_ARG (NULL ctx, unwritable cache), DG_ERR_OOM (scratch), DG_ERR_CUDA. */
dg_status dg_autotune(dg_ctx* ctx, const char* cache_path, char* report, int report_len);

/* Largest mesh (elements) that dg_conservation_noalloc accepts. */
#define DG_CONSERVATION_NOALLOC_MAX_ELEMS 65536

/* The paper has no counterpart to this call; it is a service for callers that cannot allocate.
 * The same sums as dg_conservation, written to out_dev[4] (caller-owned device memory, FP64)
 * asynchronously on `stream`, without allocating device memory (no cudaMalloc, cudaFree or
 * allocating library call) and without a host copy or synchronisation. It is meant for callers
 * that must not allocate while they run: a process whose memory pool has already claimed the
 * device, or a time-critical loop in which an allocation would stall the device.
 * Scratch: the per-element partial sums go to one static device array of
 * 4 x DG_CONSERVATION_NOALLOC_MAX_ELEMS doubles (2 MiB) that the library module carries.
 * Nothing in it has to start at zero. Every call in the process on that device shares it, so
 * calls whose work overlaps on the GPU (other streams, other threads) race and give wrong
 * sums: serialise them. The first call on a device looks up the array's device address (which
 * can load the library's device code), so make that first call before any stream capture.
 * Errors: DG_ERR_ARG for a NULL pointer or a mesh of more than
 * DG_CONSERVATION_NOALLOC_MAX_ELEMS elements; DG_ERR_UNSUPPORTED under model 1; DG_ERR_CUDA
 * if the look-up or a launch fails.
 * The device error word is not read (see dg_check_device). The final sum runs in a fixed
 * order on the device, so it may differ from dg_conservation's host sum by rounding. */
dg_status dg_conservation_noalloc(dg_ctx* ctx, const double* R_dev, double* out_dev, void* stream);

/* Two-component Gaussian mixture on the node features (Q_S, R_S, Q_Omega) of Sec. 2.1. The
 * mixture is fitted outside the library (on snapshots of developed flow); any per-feature
 * scaling used in that fit folds into the means and covariances. */
typedef struct {
  double weight[2];     /* mixture weights, positive (they need not sum to 1)        */
  double mean[2][3];    /* component means, in (Q_S, R_S, Q_Omega) order              */
  double cov[2][3][3];  /* component covariances, symmetric positive definite        */
  int viscous;          /* 0 or 1: the component of the viscous/rotational region    */
  int precision;        /* 0 FP64 (the state's precision; the decision of the FP64
                           oracle), 1 FP32: the velocity rounded to FP32, the gradient,
                           features, memberships and element means in FP32 (the pass is
                           then bound by HBM, not the FP64 pipe); flags can differ from
                           the FP64 decision only for elements whose two means lie within
                           the FP32 error of each other                               */
} dg_gmm;

/* Viscous/inviscid region detection (Sec. 2.1), on the device, from the state q_dev
 * ([4][total_nodes] FP64, the current mesh and orders):
 *   1. at every node, the gradient of the element's velocity polynomial, J_ck = du_c/dx_k, by
 *      the chain rule with the element's metric terms (no interface terms); the nodes are the
 *      context's (dg_params.nodes: Gauss-Lobatto, or the Gauss points the paper uses);
 *   2. S = (J + J^T)/2, Omega = (J - J^T)/2, Q_S = (tr(S)^2 - tr(S^2))/2, R_S = -det(S)/3,
 *      Q_Omega = -tr(Omega^2)/2;
 *   3. the posterior probabilities p_v, p_i of the viscous and the other component of `gmm`
 *      at the node's features (the mixture's E-step);
 *   4. per element, the means of p_v and p_i over its (N+1)^3 nodes, and the region with the
 *      larger mean (1 viscous/NS, 0 inviscid/Euler; a tie is viscous).
 * FP64 throughout (gmm.precision 0) or FP32 (gmm.precision 1). Outputs, caller-owned device
 * memory, NULL to skip (at least one given):
 *   flags_dev    [n_elements] uint8, element order: ready for dg_set_element_flags once copied
 *                to the host (this call does not change the context's flags);
 *   pbar_dev     [2][n_elements] FP64: mean p_v, then mean p_i;
 *   features_dev [4][total_nodes] FP64: Q_S, R_S, Q_Omega, p_v per node (node layout of q).
 * Asynchronous on `stream`. Errors: DG_ERR_ARG for a NULL ctx, q_dev or gmm, no output, a
 * non-positive or non-finite weight, a covariance that is not symmetric (to 1e-12 of its
 * largest entry) or not positive definite, viscous outside {0, 1}, precision outside {0, 1};
 * DG_ERR_UNSUPPORTED under model 1 (q holds momenta there); DG_ERR_CUDA if a launch fails. */
dg_status dg_detect_regions(dg_ctx* ctx, const double* q_dev, const dg_gmm* gmm, uint8_t* flags_dev,
                            double* pbar_dev, double* features_dev, void* stream);

/* Failure detection of the pipelined reduced-precision passes (precision 1..3; the paper has
 * no counterpart). Each of their warps waits on an mbarrier for a staged tile (consumers) or
 * for a free buffer (the producer) with a bounded number of polls; when the budget runs out
 * the warp records DG_ERR_TIMEOUT in the device error word (read by dg_check_device, which
 * names the site: 1 inviscid consumers, 2 inviscid producer, 3 viscous consumers, 4 viscous
 * producer, 5 the grid barrier of the persistent stage kernel, 6 the producer's wait for the
 * finished viscous tiles in the one-launch stage kernel with tile queues) and returns, leaving
 * the CUDA context usable; dg_check_device also resets that grid barrier and those queues.
 *   polls      poll budget of every such wait, 1 .. 2^31 - 1; 0 restores the default 2^22.
 *   stop_tile  test hook: -1 off; k >= 0 makes the producer warp of block 0 of every pipelined
 *              launch return before staging its k-th tile, so that block's consumers wait for
 *              data that never comes until their budget runs out. Everything staged before
 *              was waited for by those consumers, so no copy is left in flight when they return.
 *              -2: block 0 of the persistent stage kernel (see dg_autotune) does not arrive at
 *              its grid barrier, so every block's bounded wait there runs out (site 5).
 * Applies to every later launch (the captured step graph is rebuilt). Results computed while
 * stop_tile != -1 are wrong by design. Errors: DG_ERR_ARG for a NULL ctx or out-of-range value. */
dg_status dg_set_wait_limit(dg_ctx* ctx, int64_t polls, int stop_tile);

/* Overlapped launches of the pipelined reduced-precision passes (precision 1..3, box and affine
 * elements; the paper has no counterpart). With enable = 1 (the default) each of their launches
 * carries programmatic stream serialisation: its blocks may be scheduled while the kernel before
 * it in the stream drains, and every thread waits in the kernel (griddepcontrol.wait) for that
 * kernel to complete before it touches memory the kernel may write or read. An inviscid launch
 * that directly follows the viscous pass of its stage runs the Euler elements that have no NS
 * neighbour and no mortar face first, without that wait. Results are identical either way;
 * enable = 0 gives plain launches (for comparison). dg_phase_times always uses plain launches.
 * Applies to every later launch (the captured step graph is rebuilt). Errors: DG_ERR_ARG for a
 * NULL ctx or enable outside {0, 1}. */
dg_status dg_set_launch_overlap(dg_ctx* ctx, int enable);

/* Synchronise `stream`, then read and clear the device error word. */
dg_status dg_check_device(dg_ctx* ctx, void* stream);

/* Phases of one residual evaluation / Runge-Kutta stage, in launch order. */
#define DG_NPHASES 5 /* 0 traces, 1 mortar lifting, 2 viscous, 3 mortar flux, 4 inviscid+update */

/* Tracing: run `reps` Runge-Kutta stages (stage index cycling 0, 1, 2) in place on q, g with
 * CUDA events recorded on `stream` between the phases, synchronise, and return the mean
 * time of each phase in milliseconds (a phase with no work reports 0). Advances q and g
 * exactly like dg_rk_step. */
dg_status dg_phase_times(dg_ctx* ctx, double* q_dev, double* g_dev, double dt, int reps,
                         double out_ms[DG_NPHASES], void* stream);

/* Algorithmic DRAM bytes of each phase, averaged over the three stages of one Runge-Kutta
 * step, on the current mesh, orders, flags and precision: every value a phase must read or
 * write once (state, RK register, traces, viscous buffers, metric terms), none re-read. The
 * roofline of a phase is these bytes over its mean time from dg_phase_times. The step is one on
 * its own, as dg_phase_times runs it: the trace kernel in stage 0, the updates of stages 0 and 1
 * writing the next stage's traces. In a dg_rk_step call of several steps every update writes
 * traces (stage 2 those of the next step) and only the first step runs the trace kernel. */
dg_status dg_phase_bytes(const dg_ctx* ctx, double out_bytes[DG_NPHASES]);

/* Number of kernel launches the last dg_residual / one dg_rk_step step issued, and one step
 * that follows another in the same dg_rk_step call (0 before any such call). */
int dg_launches_per_residual(const dg_ctx* ctx);
int dg_launches_per_step(const dg_ctx* ctx);
int dg_launches_per_chained_step(const dg_ctx* ctx);

/* Thread-local message describing the last failure on this thread. */
const char* dg_last_error(void);

/* Free every library-owned buffer. NULL is allowed. */
void dg_destroy(dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
