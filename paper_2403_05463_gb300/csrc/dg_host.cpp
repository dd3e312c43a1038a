// dg_host.cpp -- host side of the C ABI (include/dg.h): mesh ingestion, face matching and
// orientation, geometry (curl-form metrics), per-order buckets, device buffers, launch
// sequencing and CUDA-graph capture of the Runge-Kutta step.
#include "../../include/dg.h"
#include "dg_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

using namespace dgk;

namespace {

thread_local std::string g_last_error;

dg_status fail(dg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e__ = (call);                                                           \
    if (e__ != cudaSuccess)                                                             \
      return fail(e__ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(e__));                                      \
  } while (0)

// ---------------------------------------------------------------------------------------
// 1D Gauss-Lobatto operators. Interior nodes: zeros of P_N', found by Newton iteration with
// P_N'' from Legendre's equation (1-x^2) P'' = 2x P' - N(N+1) P. D by the closed form for
// Lobatto points (Canuto et al. 2006, Sec. 2.3), interpolation in barycentric form and the
// L2 projection by truncating the Legendre expansion.
// ---------------------------------------------------------------------------------------
void legendre_and_derivative(int N, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double d2 = d0 + (2 * k + 1) * p1;  // P'_{k+1} = P'_{k-1} + (2k+1) P_k
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  P = p1;
  dP = d1;
}

struct Rule {
  int N;
  std::vector<double> x, w, D;  // D row-major n x n
};

Rule make_rule(int N) {
  Rule r;
  r.N = N;
  const int n = N + 1;
  r.x.assign(n, 0.0);
  r.w.assign(n, 0.0);
  r.x[0] = -1.0;
  r.x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double x = -std::cos(M_PI * j / N);  // Chebyshev-Lobatto starting guess
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_and_derivative(N, x, P, dP);
      double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    r.x[j] = x;
  }
  for (int j = 0; j <= N / 2; ++j) {  // symmetrise
    double m = 0.5 * (r.x[N - j] - r.x[j]);
    r.x[j] = -m;
    r.x[N - j] = m;
  }
  if (N % 2 == 0) r.x[N / 2] = 0.0;
  std::vector<double> PN(n);
  for (int j = 0; j < n; ++j) {
    double P, dP;
    legendre_and_derivative(N, r.x[j], P, dP);
    PN[j] = P;
    r.w[j] = 2.0 / (N * (N + 1.0) * P * P);
  }
  r.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (i != j) r.D[i * n + j] = PN[i] / (PN[j] * (r.x[i] - r.x[j]));
    }
  r.D[0] = -N * (N + 1.0) / 4.0;
  r.D[N * n + N] = N * (N + 1.0) / 4.0;
  return r;
}

// Gauss-Legendre rule of N+1 points (App. B's quadrature): the roots of P_{N+1}, by Newton from
// the Chebyshev-Gauss guesses cos(pi (2j+1) / (2N+2)), weights 2 / ((1 - x^2) P'_{N+1}^2);
// D_ij = l_j'(x_i) from the barycentric weights.
Rule make_gl_rule(int N) {
  Rule r;
  r.N = N;
  const int n = N + 1;
  r.x.assign(n, 0.0);
  r.w.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double x = -std::cos(M_PI * (2.0 * j + 1.0) / (2.0 * n));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_and_derivative(n, x, P, dP);
      const double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    r.x[j] = x;
  }
  for (int j = 0; j < n / 2; ++j) {  // symmetrise
    const double m = 0.5 * (r.x[N - j] - r.x[j]);
    r.x[j] = -m;
    r.x[N - j] = m;
  }
  if (n % 2 == 1) r.x[N / 2] = 0.0;
  for (int j = 0; j < n; ++j) {
    double P, dP;
    legendre_and_derivative(n, r.x[j], P, dP);
    r.w[j] = 2.0 / ((1.0 - r.x[j] * r.x[j]) * dP * dP);
  }
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (r.x[j] - r.x[k]);
  r.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) {
        r.D[i * n + j] = lam[j] / (lam[i] * (r.x[i] - r.x[j]));
        diag -= r.D[i * n + j];
      }
    r.D[i * n + i] = diag;
  }
  return r;
}

// barycentric Lagrange interpolation matrix from nodes xs to points xd: I[i][j]
std::vector<double> interp_matrix(const std::vector<double>& xs, const std::vector<double>& xd) {
  const int ns = (int)xs.size(), nd = (int)xd.size();
  std::vector<double> lam(ns, 1.0), I(nd * ns, 0.0);
  for (int j = 0; j < ns; ++j)
    for (int k = 0; k < ns; ++k)
      if (k != j) lam[j] /= (xs[j] - xs[k]);
  for (int i = 0; i < nd; ++i) {
    int hit = -1;
    for (int j = 0; j < ns; ++j)
      if (xd[i] == xs[j]) hit = j;
    if (hit >= 0) {
      I[i * ns + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < ns; ++j) den += lam[j] / (xd[i] - xs[j]);
    for (int j = 0; j < ns; ++j) I[i * ns + j] = lam[j] / (xd[i] - xs[j]) / den;
  }
  return I;
}

// L2 projection of a degree-Nh polynomial (values at the nodes of `hi`) onto degree Nl:
// Legendre coefficients by the rule of `hi` (exact for the modes kept: degree k + Nh <=
// 2 Nh - 1 for k < Nh on Lobatto nodes, <= 2 Nh + 1 on Gauss points), truncation,
// evaluation at the nodes of `lo`.
std::vector<double> projection_matrix(const Rule& hi, const Rule& lo) {
  const int nh = hi.N + 1, nl = lo.N + 1;
  std::vector<double> P(nl * nh, 0.0);
  if (hi.N == lo.N) {
    for (int i = 0; i < nl; ++i) P[i * nh + i] = 1.0;
    return P;
  }
  auto leg = [](int k, double x) {
    double P, dP;
    legendre_and_derivative(k, x, P, dP);
    return P;
  };
  for (int i = 0; i < nl; ++i)
    for (int j = 0; j < nh; ++j) {
      double s = 0.0;
      for (int k = 0; k <= lo.N; ++k) s += (k + 0.5) * leg(k, hi.x[j]) * leg(k, lo.x[i]);
      P[i * nh + j] = s * hi.w[j];
    }
  return P;
}

struct OpTables {
  Rule rule[NP];
  Rule gl[NP];                          // Gauss-Legendre rules (element nodes with nodes = 1)
  double glb[NP][2][NP] = {};           // Gauss-Legendre l_i(-1), l_i(+1)
  std::vector<double> interp, proj;  // [(a*NP+b)*NP*NP + i*NP + j]
  std::vector<double> interp_gl;     // Gauss-Lobatto of degree a -> Gauss-Legendre of order b
  std::vector<double> interp_g, proj_g;  // the same as interp, proj between Gauss point sets
  std::vector<double> lb_g;              // [(N*2+s)*NP + i] = glb[N][s][i]
  OpTables() {
    for (int N = 1; N <= MAXN; ++N) rule[N] = make_rule(N);
    for (int N = 1; N <= MAXN; ++N) {
      gl[N] = make_gl_rule(N);
      const std::vector<double> ends = {-1.0, 1.0};
      const std::vector<double> E = interp_matrix(gl[N].x, ends);
      for (int s = 0; s < 2; ++s)
        for (int i = 0; i <= N; ++i) glb[N][s][i] = E[s * (N + 1) + i];
    }
    interp_gl.assign(NP * NP * NP * NP, 0.0);
    for (int a = 1; a <= MAXN; ++a)
      for (int b = 1; b <= MAXN; ++b) {
        auto I = interp_matrix(rule[a].x, gl[b].x);
        for (int i = 0; i <= b; ++i)
          for (int j = 0; j <= a; ++j) interp_gl[(a * NP + b) * NP * NP + i * NP + j] = I[i * (a + 1) + j];
      }
    lb_g.assign(NP * 2 * NP, 0.0);
    for (int N = 1; N <= MAXN; ++N)
      for (int s = 0; s < 2; ++s)
        for (int i = 0; i <= N; ++i) lb_g[(N * 2 + s) * NP + i] = glb[N][s][i];
    fill_mortar_tables(rule, interp, proj);
    fill_mortar_tables(gl, interp_g, proj_g);
  }
  // interpolation a -> b and projection a -> b <= a between the node sets of one rule family
  static void fill_mortar_tables(const Rule* r, std::vector<double>& interp, std::vector<double>& proj) {
    interp.assign(NP * NP * NP * NP, 0.0);
    proj.assign(NP * NP * NP * NP, 0.0);
    for (int a = 1; a <= MAXN; ++a)
      for (int b = 1; b <= MAXN; ++b) {
        auto I = interp_matrix(r[a].x, r[b].x);
        for (int i = 0; i <= b; ++i)
          for (int j = 0; j <= a; ++j) interp[(a * NP + b) * NP * NP + i * NP + j] = I[i * (a + 1) + j];
        if (b <= a) {
          auto P = projection_matrix(r[a], r[b]);
          for (int i = 0; i <= b; ++i)
            for (int j = 0; j <= a; ++j) proj[(a * NP + b) * NP * NP + i * NP + j] = P[i * (a + 1) + j];
        }
      }
  }
};

const OpTables& ops() {
  static OpTables t;
  return t;
}

// face f = 2d+s: tangential directions and hexahedron corner of face corner (ca, cb)
void tangents(int d, int& t0, int& t1) {
  t0 = d == 0 ? 1 : 0;
  t1 = d == 2 ? 1 : 2;
}
int face_corner_index(int f, int ca, int cb) {
  int d = f >> 1, t0, t1, c[3];
  tangents(d, t0, t1);
  c[d] = f & 1;
  c[t0] = ca;
  c[t1] = cb;
  return c[0] + 2 * c[1] + 4 * c[2];
}
void orient_fwd(int o, int M, int a1, int b1, int& a0, int& b0) {
  int x = (o & 1) ? b1 : a1, y = (o & 1) ? a1 : b1;
  a0 = (o & 2) ? M - x : x;
  b0 = (o & 4) ? M - y : y;
}

struct Key4 {
  int64_t k[4];
  bool operator==(const Key4& o) const { return std::memcmp(k, o.k, sizeof k) == 0; }
};
struct Key4Hash {
  size_t operator()(const Key4& a) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 4; ++i) {
      h ^= (uint64_t)a.k[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

}  // namespace

// ---------------------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;  // one step on its own: trace kernel, stages 0..2
  // chained steps (nsteps > 1): [0] the first step, whose three stages all write the next
  // stage's traces; [1], [2] a later step of trace-buffer parity 0 or 1, without the trace kernel
  cudaGraphExec_t chain[3] = {nullptr, nullptr, nullptr};
  int chain_launches = 0;          // launches of a later chained step
  const double* q = nullptr;
  const double* g = nullptr;
  double dt = 0.0;
  uint64_t version = 0;
};

struct dg_ctx {
  int device = 0;
  int64_t ne = 0;
  int gdeg = 1;
  std::vector<int64_t> hex;
  std::vector<double> gnodes;   // [E][(g+1)^3][3]
  std::vector<int8_t> bc;       // [E][6]
  dg_params prm{};
  std::vector<int8_t> order;
  std::vector<uint8_t> flag;
  std::vector<int64_t> off, troff;
  int64_t total = 0, tr_total = 0;
  // topology (order independent)
  std::vector<int32_t> nb;      // [E*6] neighbour or -1
  std::vector<uint8_t> nbf, nbo;
  // device
  std::map<std::string, DevBuf> buf;
  DevMesh M{};
  std::vector<Bucket> all_buckets;  // per (N, geometry kind): every element
  std::vector<std::vector<int32_t>> all_lists;  // host copies of the all_buckets lists
  std::vector<Bucket> ns_buckets;   // per (N, curved): NS elements
  std::vector<Bucket> ord_buckets;  // per N (traces, coordinates, sums)
  int32_t* mortar_all = nullptr;    // device slots e*6+f of every mortar face
  int n_mortar_all = 0;
  int32_t* mortar_ns = nullptr;     // mortar slots of NS elements (lifting)
  int n_mortar_ns = 0;
  // both lists are sorted by mortar order: [mo_start[MO], mo_start[MO + 1]) holds order MO
  int mortar_all_mo[MAXN + 2] = {};
  int mortar_ns_mo[MAXN + 2] = {};
  int32_t* mortar_face = nullptr;   // one slot per mortar face: the side of the larger order
  int mortar_face_mo[MAXN + 2] = {};
  std::vector<ElemConst> ec;
  std::vector<uint8_t> geo_kind;  // 0 axis-aligned box, 1 affine, 2 curved
  bool any_curved = false;
  cudaStream_t cap_stream = nullptr;
  // host-buffer variants: the transfers are split over kCopyStreams streams (created on first
  // use), each piece ordered after the caller's stream and joined back into it
  static constexpr int kCopyStreams = 4;
  cudaStream_t copy_stream[kCopyStreams] = {};
  cudaEvent_t copy_fork = nullptr, copy_done[kCopyStreams] = {};
  GraphCache graph;
  uint64_t version = 1;
  int launches_residual = 0, launches_step = 0;
  // while a chained RK step is captured: the trace-buffer parity of its stage 0, whether stage 2
  // writes the next stage's traces too, and whether the trace kernel is left out
  int cap_parity = 0, cap_write_all = 0, cap_no_traces = 0;
  // the last phase that launched anything was the viscous pass (phase 2): the inviscid launch
  // that follows it may start its independent entries before that pass has completed
  bool visc_last = false;
  // host-variant staging
  double* trace_buf[2] = {nullptr, nullptr};
  double* stage_q = nullptr;
  double* stage_r = nullptr;
  double* partial = nullptr;
  std::vector<double> partial_host;
  // autotuned launch choices of the reduced-precision passes, key (pass, N, geometry kind) with
  // pass 0 inviscid, 1 viscous; value (tile_alt, bps, visc_alt)
  std::map<std::array<int, 3>, std::array<int, 3>> tuning;
  // orders and node offsets before the last successful dg_set_orders (for dg_project_state)
  std::vector<int8_t> prev_order;
  std::vector<int64_t> prev_off;
};

namespace {

void free_buf(dg_ctx* c, const std::string& name) {
  auto it = c->buf.find(name);
  if (it != c->buf.end()) {
    cudaFree(it->second.p);
    c->buf.erase(it);
  }
}

template <typename T>
dg_status dev_alloc(dg_ctx* c, const std::string& name, size_t count, T** out) {
  free_buf(c, name);
  // 256 bytes of slack: bulk copies read whole 16-byte blocks around the wanted range
  size_t bytes = count * sizeof(T) + 256;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(DG_ERR_OOM, "cudaMalloc(%s, %zu bytes): %s", name.c_str(), bytes, cudaGetErrorString(e));
  c->buf[name] = DevBuf{p, bytes};
  *out = (T*)p;
  return DG_OK;
}

template <typename T>
dg_status dev_upload(dg_ctx* c, const std::string& name, const std::vector<T>& v, T** out) {
  dg_status st = dev_alloc(c, name, v.size(), out);
  if (st != DG_OK) return st;
  if (!v.empty()) CU(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DG_OK;
}

dg_status check_params(const dg_params* p) {
  if (!p) return fail(DG_ERR_ARG, "params is NULL");
  if (!(p->c0sq > 0.0) || !(p->nu >= 0.0) || !(p->cs >= 0.0) || !(p->cv >= 0.0))
    return fail(DG_ERR_ARG, "need c0sq > 0 and nu, cs, cv >= 0");
  if (p->closure < 0 || p->closure > 1) return fail(DG_ERR_ARG, "closure must be 0 or 1");
  if (p->riemann < 0 || p->riemann > 1) return fail(DG_ERR_ARG, "riemann must be 0 or 1");
  if (p->precision < 0 || p->precision > 3) return fail(DG_ERR_UNSUPPORTED, "precision %d not built", p->precision);
  if (p->mixed_face < 0 || p->mixed_face > 1) return fail(DG_ERR_ARG, "mixed_face must be 0 or 1");
  if (p->split < 0 || p->split > 1) return fail(DG_ERR_ARG, "split must be 0 or 1");
  if (p->model < 0 || p->model > 1) return fail(DG_ERR_ARG, "model must be 0 or 1");
  if (p->nodes < 0 || p->nodes > 1) return fail(DG_ERR_ARG, "nodes must be 0 or 1");
  if (p->fp64_divergence < 0 || p->fp64_divergence > 1) return fail(DG_ERR_ARG, "fp64_divergence must be 0 or 1");
  if (p->nodes == 1 && (p->precision != 0 || p->split != 0))
    return fail(DG_ERR_UNSUPPORTED, "Gauss-Legendre nodes run in FP64 with the standard volume term only");
  if (p->model == 1) {
    if (p->precision != 0) return fail(DG_ERR_UNSUPPORTED, "the compressible form runs in FP64 (precision 0) only");
    if (p->split != 0) return fail(DG_ERR_UNSUPPORTED, "the compressible form has the standard volume term only");
    if (!(p->gamma > 1.0) || !(p->prandtl > 0.0) || !(p->prandtl_t > 0.0))
      return fail(DG_ERR_ARG, "the compressible form needs gamma > 1 and positive Prandtl numbers");
  }
  return DG_OK;
}

// variables of the state: 4 (incompressible), 5 (compressible)
int nvar(const dg_ctx* c) { return c->prm.model == 1 ? 5 : 4; }

// the element's node rule: Gauss-Lobatto, or Gauss-Legendre with nodes = 1
const Rule& node_rule(const dg_ctx* c, int N) { return c->prm.nodes == 1 ? ops().gl[N] : ops().rule[N]; }

void apply_params(dg_ctx* c) {
  c->M.nu = c->prm.nu;
  c->M.c0sq = c->prm.c0sq;
  c->M.cs = c->prm.cs;
  c->M.cv = c->prm.cv;
  c->M.closure = c->prm.closure;
  c->M.riemann = c->prm.riemann;
  c->M.mixed_face = c->prm.mixed_face;
  c->M.split = c->prm.split;
  c->M.model = c->prm.model;
  c->M.nodes = c->prm.nodes;
  c->M.gamma = c->prm.gamma;
  c->M.prandtl = c->prm.prandtl;
  c->M.prandtl_t = c->prm.prandtl_t;
  c->M.p_inf = c->prm.p_inf;
  // precisions 2 and 3 are the FP32 path (same data layout) with the inviscid volume
  // contraction on the tensor cores (3xTF32, plain TF32)
  c->M.precision = c->prm.precision >= 1 ? 1 : 0;
  c->M.tc = c->prm.precision == 2 ? 1 : (c->prm.precision == 3 ? 2 : 0);
  c->M.div64 = c->prm.fp64_divergence;
  c->M.nu32 = (float)c->prm.nu;
  c->M.c0sq32 = (float)c->prm.c0sq;
  c->M.cs32 = (float)c->prm.cs;
  c->M.cv32 = (float)c->prm.cv;
  for (int i = 0; i < 4; ++i) c->M.inflow[i] = c->prm.inflow[i];
  c->version++;
}

// Geometry of element e at order N. Affine (parallelepiped) elements: Ja^d = a_{d+1} x a_{d+2}
// with a_d = dX/dxi_d (constant). Otherwise the curl form of the metric identities
// (Kopriva 2006) at the geometry degree g, interpolated to the element's nodes.
struct ElemGeo {
  bool affine;
  double Ja[9], J;                  // affine
  std::vector<double> Jan, Jn;      // curved: [9][n3], [n3]
};

bool is_affine(const dg_ctx* c, int64_t e, double a[3][3], double x0[3]) {
  const int g = c->gdeg, ng = g + 1, ng3 = ng * ng * ng;
  const double* X = &c->gnodes[(size_t)e * ng3 * 3];
  auto node = [&](int i, int j, int k) { return X + 3 * (i + ng * (j + ng * k)); };
  const double* p0 = node(0, 0, 0);
  const double* px = node(g, 0, 0);
  const double* py = node(0, g, 0);
  const double* pz = node(0, 0, g);
  double scale = 0.0;
  for (int k = 0; k < 3; ++k) {
    x0[k] = p0[k];
    a[0][k] = 0.5 * (px[k] - p0[k]);
    a[1][k] = 0.5 * (py[k] - p0[k]);
    a[2][k] = 0.5 * (pz[k] - p0[k]);
    scale = std::max({scale, std::fabs(a[0][k]), std::fabs(a[1][k]), std::fabs(a[2][k])});
  }
  const std::vector<double>& t = ops().rule[std::max(g, 1)].x;  // reference points of degree g
  for (int kk = 0; kk < ng; ++kk)
    for (int jj = 0; jj < ng; ++jj)
      for (int ii = 0; ii < ng; ++ii) {
        const double* p = node(ii, jj, kk);
        for (int k = 0; k < 3; ++k) {
          double ref = x0[k] + (t[ii] + 1.0) * a[0][k] + (t[jj] + 1.0) * a[1][k] + (t[kk] + 1.0) * a[2][k];
          if (std::fabs(p[k] - ref) > 1e-13 * scale) return false;
        }
      }
  return true;
}

void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

void elem_geometry(const dg_ctx* c, int64_t e, int N, ElemGeo& G) {
  double a[3][3], x0[3];
  const int g = c->gdeg, ng = g + 1, ng3 = ng * ng * ng;
  if (is_affine(c, e, a, x0)) {
    G.affine = true;
    double t[3];
    cross(a[1], a[2], t);
    for (int k = 0; k < 3; ++k) G.Ja[0 * 3 + k] = t[k];
    cross(a[2], a[0], t);
    for (int k = 0; k < 3; ++k) G.Ja[1 * 3 + k] = t[k];
    cross(a[0], a[1], t);
    for (int k = 0; k < 3; ++k) G.Ja[2 * 3 + k] = t[k];
    G.J = a[0][0] * G.Ja[0] + a[0][1] * G.Ja[1] + a[0][2] * G.Ja[2];
    return;
  }
  G.affine = false;
  const Rule& rg = ops().rule[g];
  const Rule& rn = node_rule(c, N);
  const int n = N + 1, n3 = n * n * n;
  const double* X = &c->gnodes[(size_t)e * ng3 * 3];
  // derivative along direction d on the ng^3 grid
  auto deriv = [&](const std::vector<double>& u, int d) {
    std::vector<double> out(ng3, 0.0);
    for (int k = 0; k < ng; ++k)
      for (int j = 0; j < ng; ++j)
        for (int i = 0; i < ng; ++i) {
          int idx[3] = {i, j, k};
          double acc = 0.0;
          for (int m = 0; m < ng; ++m) {
            int q[3] = {i, j, k};
            q[d] = m;
            acc += rg.D[idx[d] * ng + m] * u[q[0] + ng * (q[1] + ng * q[2])];
          }
          out[i + ng * (j + ng * k)] = acc;
        }
    return out;
  };
  std::vector<double> I = interp_matrix(rg.x, rn.x);  // n x ng
  auto to_nodes = [&](const std::vector<double>& u) {
    // separable interpolation, one direction at a time
    std::vector<double> t1(n * ng * ng), t2(n * n * ng), out(n3);
    for (int k = 0; k < ng; ++k)
      for (int j = 0; j < ng; ++j)
        for (int i = 0; i < n; ++i) {
          double s = 0.0;
          for (int m = 0; m < ng; ++m) s += I[i * ng + m] * u[m + ng * (j + ng * k)];
          t1[i + n * (j + ng * k)] = s;
        }
    for (int k = 0; k < ng; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double s = 0.0;
          for (int m = 0; m < ng; ++m) s += I[j * ng + m] * t1[i + n * (m + ng * k)];
          t2[i + n * (j + n * k)] = s;
        }
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double s = 0.0;
          for (int m = 0; m < ng; ++m) s += I[k * ng + m] * t2[i + n * (j + n * m)];
          out[i + n * (j + n * k)] = s;
        }
    return out;
  };
  std::vector<double> Xc[3];
  for (int k = 0; k < 3; ++k) {
    Xc[k].resize(ng3);
    for (int p = 0; p < ng3; ++p) Xc[k][p] = X[3 * p + k];
  }
  std::vector<double> dX[3][3];  // dX[k][d] = d X_k / d xi_d
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) dX[k][d] = deriv(Xc[k], d);
  // J at the nodes
  std::vector<double> dXn[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) dXn[k][d] = to_nodes(dX[k][d]);
  G.Jn.assign(n3, 0.0);
  for (int p = 0; p < n3; ++p) {
    double m[3][3];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) m[k][d] = dXn[k][d][p];
    G.Jn[p] = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
              m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
  }
  // curl form: Ja^i_k = -(curl_xi v^k)_i with v^k_d = X_l dX_m/dxi_d, (k, m, l) cyclic
  G.Jan.assign(9 * n3, 0.0);
  for (int k = 0; k < 3; ++k) {
    const int m = (k + 1) % 3, l = (k + 2) % 3;
    std::vector<double> v[3];
    for (int d = 0; d < 3; ++d) {
      v[d].resize(ng3);
      for (int p = 0; p < ng3; ++p) v[d][p] = Xc[l][p] * dX[m][d][p];
    }
    // (curl v)_0 = d1 v2 - d2 v1, (curl v)_1 = d2 v0 - d0 v2, (curl v)_2 = d0 v1 - d1 v0
    for (int i = 0; i < 3; ++i) {
      const int j1 = (i + 1) % 3, j2 = (i + 2) % 3;
      std::vector<double> a1 = deriv(v[j2], j1), a2 = deriv(v[j1], j2), w(ng3);
      for (int p = 0; p < ng3; ++p) w[p] = -(a1[p] - a2[p]);
      std::vector<double> wn = to_nodes(w);
      for (int p = 0; p < n3; ++p) G.Jan[(i * 3 + k) * n3 + p] = wn[p];
    }
  }
}

void destroy_graph(dg_ctx* c) {
  if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
  for (cudaGraphExec_t& e : c->graph.chain)
    if (e) cudaGraphExecDestroy(e);
  c->graph = GraphCache{};
}

void build_buckets(const std::vector<int32_t>& elems, const std::vector<int8_t>& order,
                   const std::vector<uint8_t>& geo_kind, bool split_geo,
                   std::vector<std::vector<int32_t>>& lists, std::vector<std::pair<int, int>>& keys) {
  std::map<std::pair<int, int>, std::vector<int32_t>> m;
  for (int32_t e : elems) m[{order[e], split_geo ? (int)geo_kind[e] : 1}].push_back(e);
  lists.clear();
  keys.clear();
  for (auto& kv : m) {
    keys.push_back(kv.first);
    lists.push_back(kv.second);
  }
}

dg_status upload_buckets(dg_ctx* c, const std::string& prefix, const std::vector<int32_t>& elems, bool split_curved,
                         bool ns, std::vector<Bucket>& out, std::vector<std::vector<int32_t>>* host_lists = nullptr) {
  std::vector<std::vector<int32_t>> lists;
  std::vector<std::pair<int, int>> keys;
  build_buckets(elems, c->order, c->geo_kind, split_curved, lists, keys);
  out.clear();
  for (size_t i = 0; i < lists.size(); ++i) {
    Bucket b;
    b.N = keys[i].first;
    b.geo = keys[i].second;
    b.curved = b.geo == 2;
    b.ns = ns;
    b.count = (int)lists[i].size();
    dg_status st = dev_upload(c, prefix + std::to_string(i), lists[i], &b.list);
    if (st != DG_OK) return st;
    if (host_lists) {
      std::vector<int64_t> bo(lists[i].size()), bt(lists[i].size());
      for (size_t j = 0; j < lists[i].size(); ++j) {
        bo[j] = c->off[lists[i][j]];
        bt[j] = c->troff[lists[i][j]];
      }
      int64_t* d;
      if ((st = dev_upload(c, prefix + "o" + std::to_string(i), bo, &d)) != DG_OK) return st;
      b.boff = d;
      if ((st = dev_upload(c, prefix + "t" + std::to_string(i), bt, &d)) != DG_OK) return st;
      b.btr = d;
    }
    out.push_back(b);
  }
  if (host_lists) *host_lists = lists;
  return DG_OK;
}

// Copy the autotuned choices onto the buckets they apply to (buckets are rebuilt with the
// orders and flags; the choices are kept per (pass, order, geometry kind)).
void apply_tuning(dg_ctx* c) {
  for (Bucket& b : c->all_buckets) {
    auto it = c->tuning.find({0, b.N, b.geo});
    b.tile_alt = it == c->tuning.end() ? 0 : it->second[0];
    b.bps = it == c->tuning.end() ? 0 : it->second[1];
    b.visc_alt = 0;
    auto st = c->tuning.find({2, b.N, b.geo});
    b.vsplit = st == c->tuning.end() || st->second[0] != 2 ? 0 : std::min(std::max(st->second[1], 0), 3);
  }
  for (Bucket& b : c->ns_buckets) {
    auto it = c->tuning.find({1, b.N, b.geo});
    b.tile_alt = it == c->tuning.end() ? 0 : it->second[0];
    b.bps = it == c->tuning.end() ? 0 : it->second[1];
    b.visc_alt = it == c->tuning.end() ? 0 : it->second[2];
  }
}

// Per-entry tables of a set of buckets, in bucket order: the element's 6 face links, its flag
// and its 32-byte record (read by the pipelined passes instead of chasing the element id).
dg_status upload_entry_tables(dg_ctx* c, const std::string& prefix, const std::vector<std::vector<int32_t>>& lists,
                              const std::vector<FaceLink>& link, std::vector<Bucket>& buckets) {
  dg_status st = DG_OK;
  for (size_t i = 0; i < buckets.size() && i < lists.size(); ++i) {
    const std::vector<int32_t>& L = lists[i];
    std::vector<FaceLink> bl(L.size() * 6);
    std::vector<uint8_t> bf(L.size());
    std::vector<EntryMeta> bm(L.size());
    for (size_t j = 0; j < L.size(); ++j) {
      for (int f = 0; f < 6; ++f) bl[j * 6 + f] = link[(size_t)L[j] * 6 + f];
      bf[j] = c->flag[L[j]];
      bm[j].off = c->off[L[j]];
      bm[j].troff = c->troff[L[j]];
      bm[j].elem = L[j];
      bm[j].flag = c->flag[L[j]];
      bm[j].has_mortar = 0;
      for (int f = 0; f < 6; ++f) bm[j].has_mortar |= link[(size_t)L[j] * 6 + f].kind == FK_MORTAR ? 1 : 0;
      bm[j].pad = 0;
    }
    FaceLink* dbl;
    uint8_t* dbf;
    EntryMeta* dbm;
    if ((st = dev_upload(c, prefix + "l" + std::to_string(i), bl, &dbl)) != DG_OK) return st;
    if ((st = dev_upload(c, prefix + "f" + std::to_string(i), bf, &dbf)) != DG_OK) return st;
    if ((st = dev_upload(c, prefix + "m" + std::to_string(i), bm, &dbm)) != DG_OK) return st;
    buckets[i].blink = dbl;
    buckets[i].bflag = dbf;
    buckets[i].bmeta = dbm;
  }
  return st;
}

// flag-dependent tables: links' neighbour flags, NS buckets, mortar lifting slots
dg_status rebuild_flags(dg_ctx* c) {
  std::vector<FaceLink> link(c->ne * 6);
  std::vector<int32_t> mall, mns, ns_elems;
  for (int64_t e = 0; e < c->ne; ++e) {
    if (c->flag[e]) ns_elems.push_back((int32_t)e);
    for (int f = 0; f < 6; ++f) {
      FaceLink L{};
      int32_t nb = c->nb[e * 6 + f];
      L.nbr = nb;
      if (nb >= 0) {
        L.nface = c->nbf[e * 6 + f];
        L.orient = c->nbo[e * 6 + f];
        L.kind = c->order[nb] == c->order[e] ? FK_CONF : FK_MORTAR;
        L.nflag = c->flag[nb];
        const int64_t nn1 = c->order[nb] + 1;
        L.nslot = c->troff[nb] + (int64_t)L.nface * nn1 * nn1;
        if (L.nslot < 0 || L.nslot + nn1 * nn1 > c->tr_total)
          return fail(DG_ERR_MESH, "internal: trace slot of element %lld face %d out of range", (long long)e, f);
        if (L.kind == FK_MORTAR) {
          mall.push_back((int32_t)(e * 6 + f));
          if (c->flag[e]) mns.push_back((int32_t)(e * 6 + f));
        }
      } else {
        L.nbr = -1;
        const int tag = c->bc[e * 6 + f];
        L.kind = tag == 1 ? FK_INFLOW : (tag == 2 ? FK_OUTFLOW : (tag == 3 ? FK_WALL : FK_SLIP));
      }
      link[e * 6 + f] = L;
    }
  }
  FaceLink* dl;
  dg_status st = dev_upload(c, "link", link, &dl);
  if (st != DG_OK) return st;
  c->M.link = dl;
  // all-element buckets in four groups, each in element order: Euler elements with no NS
  // neighbour and no mortar face (independent of the viscous and mortar passes: the inviscid
  // pass runs them while those passes drain), the NS elements, the other Euler elements, and
  // last about two rounds of tiles' worth of independent elements held back from the first
  // group (the lightest tiles end the stage, so its last round is short). n_indep counts the
  // first group only. A tile of the pipelined passes then holds elements of one flag but at the
  // boundaries between the groups.
  auto dep_class = [&](int32_t e) {
    if (c->flag[e]) return 1;
    for (int f = 0; f < 6; ++f) {
      const int32_t nb = c->nb[(int64_t)e * 6 + f];
      if (nb >= 0 && (c->flag[nb] || c->order[nb] != c->order[e])) return 2;
    }
    return 0;
  };
  std::vector<uint8_t> cls(c->ne, 0);
  for (int64_t e = 0; e < c->ne; ++e) cls[e] = (uint8_t)dep_class((int32_t)e);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) sms = 0;
  for (size_t i = 0; i < c->all_buckets.size() && i < c->all_lists.size(); ++i) {
    std::vector<int32_t>& L = c->all_lists[i];
    std::stable_sort(L.begin(), L.end(), [&](int32_t x, int32_t y) { return cls[x] < cls[y]; });
    const int n0 = (int)std::count_if(L.begin(), L.end(), [&](int32_t e) { return cls[e] == 0; });
    // two rounds of the persistent grid (about three blocks per SM) at this order's tile size
    const int tail = n0 < (int)L.size() ? std::min(n0 / 4, 2 * 3 * sms * tile_epb32(c->all_buckets[i].N, 0)) : 0;
    std::rotate(L.begin() + (n0 - tail), L.begin() + n0, L.end());
    c->all_buckets[i].n_indep = n0 - tail;
    std::vector<int64_t> bo(L.size()), bt(L.size());
    for (size_t j = 0; j < L.size(); ++j) {
      bo[j] = c->off[L[j]];
      bt[j] = c->troff[L[j]];
    }
    Bucket& b = c->all_buckets[i];
    int64_t* d;
    if ((st = dev_upload(c, "allb" + std::to_string(i), L, &b.list)) != DG_OK) return st;
    if ((st = dev_upload(c, "allbo" + std::to_string(i), bo, &d)) != DG_OK) return st;
    b.boff = d;
    if ((st = dev_upload(c, "allbt" + std::to_string(i), bt, &d)) != DG_OK) return st;
    b.btr = d;
  }
  // per-entry link and flag tables of the all-element buckets
  if ((st = upload_entry_tables(c, "allb", c->all_lists, link, c->all_buckets)) != DG_OK) return st;
  uint8_t* df;
  if ((st = dev_upload(c, "flag", c->flag, &df)) != DG_OK) return st;
  c->M.flag = df;
  // group the mortar slots by mortar order (one launch per order, sized for its points)
  auto by_order = [&](std::vector<int32_t>& v, int* start) {
    auto mo = [&](int32_t es) {
      const int64_t e = es / 6, nb = c->nb[es];
      return (int)std::max(c->order[e], c->order[nb]);
    };
    std::stable_sort(v.begin(), v.end(), [&](int32_t x, int32_t y) { return mo(x) < mo(y); });
    for (int k = 0; k <= MAXN + 1; ++k) start[k] = 0;
    for (int32_t es : v) ++start[mo(es) + 1];
    for (int k = 1; k <= MAXN + 1; ++k) start[k] += start[k - 1];
  };
  by_order(mall, c->mortar_all_mo);
  by_order(mns, c->mortar_ns_mo);
  std::vector<int32_t> mface;
  for (int32_t es : mall)
    if (c->order[es / 6] > c->order[c->nb[es]]) mface.push_back(es);
  by_order(mface, c->mortar_face_mo);
  if ((st = dev_upload(c, "mortar_face", mface, &c->mortar_face)) != DG_OK) return st;
  if ((st = dev_upload(c, "mortar_all", mall, &c->mortar_all)) != DG_OK) return st;
  c->n_mortar_all = (int)mall.size();
  if ((st = dev_upload(c, "mortar_ns", mns, &c->mortar_ns)) != DG_OK) return st;
  c->n_mortar_ns = (int)mns.size();
  for (auto it = c->buf.begin(); it != c->buf.end();) {
    if (it->first.rfind("nsb", 0) == 0) {
      cudaFree(it->second.p);
      it = c->buf.erase(it);
    } else {
      ++it;
    }
  }
  std::vector<std::vector<int32_t>> ns_lists;
  if ((st = upload_buckets(c, "nsb", ns_elems, true, true, c->ns_buckets, &ns_lists)) != DG_OK) return st;
  if ((st = upload_entry_tables(c, "nsbx", ns_lists, link, c->ns_buckets)) != DG_OK) return st;
  // viscous traces of Euler elements are never written: keep them at zero
  if (c->M.Tv) CU(cudaMemset(c->M.Tv, 0, sizeof(double) * (nvar(c) - 1) * std::max<int64_t>(c->tr_total, 1)));
  apply_tuning(c);
  c->version++;
  destroy_graph(c);
  return DG_OK;
}

// The compressible form needs a far field at its inflow and outflow faces.
dg_status check_model_mesh(const dg_ctx* c) {
  if (c->prm.model != 1) return DG_OK;
  for (int64_t s = 0; s < c->ne * 6; ++s)
    if (c->nb[s] < 0 && (c->bc[s] == 1 || c->bc[s] == 2) && !(c->prm.inflow[0] > 0.0 && c->prm.p_inf > 0.0))
      return fail(DG_ERR_ARG, "compressible form: inflow/outflow faces need a far-field density inflow[0] > 0 and p_inf > 0");
  return DG_OK;
}

// order-dependent layout, geometry, buffers
dg_status rebuild_orders(dg_ctx* c) {
  const int64_t E = c->ne;
  dg_status cm = check_model_mesh(c);
  if (cm != DG_OK) return cm;
  c->off.assign(E + 1, 0);
  c->troff.assign(E + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    const int n = c->order[e] + 1;
    c->off[e + 1] = c->off[e] + (int64_t)n * n * n;
    c->troff[e + 1] = c->troff[e] + 6LL * n * n;
  }
  c->total = c->off[E];
  c->tr_total = c->troff[E];
  if (c->total * 4 > INT64_C(1) << 40) return fail(DG_ERR_UNSUPPORTED, "mesh too large");
  // geometry
  c->ec.assign(E, ElemConst{});
  c->geo_kind.assign(E, 1);
  std::vector<double> geo;
  c->any_curved = false;
  std::vector<ElemGeo> curved_geo;
  std::vector<int64_t> curved_ids;
  for (int64_t e = 0; e < E; ++e) {
    ElemGeo G;
    const int N = c->order[e], n = N + 1, n3 = n * n * n;
    elem_geometry(c, e, N, G);
    ElemConst& k = c->ec[e];
    const Rule& r = node_rule(c, N);
    double vol = 0.0;
    if (G.affine) {
      if (!(G.J > 0.0)) return fail(DG_ERR_MESH, "element %lld has a non-positive Jacobian", (long long)e);
      for (int i = 0; i < 9; ++i) k.Ja[i] = G.Ja[i];
      k.J = G.J;
      k.invJ = 1.0 / G.J;
      k.curved = 0.0;
      // axis-aligned box: diagonal metric with positive entries
      double mx = 0.0, off_diag = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          mx = std::max(mx, std::fabs(G.Ja[i * 3 + j]));
          if (i != j) off_diag = std::max(off_diag, std::fabs(G.Ja[i * 3 + j]));
        }
      if (off_diag <= 1e-14 * mx && G.Ja[0] > 0.0 && G.Ja[4] > 0.0 && G.Ja[8] > 0.0) {
        c->geo_kind[e] = 0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            if (i != j) k.Ja[i * 3 + j] = 0.0;
      }
      vol = 8.0 * G.J;
    } else {
      for (int p = 0; p < n3; ++p) {
        if (!(G.Jn[p] > 0.0)) return fail(DG_ERR_MESH, "element %lld has a non-positive Jacobian", (long long)e);
        vol += r.w[p % n] * r.w[(p / n) % n] * r.w[p / (n * n)] * G.Jn[p];
      }
      k.curved = 1.0;
      c->geo_kind[e] = 2;
      c->any_curved = true;
      curved_ids.push_back(e);
      curved_geo.push_back(std::move(G));
    }
    k.delta = std::cbrt(vol) / n;
  }
  if (c->any_curved) {
    geo.assign((size_t)10 * c->total, 0.0);
    for (size_t i = 0; i < curved_ids.size(); ++i) {
      const int64_t e = curved_ids[i];
      const int n = c->order[e] + 1, n3 = n * n * n;
      const ElemGeo& G = curved_geo[i];
      for (int k = 0; k < 9; ++k)
        for (int p = 0; p < n3; ++p) geo[(size_t)k * c->total + c->off[e] + p] = G.Jan[k * n3 + p];
      for (int p = 0; p < n3; ++p) geo[(size_t)9 * c->total + c->off[e] + p] = G.Jn[p];
    }
  }
  dg_status st;
  int64_t* d64;
  if ((st = dev_upload(c, "elem_off", c->off, &d64)) != DG_OK) return st;
  c->M.elem_off = d64;
  if ((st = dev_upload(c, "tr_off", c->troff, &d64)) != DG_OK) return st;
  c->M.tr_off = d64;
  int8_t* d8;
  if ((st = dev_upload(c, "order", c->order, &d8)) != DG_OK) return st;
  c->M.order = d8;
  ElemConst* dec;
  if ((st = dev_upload(c, "ec", c->ec, &dec)) != DG_OK) return st;
  c->M.ec = dec;
  std::vector<ElemConst32> ec32(E);
  for (int64_t e = 0; e < E; ++e) {
    for (int k = 0; k < 9; ++k) ec32[e].Ja[k] = (float)c->ec[e].Ja[k];
    ec32[e].invJ = (float)c->ec[e].invJ;
    ec32[e].delta = (float)c->ec[e].delta;
    ec32[e].curved = (float)c->ec[e].curved;
  }
  ElemConst32* dec32;
  if ((st = dev_upload(c, "ec32", ec32, &dec32)) != DG_OK) return st;
  c->M.ec32 = dec32;
  double* dgeo = nullptr;
  float* dgeo32 = nullptr;
  if (c->any_curved) {
    if ((st = dev_upload(c, "geo", geo, &dgeo)) != DG_OK) return st;
    std::vector<float> g32(geo.size());
    for (size_t i = 0; i < (size_t)9 * c->total; ++i) g32[i] = (float)geo[i];
    for (int64_t i = 0; i < c->total; ++i)
      g32[(size_t)9 * c->total + i] = geo[(size_t)9 * c->total + i] != 0.0 ? (float)(1.0 / geo[(size_t)9 * c->total + i]) : 0.f;
    if ((st = dev_upload(c, "geo32", g32, &dgeo32)) != DG_OK) return st;
  } else {
    free_buf(c, "geo");
    free_buf(c, "geo32");
  }
  c->M.geo = dgeo;
  c->M.geo32 = dgeo32;
  c->M.n_elem = E;
  c->M.total = c->total;
  c->M.tr_total = c->tr_total;
  const int nv = nvar(c), nvv = nv - 1;  // state planes; viscous planes (momentum, + energy)
  if ((st = dev_alloc(c, "Tq", nv * c->tr_total, &c->trace_buf[0])) != DG_OK) return st;
  if ((st = dev_alloc(c, "Tq2", nv * c->tr_total, &c->trace_buf[1])) != DG_OK) return st;
  c->M.Tq = c->trace_buf[0];
  c->M.Tq_next = c->trace_buf[1];
  if ((st = dev_alloc(c, "Tv", nvv * c->tr_total, &c->M.Tv)) != DG_OK) return st;
  if ((st = dev_alloc(c, "rv", nvv * c->total, &c->M.rv)) != DG_OK) return st;
  bool has_mortar = false;
  for (int64_t s = 0; s < E * 6 && !has_mortar; ++s)
    has_mortar = c->nb[s] >= 0 && c->order[c->nb[s]] != c->order[s / 6];
  const int64_t mort = has_mortar ? c->tr_total : 0;
  const int64_t lu_planes = c->prm.model == 1 ? 12 : 9;  // phi*_c S_k: phi = (v, T) or u
  if ((st = dev_alloc(c, "LU", lu_planes * mort, &c->M.LU)) != DG_OK) return st;
  if ((st = dev_alloc(c, "LH", (int64_t)nvar(c) * mort, &c->M.LH)) != DG_OK) return st;
  CU(cudaMemset(c->M.Tv, 0, sizeof(double) * nvv * std::max<int64_t>(c->tr_total, 1)));
  if ((st = dev_alloc(c, "partial", 5 * E, &c->partial)) != DG_OK) return st;
  c->partial_host.assign(5 * E, 0.0);
  free_buf(c, "stage_q");
  free_buf(c, "stage_r");
  c->stage_q = c->stage_r = nullptr;
  // buckets over all elements
  for (auto it = c->buf.begin(); it != c->buf.end();) {
    if (it->first.rfind("allb", 0) == 0 || it->first.rfind("ordb", 0) == 0) {
      cudaFree(it->second.p);
      it = c->buf.erase(it);
    } else {
      ++it;
    }
  }
  std::vector<int32_t> every(E);
  for (int64_t e = 0; e < E; ++e) every[e] = (int32_t)e;
  if ((st = upload_buckets(c, "allb", every, true, false, c->all_buckets, &c->all_lists)) != DG_OK) return st;
  if ((st = upload_buckets(c, "ordb", every, false, false, c->ord_buckets)) != DG_OK) return st;
  return rebuild_flags(c);
}

// One phase of a residual evaluation (mode RESIDUAL) or of an RK stage (mode RK) on stream s.
// Traces are double-buffered: stage s reads buffer s % 2; in RK mode the update of stages 0
// and 1 writes the traces of the new state into the other buffer, so only stage 0 (and a
// residual evaluation) launches the trace kernel.
// The persistent stage kernel (viscous pass, grid barrier, inviscid pass and update in one
// cooperative launch) applies to a reduced-precision context with FP32 contractions whose mesh
// is one (order, box or affine) bucket without mortar faces, on the default tile shapes and the
// pipelined viscous kernel.
bool stage_fusable(const dg_ctx* c) {
  const DevMesh& M = c->M;
  // (with the FP64 divergence only the kernel with tile queues applies, see stage_fused)
  if (M.precision != 1 || M.tc || M.split || M.model || M.nodes) return false;
  if (c->all_buckets.size() != 1 || c->n_mortar_all) return false;
  // (the one-launch kernels use the default tile shapes whatever the separate launches use)
  const Bucket& bi = c->all_buckets[0];
  if (bi.geo > 1) return false;
  if (c->ns_buckets.size() > 1) return false;
  if (c->ns_buckets.size() == 1) {
    const Bucket& bv = c->ns_buckets[0];
    if (bv.count > 0 && (bv.N != bi.N || bv.geo != bi.geo)) return false;
  }
  return true;
}

// ... and is used where the autotuner chose it: 0 separate launches, 1 the persistent kernel
// with a grid barrier, 2 the one-launch kernel with tile queues
int stage_fused(const dg_ctx* c) {
  if (!stage_fusable(c)) return 0;
  auto it = c->tuning.find({2, c->all_buckets[0].N, c->all_buckets[0].geo});
  const int v = it != c->tuning.end() && (it->second[0] == 1 || it->second[0] == 2) ? it->second[0] : 0;
  return c->M.div64 && v == 1 ? 0 : v;
}

cudaError_t launch_stage(const dg_ctx* c, const DevMesh& M, const double* q, double* out, double* g, int stage,
                         int write_tr, int kind, cudaStream_t s) {
  Bucket bv{};
  if (!c->ns_buckets.empty()) bv = c->ns_buckets[0];
  return launch_stage32(M, bv, c->all_buckets[0], q, out, g, stage, write_tr, kind == 2 ? 1 : 0, s);
}

dg_status issue_phase_impl(dg_ctx* c, int phase, const double* q, double* out, double* g, int mode, int stage,
                           double dt, cudaStream_t s, int* nlaunch) {
  int nl = 0;
  DevMesh M = c->M;
  // the inviscid launch directly after this stage's viscous pass (no mortar pass between)
  M.after_visc = phase == 4 && c->visc_last && c->n_mortar_all == 0 && M.overlap ? 1 : 0;
  const int cur = (mode == MODE_RK) ? (stage + c->cap_parity) % 2 : 0;
  M.Tq = c->trace_buf[cur];
  M.Tq_next = c->trace_buf[1 - cur];
  const int write_tr = (mode == MODE_RK && (stage < 2 || c->cap_write_all)) ? 1 : 0;
  // a chained step's traces come from the previous step's last update
  if (phase == 0 && mode == MODE_RK && c->cap_no_traces) {
    if (nlaunch) *nlaunch += nl;
    return DG_OK;
  }
  if (M.nodes == 1 && M.model == 1) {  // compressible form on Gauss-Legendre nodes
    if (phase == 0 && !(mode == MODE_RK && stage > 0)) {
      for (const Bucket& b : c->ord_buckets) {
        CU(launch_traces_cns_gl(M, b, q, s));
        ++nl;
      }
    } else if (phase == 1 && c->n_mortar_ns) {
      CU(launch_mortar_lift_cns(M, c->mortar_ns, c->n_mortar_ns, s));
      ++nl;
    } else if (phase == 3 && c->n_mortar_all) {
      CU(launch_mortar_flux_cns(M, c->mortar_all, c->n_mortar_all, s));
      ++nl;
    } else if (phase == 2) {
      for (const Bucket& b : c->ns_buckets) {
        CU(launch_viscous_cns_gl(M, b, q, s));
        ++nl;
      }
    } else if (phase == 4) {
      for (const Bucket& b : c->all_buckets) {
        CU(launch_inviscid_cns_gl(M, b, q, out, g, mode, stage, dt, write_tr, s));
        ++nl;
      }
    }
    if (nlaunch) *nlaunch += nl;
    return DG_OK;
  }
  if (M.nodes == 1) {  // Gauss-Legendre nodes: the mortar kernels take the Gauss-point tables
    if (phase == 0 && !(mode == MODE_RK && stage > 0)) {
      for (const Bucket& b : c->ord_buckets) {
        CU(launch_traces_gl(M, b, q, s));
        ++nl;
      }
    } else if (phase == 1 && c->n_mortar_ns) {
      CU(launch_mortar_lift(M, c->mortar_ns, c->mortar_ns_mo, &nl, s));
    } else if (phase == 3 && c->n_mortar_all) {
      CU(launch_mortar_flux(M, c->mortar_face, c->mortar_face_mo, &nl, s));
    } else if (phase == 2) {
      for (const Bucket& b : c->ns_buckets) {
        CU(launch_viscous_gl(M, b, q, s));
        ++nl;
      }
    } else if (phase == 4) {
      for (const Bucket& b : c->all_buckets) {
        CU(launch_inviscid_gl(M, b, q, out, g, mode, stage, dt, write_tr, s));
        ++nl;
      }
    }
    if (nlaunch) *nlaunch += nl;
    return DG_OK;
  }
  if (M.model == 1) {  // compressible form: five-variable kernels and mortars
    if (phase == 0 && !(mode == MODE_RK && stage > 0)) {
      for (const Bucket& b : c->ord_buckets) {
        CU(launch_traces_cns(M, b, q, s));
        ++nl;
      }
    } else if (phase == 1 && c->n_mortar_ns) {
      CU(launch_mortar_lift_cns(M, c->mortar_ns, c->n_mortar_ns, s));
      ++nl;
    } else if (phase == 3 && c->n_mortar_all) {
      CU(launch_mortar_flux_cns(M, c->mortar_all, c->n_mortar_all, s));
      ++nl;
    } else if (phase == 2) {
      for (const Bucket& b : c->ns_buckets) {
        CU(launch_viscous_cns(M, b, q, s));
        ++nl;
      }
    } else if (phase == 4) {
      for (const Bucket& b : c->all_buckets) {
        CU(launch_inviscid_cns(M, b, q, out, g, mode, stage, dt, write_tr, s));
        ++nl;
      }
    }
    if (nlaunch) *nlaunch += nl;
    return DG_OK;
  }
  switch (phase) {
    case 0:
      if (mode == MODE_RK && stage > 0) break;
      for (const Bucket& b : c->ord_buckets) {
        CU(launch_traces(M, b, q, M.precision, s));
        ++nl;
      }
      break;
    case 1:
      if (c->n_mortar_ns) CU(launch_mortar_lift(M, c->mortar_ns, c->mortar_ns_mo, &nl, s));
      break;
    case 2:
      if (mode == MODE_RK && stage_fused(c)) break;  // the stage kernel runs it in phase 4
      for (const Bucket& b : c->ns_buckets) {
        CU(launch_viscous(M, b, q, M.precision, s));
        ++nl;
      }
      break;
    case 3:
      if (c->n_mortar_all) CU(launch_mortar_flux(M, c->mortar_face, c->mortar_face_mo, &nl, s));
      break;
    default:
      if (mode == MODE_RK && stage_fused(c)) {
        CU(launch_stage(c, M, q, out, g, stage, write_tr, stage_fused(c), s));
        ++nl;
        break;
      }
      for (const Bucket& b : c->all_buckets) {
        CU(launch_inviscid(M, b, q, out, g, mode, stage, dt, write_tr, M.precision, s));
        ++nl;
      }
  }
  if (nlaunch) *nlaunch += nl;
  return DG_OK;
}

// Every phase is issued through here: it records whether the last launching phase was the
// viscous pass, which the next phase-4 launch may overlap.
dg_status issue_phase(dg_ctx* c, int phase, const double* q, double* out, double* g, int mode, int stage, double dt,
                      cudaStream_t s, int* nlaunch) {
  int nl = 0;
  const dg_status st = issue_phase_impl(c, phase, q, out, g, mode, stage, dt, s, &nl);
  if (nl > 0) c->visc_last = phase == 2;
  if (nlaunch) *nlaunch += nl;
  return st;
}

dg_status issue_stage(dg_ctx* c, const double* q, double* out, double* g, int mode, int stage, double dt,
                      cudaStream_t s, int* nlaunch) {
  for (int ph = 0; ph < DG_NPHASES; ++ph) {
    dg_status st = issue_phase(c, ph, q, out, g, mode, stage, dt, s, nlaunch);
    if (st != DG_OK) return st;
  }
  return DG_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

const char* dg_last_error(void) { return g_last_error.c_str(); }

dg_status dg_create_mesh(const dg_mesh_desc* mesh, const dg_params* params, int device, dg_ctx** out) {
  if (!out) return fail(DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !mesh->hex || !mesh->geom_xyz) return fail(DG_ERR_ARG, "mesh, hex or geom_xyz is NULL");
  if (mesh->n_elem <= 0 || mesh->n_elem > INT32_MAX / 6) return fail(DG_ERR_ARG, "n_elem out of range");
  if (mesh->geom_degree < 1 || mesh->geom_degree > 2) return fail(DG_ERR_UNSUPPORTED, "geometry degree must be 1 or 2");
  dg_status st = check_params(params);
  if (st != DG_OK) return st;
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(DG_ERR_ARG, "device %d not present (%d devices)", device, ndev);
  CU(cudaSetDevice(device));
  dg_ctx* c = new dg_ctx();
  c->device = device;
  c->ne = mesh->n_elem;
  c->gdeg = mesh->geom_degree;
  const int ng3 = (c->gdeg + 1) * (c->gdeg + 1) * (c->gdeg + 1);
  c->hex.assign(mesh->hex, mesh->hex + c->ne * 8);
  c->gnodes.assign(mesh->geom_xyz, mesh->geom_xyz + c->ne * ng3 * 3);
  c->bc.assign(c->ne * 6, -1);
  if (mesh->bc_tag) c->bc.assign(mesh->bc_tag, mesh->bc_tag + c->ne * 6);
  for (int64_t i = 0; i < c->ne * 6; ++i)
    if (c->bc[i] == 0 || c->bc[i] < -1 || c->bc[i] > 4) {
      const int tag = c->bc[i];
      delete c;
      return fail(DG_ERR_ARG, "element %lld face %d: boundary tag %d is not -1, 1, 2, 3 or 4", (long long)(i / 6),
                  (int)(i % 6), tag);
    }
  c->prm = *params;
  // face matching on sorted corner ids
  c->nb.assign(c->ne * 6, -1);
  c->nbf.assign(c->ne * 6, 0);
  c->nbo.assign(c->ne * 6, 0);
  std::unordered_map<Key4, std::vector<int64_t>, Key4Hash> faces;
  faces.reserve((size_t)c->ne * 4);
  for (int64_t e = 0; e < c->ne; ++e)
    for (int f = 0; f < 6; ++f) {
      Key4 k;
      for (int i = 0; i < 4; ++i) k.k[i] = c->hex[e * 8 + face_corner_index(f, i & 1, i >> 1)];
      std::sort(k.k, k.k + 4);
      for (int i = 0; i < 3; ++i)
        if (k.k[i] == k.k[i + 1]) {
          delete c;
          return fail(DG_ERR_MESH, "element %lld face %d repeats a vertex id", (long long)e, f);
        }
      faces[k].push_back(e * 6 + f);
    }
  for (auto& kv : faces) {
    const auto& v = kv.second;
    if (v.size() > 2) {
      delete c;
      return fail(DG_ERR_MESH, "a face is shared by %zu elements", v.size());
    }
    if (v.size() == 1) {
      int64_t s = v[0];
      if (c->bc[s] < 1) {
        delete c;
        return fail(DG_ERR_MESH, "element %lld face %d is unmatched and has no boundary tag", (long long)(s / 6),
                    (int)(s % 6));
      }
      continue;
    }
    for (int side = 0; side < 2; ++side) {
      const int64_t s0 = v[side], s1 = v[1 - side];
      const int64_t e0 = s0 / 6, e1 = s1 / 6;
      const int f0 = (int)(s0 % 6), f1 = (int)(s1 % 6);
      if (c->bc[s0] >= 1) {
        delete c;
        return fail(DG_ERR_MESH, "element %lld face %d is interior but tagged as boundary", (long long)e0, f0);
      }
      int found = -1;
      for (int o = 0; o < 8 && found < 0; ++o) {
        bool ok = true;
        for (int cb = 0; cb < 2 && ok; ++cb)
          for (int ca = 0; ca < 2 && ok; ++ca) {
            int a0, b0;
            orient_fwd(o, 1, ca, cb, a0, b0);
            ok = c->hex[e1 * 8 + face_corner_index(f1, ca, cb)] == c->hex[e0 * 8 + face_corner_index(f0, a0, b0)];
          }
        if (ok) found = o;
      }
      if (found < 0) {
        delete c;
        return fail(DG_ERR_MESH, "no orientation matches element %lld face %d", (long long)e0, f0);
      }
      c->nb[s0] = (int32_t)e1;
      c->nbf[s0] = (uint8_t)f1;
      c->nbo[s0] = (uint8_t)found;
    }
  }
  // constants, default orders and flags
  Ops1D o1{};
  const OpTables& T = ops();
  for (int N = 1; N <= MAXN; ++N) {
    const int n = N + 1;
    for (int i = 0; i < n * n; ++i) o1.D[N][i] = T.rule[N].D[i];
    for (int i = 0; i < n; ++i) {
      o1.w[N][i] = T.rule[N].w[i];
      o1.x[N][i] = T.rule[N].x[i];
    }
    for (int i = 0; i < n * n; ++i) o1.Dg[N][i] = T.gl[N].D[i];
    for (int i = 0; i < n; ++i) {
      o1.wg[N][i] = T.gl[N].w[i];
      o1.lbg[N][0][i] = T.glb[N][0][i];
      o1.lbg[N][1][i] = T.glb[N][1][i];
    }
  }
  cudaError_t ce = upload_ops(o1);
  if (ce == cudaSuccess) ce = prepare_kernels();
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    delete c;
    return fail(DG_ERR_CUDA, "CUDA setup failed: %s", cudaGetErrorString(ce));
  }
  double* dtab = nullptr;
  if ((st = dev_upload(c, "interp", T.interp, &dtab)) != DG_OK) {
    dg_destroy(c);
    return st;
  }
  c->M.interp = dtab;
  if ((st = dev_upload(c, "proj", T.proj, &dtab)) != DG_OK) {
    dg_destroy(c);
    return st;
  }
  c->M.proj = dtab;
  if ((st = dev_upload(c, "interp_gl", T.interp_gl, &dtab)) != DG_OK) {
    dg_destroy(c);
    return st;
  }
  c->M.interp_gl = dtab;
  const char* gnames[3] = {"interp_g", "proj_g", "lb_g"};
  const std::vector<double>* gtabs[3] = {&T.interp_g, &T.proj_g, &T.lb_g};
  const double** gdst[3] = {&c->M.interp_g, &c->M.proj_g, &c->M.lb_g};
  for (int i = 0; i < 3; ++i) {
    if ((st = dev_upload(c, gnames[i], *gtabs[i], &dtab)) != DG_OK) {
      dg_destroy(c);
      return st;
    }
    *gdst[i] = dtab;
  }
  // [0..3] the device error word, [4..5] the persistent stage kernel's grid barrier, [8..11] the
  // one-launch stage kernel's tile queues
  int* derr;
  if ((st = dev_alloc(c, "err", 16, &derr)) != DG_OK) {
    dg_destroy(c);
    return st;
  }
  cudaMemset(derr, 0, 16 * sizeof(int));
  c->M.err = derr;
  c->M.wait_polls = kWaitPolls;
  c->M.stop_tile = -1;
  c->M.overlap = 1;
  c->M.after_visc = 0;
  apply_params(c);
  c->order.assign(c->ne, (int8_t)std::max(3, c->gdeg));
  c->flag.assign(c->ne, 1);
  if ((st = rebuild_orders(c)) != DG_OK) {
    dg_destroy(c);
    return st;
  }
  *out = c;
  return DG_OK;
}

dg_status dg_set_orders(dg_ctx* c, const int8_t* orders) {
  if (!c || !orders) return fail(DG_ERR_ARG, "NULL argument");
  for (int64_t e = 0; e < c->ne; ++e)
    if (orders[e] < 1 || orders[e] > MAXN || orders[e] < c->gdeg)
      return fail(DG_ERR_ARG, "element %lld: order %d outside %d..%d", (long long)e, orders[e], std::max(1, c->gdeg), MAXN);
  CU(cudaSetDevice(c->device));
  std::vector<int8_t> old = c->order;
  std::vector<int64_t> old_off = c->off;
  c->order.assign(orders, orders + c->ne);
  dg_status st = rebuild_orders(c);
  if (st != DG_OK) {
    c->order = old;
    std::string msg = g_last_error;
    rebuild_orders(c);
    g_last_error = msg;
  } else {
    c->prev_order = std::move(old);
    c->prev_off = std::move(old_off);
  }
  return st;
}

dg_status dg_project_state(dg_ctx* c, const double* q_old, double* q_new, void* stream) {
  if (!c || !q_old || !q_new) return fail(DG_ERR_ARG, "NULL argument");
  if (c->prev_order.empty()) return fail(DG_ERR_STATE, "dg_project_state needs a preceding dg_set_orders");
  // the interpolation and projection tables follow the node set (Gauss-Lobatto or Gauss points);
  // every state plane (4, or 5 for the compressible form) is re-laid out the same way
  if (q_old == q_new) return fail(DG_ERR_ARG, "q_old and q_new must not overlap");
  CU(cudaSetDevice(c->device));
  int8_t* dord = nullptr;
  int64_t* doff = nullptr;
  dg_status st;
  if ((st = dev_upload(c, "prev_order", c->prev_order, &dord)) != DG_OK) return st;
  if ((st = dev_upload(c, "prev_off", c->prev_off, &doff)) != DG_OK) return st;
  CU(launch_project_state(c->M, dord, doff, c->prev_off.back(), q_old, q_new, (cudaStream_t)stream));
  return DG_OK;
}

// Mixture constants for the detection kernel: inverse covariances by cofactors, log-weights
// with the log-determinants (Sec. 2.1; the mixture itself is an input).
static dg_status gmm_prepare(const dg_gmm& g, GmmDev& out) {
  if (g.viscous != 0 && g.viscous != 1) return fail(DG_ERR_ARG, "gmm.viscous must be 0 or 1");
  if (g.precision != 0 && g.precision != 1) return fail(DG_ERR_ARG, "gmm.precision must be 0 or 1");
  for (int k = 0; k < 2; ++k) {
    if (!std::isfinite(g.weight[k]) || !(g.weight[k] > 0.0))
      return fail(DG_ERR_ARG, "gmm.weight[%d] must be positive and finite", k);
    const double(*C)[3] = g.cov[k];
    double big = 0.0;
    for (int i = 0; i < 3; ++i) {
      if (!std::isfinite(g.mean[k][i])) return fail(DG_ERR_ARG, "gmm.mean[%d] is not finite", k);
      for (int j = 0; j < 3; ++j) {
        if (!std::isfinite(C[i][j])) return fail(DG_ERR_ARG, "gmm.cov[%d] is not finite", k);
        big = std::max(big, std::fabs(C[i][j]));
      }
    }
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (std::fabs(C[i][j] - C[j][i]) > 1e-12 * big) return fail(DG_ERR_ARG, "gmm.cov[%d] is not symmetric", k);
    // Sylvester's criterion on the leading principal minors
    const double m1 = C[0][0], m2 = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    const double c00 = C[1][1] * C[2][2] - C[1][2] * C[2][1];
    const double c01 = C[1][2] * C[2][0] - C[1][0] * C[2][2];
    const double c02 = C[1][0] * C[2][1] - C[1][1] * C[2][0];
    const double det = C[0][0] * c00 + C[0][1] * c01 + C[0][2] * c02;
    if (!(m1 > 0.0) || !(m2 > 0.0) || !(det > 0.0))
      return fail(DG_ERR_ARG, "gmm.cov[%d] is not positive definite", k);
    const double inv00 = c00 / det;
    const double inv01 = (C[0][2] * C[2][1] - C[0][1] * C[2][2]) / det;
    const double inv02 = (C[0][1] * C[1][2] - C[0][2] * C[1][1]) / det;
    const double inv11 = (C[0][0] * C[2][2] - C[0][2] * C[2][0]) / det;
    const double inv12 = (C[0][2] * C[1][0] - C[0][0] * C[1][2]) / det;
    const double inv22 = (C[0][0] * C[1][1] - C[0][1] * C[1][0]) / det;
    const double P[6] = {inv00, inv01, inv02, inv11, inv12, inv22};
    for (int i = 0; i < 6; ++i) out.P[k][i] = P[i];
    for (int i = 0; i < 3; ++i) out.mu[k][i] = g.mean[k][i];
    out.c[k] = std::log(g.weight[k]) - 0.5 * std::log(det);
    for (int i = 0; i < 6; ++i) out.P32[k][i] = (float)P[i];
    for (int i = 0; i < 3; ++i) out.mu32[k][i] = (float)g.mean[k][i];
    out.c32[k] = (float)out.c[k];
  }
  out.viscous = g.viscous;
  return DG_OK;
}

dg_status dg_detect_regions(dg_ctx* c, const double* q, const dg_gmm* gmm, uint8_t* flags, double* pbar,
                            double* feat, void* stream) {
  if (!c || !q || !gmm) return fail(DG_ERR_ARG, "NULL argument");
  if (!flags && !pbar && !feat) return fail(DG_ERR_ARG, "dg_detect_regions: no output requested");
  if (c->prm.model != 0) return fail(DG_ERR_UNSUPPORTED, "dg_detect_regions: incompressible form only");
  GmmDev g{};
  dg_status st = gmm_prepare(*gmm, g);
  if (st != DG_OK) return st;
  CU(cudaSetDevice(c->device));
  const OpTables& T = ops();
  for (const Bucket& b : c->all_buckets) {
    DMatArg D{};
    const std::vector<double>& Dn = node_rule(c, b.N).D;  // Lobatto or Gauss points
    for (size_t i = 0; i < Dn.size(); ++i) D.D[i] = Dn[i];
    CU(launch_detect_regions(c->M, b, g, D, gmm->precision, q, flags, pbar, feat, (cudaStream_t)stream));
  }
  return DG_OK;
}

dg_status dg_set_element_flags(dg_ctx* c, const uint8_t* flags) {
  if (!c || !flags) return fail(DG_ERR_ARG, "NULL argument");
  for (int64_t e = 0; e < c->ne; ++e)
    if (flags[e] > 1) return fail(DG_ERR_ARG, "element %lld: flag %d is not 0 or 1", (long long)e, flags[e]);
  CU(cudaSetDevice(c->device));
  c->flag.assign(flags, flags + c->ne);
  return rebuild_flags(c);
}

dg_status dg_set_params(dg_ctx* c, const dg_params* params) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  dg_status st = check_params(params);
  if (st != DG_OK) return st;
  CU(cudaSetDevice(c->device));
  const dg_params old = c->prm;
  c->prm = *params;
  apply_params(c);
  destroy_graph(c);
  if (params->model != old.model || params->nodes != old.nodes) {
    // the number of state planes changes the trace and viscous buffers; the node set moves
    // the nodes, their metric terms and the face tables
    st = rebuild_orders(c);
    if (st != DG_OK) {
      std::string msg = g_last_error;
      c->prm = old;
      apply_params(c);
      rebuild_orders(c);
      g_last_error = msg;
      return st;
    }
  }
  return DG_OK;
}

dg_status dg_get_layout(const dg_ctx* c, int64_t* total_nodes, const int64_t** elem_offset) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (total_nodes) *total_nodes = c->total;
  if (elem_offset) *elem_offset = c->off.data();
  return DG_OK;
}

dg_status dg_node_coords(dg_ctx* c, double* xyz, void* stream) {
  if (!c || !xyz) return fail(DG_ERR_ARG, "NULL argument");
  CU(cudaSetDevice(c->device));
  double* gn;
  dg_status st = dev_upload(c, "gnodes", c->gnodes, &gn);
  if (st != DG_OK) return st;
  for (const Bucket& b : c->ord_buckets) CU(launch_node_coords(c->M, gn, c->gdeg, b, xyz, (cudaStream_t)stream));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  free_buf(c, "gnodes");
  return DG_OK;
}

dg_status dg_residual(dg_ctx* c, const double* q, double* R, void* stream) {
  if (!c || !q || !R) return fail(DG_ERR_ARG, "NULL argument");
  const size_t bytes = sizeof(double) * nvar(c) * c->total;
  if (overlaps(q, bytes, R, bytes)) return fail(DG_ERR_ARG, "q and R overlap");
  CU(cudaSetDevice(c->device));
  int nl = 0;
  dg_status st = issue_stage(c, q, R, nullptr, MODE_RESIDUAL, 0, 0.0, (cudaStream_t)stream, &nl);
  c->launches_residual = nl;
  return st;
}

dg_status dg_rk_step(dg_ctx* c, double* q, double* g, double t, double dt, int nsteps, void* stream) {
  (void)t;
  if (!c || !q || !g) return fail(DG_ERR_ARG, "NULL argument");
  if (nsteps < 0) return fail(DG_ERR_ARG, "nsteps < 0");
  if (!std::isfinite(dt)) return fail(DG_ERR_ARG, "dt is not finite");
  const size_t bytes = sizeof(double) * nvar(c) * c->total;
  if (overlaps(q, bytes, g, bytes)) return fail(DG_ERR_ARG, "q and g overlap");
  if (nsteps == 0) return DG_OK;
  CU(cudaSetDevice(c->device));
  GraphCache& G = c->graph;
  if (!G.exec || G.q != q || G.g != g || G.dt != dt || G.version != c->version) {
    destroy_graph(c);
    c->M.dt32 = (float)dt;
    CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int nl = 0;
    dg_status st = DG_OK;
    for (int s = 0; s < 3 && st == DG_OK; ++s) st = issue_stage(c, q, q, g, MODE_RK, s, dt, c->cap_stream, &nl);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return fail(DG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      G.exec = nullptr;
      return fail(DG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    G.q = q;
    G.g = g;
    G.dt = dt;
    G.version = c->version;
    c->launches_step = nl;
  }
  if (nsteps == 1) {
    CU(cudaGraphLaunch(G.exec, (cudaStream_t)stream));
    return DG_OK;
  }
  // Several steps: the stage index runs on across steps, so the trace-buffer parity of a step's
  // stage 0 alternates; each stage's update writes the next stage's traces (stage 2 those of
  // the next step's stage 0), and only the first step runs the trace kernel.
  if (!G.chain[0]) {
    for (int k = 0; k < 3; ++k) {
      c->cap_parity = k == 0 ? 0 : k - 1;
      c->cap_write_all = 1;
      c->cap_no_traces = k == 0 ? 0 : 1;
      CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      int nl = 0;
      dg_status st = DG_OK;
      for (int s = 0; s < 3 && st == DG_OK; ++s) st = issue_stage(c, q, q, g, MODE_RK, s, dt, c->cap_stream, &nl);
      c->cap_parity = c->cap_write_all = c->cap_no_traces = 0;
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
      if (st != DG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (ce != cudaSuccess) return fail(DG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&G.chain[k], graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        G.chain[k] = nullptr;
        return fail(DG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
      }
      if (k == 1) G.chain_launches = nl;
    }
  }
  CU(cudaGraphLaunch(G.chain[0], (cudaStream_t)stream));
  for (int i = 1; i < nsteps; ++i) CU(cudaGraphLaunch(G.chain[1 + (i % 2)], (cudaStream_t)stream));
  return DG_OK;
}

static dg_status ensure_staging(dg_ctx* c) {
  dg_status st = DG_OK;
  if (!c->stage_q) st = dev_alloc(c, "stage_q", nvar(c) * c->total, &c->stage_q);
  if (st == DG_OK && !c->stage_r) st = dev_alloc(c, "stage_r", nvar(c) * c->total, &c->stage_r);
  return st;
}

// One host<->device transfer of `bytes`, split into kCopyStreams pieces issued on the copy
// streams (several copy engines can then run at once), ordered after the work already on `s`
// and before the work enqueued on `s` afterwards.
static dg_status split_copy(dg_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
  constexpr int K = dg_ctx::kCopyStreams;
  // page-locked host memory: the SMs read or write it directly, which moves more bytes per
  // second over the CPU-GPU link than the copy engines do
  const void* host = kind == cudaMemcpyHostToDevice ? src : dst;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer &&
      (uintptr_t)at.devicePointer % 16 == 0 && bytes % 8 == 0) {
    // the device's address for the page-locked buffer, as the runtime reports it
    void* dptr = at.devicePointer;
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    CU(launch_copy_sm(kind == cudaMemcpyHostToDevice ? dst : dptr, kind == cudaMemcpyHostToDevice ? dptr : src, bytes,
                      sms, s));
    return DG_OK;
  }
  cudaGetLastError();  // a host pointer the runtime does not know leaves an error to clear
  if (!c->copy_fork) {
    CU(cudaEventCreateWithFlags(&c->copy_fork, cudaEventDisableTiming));
    for (int i = 0; i < K; ++i) {
      CU(cudaStreamCreateWithFlags(&c->copy_stream[i], cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&c->copy_done[i], cudaEventDisableTiming));
    }
  }
  CU(cudaEventRecord(c->copy_fork, s));
  const size_t piece = ((bytes + K - 1) / K + 4095) & ~(size_t)4095;  // whole 4 KiB pages
  for (int i = 0; i < K; ++i) {
    const size_t off = std::min(bytes, (size_t)i * piece), len = std::min(bytes - off, piece);
    if (len == 0) continue;
    CU(cudaStreamWaitEvent(c->copy_stream[i], c->copy_fork, 0));
    CU(cudaMemcpyAsync((char*)dst + off, (const char*)src + off, len, kind, c->copy_stream[i]));
    CU(cudaEventRecord(c->copy_done[i], c->copy_stream[i]));
    CU(cudaStreamWaitEvent(s, c->copy_done[i], 0));
  }
  return DG_OK;
}

dg_status dg_residual_host(dg_ctx* c, const double* q_host, double* R_host, void* stream) {
  if (!c || !q_host || !R_host) return fail(DG_ERR_ARG, "NULL argument");
  CU(cudaSetDevice(c->device));
  dg_status st = ensure_staging(c);
  if (st != DG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * nvar(c) * c->total;
  if ((st = split_copy(c, c->stage_q, q_host, bytes, cudaMemcpyHostToDevice, s)) != DG_OK) return st;
  if ((st = dg_residual(c, c->stage_q, c->stage_r, stream)) != DG_OK) return st;
  if ((st = split_copy(c, R_host, c->stage_r, bytes, cudaMemcpyDeviceToHost, s)) != DG_OK) return st;
  CU(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_rk_step_host(dg_ctx* c, double* q_host, double* g_host, double t, double dt, int nsteps, void* stream) {
  if (!c || !q_host) return fail(DG_ERR_ARG, "NULL argument");
  CU(cudaSetDevice(c->device));
  dg_status st = ensure_staging(c);
  if (st != DG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * nvar(c) * c->total;
  if ((st = split_copy(c, c->stage_q, q_host, bytes, cudaMemcpyHostToDevice, s)) != DG_OK) return st;
  // the first stage of every step overwrites the RK register without reading it (A_0 = 0), so
  // without g_host it simply lives in the library's device buffer
  if (g_host && (st = split_copy(c, c->stage_r, g_host, bytes, cudaMemcpyHostToDevice, s)) != DG_OK) return st;
  if ((st = dg_rk_step(c, c->stage_q, c->stage_r, t, dt, nsteps, stream)) != DG_OK) return st;
  if ((st = split_copy(c, q_host, c->stage_q, bytes, cudaMemcpyDeviceToHost, s)) != DG_OK) return st;
  if (g_host && (st = split_copy(c, g_host, c->stage_r, bytes, cudaMemcpyDeviceToHost, s)) != DG_OK) return st;
  CU(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_check_device(dg_ctx* c, void* stream) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  int h[4] = {0, 0, 0, 0};
  CU(cudaMemcpy(h, c->M.err, sizeof h, cudaMemcpyDeviceToHost));
  if (h[0] != 0) {
    // also the grid barrier's and the tile queues' words: a launch that timed out can leave
    // arrivals or claims counted
    CU(cudaMemset(c->M.err, 0, 16 * sizeof(int)));
    if (h[0] == DG_ERR_TIMEOUT) return fail(DG_ERR_TIMEOUT, "a device-side wait timed out (site %d)", h[1]);
    return fail(DG_ERR_DEVICE, "device error %d at site %d", h[0], h[1]);
  }
  return DG_OK;
}

dg_status dg_set_wait_limit(dg_ctx* c, int64_t polls, int stop_tile) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (polls < 0 || polls > INT32_MAX) return fail(DG_ERR_ARG, "polls must be in [0, 2^31)");
  if (stop_tile < -2) return fail(DG_ERR_ARG, "stop_tile must be -1 (off), -2 or a tile index");
  c->M.wait_polls = polls == 0 ? kWaitPolls : (int)polls;
  c->M.stop_tile = stop_tile;
  destroy_graph(c);  // captured launches hold the previous values
  return DG_OK;
}

dg_status dg_set_launch_overlap(dg_ctx* c, int enable) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (enable != 0 && enable != 1) return fail(DG_ERR_ARG, "enable must be 0 or 1");
  c->M.overlap = enable;
  destroy_graph(c);  // captured launches hold the previous attribute
  return DG_OK;
}

dg_status dg_conservation(dg_ctx* c, const double* R, double* out, void* stream) {
  if (!c || !R || !out) return fail(DG_ERR_ARG, "NULL argument");
  CU(cudaSetDevice(c->device));
  const int nv = nvar(c);
  for (const Bucket& b : c->ord_buckets) CU(launch_conservation(c->M, b, R, nv, c->partial, (cudaStream_t)stream));
  CU(cudaMemcpyAsync(c->partial_host.data(), c->partial, sizeof(double) * nv * c->ne, cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream));
  dg_status st = dg_check_device(c, stream);
  if (st != DG_OK) return st;
  for (int v = 0; v < nv; ++v) {
    double s = 0.0;
    for (int64_t e = 0; e < c->ne; ++e) s += c->partial_host[v * c->ne + e];
    out[v] = s;
  }
  return DG_OK;
}

static_assert(DG_CONSERVATION_NOALLOC_MAX_ELEMS == kNoAllocMaxElems, "scratch limit");

// Allocates nothing: no cudaMalloc/cudaFree, no host copy. The per-element sums are those of
// dg_conservation, written to the static scratch of dg_noalloc.cu.
dg_status dg_conservation_noalloc(dg_ctx* c, const double* R, double* out_dev, void* stream) {
  if (!c || !R || !out_dev) return fail(DG_ERR_ARG, "NULL argument");
  if (c->prm.model != 0) return fail(DG_ERR_UNSUPPORTED, "dg_conservation_noalloc: incompressible form only");
  if (c->ne > kNoAllocMaxElems)
    return fail(DG_ERR_ARG, "dg_conservation_noalloc: the mesh has %lld elements, the static scratch holds %lld",
                (long long)c->ne, (long long)kNoAllocMaxElems);
  CU(cudaSetDevice(c->device));
  double* scratch = nullptr;
  CU(noalloc_scratch(c->device, &scratch));
  CU(launch_conservation_noalloc(c->M, c->ord_buckets.data(), (int)c->ord_buckets.size(), R, scratch, out_dev,
                                 (cudaStream_t)stream));
  return DG_OK;
}

dg_status dg_phase_times(dg_ctx* c, double* q, double* g, double dt, int reps, double out_ms[DG_NPHASES],
                         void* stream) {
  if (!c || !q || !g || !out_ms) return fail(DG_ERR_ARG, "NULL argument");
  if (reps <= 0) return fail(DG_ERR_ARG, "reps must be positive");
  CU(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->M.dt32 = (float)dt;
  destroy_graph(c);  // the captured step holds its own dt
  // plain launches: each phase's events bracket its own kernels only (restored on every return)
  struct KeepOverlap {
    DevMesh& M;
    int v;
    ~KeepOverlap() { M.overlap = v; }
  } keep{c->M, c->M.overlap};
  c->M.overlap = 0;
  cudaEvent_t ev[DG_NPHASES + 1];
  for (auto& e : ev) CU(cudaEventCreate(&e));
  double acc[DG_NPHASES] = {0, 0, 0, 0, 0};
  dg_status st = DG_OK;
  for (int r = 0; r < reps && st == DG_OK; ++r) {
    CU(cudaEventRecord(ev[0], s));
    for (int ph = 0; ph < DG_NPHASES && st == DG_OK; ++ph) {
      st = issue_phase(c, ph, q, q, g, MODE_RK, r % 3, dt, s, nullptr);
      CU(cudaEventRecord(ev[ph + 1], s));
    }
    CU(cudaEventSynchronize(ev[DG_NPHASES]));
    for (int ph = 0; ph < DG_NPHASES; ++ph) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]));
      acc[ph] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != DG_OK) return st;
  for (int ph = 0; ph < DG_NPHASES; ++ph) out_ms[ph] = acc[ph] / reps;
  return DG_OK;
}

// Launch-shape autotuning of the reduced-precision passes (see include/dg.h).
dg_status dg_autotune(dg_ctx* c, const char* cache_path, char* report, int report_len) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (report && report_len > 0) report[0] = 0;
  std::string rep;
  auto give_report = [&]() {
    if (report && report_len > 0) std::snprintf(report, (size_t)report_len, "%s", rep.c_str());
  };
  CU(cudaSetDevice(c->device));
  if (c->M.precision != 1) {
    rep = "precision 0: the FP64 passes have no launch choices\n";
    give_report();
    return DG_OK;
  }
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, c->device));
  std::string dev = prop.name;
  for (char& ch : dev)
    if (ch == '\t' || ch == '\n') ch = ' ';
  // cached choices for this device: "device<TAB>pass<TAB>N<TAB>geo<TAB>tile_alt<TAB>bps<TAB>visc_alt"
  std::map<std::array<int, 3>, std::array<int, 3>> cached;
  if (cache_path && *cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof line, f)) {
        const char* tab = std::strchr(line, '\t');
        if (!tab || std::string(line, (size_t)(tab - line)) != dev) continue;
        int v[6];
        if (std::sscanf(tab + 1, "%d\t%d\t%d\t%d\t%d\t%d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6)
          cached[{v[0], v[1], v[2]}] = {v[3], v[4], v[5]};
      }
      std::fclose(f);
    }
  }
  // a scratch state and output, and every buffer a pass reads, filled once for that state
  double *tq = nullptr, *tr = nullptr;
  dg_status st;
  if ((st = dev_alloc(c, "tune_q", 4 * c->total, &tq)) != DG_OK) return st;
  if ((st = dev_alloc(c, "tune_r", 4 * c->total, &tr)) != DG_OK) return st;
  {
    std::vector<double> hq(4 * c->total);
    for (int64_t i = 0; i < c->total; ++i) {
      hq[i] = 0.01 * std::sin(0.001 * (double)i);
      hq[c->total + i] = 1.0;
      hq[2 * c->total + i] = 0.1 * std::cos(0.002 * (double)i);
      hq[3 * c->total + i] = -0.1;
    }
    CU(cudaMemcpy(tq, hq.data(), sizeof(double) * hq.size(), cudaMemcpyHostToDevice));
  }
  cudaStream_t s = c->cap_stream;
  for (int ph = 0; ph < DG_NPHASES; ++ph)
    if ((st = issue_phase(c, ph, tq, tr, tr, MODE_RESIDUAL, 0, 0.0, s, nullptr)) != DG_OK) return st;
  CU(cudaMemsetAsync(tr, 0, sizeof(double) * 4 * c->total, s));  // the scratch RK register
  DevMesh M = c->M;
  M.Tq = c->trace_buf[0];
  M.Tq_next = c->trace_buf[1];
  M.dt32 = 1e-9f;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  auto timed = [&](auto&& launch, float& ms) -> cudaError_t {
    cudaError_t r = launch();
    if (r != cudaSuccess) return r;
    if ((r = cudaEventRecord(e0, s)) != cudaSuccess) return r;
    for (int k = 0; k < 5 && r == cudaSuccess; ++k) r = launch();
    if (r != cudaSuccess) return r;
    if ((r = cudaEventRecord(e1, s)) != cudaSuccess) return r;
    if ((r = cudaEventSynchronize(e1)) != cudaSuccess) return r;
    if ((r = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return r;
    ms /= 5.f;
    return cudaSuccess;
  };
  cudaError_t ce = cudaSuccess;
  char buf[256];
  for (Bucket& b : c->all_buckets) {
    if (ce != cudaSuccess) break;
    const std::array<int, 3> key = {0, b.N, b.geo};
    auto hit = cached.find(key);
    if (hit != cached.end()) {
      c->tuning[key] = hit->second;
      std::snprintf(buf, sizeof buf, "inviscid N=%d geo=%d: cached, %d elements/tile, %d blocks/SM (0 = max)\n", b.N,
                    b.geo, tile_epb32(b.N, hit->second[0]), hit->second[1]);
      rep += buf;
      continue;
    }
    std::array<int, 3> best = {0, 0, 0};
    float best_ms = 0.f, default_ms = 0.f;
    for (int alt = 0; alt < 2 && ce == cudaSuccess; ++alt) {
      if (alt == 1 && tile_epb32(b.N, 1) == tile_epb32(b.N, 0)) continue;
      for (int bps = 0; bps < 3 && ce == cudaSuccess; ++bps) {
        b.tile_alt = alt;
        b.bps = bps;
        float ms = 0.f;
        // the RK form of the pass (stage 1: reads g, writes q, g and the next traces) on the
        // scratch state, with g in the scratch output buffer
        ce = timed([&]() { return launch_inviscid(M, b, tq, tq, tr, MODE_RK, 1, 1e-9, 1, 1, s); }, ms);
        if (alt == 0 && bps == 0) default_ms = best_ms = ms;
        if (ms < best_ms) {
          best_ms = ms;
          best = {alt, bps, 0};
        }
      }
    }
    c->tuning[key] = best;
    std::snprintf(buf, sizeof buf,
                  "inviscid N=%d geo=%d: %d elements/tile, %d blocks/SM (0 = max): %.4f ms, default %.4f ms\n", b.N,
                  b.geo, tile_epb32(b.N, best[0]), best[1], best_ms, default_ms);
    rep += buf;
  }
  for (Bucket& b : c->ns_buckets) {
    if (b.geo == 2 || ce != cudaSuccess) continue;  // curved: a single kernel
    const std::array<int, 3> key = {1, b.N, b.geo};
    auto hit = cached.find(key);
    if (hit != cached.end()) {
      c->tuning[key] = hit->second;
      std::snprintf(buf, sizeof buf, "viscous N=%d geo=%d: cached, %s kernel, %d elements/tile, %d blocks/SM (0 = max)\n",
                    b.N, b.geo, hit->second[2] ? "cp.async" : "pipelined", tile_epb32(b.N, hit->second[0]),
                    hit->second[1]);
      rep += buf;
      continue;
    }
    // (tile_alt, bps, visc_alt): the pipelined kernel with the default or the alternative tile
    // shape (fewer elements per tile: a shorter last round), or the cp.async-staged kernel
    const int cand[6][3] = {{0, 0, 0}, {0, 1, 0}, {0, 2, 0}, {0, 0, 1}, {1, 0, 0}, {1, 2, 0}};
    const bool has_alt = tile_epb32(b.N, 1) != tile_epb32(b.N, 0);
    std::array<int, 3> best = {0, 0, 0};
    float best_ms = 0.f, default_ms = 0.f;
    for (int k = 0; k < 6 && ce == cudaSuccess; ++k) {
      if (cand[k][0] && !has_alt) continue;
      b.tile_alt = cand[k][0];
      b.bps = cand[k][1];
      b.visc_alt = cand[k][2];
      float ms = 0.f;
      ce = timed([&]() { return launch_viscous(M, b, tq, 1, s); }, ms);
      if (k == 0) default_ms = best_ms = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best = {cand[k][0], cand[k][1], cand[k][2]};
      }
    }
    b.tile_alt = 0;
    c->tuning[key] = best;
    std::snprintf(buf, sizeof buf,
                  "viscous N=%d geo=%d: %s kernel, %d elements/tile, %d blocks/SM (0 = max): %.4f ms, default %.4f ms\n",
                  b.N, b.geo, best[2] ? "cp.async" : "pipelined", tile_epb32(b.N, best[0]), best[1], best_ms,
                  default_ms);
    rep += buf;
  }
  // one persistent kernel per stage against the separate viscous and inviscid launches, on the
  // shapes just chosen (the RK form of stage 1 on the scratch state)
  apply_tuning(c);
  if (ce == cudaSuccess && stage_fusable(c)) {
    const Bucket& bi = c->all_buckets[0];
    const std::array<int, 3> key = {2, bi.N, bi.geo};
    auto hit = cached.find(key);
    if (hit != cached.end()) {
      c->tuning[key] = hit->second;
      std::snprintf(buf, sizeof buf, "stage N=%d geo=%d: cached, %s (split %d)\n", bi.N, bi.geo,
                    hit->second[0] == 2 ? "one launch with tile queues"
                                        : (hit->second[0] ? "one persistent kernel" : "separate launches"),
                    hit->second[1]);
      rep += buf;
    } else {
      float ms_sep = 0.f, ms_fused = 0.f;
      DevMesh Mi = M;  // as in a step: the inviscid launch overlaps the viscous pass before it
      Mi.after_visc = M.overlap;
      ce = timed(
          [&]() {
            cudaError_t r = cudaSuccess;
            for (const Bucket& b : c->ns_buckets)
              if (r == cudaSuccess) r = launch_viscous(M, b, tq, 1, s);
            if (r == cudaSuccess) r = launch_inviscid(c->ns_buckets.empty() ? M : Mi, bi, tq, tq, tr, MODE_RK, 1, 1e-9, 1, 1, s);
            return r;
          },
          ms_sep);
      float ms_queue = 0.f;
      if (ce == cudaSuccess && !M.div64) ce = timed([&]() { return launch_stage(c, M, tq, tq, tr, 1, 1, 1, s); }, ms_fused);
      // the queue kernel with each split of the blocks between the viscous and the inviscid
      // queue at the start (all blocks start with the viscous one, or k = 1..3 times its share
      // of the two queues' tiles)
      int vsplit = 0;
      Bucket& bq = c->all_buckets[0];
      for (int v = 0; v < 4 && ce == cudaSuccess; ++v) {
        if (v > 0 && (c->ns_buckets.empty() || c->ns_buckets[0].count == 0)) break;
        bq.vsplit = v;
        float ms = 0.f;
        ce = timed([&]() { return launch_stage(c, M, tq, tq, tr, 1, 1, 2, s); }, ms);
        if (v == 0 || ms < ms_queue) ms_queue = ms, vsplit = v;
      }
      bq.vsplit = 0;
      // a tie keeps the separate launches (per-pass timing and rooflines stay per kernel): a
      // one-launch form must be at least 1% faster
      int fused = 0;
      float best = ms_sep;
      if (ce == cudaSuccess && !M.div64 && ms_fused < 0.99f * best) fused = 1, best = ms_fused;
      if (ce == cudaSuccess && ms_queue < (fused ? best : 0.99f * best)) fused = 2, best = ms_queue;
      c->tuning[key] = {fused, fused == 2 ? vsplit : 0, 0};
      static const char* split_name[4] = {"all", "1x their share", "2x their share", "3x their share"};
      std::snprintf(buf, sizeof buf,
                    "stage N=%d geo=%d: %s: %.4f ms (one persistent kernel %.4f ms, one launch with tile queues %.4f "
                    "ms, separate %.4f ms; queue kernel: blocks starting with the viscous tiles: %s)\n",
                    bi.N, bi.geo,
                    fused == 2 ? "one launch with tile queues" : (fused ? "one persistent kernel" : "separate launches"),
                    best, ms_fused, ms_queue, ms_sep, split_name[vsplit]);
      rep += buf;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_buf(c, "tune_q");
  free_buf(c, "tune_r");
  apply_tuning(c);
  destroy_graph(c);
  c->version++;
  if (ce != cudaSuccess) return fail(DG_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(ce));
  if (cache_path && *cache_path) {
    // keep other devices' lines, replace this device's
    std::vector<std::string> keep;
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof line, f)) {
        const char* tab = std::strchr(line, '\t');
        if (tab && std::string(line, (size_t)(tab - line)) != dev) keep.emplace_back(line);
      }
      std::fclose(f);
    }
    FILE* f = std::fopen(cache_path, "w");
    if (!f) return fail(DG_ERR_ARG, "cannot write the tuning cache %s", cache_path);
    for (const std::string& l : keep) std::fputs(l.c_str(), f);
    for (const auto& kv : c->tuning)
      std::fprintf(f, "%s\t%d\t%d\t%d\t%d\t%d\t%d\n", dev.c_str(), kv.first[0], kv.first[1], kv.first[2], kv.second[0],
                   kv.second[1], kv.second[2]);
    std::fclose(f);
  }
  give_report();
  return DG_OK;
}

dg_status dg_phase_bytes(const dg_ctx* c, double out[DG_NPHASES]) {
  if (!c || !out) return fail(DG_ERR_ARG, "NULL argument");
  // Mean over the three stages of one RK step. State q is FP64 (8 B); traces are 8 B per
  // value (FP64, or an FP32 hi/lo pair); with precision 1 the RK register g, the viscous
  // traces and the viscous divergence are FP32 (4 B).
  const bool f32 = c->M.precision == 1;
  const double d = 8.0, sg = f32 ? 4.0 : 8.0, sv = f32 ? 4.0 : 8.0, tr = 8.0;
  // state planes, viscous planes (momentum, + energy), planes the viscous pass reads (the
  // velocity; the whole conservative state in the compressible form)
  const double nv = nvar(c), nvv = nv - 1.0, nu_in = c->prm.model == 1 ? 5.0 : 3.0;
  double b[DG_NPHASES] = {0, 0, 0, 0, 0};
  for (int64_t e = 0; e < c->ne; ++e) {
    const double n = c->order[e] + 1, n2 = n * n, n3 = n2 * n;
    const bool ns = c->flag[e] != 0;
    const bool curved = c->ec[e].curved != 0.0;
    const double geo = curved ? 10.0 * n3 * (f32 ? 4.0 : 8.0) : (f32 ? 48.0 : 112.0);
    // traces: launched in one stage out of three (q at the face nodes in, or the whole
    // element on Gauss-Legendre nodes, traces out)
    b[0] += ((c->prm.nodes == 1 ? nv * n3 * d : nv * 6.0 * n2 * d) + nv * 6.0 * n2 * tr) / 3.0;
    // inviscid + update: q in and out, g out (and in for two stages of three), geometry,
    // traces of the new state written in two stages of three
    double inv = nv * n3 * d * 2.0 + nv * n3 * sg * (1.0 + 2.0 / 3.0) + geo + (2.0 / 3.0) * nv * 6.0 * n2 * tr;
    if (ns) {
      b[2] += nu_in * n3 * d + geo + nvv * n3 * sv + 6.0 * nvv * n2 * sv;  // state in, rv and Tv out
      inv += nvv * n3 * sv;                                                // rv in
    }
    for (int f = 0; f < 6; ++f) {
      const int32_t nb = c->nb[e * 6 + f];
      if (nb < 0) continue;
      const double nn = c->order[nb] + 1;
      const bool nbns = c->flag[nb] != 0;
      if (c->order[nb] == c->order[e]) {
        if (ns) b[2] += nu_in * n2 * tr;                // neighbour trace for the lifting
        inv += nv * n2 * tr;                            // neighbour q trace
        if (ns) inv += nvv * n2 * sv;                   // own viscous trace
        if (nbns) inv += nvv * n2 * sv;                 // neighbour viscous trace
      } else {
        if (ns) {
          b[1] += 3.0 * (n2 + nn * nn) * tr + 9.0 * n2 * d;  // both velocity traces in, lifting out
          b[2] += 9.0 * n2 * d;                              // lifting in
        }
        b[3] += 4.0 * (n2 + nn * nn) * tr + (ns ? 3.0 * n2 * sv : 0.0) + (nbns ? 3.0 * nn * nn * sv : 0.0) +
                4.0 * n2 * d;
        inv += 4.0 * n2 * d + (ns ? 3.0 * n2 * sv : 0.0);   // projected flux, own viscous trace
      }
    }
    b[4] += inv;
  }
  if (stage_fused(c)) {  // one persistent kernel runs the viscous pass inside phase 4
    b[4] += b[2];
    b[2] = 0.0;
  }
  for (int ph = 0; ph < DG_NPHASES; ++ph) out[ph] = b[ph];
  return DG_OK;
}

int dg_launches_per_residual(const dg_ctx* c) { return c ? c->launches_residual : 0; }
int dg_launches_per_step(const dg_ctx* c) { return c ? c->launches_step : 0; }
int dg_launches_per_chained_step(const dg_ctx* c) { return c ? c->graph.chain_launches : 0; }

void dg_destroy(dg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  destroy_graph(c);
  for (auto& kv : c->buf) cudaFree(kv.second.p);
  c->buf.clear();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (int i = 0; i < dg_ctx::kCopyStreams; ++i) {
    if (c->copy_stream[i]) cudaStreamDestroy(c->copy_stream[i]);
    if (c->copy_done[i]) cudaEventDestroy(c->copy_done[i]);
  }
  if (c->copy_fork) cudaEventDestroy(c->copy_fork);
  delete c;
}

}  // extern "C"
