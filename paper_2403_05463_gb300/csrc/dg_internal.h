// dg_internal.h -- data shared between the host library (dg_host.cpp) and the kernels.
// Not part of the public C ABI (include/dg.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dgk {

constexpr int MAXN = 7;        // largest polynomial order with a kernel instantiation
constexpr int NP = MAXN + 1;   // table stride
constexpr int kErrTimeout = 7;  // DG_ERR_TIMEOUT in the device error word
constexpr int kWaitPolls = 1 << 22;  // default poll budget of a bounded mbarrier wait

// Kind of coupling behind one local face of an element.
enum FaceKind : uint8_t {
  FK_CONF = 0,     // same order on both sides: the flux is evaluated node by node, in place
  FK_MORTAR = 1,   // different orders: flux on the mortar of the larger order, projected back
  FK_INFLOW = 2,   // ghost state: prescribed velocity, interior pressure
  FK_OUTFLOW = 3,  // ghost state: interior velocity, zero pressure
  FK_WALL = 4,     // no-slip wall: mirror ghost with every velocity component reversed
  FK_SLIP = 5,     // free-slip wall: mirror ghost with the normal velocity reversed
};

// One entry per (element, local face). Local face f = 2 d + s lies on xi_{d+1} = s ? +1 : -1;
// its face coordinates (a, b) run along the two other directions in increasing order.
struct FaceLink {
  int32_t nbr;     // neighbour element, -1 on a boundary
  uint8_t nface;   // neighbour's local face
  uint8_t orient;  // swap | flip_a << 1 | flip_b << 2: neighbour (a1, b1) -> mine
  uint8_t kind;    // FaceKind
  uint8_t nflag;   // neighbour flag (0 Euler, 1 NS)
  int64_t nslot;   // first trace slot of the neighbour's face: tr_off[nbr] + nface n_nbr^2
};
static_assert(sizeof(FaceLink) == 16, "FaceLink layout is shared by host and device");

// Per-element constants. Affine elements carry their constant metric here; curved elements
// read per-node metric terms from DevMesh::geo.
struct ElemConst {
  double Ja[9];    // Ja[d*3+k] = J d xi_d / d x_k (affine only)
  double J, invJ;  // affine only
  double delta;    // LES filter width: cube root of the element volume / (N + 1)
  double curved;   // 1.0: metric terms per node in DevMesh::geo; 0.0: affine (Ja above)
  // (the geometry kind used for bucketing -- box, affine, curved -- is kept on the host)
};

// FP32 copy of the per-element constants for the reduced-precision passes.
struct ElemConst32 {
  float Ja[9];
  float invJ;
  float delta;
  float curved;
};

// Everything a kernel needs, passed by value.
struct DevMesh {
  int64_t n_elem, total, tr_total;
  const int64_t* elem_off;   // [E+1] node offsets
  const int64_t* tr_off;     // [E+1] face-trace offsets: element e's 6 faces x n^2 nodes
  const int8_t* order;       // [E]
  const uint8_t* flag;       // [E]
  const FaceLink* link;      // [E*6]
  const ElemConst* ec;       // [E]
  const double* geo;         // curved elements: [10][total] = Ja[9] (d*3+k) then J
  const ElemConst32* ec32;   // [E] FP32 constants
  const float* geo32;        // curved elements: [10][total] = Ja[9] then 1/J (FP32)
  double* Tq;                // face traces of q: FP64 [4][tr_total], or with precision 1 FP32
                             // (hi, lo) pairs, hi + lo = q to 2^-48 relative, interleaved per
                             // slot [tr_total][4] (one 32-byte record per face node)
  double* Tq_next;           // traces of the updated q written by the RK update for the next
                             // stage (double-buffered with Tq: neighbours still read Tq)
  double* Tv;                // outward viscous flux traces tau . S (NS elements): FP64
                             // [3][tr_total], or with precision 1 FP32 [tr_total][3]
  double* rv;                // [3][total]    J * viscous volume divergence (NS elements)
  double* LU;                // [9][tr_total] projected BR1 lifting u*_c S_k on mortar faces
                             // (compressible: [12][tr_total], phi*_c S_k with phi = (v, T))
  double* LH;                // [nvar][tr_total] projected total flux (F_e* - F_v*) . S on mortars
  const double* interp;      // [(Ns*NP+Nd)*NP*NP + i*NP + j]: Lagrange interpolation Ns -> Nd
  const double* proj;        // [(Nh*NP+Nl)*NP*NP + i*NP + j]: L2 projection Nh -> Nl
  int* err;                  // device error word [0..3]; [4], [5] the grid barrier of the
                             // persistent stage kernel (arrivals, generation); [8..11] the tile
                             // queues of the one-launch stage kernel (16 ints)
  int wait_polls;            // polls of a bounded mbarrier wait before it gives up (timeout)
  int stop_tile;             // test hook, -1 off: the producer warp of block 0 of each pipelined
                             // launch returns before staging its stop_tile-th tile; -2: block 0
                             // of the persistent stage kernel skips its grid-barrier arrival
  int overlap;               // 1: the pipelined FP32 passes are overlapped launches (programmatic
                             // stream serialisation; they wait in the kernel for the launch before)
  int after_visc;            // set per launch: this inviscid launch directly follows the viscous
                             // pass of its stage, so its bucket's independent entries need not wait
  double nu, c0sq, cs, cv;
  int closure, riemann;
  int mixed_face;            // 0 average, 1 one-sided viscous flux on NS/Euler faces
  int split;                 // 0 standard convective volume term, 1 kinetic-energy-preserving split form
  int precision;             // 0: Tv/rv hold FP64; 1: they hold FP32 (same buffers)
  int div64;                 // reduced-precision inviscid pass, box elements: the velocity
                             // divergence (pressure row, U_c du_d fluxes) in FP64
  int tc;                    // the FP32 inviscid volume contraction on tensor cores: 1 in 3xTF32,
                             // 2 in plain TF32 (one product of the rounded operands); 0 FP32 FMAs
  float nu32, c0sq32, cs32, cv32, dt32;  // FP32 copies for the reduced-precision passes
  double inflow[4];
  // governing equations: 0 incompressible (artificial compressibility, q = (p, u, v, w)),
  // 1 compressible (App. A, u = (rho, rho v, rho e); FP64, conforming periodic meshes)
  int model;
  double gamma, prandtl, prandtl_t;  // compressible: ideal gas with unit gas constant
  double p_inf;                      // compressible: far-field pressure (inflow, outflow ghosts)
  // element nodes: 0 Gauss-Lobatto, 1 Gauss-Legendre (face values interpolated; FP64,
  // incompressible)
  int nodes;
  const double* interp_gl;   // [(g*NP+N)*NP*NP + i*NP + j]: Gauss-Lobatto degree g -> Gauss-Legendre order N
  const double* interp_g;    // the layout of interp and proj, between Gauss-Legendre point sets
  const double* proj_g;      // (mortars on Gauss-Legendre nodes)
  const double* lb_g;        // [(N*2+s)*NP + i]: Gauss-Legendre l_i(-1) (s = 0), l_i(+1) (s = 1)
};

// 1D Gauss-Lobatto operators for N = 1..MAXN (uploaded to constant memory).
struct Ops1D {
  double D[NP][NP * NP];  // D[N][i*n+m]
  double w[NP][NP];       // w[N][i]
  double x[NP][NP];       // x[N][i]
  // Gauss-Legendre element nodes (nodes = 1)
  double Dg[NP][NP * NP];    // D[N][i*n+m] on the Gauss points
  double wg[NP][NP];         // Gauss weights
  double lbg[NP][2][NP];     // l_i(-1), l_i(+1)
};

// Per-entry record of a bucket (32 bytes, copied whole into shared memory by the
// pipelined inviscid pass).
struct EntryMeta {
  int64_t off;    // node offset of the element
  int64_t troff;  // first face-trace slot of the element
  int32_t elem;   // element id
  int32_t flag;   // 0 Euler, 1 NS
  int32_t has_mortar;  // 1: one of its faces is a mortar face
  int32_t pad;
};
static_assert(sizeof(EntryMeta) == 32, "EntryMeta is copied in 16-byte blocks");

// Element lists of one kernel launch.
struct Bucket {
  int N;
  int geo;            // 0 axis-aligned box, 1 affine, 2 curved
  bool curved;        // geo == 2
  bool ns;            // true: only NS elements (viscous pass)
  int32_t* list;      // device: element ids
  int count;
  // per-entry tables in bucket order (device), for the pipelined inviscid pass
  const int64_t* boff = nullptr;    // node offset of the entry's element
  const int64_t* btr = nullptr;     // first face-trace slot of the entry's element
  const FaceLink* blink = nullptr;  // the element's 6 face links
  const uint8_t* bflag = nullptr;   // the element's flag
  const EntryMeta* bmeta = nullptr; // the entry's record
  // launch choices of the reduced-precision passes (set by the autotuner; 0 = default)
  int tile_alt = 0;   // inviscid: 1 = the alternative elements-per-tile shape
  int bps = 0;        // pipelined passes: resident blocks per SM (0 = as many as fit)
  int visc_alt = 0;   // viscous, box/affine: 1 = the cp.async-staged kernel instead of the pipelined one
  // all-element buckets: the first n_indep entries are Euler elements with no NS neighbour and
  // no mortar face (their inviscid pass touches nothing the viscous or mortar passes write)
  int n_indep = 0;
  // one-launch stage kernel with tile queues: 0, every block starts with the viscous queue; k =
  // 1..3, the share k * (viscous tiles) / (viscous + independent inviscid tiles) of the grid
  // does (lowest indices first, at most all) and the others start with the independent tiles
  int vsplit = 0;
};

enum StageMode { MODE_RESIDUAL = 0, MODE_RK = 1 };

// Allocation-free conservation sums (dg_noalloc.cu): largest mesh its static scratch holds.
constexpr int64_t kNoAllocMaxElems = 65536;

// Launchers (dg_kernels.cu). All return cudaGetLastError() of their launches.
cudaError_t upload_ops(const Ops1D& ops);
cudaError_t launch_traces(const DevMesh& M, const Bucket& b, const double* q, int precision, cudaStream_t s);
cudaError_t launch_project_state(const DevMesh& M, const int8_t* old_order, const int64_t* old_off, int64_t total_old,
                                 const double* qo, double* qn, cudaStream_t s);
// mortar kernels of the incompressible form: slots sorted by mortar order, mo_start[MO] ..
// mo_start[MO + 1] (host array of MAXN + 2) those of order MO; *nlaunch counts the launches.
// Lifting: one slot per mortar side of an NS element. Flux: one slot per mortar face, the side
// of the larger order (the kernel writes both sides).
cudaError_t launch_mortar_lift(const DevMesh& M, const int32_t* slots, const int* mo_start, int* nlaunch,
                               cudaStream_t s);
cudaError_t launch_mortar_flux(const DevMesh& M, const int32_t* slots, const int* mo_start, int* nlaunch,
                               cudaStream_t s);
cudaError_t launch_viscous(const DevMesh& M, const Bucket& b, const double* q, int precision,
                           cudaStream_t s);
cudaError_t launch_inviscid(const DevMesh& M, const Bucket& b, const double* q, double* out,
                            double* g, int mode, int stage, double dt, int write_tr, int precision,
                            cudaStream_t s);
cudaError_t launch_node_coords(const DevMesh& M, const double* geom_nodes, int geom_degree,
                               const Bucket& b, double* xyz, cudaStream_t s);
cudaError_t launch_conservation(const DevMesh& M, const Bucket& b, const double* R, int nvar,
                                double* partial, cudaStream_t s);
cudaError_t prepare_kernels();
// Copy between page-locked host memory and device memory with the SMs (16-byte aligned
// pointers, a whole number of doubles); cudaErrorInvalidValue otherwise.
cudaError_t launch_copy_sm(void* dst, const void* src, size_t bytes, int sms, cudaStream_t s);
// FP32-arithmetic variants (dg_kernels_f32.cu)
cudaError_t upload_ops32(const Ops1D& ops);
cudaError_t prepare_kernels32();
cudaError_t launch_viscous32(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s);
cudaError_t launch_traces32(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s);
cudaError_t launch_inviscid32(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                              int mode, int stage, int write_tr, cudaStream_t s);

// One persistent launch per RK stage of a single (order, box/affine) bucket: the viscous pass over
// bv's NS elements, then the inviscid pass and update over bi (the default tile shape, FP32
// contractions). queue 0: static tile order with a bounded grid barrier between the passes
// (cooperative launch; err[4], err[5]); queue 1: tiles from queues, the inviscid tiles that read
// viscous results waiting on a counter of finished viscous tiles (overlapped launch; err[8..11]).
cudaError_t launch_stage32(const DevMesh& M, const Bucket& bv, const Bucket& bi, const double* q, double* out,
                           double* g, int stage, int write_tr, int queue, cudaStream_t s);

// elements per tile of the FP32 inviscid pass at order N: the default shape or the alternative
int tile_epb32(int N, int alt);

// Compressible form (dg_cns.cu), FP64: traces [5][tr_total] in Tq, viscous traces Fv . S
// [4][tr_total] in Tv (momentum, energy), J r_v [4][total] in rv.
cudaError_t upload_ops_cns(const Ops1D& ops);
cudaError_t prepare_kernels_cns();
cudaError_t launch_mortar_lift_cns(const DevMesh& M, const int32_t* slots, int count, cudaStream_t s);
cudaError_t launch_mortar_flux_cns(const DevMesh& M, const int32_t* slots, int count, cudaStream_t s);
cudaError_t launch_traces_cns(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s);
cudaError_t launch_viscous_cns(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s);
cudaError_t launch_inviscid_cns(const DevMesh& M, const Bucket& b, const double* u, double* out, double* g,
                                int mode, int stage, double dt, int write_tr, cudaStream_t s);

// Compressible form on Gauss-Legendre element nodes (dg_cns_gl.cu), FP64: the buffers of the
// compressible form, with the face values and viscous traces interpolated to the face points.
cudaError_t upload_ops_cns_gl(const Ops1D& ops);
cudaError_t prepare_kernels_cns_gl();
cudaError_t launch_traces_cns_gl(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s);
cudaError_t launch_viscous_cns_gl(const DevMesh& M, const Bucket& b, const double* u, cudaStream_t s);
cudaError_t launch_inviscid_cns_gl(const DevMesh& M, const Bucket& b, const double* u, double* out, double* g,
                                   int mode, int stage, double dt, int write_tr, cudaStream_t s);

// Gauss-Legendre element nodes (dg_gl.cu), FP64, incompressible form: traces are the face values
// interpolated along the normal lines; face terms are lifted with l_i(+-1) / w_i.
cudaError_t upload_ops_gl(const Ops1D& ops);
cudaError_t prepare_kernels_gl();
cudaError_t launch_traces_gl(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s);
cudaError_t launch_viscous_gl(const DevMesh& M, const Bucket& b, const double* q, cudaStream_t s);
cudaError_t launch_inviscid_gl(const DevMesh& M, const Bucket& b, const double* q, double* out, double* g,
                               int mode, int stage, double dt, int write_tr, cudaStream_t s);

// Region detection (dg_regions.cu): the mixture as the kernel uses it.
struct GmmDev {
  double P[2][6];   // inverse covariance of component k, upper triangle: 00 01 02 11 12 22
  double mu[2][3];  // means
  double c[2];      // log w_k - log det(C_k) / 2 (the common -3/2 log 2 pi cancels)
  int viscous;      // index of the viscous component
  // FP32 copies for the FP32 pass
  float P32[2][6], mu32[2][3], c32[2];
};
struct DMatArg {
  double D[NP * NP];  // D of one order, row-major [i * n + m], n = N + 1
};
cudaError_t launch_detect_regions(const DevMesh& M, const Bucket& b, const GmmDev& g, const DMatArg& D, int fp32,
                                  const double* q, uint8_t* flags, double* pbar, double* feat, cudaStream_t s);

// Allocation-free conservation sums (dg_noalloc.cu)
cudaError_t noalloc_scratch(int device, double** ptr);
cudaError_t launch_conservation_noalloc(const DevMesh& M, const Bucket* buckets, int n_buckets, const double* R,
                                        double* scratch, double* out, cudaStream_t s);

}  // namespace dgk
