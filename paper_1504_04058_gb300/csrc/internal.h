// internal.h -- host-side state of a libasp handle and the launch interfaces
// between the translation units.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "asp.h"

namespace asp {

// Subproblem kinds (Section 3.1): H_q^M, H_p^R, H_p^L.
enum SubKind : int { KIND_M = 0, KIND_R = 1, KIND_L = 2 };

// One layer subproblem on its padded grid [lo, lo+w-1] along x2 (global
// 1-based), full x1 range.  Ordered x2-fastest ("quasi-1D", Section 3.1) it is
// block tridiagonal with n blocks (one per x1 node) of size w x w.
struct SubDesc {
  int kind;          // KIND_M / KIND_R / KIND_L
  int p;             // layer index, 1-based
  int lo;            // global x2 index of local column 0
  int w;             // padded width (columns along x2)
  int wp;            // leading dimension of a stored w x w block (>= w)
  int xoff;          // X_p = local columns [xoff, xoff + xw)
  int xw;
  int prof;          // offset of this subproblem's sweep-axis coefficients
  int bs;            // elements per stored block: w*wp, or with packed factors
                     // (ASP_PREC_C64_SYM) the upper triangle of the symmetric
                     // W_k Delta (packed_block_elems)
  long long woff;    // element offset of block 0 of its factor
  long long toff;    // element offset of its trace-transfer map (-1: none)
};

// With ASP_PREC_C64_SYM, 2D factors are stored as the upper triangle of W'_k = W_k Delta,
// Delta = diag(s2_j) the subproblem's sweep-axis PML weights: D^-1 H is
// complex symmetric for D = diag(s1_k s2_j) (Section 3.1, practical remark 4),
// and by induction over the block recursion so is every S_k^-1 D_k, i.e. W'_k.
// Entry (i, j), i <= j, sits at j (j + 1) / 2 + i; the block is padded to an
// even count (16-byte aligned blocks).  W_k = W'_k Delta^-1.
__host__ __device__ inline int packed_block_elems(int w) { return ((w * (w + 1) / 2) + 1) & ~1; }
__host__ __device__ inline int packed_index(int i, int j) {
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  return hi * (hi + 1) / 2 + lo;
}

// Solve modes of the batched block-tridiagonal solver (btsolve.cuh).
enum SolveMode : int {
  MODE_EMBED = 0,   // G~_q^M: right-hand side = input restricted to X_q
  MODE_FILL_R = 1,  // G~_p^R: right-hand side = -(1/h^2) accR[p-1] on local column 0
  MODE_FILL_L = 2,  // G~_p^L: right-hand side = -(1/h^2) accL[p+1] on local column w-1
  MODE_TMAP_R = 3,  // transfer map of G~_p^R: unit boundary data, keep last column of X_p
  MODE_TMAP_L = 4,  // transfer map of G~_p^L: unit boundary data, keep first column of X_p
  MODE_SUB = 5,     // plain H^-1 g on the whole padded grid (checking entry point)
};

struct Job {
  int sub;   // index into the SubDesc table
  int mode;  // SolveMode
  int rhs0;  // first right-hand side of this job
  int nr;    // number of right-hand sides in this job
};

// Coefficients of the sweep-axis (x2) second difference of one subproblem,
// local column j: up[j] couples j -> j+1, dn[j] couples j -> j-1, dg[j] is the
// x2 part of the diagonal (Eq. (4) with the subproblem's s-profile).
struct SweepCoef {
  double2 up, dn, dg;
};

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using T = float2; };
template <> struct CplxOf<double> { using T = double2; };

// Coefficients of the layer operators in the factor precision R: the x1
// stencil weights a_k, c_k, d_k per x1 node, omega^2/c^2 (natural order) and
// the sweep-axis weights of every subproblem column (concatenated, SubDesc::prof).
template <typename R> struct FactorCoefs {
  using C = typename CplxOf<R>::T;
  const C* s1 = nullptr;     // s at the x1 nodes (boundary PML), and its reciprocal
  const C* s1inv = nullptr;
  const C* s2 = nullptr;     // s of every subproblem column (SubDesc::prof), and its reciprocal
  const C* s2inv = nullptr;
  const C* ca = nullptr;
  const C* cc = nullptr;
  const C* cd = nullptr;
  const R* k2 = nullptr;
  const C* up = nullptr;
  const C* dn = nullptr;
  const C* dg = nullptr;
};

struct SolveParams {
  const SubDesc* subs;
  const Job* jobs;
  int njobs;
  int n;            // blocks per subproblem (= x1 nodes)
  int ldv;          // right-hand-side stride of the vectors (= nrhs of the call)
  int ldacc;        // right-hand-side stride of the trace buffers (nrhs rounded up to even)
  int ldT;          // row stride of the transfer maps (n rounded up to even)
  double inv_h2;
  const void* W;    // factor blocks W_k = S_k^-1
  const void* ca;   // a_k: coupling of block k to block k-1 (x1 stencil), factor precision
  const void* cc;   // c_k: coupling of block k to block k+1, factor precision
  const void* s2inv;  // 1 / s2 of every subproblem column (complex64: packed factors), factor precision
  const void* in;   // EMBED / SUB input (factor precision, RHS-interleaved)
  void* outM;       // EMBED output restricted to X_q (factor precision)
  void* outR;       // FILL_R output
  void* outL;       // FILL_L output
  void* accR;       // [m+1][n][ldacc] right traces / accumulated right-going traces
  void* accL;       // [m+1][n][ldacc] left traces
  void* tmap;       // transfer maps base
  void* outSub;     // MODE_SUB output (complex128, [w][n][ldv])
  void* zscr;       // forward-pass scratch, one slot per resident CTA
  long long zslot;  // elements per slot
  int zslots;       // number of slots (upper bound on the grid)
  int* err;
};

// One trace-transfer map built on the tensor cores (tmap_tc.cu): complex64
// factors, padded subproblem width <= kTmapTcMaxW.
constexpr int kTmapTcMaxW = 32;
struct TmMap {
  long long woff;  // element offset of its subproblem's factor blocks
  long long toff;  // element offset of the map
  long long goff;  // element offset of its diagonal-block columns ([n][2][32])
  int w, wp;       // padded width and block leading dimension of the subproblem
  int bs, prof;    // elements per stored (packed) block; its sweep coefficients' offset
  int jin, keep;   // boundary-data column and traced column (local)
  float2 rho;      // s2(keep) / s2(in) of the subproblem's sweep profile
};

struct ChainParams {
  int n, m, ldacc, ldT, nrhs;
  const void* tmap;        // maps
  const long long* toffR;  // [m+1] element offset of T_p^R (p = 2..m-1)
  const long long* toffL;  // [m+1] element offset of T_p^L
  void* accR;              // [m+1][n][ldacc]
  void* accL;
  unsigned int* bar;       // two grid-barrier counters (R, L), zeroed before launch
  int* err;
};

// ---- 3D (Section 4): slab subproblems
// A slab is a subproblem on the padded sweep range [lo, lo+w-1] along x3 with
// the full x1 and x2 ranges.  With x2 as the block index and the local index
// j = i3l*n + i1 inside a block (x1 fastest), it is block tridiagonal: n dense
// diagonal blocks T_k of size nb = n*w (the x1/x3 stencil of plane x2 = k),
// coupled to the neighbouring planes by the x2 weights times the identity.
struct Slab {
  int kind, p;
  int lo, w;          // padded sweep range (global 1-based x3)
  int xoff, xw;       // X_p = local planes [xoff, xoff + xw)
  int prof;           // offset of its sweep-axis coefficients (SweepCoef table)
  int nb;             // block size n*w
  int ld;             // row stride of a stored block (nb rounded up to 4)
  int np;             // Gauss-Jordan steps: columns [0, np), pivots from rows [0, np) (nb: a full inversion)
  int src_plane;      // FILL modes: 0-based global x3 plane of the incoming trace
  int src_sweep;      // FILL modes: 1 if the trace includes the sweep field there
  long long woff;     // element offset of block 0 of its factor (n blocks of nb x ld)
  long long aoff;     // element offset of its factor-time work area (slab_work_elems)
  long long zbo;      // offset of the work area's pivot-row buffers from aoff (2*nb*ld for a slab)
  long long poff;     // int offset of its pivot tables (3 * nb)
  long long zoff;     // element offset of its solve scratch (n * nb * max_rhs)
};

// Blocked Gauss-Jordan of the 3D factor: inner panels of kSlabPanel columns
// inside outer blocks of kSlabOuter columns.  Per slab the factor-time work
// area holds two nb x ld matrices, the outer block's pivot rows (kSlabOuter x
// ld) and the inner panel's pivot rows inside the outer block (kSlabPanel x
// kSlabOuter).
constexpr int kSlabPanel = 32;
constexpr int kSlabOuter = 256;

// Most map rows one CTA of the 2D sweep chain holds.  The chain runs one CTA
// per SM, half of the SMs per sweep direction, so 2D problems take
// n <= kChainMaxRows * (SMs / 2): 1216 on 152 SMs.
constexpr int kChainMaxRows = 16;
inline long long slab_work_elems(int nb, int ld) {
  return 2LL * nb * ld + (long long)kSlabOuter * ld + (long long)kSlabPanel * kSlabOuter;
}

struct Slab3Params {
  const Slab* slabs;
  const int* list;    // slab indices of this launch
  int nlist;
  int n;
  void* W;            // factors
  void* A;            // work matrices
  int* piv;           // pivot tables: piv_row[nb], col_of_row[nb], row_step[nb]
  int* err;
};

// ---- 3D slab subproblems by nested dissection (nd3d.cu; Section 4: the
// unknowns of a slab are grouped along x3 into columns, and the n x n grid of
// columns is ordered by nested dissection).  The separator tree depends on n
// only; a slab of width w has w unknowns per column.  Node fields, kNdNodeInts
// ints per node: I columns, B columns, offset of its columns (I then B, each
// ascending by id i2*n + i1), offset of its child map (the parent front column
// position of each of its B columns; -1 for the root), first and second child
// (-1: none), depth.
constexpr int kNdNodeInts = 8;
enum NdNodeField : int { ND_NCI = 0, ND_NCB, ND_OFFC, ND_OFFM, ND_C0, ND_C1, ND_DEPTH };
constexpr int kNdLeafCols = 8;   // a region of at most this many columns is a leaf

struct NdTree {
  int n = 0, nn = 0, maxdepth = 0;
  std::vector<int> node;   // nn * kNdNodeInts
  std::vector<int> cols;
  std::vector<int> cmap;
  std::vector<std::vector<int>> at_depth;
  int nc(int t) const { return node[t * kNdNodeInts + ND_NCI] + node[t * kNdNodeInts + ND_NCB]; }
};

// One node of one slab: front f = slab_rank * nn + node, with slab_rank the
// slab's position in the handle's slab list.
struct NdFront {
  int slab, node, w, lds, ldb, pad;
  long long xl;   // factor offset of [X; L] (ns x lds): X = F_II^-1, L = F_BI X
  long long pf;   // factor offset of P = X F_IB (s x ldb)
  long long zu;   // solve scratch: z (s rows) then u (B rows), max_rhs columns
};

struct NdSizes {
  long long factor_elems = 0, work_elems = 0, piv_ints = 0, zu_elems = 0, nfronts = 0;
  long long tc_floats = 0;  // complex64: tensor-core operand areas of the large-front levels
  int max_front = 0;
};
// Levels whose largest front has at least this many unknowns run their
// rank-256 updates on the tensor cores (complex64).
constexpr int kNdTcMinFront = 512;
// Builds the separator tree of an n x n grid of columns; returns false (with
// *why) if a child column is missing from its parent's front.
bool nd_build_tree(int n, NdTree& T, std::string* why);
// Factor, work, pivot and scratch sizes of the nested-dissection path for the
// given slab widths and kinds (in slab order) and factor element size;
// chunk[i] receives the factor chunk of slab i within its group (the slabs of
// one chunk are factored together).
NdSizes nd_sizes(const NdTree& T, const std::vector<int>& widths, const std::vector<int>& kinds, int max_rhs,
                 int esz, std::vector<int>* chunk);

// Operand area and tensor maps of the tensor-core update (tcupdate.cu) for
// one slab group.
struct TcGroup {
  float* ahi = nullptr;
  float* alo = nullptr;
  float* bhi = nullptr;
  float* blo = nullptr;
  void* maps = nullptr;        // host copy of the four CUtensorMaps
  long long* rowA = nullptr;   // device: first operand row of each slab of the group list
};

struct Solve3Job {
  int slab, mode, rhs0, nr;
  int item0;          // first work item of this job (prefix over the launch)
};

struct Solve3Params {
  const Slab* slabs;
  const Solve3Job* jobs;
  int njobs;
  int nitems;         // total work items (row chunks) per block step
  int n, ldv;
  double inv_h2;
  const void* W;
  const void* ca;     // x2 weights a_k (block k -> k-1), factor precision
  const void* cc;     // x2 weights c_k (block k -> k+1)
  const void* in;
  void* outM;
  void* outR;
  void* outL;
  void* outSub;       // MODE_SUB output (complex128, [w][n][n][ldv])
  void* z;            // per-slab scratch base
  unsigned int* bar;
  int* err;
};

struct Handle;

enum Phase : int {
  PH_FACTOR = 0, PH_TMAP = 1, PH_EMBED = 2, PH_CHAIN = 3, PH_FILL = 4, PH_SUM = 5, PH_MATVEC = 6,
  PH_KRYLOV = 7, PH_SCHUR = 8, PH_TDIAG = 9, PH_COUNT = 10
};

// Records CUDA events around launches when phase timing is enabled.
struct PhaseTok {
  int phase = -1;
  cudaEvent_t a = nullptr;
};
PhaseTok phase_begin(Handle& H, int phase, cudaStream_t s);
void phase_end(Handle& H, PhaseTok t, cudaStream_t s);

// ---- launchers (one translation unit each) ----
cudaError_t launch_matvec(const Handle& H, const double2* x, double2* y, int nrhs, cudaStream_t s);
cudaError_t launch_factor(Handle& H, int first, int count, cudaStream_t s);
cudaError_t launch_btsolve_apply(Handle& H, const SolveParams& P, int cls, int cap, int variant, int wmax,
                                 cudaStream_t s);
cudaError_t launch_btsolve_aux(Handle& H, const SolveParams& P, int cls, int cap, int wmax, cudaStream_t s);
int btsolve_rhs_capacity(int nrhs, int wmax, int prec, bool tmap);
cudaError_t launch_chain(Handle& H, const ChainParams& P, cudaStream_t s);
cudaError_t launch_tmap_diag(Handle& H, cudaStream_t s);
cudaError_t launch_tmap_tc(Handle& H, cudaStream_t s);
cudaError_t launch_to_prec(const double2* in, void* out, long long count, int prec, cudaStream_t s);
// z = a + b (planes >= r_from) + c (planes < l_below), planes of per_col elements
cudaError_t launch_sum3(const void* a, const void* b, const void* c, double2* z, long long per_col, int ncols,
                        int r_from, int l_below, int prec, cudaStream_t s);
cudaError_t launch_matvec3d(const Handle& H, const double2* x, double2* y, int nrhs, cudaStream_t s);
int factor3d(Handle& H, cudaStream_t s);
// the Gauss-Jordan steps on columns [0, np) of every matrix of P.list (factor3d.cu)
cudaError_t gj_partial(Handle& H, const Slab3Params& P, int nbmax, int npmax, const TcGroup* tc, cudaStream_t s);
int nd_setup(Handle& H);
int nd_factor(Handle& H, cudaStream_t s);
void nd_release(Handle& H);
// the slab solves of one batch (P.jobs) by the nested-dissection factors
cudaError_t nd_solve(Handle& H, const Solve3Params& P, int NR, int nbmax, cudaStream_t s);
int apply3d(Handle& H, const double2* r, double2* z, int nrhs, cudaStream_t s);
int subsolve3d(Handle& H, int slab, const double2* g, double2* v, int nrhs, cudaStream_t s);
void release_jobs3(const Handle* H);
long long tc_group_floats(long long rows);
int tc_group_setup(TcGroup& G, float* area, const std::vector<long long>& rowA_host, long long rows);
void tc_group_release(TcGroup& G);
cudaError_t launch_tc_update(const TcGroup& G, const Slab3Params& P, int nbmax, int C0, int buf, cudaStream_t s);

// ---- handle ----
struct Handle {
  asp_params prm{};
  int dim = 2;
  int n = 0, m = 0, prec = 0, gamma = 0, gamma_a = 0, b = 0;
  bool packed = false;  // complex64 blocks stored as packed symmetric triangles (ASP_PREC_C64_SYM)
  double h = 0, inv_h2 = 0;
  long long N = 0;  // n^dim grid points

  // partition (host), 1-based arrays sized m+1
  std::vector<int> x_lo, x_hi, alpha, beta;

  // device: velocity term omega^2/c^2 (natural order), global x1/x2 stencil
  // coefficients per node (the same profile on both axes)
  double* k2 = nullptr;
  double* dgre = nullptr;  // 2D: Re of the operator's diagonal, d_{i1}.x + d_{i2}.x + k2 (natural order)
  double2* ca = nullptr;  // a_k = s_k s_{k-1/2} / h^2
  double2* cc = nullptr;  // c_k = s_k s_{k+1/2} / h^2
  double2* cd = nullptr;  // d_k = -s_k (s_{k+1/2} + s_{k-1/2}) / h^2
  // nodes [real_lo, real_hi) of an axis where a_k, c_k, d_k are real (outside the PML)
  int real_lo = 0, real_hi = 0;

  // the same coefficients in the factor precision (owned device buffers)
  FactorCoefs<float> fc32;
  FactorCoefs<double> fc64;
  std::vector<void*> coef_bufs;

  // subproblems
  std::vector<SubDesc> subs;
  SubDesc* d_subs = nullptr;
  std::vector<SweepCoef> coef;  // concatenated sweep-axis coefficients
  SweepCoef* d_coef = nullptr;
  std::vector<int> subM, subR, subL;  // subproblem index per layer (-1 if none), size m+1
  int wmax = 0, wmaxRL = 0;

  // factors and transfer maps
  void* W = nullptr;
  size_t W_elems = 0;
  void* tmap = nullptr;
  size_t tmap_elems = 0;
  int ldT = 0;  // row stride of a transfer map (n rounded up to even)
  std::vector<long long> toffR, toffL;
  long long* d_toffR = nullptr;
  long long* d_toffL = nullptr;
  // maps built on the tensor cores (empty: the maps come from CLS_TMAP solves)
  std::vector<TmMap> tm_host;
  TmMap* d_tm = nullptr;
  void* gdiag = nullptr;  // diagonal-block columns of every such map
  bool factored = false;

  // apply workspace (factor precision), sized for max_rhs
  void* r_lo = nullptr;   // converted input (c64 path only)
  void* uM = nullptr;
  void* uR = nullptr;
  void* uL = nullptr;
  void* accR = nullptr;
  void* accL = nullptr;
  void* zscr = nullptr;
  long long zslot = 0;
  int zslots = 0;
  unsigned int* bar = nullptr;
  Job* d_jobs = nullptr;
  int jobs_cap = 0;

  // Krylov workspace (complex128)
  double2* V = nullptr;   // (restart+1) vectors
  double2* Z = nullptr;   // restart vectors
  double2* wv = nullptr;  // work vector
  double* red = nullptr;  // reduction partials
  double2* hess = nullptr;
  double* kstate = nullptr;
  int* kflags = nullptr;
  int* h_flags = nullptr;  // pinned
  double* h_state = nullptr;

  int* err = nullptr;  // device error word [2]
  long long launches = 0;
  int num_sms = 0;

  // phase timing
  bool timing = false;
  struct Rec { int phase; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> evpool;
  std::mutex rec_mu;

  // 3D slabs (subM/subR/subL index into slabs when dim == 3)
  std::vector<Slab> slabs;
  Slab* d_slabs = nullptr;
  int* d_slab_lists = nullptr;  // [M slabs | R and L slabs]
  int nbmaxM = 0, nbmaxRL = 0;
  void* A3 = nullptr;           // factor-time work matrices
  int* piv3 = nullptr;
  void* z3 = nullptr;           // solve scratch
  float* tc_area = nullptr;     // tensor-core update operands (complex64 factors)
  // factor groups: contiguous ranges of the slab list, each factored on its own
  // stream so that one group's latency-bound panels overlap another's updates
  struct FGroup {
    int first = 0, count = 0, nbmax = 0;
    TcGroup tc;
    cudaStream_t stream = nullptr;  // owned (nullptr: the caller's stream)
    cudaEvent_t done = nullptr;
  };
  std::vector<FGroup> fgroups;

  // nested dissection (slab_solver == ASP_SLAB_ND)
  bool nd = false;
  NdTree ndt;
  int* d_ndtab = nullptr;       // node table, columns, child maps
  NdFront* d_ndf = nullptr;     // every front [slab * nn + node]
  Slab* d_ndslab = nullptr;     // engine view of every front (nb = front size, np = s)
  int* d_ndlist = nullptr;      // front lists per (chunk, depth)
  struct NdLevel { int off = 0, count = 0, nbmax = 0, npmax = 0, bmax = 0, depth = 0, group = 0, tc = -1; };
  std::vector<NdLevel> nd_levels;   // in factor order: per group, per chunk, deepest depth first
  std::vector<NdFront> ndf_host;
  void* nd_zu = nullptr;        // solve scratch of every front
  // complex64: tensor-core update operands of the levels with large fronts
  // (NdLevel::tc indexes nd_tcg; one operand area per factor group)
  std::vector<TcGroup> nd_tcg;
  float* nd_tc_area[2] = {nullptr, nullptr};
  int nd_maxfront = 0;
  // per depth: offset of its node list in d_ndtab, and the largest column
  // counts (I + B, I, B) of its nodes
  std::vector<int> nd_dep_off, nd_dep_nc, nd_dep_nci, nd_dep_ncb;

  // second stream for work that overlaps the caller's stream (factor time)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

void set_detail(const std::string& s);
// Device allocation of the setup paths: cudaMalloc, unless the test hook
// (asp_testhook_fail_device_alloc) has armed a failure for this allocation.
cudaError_t dev_malloc(void** p, size_t bytes);
// Raises a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it).
cudaError_t ensure_dyn_smem(const void* func, size_t bytes);
int fail(int code, const std::string& detail);

}  // namespace asp

struct asp_handle {
  asp::Handle h;
};
