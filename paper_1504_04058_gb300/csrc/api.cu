// api.cu -- the C ABI of libasp (include/asp.h): setup, factor, apply,
// matvec, FGMRES, and the small element-wise kernels of the apply.
//
// Setup builds, on the host in FP64, everything the kernels read:
//  * the layer partition of Section 3.1 (X_p, X_q^M, X_p^R, X_p^L) with
//    m = floor(P/b) layers over the P = n+2-2*gamma physical columns, the last
//    layer taking the remainder;
//  * the PML functions sigma(x) = (C/eta)(d/eta)^2, s = (1 + i sigma/omega)^-1
//    (Section 2), for the boundary PML on both axes and for the auxiliary
//    profiles sigma_q^M, sigma_p^R, sigma_p^L of every subproblem;
//  * the stencil weights s_i s_{i+-1/2}/h^2 of Eq. (2)/(4) at every node.
// All device memory of a handle is allocated here (asp_footprint_bytes gives
// the total in advance) and released by asp_destroy.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "btsolve.cuh"
#include "common.cuh"
#include "internal.h"

namespace asp {

int gmres_run(Handle& H, const double2* f, double2* u, int nrhs, double tol, int restart, int maxit,
              asp_solve_info* info, cudaStream_t s);
size_t krylov_state_bytes(int restart, int nrhs, size_t* n2, size_t* nd, size_t* ni);

static thread_local std::string g_detail;

static cudaEvent_t pool_event(Handle& H) {
  std::lock_guard<std::mutex> lock(H.rec_mu);
  if (!H.evpool.empty()) {
    cudaEvent_t e = H.evpool.back();
    H.evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

PhaseTok phase_begin(Handle& H, int phase, cudaStream_t s) {
  PhaseTok t;
  if (!H.timing) return t;
  t.phase = phase;
  t.a = pool_event(H);
  if (t.a) cudaEventRecord(t.a, s);
  return t;
}

void phase_end(Handle& H, PhaseTok t, cudaStream_t s) {
  if (!H.timing || t.phase < 0 || !t.a) return;
  cudaEvent_t b = pool_event(H);
  std::lock_guard<std::mutex> lock(H.rec_mu);
  if (b) {
    cudaEventRecord(b, s);
    H.recs.push_back({t.phase, t.a, b});
  } else {
    H.evpool.push_back(t.a);
  }
}

// The dynamic shared-memory limit is a property of the kernel, shared by every
// host thread; concurrent handles of different sizes must never lower it under
// each other's launches, so it only ever grows.
cudaError_t ensure_dyn_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set_to;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(dev, func);
  auto it = set_to.find(key);
  if (it != set_to.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set_to[key] = bytes;
  return e;
}

void set_detail(const std::string& s) { g_detail = s; }

// allocations left before the injected failure (-1: the hook is disarmed)
std::atomic<int> g_alloc_fail_after{-1};

cudaError_t dev_malloc(void** p, size_t bytes) {
  int left = g_alloc_fail_after.load();
  while (left >= 0) {
    if (g_alloc_fail_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {  // this allocation fails; the hook is now disarmed (-1)
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}
int fail(int code, const std::string& detail) {
  g_detail = detail;
  return code;
}

namespace {

// ---------------------------------------------------------------- PML
// sigma = 0 on [lo_edge, hi_edge]; (C/eta)(d/eta)^2 at distance d outside, on the
// sides that carry a layer.
struct Profile {
  bool lo_on = false, hi_on = false;
  double lo_edge = 0, hi_edge = 0, eta_lo = 1, eta_hi = 1, C = 0;
  double sigma(double x) const {
    if (lo_on && x < lo_edge) {
      const double d = lo_edge - x;
      return (C / eta_lo) * (d / eta_lo) * (d / eta_lo);
    }
    if (hi_on && x > hi_edge) {
      const double d = x - hi_edge;
      return (C / eta_hi) * (d / eta_hi) * (d / eta_hi);
    }
    return 0.0;
  }
  // s = 1 / (1 + i sigma/omega)
  double2 s(double x, double omega) const {
    const double t = sigma(x) / omega;
    const double den = 1.0 + t * t;
    return make_double2(1.0 / den, -t / den);
  }
};

double2 hmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
double2 hscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
double2 hadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

struct Sizes {
  int m = 0, wmax = 0, wmaxRL = 0, nsub = 0;
  size_t W_elems = 0, tmap_elems = 0, coef = 0;
  size_t A_elems = 0, piv_elems = 0, z3_elems = 0, tc_floats = 0;  // 3D
  int nbmaxM = 0, nbmaxRL = 0;                       // 3D
  size_t esz = 0;
  long long N = 0;
  size_t zslot = 0;
  int zslots = 0;
  size_t bytes = 0;
};

// Physical layer widths b_1..b_m (Section 3.1, practical remark 3: arbitrary
// widths).  With widths == nullptr: floor(P/b) layers of b columns, the last
// one absorbing the remainder, P = n + 2 - 2*gamma.  Empty on invalid input.
std::vector<int> layer_widths(const asp_params* p, const int* widths, int m, std::string* why) {
  std::vector<int> w;
  const int P = p->n + 2 - 2 * p->pml;
  if (!widths) {
    const int mm = p->b >= 1 ? P / p->b : 0;
    if (mm < 1) { *why = "n too small for the PML width and layer width (need n >= 2*gamma + b - 2)"; return w; }
    w.assign(mm, p->b);
    w[mm - 1] += P - mm * p->b;
    return w;
  }
  if (m < 1 || m > P) { *why = "number of layers out of range [1, n + 2 - 2*gamma]"; return w; }
  long long sum = 0;
  for (int i = 0; i < m; ++i) {
    if (widths[i] < 1) { *why = "every layer width must be >= 1"; return w; }
    sum += widths[i];
  }
  if (sum != P) { *why = "layer widths must sum to n + 2 - 2*gamma = " + std::to_string(P); return w; }
  w.assign(widths, widths + m);
  return w;
}

bool valid(const asp_params* p, std::string* why, const std::vector<int>* widths = nullptr) {
  if (!p) { *why = "null params"; return false; }
  if (p->dim != 2 && p->dim != 3) { *why = "dim must be 2 or 3"; return false; }
  if (p->dim == 2 && (p->n < 3 || p->n > 16383)) { *why = "n out of range [3, 16383]"; return false; }
  if (p->dim == 3 && (p->n < 3 || p->n > 1023)) { *why = "n out of range [3, 1023] in 3D"; return false; }
  if (!(p->omega > 0) || !isfinite(p->omega)) { *why = "omega must be positive and finite"; return false; }
  if (p->pml < 2) { *why = "pml (gamma) must be >= 2"; return false; }
  if (p->pml_aux < 0) { *why = "pml_aux must be >= 0"; return false; }
  if (p->b < 1) { *why = "b must be >= 1"; return false; }
  if (!(p->C > 0) || !isfinite(p->C)) { *why = "C must be positive and finite"; return false; }
  if (p->factor_prec != ASP_PREC_C128 && p->factor_prec != ASP_PREC_C64 && p->factor_prec != ASP_PREC_C64_SYM) {
    *why = "bad factor_prec";
    return false;
  }
  if (p->max_rhs < 1 || p->max_rhs > 256) { *why = "max_rhs out of range [1, 256]"; return false; }
  if (p->restart < 1 || p->restart > 64) { *why = "restart out of range [1, 64]"; return false; }
  if (p->slab_solver != ASP_SLAB_BLOCK && p->slab_solver != ASP_SLAB_ND) { *why = "bad slab_solver"; return false; }
  if (p->slab_solver == ASP_SLAB_ND && p->dim != 3) { *why = "slab_solver ASP_SLAB_ND is 3D only"; return false; }
  const int P = p->n + 2 - 2 * p->pml;
  if (!widths && P < p->b) { *why = "n too small for the PML width and layer width (need n >= 2*gamma + b - 2)"; return false; }
  const int ga = p->pml_aux ? p->pml_aux : p->pml;
  // the auxiliary padding of X_2^M and X_{m-1}^M must stay inside [1, n]
  const int bmin = widths ? std::min(widths->front(), widths->back()) : p->b;
  if (ga > p->pml + bmin) { *why = "pml_aux too wide for the layer width"; return false; }
  return true;
}

// ASP_PREC_C64_SYM is complex64 arithmetic with packed symmetric factor
// storage: the rest of the library sees ASP_PREC_C64 and the `packed` flag.
asp_params normalized(const asp_params* p, bool* packed) {
  asp_params q = *p;
  *packed = q.factor_prec == ASP_PREC_C64_SYM;
  if (*packed) q.factor_prec = ASP_PREC_C64;
  return q;
}

struct Part {
  int m;
  std::vector<int> x_lo, x_hi, alpha, beta, m_lo, m_hi;
};

// Layers of the given physical widths: alpha_p = gamma + b_1 + ... + b_{p-1},
// beta_p = alpha_p + b_p - 1 (beta_m = n + 1 - gamma when the widths sum to P).
Part partition(int n, int gamma, int ga, const std::vector<int>& widths) {
  Part P;
  P.m = (int)widths.size();
  const int m = P.m;
  P.x_lo.assign(m + 1, 0); P.x_hi = P.x_lo; P.alpha = P.x_lo; P.beta = P.x_lo; P.m_lo = P.x_lo; P.m_hi = P.x_lo;
  int a = gamma;
  for (int p = 1; p <= m; ++p) {
    P.alpha[p] = a;
    P.beta[p] = (p < m) ? a + widths[p - 1] - 1 : n + 1 - gamma;
    a = P.beta[p] + 1;
    P.x_lo[p] = (p == 1) ? 1 : P.alpha[p];
    P.x_hi[p] = (p == m) ? n : P.beta[p];
    P.m_lo[p] = (p == 1) ? 1 : P.alpha[p] - ga + 1;
    P.m_hi[p] = (p == m) ? n : P.beta[p] + ga - 1;
  }
  return P;
}

// Largest 3D block size (n * padded width) the slab kernels take.
constexpr int kMaxNb3 = 3072;

// SM count assumed by size and support queries made without a device (GB300).
constexpr int kDefaultSms = 152;

// Valid problems that this build does not handle on a GPU with `sms` SMs: 2D
// padded layers wider than 64 columns, 2D grids with more than
// kChainMaxRows * (sms / 2) points per side (sweep chain with three or more
// layers), 3D blocks larger than kMaxNb3.
bool supported(const asp_params* p, const Part& P, std::string* why, int sms) {
  int wmax = 0;
  for (int q = 1; q <= P.m; ++q) wmax = std::max(wmax, P.m_hi[q] - P.m_lo[q] + 1);
  if (p->dim == 2 && wmax > 64) {
    *why = "padded layer width 2*gamma_a + b - 2 (+ remainder) exceeds 64 columns";
    return false;
  }
  const int max_n2 = kChainMaxRows * (sms / 2);
  if (p->dim == 2 && P.m >= 3 && p->n > max_n2) {
    *why = "2D n exceeds " + std::to_string(max_n2) + " on " + std::to_string(sms) +
           " SMs (the sweep chain holds at most " + std::to_string(kChainMaxRows) +
           " map rows per CTA on half of the SMs)";
    return false;
  }
  if (p->dim == 3 && p->slab_solver == ASP_SLAB_BLOCK && (long long)p->n * wmax > kMaxNb3) {
    *why = "3D block size n * (padded slab width) exceeds " + std::to_string(kMaxNb3);
    return false;
  }
  if (p->dim == 3 && p->slab_solver == ASP_SLAB_ND) {
    // the nested-dissection solve stages a front's vector (4 right-hand sides) in shared memory
    NdTree T;
    std::string w2;
    if (!nd_build_tree(p->n, T, &w2)) { *why = w2; return false; }
    int ncmax = 0;
    for (int t = 0; t < T.nn; ++t) ncmax = std::max(ncmax, T.nc(t));
    const long long esz = p->factor_prec == ASP_PREC_C128 ? 16 : 8;
    if ((long long)ncmax * wmax * 4 * esz > 200 * 1024) {
      *why = "nested-dissection front of " + std::to_string((long long)ncmax * wmax) +
             " unknowns exceeds the solve's shared-memory stage";
      return false;
    }
  }
  return true;
}

int fmax_rhs_cap(int prec) { return prec == ASP_PREC_C64 ? 64 : 16; }

// complex64 maps of padded width <= kTmapTcMaxW are built on the tensor cores
// (tmap_tc.cu) and need no forward-pass scratch of their own.
bool tc_maps(int dim, int prec, int m, int wmaxRL) {
  return dim == 2 && prec == ASP_PREC_C64 && m >= 3 && wmaxRL <= kTmapTcMaxW;
}

// Right-hand sides per scratch slot: the widest solve instance that uses the slot.
int zslot_cols(int dim, int prec, int m, int wmaxRL) {
  if (prec == ASP_PREC_C64) return tc_maps(dim, prec, m, wmaxRL) ? 32 : 64;
  return 16;
}

Sizes sizes_for3(const asp_params* p, const Part& P, int num_sms) {
  Sizes Z;
  const int n = p->n;
  Z.m = P.m;
  Z.esz = p->factor_prec == ASP_PREC_C128 ? 16 : 8;
  Z.N = (long long)n * n * n;
  const long long mr = p->max_rhs;
  auto addslab = [&](int lo, int hi, bool rl) {
    const int w = hi - lo + 1;
    const int nb = n * w, ld = (nb + 3) & ~3;
    Z.W_elems += (size_t)n * nb * ld;
    Z.A_elems += (size_t)slab_work_elems(nb, ld);
    Z.piv_elems += (size_t)3 * nb;
    Z.z3_elems += (size_t)n * nb * mr;
    Z.coef += w;
    Z.wmax = std::max(Z.wmax, w);
    if (rl) Z.nbmaxRL = std::max(Z.nbmaxRL, nb);
    else Z.nbmaxM = std::max(Z.nbmaxM, nb);
    Z.nsub++;
  };
  long long tc_rows_M = 0, tc_rows_RL = 0;
  auto padr = [&](int lo, int hi) { return (long long)((n * (hi - lo + 1) + 127) / 128 * 128); };
  std::vector<int> sw, sk;  // slab widths and kinds in slab order
  for (int q = 1; q <= P.m; ++q) {
    addslab(P.m_lo[q], P.m_hi[q], false); tc_rows_M += padr(P.m_lo[q], P.m_hi[q]);
    sw.push_back(P.m_hi[q] - P.m_lo[q] + 1); sk.push_back(KIND_M);
  }
  for (int q = 2; q <= P.m; ++q) {
    addslab(P.alpha[q], P.m_hi[q], true); tc_rows_RL += padr(P.alpha[q], P.m_hi[q]);
    sw.push_back(P.m_hi[q] - P.alpha[q] + 1); sk.push_back(KIND_R);
  }
  for (int q = 1; q <= P.m - 1; ++q) {
    addslab(P.m_lo[q], P.beta[q], true); tc_rows_RL += padr(P.m_lo[q], P.beta[q]);
    sw.push_back(P.beta[q] - P.m_lo[q] + 1); sk.push_back(KIND_L);
  }
  size_t nd_extra = 0;
  if (p->slab_solver == ASP_SLAB_ND) {
    // nested dissection: its factors, work, pivots and tensor-core operand
    // areas replace the block path's
    NdTree T;
    std::string why;
    nd_build_tree(n, T, &why);
    const NdSizes ND = nd_sizes(T, sw, sk, (int)mr, (int)Z.esz, nullptr);
    Z.W_elems = (size_t)ND.factor_elems;
    Z.A_elems = (size_t)ND.work_elems;
    Z.piv_elems = (size_t)ND.piv_ints;
    nd_extra = (size_t)ND.zu_elems * Z.esz + (size_t)ND.tc_floats * sizeof(float) +
               (size_t)ND.nfronts * (sizeof(NdFront) + sizeof(Slab) + sizeof(int)) +
               (T.node.size() + T.cols.size() + T.cmap.size() + T.nn) * sizeof(int);
  } else if (p->factor_prec == ASP_PREC_C64) {
    Z.tc_floats = tc_group_floats(tc_rows_M) + tc_group_floats(tc_rows_RL);
  }
  const long long R = p->restart;
  size_t n2, nd, ni;
  const size_t kst = krylov_state_bytes(p->restart, p->max_rhs, &n2, &nd, &ni);
  const size_t rsz = Z.esz / 2;  // real type of the factor precision
  size_t bytes = 0;
  bytes += Z.N * (sizeof(double) + rsz) + 3 * (size_t)n * (sizeof(double2) + Z.esz);  // k2, ca, cc, cd (both)
  bytes += Z.coef * (sizeof(SweepCoef) + 5 * Z.esz) + Z.nsub * sizeof(Slab) + Z.nsub * sizeof(int);
  bytes += (size_t)n * 2 * Z.esz;  // s1, 1/s1
  bytes += (Z.W_elems + Z.A_elems + Z.z3_elems) * Z.esz + Z.piv_elems * sizeof(int);
  bytes += Z.tc_floats * sizeof(float);
  bytes += nd_extra;
  bytes += (size_t)Z.N * mr * Z.esz * (3 + (Z.esz == 8 ? 1 : 0));                 // uM uR uL (+ r_lo)
  bytes += (size_t)(2 * R + 2) * Z.N * mr * sizeof(double2);                        // V, Z, work
  bytes += (size_t)num_sms * 4 * 9 * mr * sizeof(double2);                          // dot partials
  bytes += kst + 64;
  Z.bytes = bytes;
  return Z;
}

// p->factor_prec is ASP_PREC_C128 or ASP_PREC_C64 here (see normalized());
// packed: complex64 blocks stored as packed symmetric triangles.
Sizes sizes_for(const asp_params* p, const Part& P, int num_sms, bool packed) {
  if (p->dim == 3) return sizes_for3(p, P, num_sms);
  Sizes Z;
  const int n = p->n;
  Z.m = P.m;
  Z.esz = p->factor_prec == ASP_PREC_C128 ? 16 : 8;
  Z.N = (long long)n * n;
  auto addsub = [&](int lo, int hi, bool rl) {
    const int w = hi - lo + 1;
    const int wp = (p->factor_prec == ASP_PREC_C64) ? ((w + 1) & ~1) : w;
    Z.W_elems += (size_t)n * (packed ? packed_block_elems(w) : w * wp);
    Z.coef += w;
    Z.wmax = std::max(Z.wmax, w);
    if (rl) Z.wmaxRL = std::max(Z.wmaxRL, w);
    Z.nsub++;
  };
  for (int q = 1; q <= P.m; ++q) addsub(P.m_lo[q], P.m_hi[q], false);
  for (int q = 2; q <= P.m; ++q) addsub(P.alpha[q], P.m_hi[q], true);
  for (int q = 1; q <= P.m - 1; ++q) addsub(P.m_lo[q], P.beta[q], true);
  const int ldT = (n + 1) & ~1;
  Z.tmap_elems = P.m >= 3 ? (size_t)2 * (P.m - 2) * n * ldT : 0;
  Z.zslots = std::max(1, 4 * num_sms);
  Z.zslot = (size_t)n * Z.wmax * zslot_cols(2, p->factor_prec, P.m, Z.wmaxRL);
  const bool tcm = tc_maps(2, p->factor_prec, P.m, Z.wmaxRL);
  const long long R = p->restart;
  const long long mr = p->max_rhs;
  size_t n2, nd, ni;
  const size_t kst = krylov_state_bytes(p->restart, p->max_rhs, &n2, &nd, &ni);
  size_t bytes = 0;
  bytes += 2 * Z.N * sizeof(double) + 3 * (size_t)n * sizeof(double2);          // k2, dgre, ca, cc, cd
  bytes += Z.coef * sizeof(SweepCoef) + Z.nsub * sizeof(SubDesc);
  bytes += Z.W_elems * Z.esz + Z.tmap_elems * Z.esz;
  if (tcm) bytes += (size_t)2 * (P.m - 2) * (n * 2 * 32 * sizeof(float2) + sizeof(TmMap));  // Gamma columns, map table
  bytes += (size_t)n * 2 * sizeof(float2) + Z.coef * 2 * Z.esz;                    // s1, 1/s1, s2, 1/s2
  bytes += (size_t)Z.N * mr * Z.esz * (3 + (Z.esz == 8 ? 1 : 0));              // uM uR uL (+ r_lo)
  bytes += (size_t)2 * (P.m + 1) * n * ((mr + 1) & ~1) * Z.esz;                   // accR, accL
  bytes += (size_t)Z.zslots * Z.zslot * Z.esz;                                   // forward scratch
  bytes += (size_t)(2 * R + 2) * Z.N * mr * sizeof(double2);                     // V, Z, work
  bytes += (size_t)num_sms * 4 * 9 * mr * sizeof(double2);                       // dot partials
  bytes += kst + 64;
  Z.bytes = bytes;
  return Z;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// ---------------------------------------------------------------- small kernels
template <typename R>
__global__ void to_prec_kernel(const double2* __restrict__ in, Cx<R>* __restrict__ out, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = cvt<R>(in[e]);
}

// z = uM + uR (except on X_1, where there is no right-going part) + uL (except
// on X_m).  Grid: blockIdx.y = sweep-axis index (x2 column in 2D, x3 plane in
// 3D), blockIdx.x = chunk of its per_col elements.  The sum is taken in the
// factor precision R and widened once: in complex64 the three parts carry the
// layer solves' own relative error (far above FP32 rounding), and widening
// each part to FP64 first would put six conversions and four additions per
// element on GB300's narrow FP64 pipe.
template <typename R>
__global__ void sum3_kernel(const Cx<R>* __restrict__ a, const Cx<R>* __restrict__ b, const Cx<R>* __restrict__ c,
                            double2* __restrict__ z, long long per_col, int r_from, int l_below) {
  const long long er = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (er >= per_col) return;
  const int col = blockIdx.y;  // 0-based x2 index
  const long long e = (long long)col * per_col + er;
  Cx<R> v = a[e];
  if (col >= r_from) { const Cx<R> vb = b[e]; v.x += vb.x; v.y += vb.y; }
  if (col < l_below) { const Cx<R> vc = c[e]; v.x += vc.x; v.y += vc.y; }
  z[e] = make_double2((double)v.x, (double)v.y);
}

int vec_grid(long long count, int sms) {
  long long g = (count + 255) / 256;
  g = std::min<long long>(g, (long long)std::max(sms, 1) * 8);
  return (int)std::max<long long>(g, 1);
}

}  // namespace

cudaError_t launch_to_prec(const double2* in, void* out, long long count, int prec, cudaStream_t s) {
  if (prec == ASP_PREC_C64)
    to_prec_kernel<float><<<vec_grid(count, 152), 256, 0, s>>>(in, (float2*)out, count);
  else
    to_prec_kernel<double><<<vec_grid(count, 152), 256, 0, s>>>(in, (double2*)out, count);
  return cudaGetLastError();
}

cudaError_t launch_sum3(const void* a, const void* b, const void* c, double2* z, long long per_col, int ncols,
                        int r_from, int l_below, int prec, cudaStream_t s) {
  const dim3 sgrid((unsigned)((per_col + 255) / 256), (unsigned)ncols);
  if (prec == ASP_PREC_C64)
    sum3_kernel<float><<<sgrid, 256, 0, s>>>((const float2*)a, (const float2*)b, (const float2*)c, z, per_col, r_from,
                                             l_below);
  else
    sum3_kernel<double><<<sgrid, 256, 0, s>>>((const double2*)a, (const double2*)b, (const double2*)c, z, per_col,
                                              r_from, l_below);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- job lists
namespace {

struct JobList {
  Job* d = nullptr;
  int n = 0, cap = 0, wmax = 0, variant = 0;
};

// A layer-solve launch shape: right-hand sides per job (the tile's column
// capacity) and the instance variant of launch_btsolve_apply.
struct Shape {
  int cap = 0, variant = 0;
};

struct JobCache {
  std::map<int, JobList> embed, fill;
  std::map<int, Shape> tuned_embed, tuned_fill;  // asp_autotune's choices per nrhs
  std::map<long long, JobList> sub;  // key: subproblem index * 1024 + nrhs
  JobList tmap;
  bool have_tmap = false;
  std::vector<void*> owned;
  ~JobCache() {
    for (void* p : owned) cudaFree(p);
  }
};

// Job lists per handle.  Handles may be used from different host threads at
// the same time (one thread per handle), so the map itself is guarded.
std::mutex& caches_mu() {
  static std::mutex mu;
  return mu;
}
std::map<const Handle*, JobCache>& caches() {
  static std::map<const Handle*, JobCache> c;
  return c;
}
JobCache& cache_of(const Handle* h) {
  std::lock_guard<std::mutex> lock(caches_mu());
  return caches()[h];
}

int upload_jobs(Handle& H, const std::vector<Job>& jobs, int cap, int wmax, JobList* out, int variant = 0) {
  out->n = (int)jobs.size();
  out->cap = cap;
  out->wmax = wmax;
  out->variant = variant;
  if (jobs.empty()) return ASP_OK;
  void* d = nullptr;
  if (cudaMalloc(&d, jobs.size() * sizeof(Job)) != cudaSuccess) return fail(ASP_ERR_OOM, "job list allocation");
  if (cudaMemcpy(d, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return fail(ASP_ERR_CUDA, "job list upload");
  }
  cache_of(&H).owned.push_back(d);
  out->d = (Job*)d;
  return ASP_OK;
}

int embed_wmax(const Handle& H) {
  int wm = 0;
  for (int q = 1; q <= H.m; ++q) wm = std::max(wm, H.subs[H.subM[q]].w);
  return wm;
}

int build_embed_jobs(Handle& H, int nrhs, Shape sh, JobList* L) {
  std::vector<Job> jobs;
  for (int q = 1; q <= H.m; ++q)
    for (int r0 = 0; r0 < nrhs; r0 += sh.cap) jobs.push_back({H.subM[q], MODE_EMBED, r0, std::min(sh.cap, nrhs - r0)});
  return upload_jobs(H, jobs, sh.cap, embed_wmax(H), L, sh.variant);
}

int build_fill_jobs(Handle& H, int nrhs, Shape sh, JobList* L) {
  std::vector<Job> jobs;
  for (int p = 1; p <= H.m; ++p) {
    for (int r0 = 0; r0 < nrhs; r0 += sh.cap) {
      if (p >= 2) jobs.push_back({H.subR[p], MODE_FILL_R, r0, std::min(sh.cap, nrhs - r0)});
      if (p <= H.m - 1) jobs.push_back({H.subL[p], MODE_FILL_L, r0, std::min(sh.cap, nrhs - r0)});
    }
  }
  return upload_jobs(H, jobs, sh.cap, std::max(1, H.wmaxRL), L, sh.variant);
}

// The launch shape of the M-solves / fills for nrhs right-hand sides: the
// autotuner's choice if asp_autotune ran for this nrhs, else the default
// capacity for the count.
Shape shape_for(Handle& H, JobCache& c, int cls, int nrhs) {
  const auto& tuned = cls == CLS_EMBED ? c.tuned_embed : c.tuned_fill;
  auto it = tuned.find(nrhs);
  if (it != tuned.end()) return it->second;
  Shape sh;
  sh.cap = btsolve_rhs_capacity(nrhs, cls == CLS_EMBED ? embed_wmax(H) : std::max(1, H.wmaxRL), H.prec, false);
  return sh;
}

int get_embed_jobs(Handle& H, int nrhs, JobList** out) {
  JobCache& c = cache_of(&H);
  auto it = c.embed.find(nrhs);
  if (it == c.embed.end()) {
    JobList L;
    int rc = build_embed_jobs(H, nrhs, shape_for(H, c, CLS_EMBED, nrhs), &L);
    if (rc != ASP_OK) return rc;
    it = c.embed.emplace(nrhs, L).first;
  }
  *out = &it->second;
  return ASP_OK;
}

int get_fill_jobs(Handle& H, int nrhs, JobList** out) {
  JobCache& c = cache_of(&H);
  auto it = c.fill.find(nrhs);
  if (it == c.fill.end()) {
    JobList L;
    int rc = build_fill_jobs(H, nrhs, shape_for(H, c, CLS_FILL, nrhs), &L);
    if (rc != ASP_OK) return rc;
    it = c.fill.emplace(nrhs, L).first;
  }
  *out = &it->second;
  return ASP_OK;
}

SolveParams base_params(Handle& H, int ldv) {
  SolveParams P{};
  P.subs = H.d_subs;
  P.n = H.n;
  P.ldv = ldv;
  P.ldacc = (ldv + 1) & ~1;
  P.ldT = H.ldT;
  P.inv_h2 = H.inv_h2;
  P.W = H.W;
  P.ca = H.prec == ASP_PREC_C64 ? (const void*)H.fc32.ca : (const void*)H.fc64.ca;
  P.cc = H.prec == ASP_PREC_C64 ? (const void*)H.fc32.cc : (const void*)H.fc64.cc;
  P.s2inv = H.prec == ASP_PREC_C64 ? (const void*)H.fc32.s2inv : (const void*)H.fc64.s2inv;
  P.outM = H.uM;
  P.outR = H.uR;
  P.outL = H.uL;
  P.accR = H.accR;
  P.accL = H.accL;
  P.tmap = H.tmap;
  P.zscr = H.zscr;
  P.zslot = H.zslot;
  P.zslots = H.zslots;
  P.err = H.err;
  return P;
}

// Self-test of the bounded-wait path: an mbarrier that nothing arrives on, waited
// for with the library's wait helper and a short poll limit.  The wait must give
// up and record ASP_ERR_TIMEOUT in the error word; no copy is in flight, so the
// CTA then simply exits.
__global__ void wait_selftest_kernel(int* err, uint32_t limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool done = mbar_wait(&bar, 0u, limit);  // phase 0 never completes
  if (!done && threadIdx.x == 0) record_error(err, ASP_ERR_TIMEOUT, 0);
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(&bar);
}

int check_err(Handle& H, cudaStream_t s, const char* what) {
  int e[2] = {0, 0};
  if (cudaMemcpyAsync(e, H.err, sizeof(e), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(ASP_ERR_CUDA, std::string(what) + ": ") ;
  if (e[0] != 0) {
    cudaMemsetAsync(H.err, 0, 2 * sizeof(int), s);
    return fail(e[0], std::string(what) + ": device reported " + asp_error_string(e[0]) + " (detail " +
                          std::to_string(e[1]) + ")");
  }
  return ASP_OK;
}

}  // namespace

int apply_precond(Handle& H, const double2* r, double2* z, int nrhs, cudaStream_t s) {
  if (H.dim == 3) return apply3d(H, r, z, nrhs, s);
  if (!H.factored) return fail(ASP_ERR_STATE, "apply before factor");
  const long long count = H.N * nrhs;
  const void* in = r;
  if (H.prec == ASP_PREC_C64) {
    PhaseTok tk = phase_begin(H, PH_SUM, s);
    if (launch_to_prec(r, H.r_lo, count, H.prec, s) != cudaSuccess) return fail(ASP_ERR_CUDA, "to_prec launch");
    phase_end(H, tk, s);
    H.launches += 1;
    in = H.r_lo;
  }
  JobList *je = nullptr, *jf = nullptr;
  int rc = get_embed_jobs(H, nrhs, &je);
  if (rc != ASP_OK) return rc;
  rc = get_fill_jobs(H, nrhs, &jf);
  if (rc != ASP_OK) return rc;
  // 1. M-solves of every layer (Algorithm 2, first loop) + traces
  SolveParams P = base_params(H, nrhs);
  P.in = in;
  P.jobs = je->d;
  P.njobs = je->n;
  PhaseTok tk = phase_begin(H, PH_EMBED, s);
  cudaError_t ce = launch_btsolve_apply(H, P, CLS_EMBED, je->cap, je->variant, je->wmax, s);
  phase_end(H, tk, s);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("M-solve launch: ") + cudaGetErrorString(ce));
  // 2. accumulated traces of both sweeps (Algorithm 2, second and third loops)
  const size_t esz = H.prec == ASP_PREC_C128 ? sizeof(double2) : sizeof(float2);
  for (int r0 = 0; r0 < nrhs; r0 += 32) {
    ChainParams C{};
    C.n = H.n; C.m = H.m; C.ldacc = (nrhs + 1) & ~1; C.ldT = H.ldT; C.nrhs = std::min(32, nrhs - r0);
    C.tmap = H.tmap; C.toffR = H.d_toffR; C.toffL = H.d_toffL;
    C.accR = (char*)H.accR + r0 * esz;
    C.accL = (char*)H.accL + r0 * esz;
    C.bar = H.bar; C.err = H.err;
    tk = phase_begin(H, PH_CHAIN, s);
    ce = launch_chain(H, C, s);
    phase_end(H, tk, s);
    if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("sweep chain launch: ") + cudaGetErrorString(ce));
  }
  // 3. the right- and left-going layer fields from the accumulated traces
  P.jobs = jf->d;
  P.njobs = jf->n;
  tk = phase_begin(H, PH_FILL, s);
  ce = launch_btsolve_apply(H, P, CLS_FILL, jf->cap, jf->variant, jf->wmax, s);
  phase_end(H, tk, s);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("fill launch: ") + cudaGetErrorString(ce));
  // 4. u~_p = u~_{p,1:p-1} + u~_{p,p} + u~_{p,p+1:m}
  tk = phase_begin(H, PH_SUM, s);
  ce = launch_sum3(H.uM, H.uR, H.uL, z, (long long)H.n * nrhs, H.n, H.x_hi[1], H.x_lo[H.m] - 1, H.prec, s);
  phase_end(H, tk, s);
  H.launches += 1;
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("sum launch: ") + cudaGetErrorString(ce));
  return ASP_OK;
}

// Candidate launch shapes of the M-solves (cls CLS_EMBED) or fills for nrhs
// right-hand sides: the default capacity, its variant where one is compiled
// (complex64 at 32 and 1 right-hand sides), and the next smaller capacity
// (more, narrower jobs).  At most kTuneCands.
constexpr int kTuneCands = 3;
std::vector<Shape> tune_candidates(const Handle& H, int nrhs, int wmax) {
  std::vector<Shape> c;
  const int def = btsolve_rhs_capacity(nrhs, wmax, H.prec, false);
  c.push_back({def, 0});
  if (H.prec == ASP_PREC_C64 && (def == 32 || def == 1)) c.push_back({def, 1});
  static const int caps[] = {32, 16, 8, 4, 2, 1};
  for (int cp : caps)
    if (cp < def) {
      c.push_back({cp, 0});
      break;
    }
  return c;
}

int autotune(Handle& H, int nrhs, int* choice, double* ms_out, cudaStream_t s) {
  if (!H.factored) return fail(ASP_ERR_STATE, "autotune before factor");
  if (ms_out)
    for (int i = 0; i < 2 * kTuneCands; ++i) ms_out[i] = 0.0;
  if (H.dim != 2) return ASP_OK;  // the 3D slab solves have one launch shape
  JobCache& c = cache_of(&H);
  SolveParams P = base_params(H, nrhs);
  P.in = H.prec == ASP_PREC_C64 ? (const void*)H.r_lo : (const void*)H.wv;  // contents do not matter for timing
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(ASP_ERR_CUDA, "autotune: event creation");
  }
  int rc = ASP_OK;
  for (int k = 0; k < 2 && rc == ASP_OK; ++k) {
    const int cls = k == 0 ? CLS_EMBED : CLS_FILL;
    const int wm = cls == CLS_EMBED ? embed_wmax(H) : std::max(1, H.wmaxRL);
    const std::vector<Shape> cands = tune_candidates(H, nrhs, wm);
    Shape best = cands[0];
    double best_ms = 1e300;
    for (size_t i = 0; i < cands.size() && rc == ASP_OK; ++i) {
      JobList L;
      rc = cls == CLS_EMBED ? build_embed_jobs(H, nrhs, cands[i], &L) : build_fill_jobs(H, nrhs, cands[i], &L);
      if (rc != ASP_OK) break;
      P.jobs = L.d;
      P.njobs = L.n;
      // one untimed launch, then three timed ones on the handle's own factors
      cudaError_t ce = launch_btsolve_apply(H, P, cls, L.cap, L.variant, L.wmax, s);
      if (ce != cudaSuccess) {  // a shape this width does not fit: not a candidate
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) ce = launch_btsolve_apply(H, P, cls, L.cap, L.variant, L.wmax, s);
      cudaEventRecord(e1, s);
      float t = 0.f;
      if (ce != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
        rc = fail(ASP_ERR_CUDA, "autotune: timed launches");
        break;
      }
      H.launches += 4;
      const double ms = t / 3.0;
      if (ms_out) ms_out[k * kTuneCands + i] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best = cands[i];
      }
    }
    if (rc != ASP_OK) break;
    (cls == CLS_EMBED ? c.tuned_embed : c.tuned_fill)[nrhs] = best;
    (cls == CLS_EMBED ? c.embed : c.fill).erase(nrhs);  // the next apply builds its jobs with the choice
    if (choice) {
      choice[2 * k] = best.cap;
      choice[2 * k + 1] = best.variant;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == ASP_OK) rc = check_err(H, s, "autotune");
  return rc;
}

int set_solve_shape(Handle& H, int nrhs, int kind, int cap, int variant) {
  if (H.dim != 2) return fail(ASP_ERR_UNSUPPORTED, "3D slab solves have one launch shape");
  if (kind != 0 && kind != 1) return fail(ASP_ERR_INVALID, "kind must be 0 (M-solves) or 1 (fills)");
  const int wm = kind == 0 ? embed_wmax(H) : std::max(1, H.wmaxRL);
  for (const Shape& c : tune_candidates(H, nrhs, wm))
    if (c.cap == cap && c.variant == variant) {
      JobCache& jc = cache_of(&H);
      (kind == 0 ? jc.tuned_embed : jc.tuned_fill)[nrhs] = c;
      (kind == 0 ? jc.embed : jc.fill).erase(nrhs);  // the next apply builds its jobs with it
      return ASP_OK;
    }
  return fail(ASP_ERR_INVALID, "not a launch shape of this handle at this nrhs");
}

}  // namespace asp

using namespace asp;

extern "C" {

int asp_set_solve_shape(asp_handle* hd, int nrhs, int kind, int cap, int variant) {
  if (!hd) return fail(ASP_ERR_INVALID, "null handle");
  Handle& H = hd->h;
  if (nrhs < 1 || nrhs > H.prm.max_rhs) return fail(ASP_ERR_INVALID, "nrhs out of range");
  return set_solve_shape(H, nrhs, kind, cap, variant);
}

int asp_autotune(asp_handle* hd, int nrhs, int* choice_host, double* ms_host, void* stream) {
  if (!hd) return fail(ASP_ERR_INVALID, "null handle");
  Handle& H = hd->h;
  if (nrhs < 1 || nrhs > H.prm.max_rhs) return fail(ASP_ERR_INVALID, "nrhs out of range");
  return autotune(H, nrhs, choice_host, ms_host, (cudaStream_t)stream);
}

const char* asp_error_string(int code) {
  switch (code) {
    case ASP_OK: return "ASP_OK";
    case ASP_ERR_INVALID: return "ASP_ERR_INVALID";
    case ASP_ERR_OOM: return "ASP_ERR_OOM";
    case ASP_ERR_CUDA: return "ASP_ERR_CUDA";
    case ASP_ERR_SMALL_PIVOT: return "ASP_ERR_SMALL_PIVOT";
    case ASP_ERR_NOT_CONVERGED: return "ASP_ERR_NOT_CONVERGED";
    case ASP_ERR_TIMEOUT: return "ASP_ERR_TIMEOUT";
    case ASP_ERR_STATE: return "ASP_ERR_STATE";
    case ASP_ERR_UNSUPPORTED: return "ASP_ERR_UNSUPPORTED";
  }
  return "ASP_ERR_UNKNOWN";
}

const char* asp_last_error_detail(void) { return g_detail.c_str(); }

size_t asp_footprint_bytes_layers(const asp_params* pin, const int* widths, int m) {
  std::string why;
  if (!pin) return 0;
  if (!valid(pin, &why)) return 0;
  bool packed = false;
  const asp_params q = normalized(pin, &packed);
  const asp_params* p = &q;
  if (packed && p->dim != 2) return 0;
  int sms = device_sms();
  if (sms <= 0) sms = kDefaultSms;
  const std::vector<int> w = layer_widths(p, widths, m, &why);
  if (w.empty() || !valid(p, &why, &w)) return 0;
  const Part P = partition(p->n, p->pml, p->pml_aux ? p->pml_aux : p->pml, w);
  if (!supported(p, P, &why, sms)) return 0;
  return sizes_for(p, P, sms, packed).bytes;
}

size_t asp_footprint_bytes(const asp_params* p) { return asp_footprint_bytes_layers(p, nullptr, 0); }

int asp_layer_widths_from_velocity(const asp_params* p, const double* c, int b_min, int b_max, int* widths,
                                   int capacity) {
  if (!p || !c || !widths) return fail(ASP_ERR_INVALID, "null argument");
  if ((p->dim != 2 && p->dim != 3) || p->n < 3 || p->pml < 2) return fail(ASP_ERR_INVALID, "bad dim, n or pml");
  const int n = p->n, gamma = p->pml, ga = p->pml_aux ? p->pml_aux : p->pml;
  const int P = n + 2 - 2 * gamma;
  // a padded M-layer is 2*gamma_a + b - 2 columns wide and the 2D kernels take 64
  const int b_cap = p->dim == 2 ? 66 - 2 * ga : P;
  if (b_min < 1 || b_max < b_min || b_min > b_cap || P < b_min)
    return fail(ASP_ERR_INVALID, "need 1 <= b_min <= b_max, b_min <= n + 2 - 2*gamma and a padded width <= 64");
  b_max = std::min(b_max, b_cap);
  const long long T = p->dim == 3 ? (long long)n * n : n;  // transverse points per sweep column
  // relative velocity jump between sweep columns j and j+1 (1-based j), worst over the column
  std::vector<double> v(n + 2, 0.0);
  for (int j = 1; j < n; ++j) {
    double worst = 0.0;
    const double* a = c + (long long)(j - 1) * T;
    const double* b = c + (long long)j * T;
    for (long long t = 0; t < T; ++t) {
      if (!(a[t] > 0) || !(b[t] > 0) || !isfinite(a[t]) || !isfinite(b[t]))
        return fail(ASP_ERR_INVALID, "velocity must be positive and finite");
      worst = std::max(worst, fabs(b[t] - a[t]) / std::min(a[t], b[t]));
    }
    v[j] = worst;
  }
  // "heavy" variation: well above the typical jump inside the physical region
  std::vector<double> vs(v.begin() + gamma, v.begin() + (n + 1 - gamma));
  double tau = 1e-3;
  if (!vs.empty()) {
    std::nth_element(vs.begin(), vs.begin() + vs.size() / 2, vs.end());
    tau = std::max(tau, 4.0 * vs[vs.size() / 2]);
  }
  // left to right: at least b_min columns; a layer does not end between two
  // columns with a heavy jump unless it has reached b_max; the last layer
  // takes what is left when that is less than b_min more
  std::vector<int> w;
  int a = gamma;  // first physical column of the next layer
  const int last = n + 1 - gamma;
  while (a <= last) {
    int e = a + b_min - 1;  // last column of this layer
    while (e < last && e - a + 1 < b_max && v[e] > tau) ++e;
    if (last - e < b_min) {
      if (last - a + 1 <= b_cap) e = last;               // absorb the remainder
      else e = std::min(e, last - b_min);                 // keep the padded width in range
    }
    e = std::min(e, last);
    w.push_back(e - a + 1);
    a = e + 1;
  }
  if ((int)w.size() > capacity) return fail(ASP_ERR_INVALID, "capacity below the number of layers");
  for (size_t i = 0; i < w.size(); ++i) widths[i] = w[i];
  return (int)w.size();
}

int asp_num_layers(const asp_handle* h) { return h ? h->h.m : ASP_ERR_INVALID; }

int asp_layer_range(const asp_handle* h, int p, int* x_lo, int* x_hi) {
  if (!h || p < 1 || p > h->h.m) return fail(ASP_ERR_INVALID, "layer index out of range");
  if (x_lo) *x_lo = h->h.x_lo[p];
  if (x_hi) *x_hi = h->h.x_hi[p];
  return ASP_OK;
}

int asp_set_phase_timing(asp_handle* hd, int enable) {
  if (!hd) return fail(ASP_ERR_INVALID, "null handle");
  hd->h.timing = enable != 0;
  return ASP_OK;
}

int asp_phase_times(asp_handle* hd, double* ms, long long* launches, int nphases) {
  if (!hd || nphases < 0 || nphases > ASP_NUM_PHASES) return fail(ASP_ERR_INVALID, "bad arguments");
  Handle& H = hd->h;
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(ASP_ERR_CUDA, "synchronize for phase times");
  for (int i = 0; i < nphases; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  std::lock_guard<std::mutex> lock(H.rec_mu);
  for (auto& r : H.recs) {
    float t = 0.f;
    if (r.phase < nphases && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      if (ms) ms[r.phase] += t;
      if (launches) launches[r.phase] += 1;
    }
    H.evpool.push_back(r.a);
    H.evpool.push_back(r.b);
  }
  H.recs.clear();
  return ASP_OK;
}

void asp_destroy(asp_handle* hd) {
  if (!hd) return;
  Handle& H = hd->h;
  for (auto& r : H.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : H.evpool) cudaEventDestroy(e);
  {
    std::lock_guard<std::mutex> lock(caches_mu());
    caches().erase(&H);
  }
  release_jobs3(&H);
  nd_release(H);
  for (auto& g : H.fgroups) {
    tc_group_release(g.tc);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.done) cudaEventDestroy(g.done);
  }
  void* ptrs[] = {H.k2, H.dgre, H.ca, H.cc, H.cd, H.d_subs, H.d_coef, H.W, H.tmap, H.d_toffR, H.d_toffL, H.d_tm, H.gdiag, H.r_lo,
                  H.uM, H.uR, H.uL, H.accR, H.accL, H.zscr, H.bar, H.V, H.Z, H.wv, H.red, H.hess, H.kstate,
                  H.kflags, H.err, H.d_slabs, H.d_slab_lists, H.A3, H.piv3, H.z3, H.tc_area};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : H.coef_bufs)
    if (p) cudaFree(p);
  if (H.h_flags) cudaFreeHost(H.h_flags);
  if (H.ev_fork) cudaEventDestroy(H.ev_fork);
  if (H.ev_join) cudaEventDestroy(H.ev_join);
  if (H.aux) cudaStreamDestroy(H.aux);
  delete hd;
}

int asp_setup(const asp_params* p, const double* c, int c_is_device, asp_handle** out) {
  return asp_setup_layers(p, nullptr, 0, c, c_is_device, out);
}

int asp_setup_layers(const asp_params* pin, const int* widths, int nwidths, const double* c, int c_is_device,
                     asp_handle** out) {
  std::string why;
  if (!out) return fail(ASP_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!pin) return fail(ASP_ERR_INVALID, "null params");
  if (!valid(pin, &why)) return fail(ASP_ERR_INVALID, why);
  bool packed = false;
  const asp_params q = normalized(pin, &packed);
  const asp_params* p = &q;
  if (packed && p->dim != 2) return fail(ASP_ERR_UNSUPPORTED, "packed symmetric factors are 2D only");
  const std::vector<int> lw = layer_widths(p, widths, nwidths, &why);
  if (lw.empty()) return fail(ASP_ERR_INVALID, why);
  if (!valid(p, &why, &lw)) return fail(ASP_ERR_INVALID, why);
  const int sms = device_sms();
  const Part P = partition(p->n, p->pml, p->pml_aux ? p->pml_aux : p->pml, lw);
  if (!supported(p, P, &why, sms > 0 ? sms : kDefaultSms)) return fail(ASP_ERR_UNSUPPORTED, why);
  if (!c) return fail(ASP_ERR_INVALID, "velocity pointer is null");
  const int n = p->n;
  const long long N = p->dim == 3 ? (long long)n * n * n : (long long)n * n;
  std::vector<double> ch(N);
  if (c_is_device) {
    if (cudaMemcpy(ch.data(), c, N * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ASP_ERR_CUDA, "copying the velocity from the device");
  } else {
    memcpy(ch.data(), c, N * sizeof(double));
  }
  for (long long i = 0; i < N; ++i)
    if (!(ch[i] > 0) || !isfinite(ch[i])) return fail(ASP_ERR_INVALID, "velocity must be positive and finite");
  if (sms <= 0) return fail(ASP_ERR_CUDA, "no CUDA device");

  asp_handle* hd = new asp_handle();
  Handle& H = hd->h;
  H.prm = *p;
  H.dim = p->dim;
  H.n = n;
  H.N = N;
  H.prec = p->factor_prec;
  H.gamma = p->pml;
  H.gamma_a = p->pml_aux ? p->pml_aux : p->pml;
  H.b = p->b;
  H.h = 1.0 / (n + 1);
  H.inv_h2 = 1.0 / (H.h * H.h);
  H.num_sms = sms;
  const double h = H.h, omega = p->omega, ih2 = H.inv_h2;
  H.m = P.m;
  H.x_lo = P.x_lo; H.x_hi = P.x_hi; H.alpha = P.alpha; H.beta = P.beta;
  const int m = H.m;
  H.packed = packed;
  H.nd = p->dim == 3 && p->slab_solver == ASP_SLAB_ND;
  Sizes Z = sizes_for(p, P, sms, packed);

  // ---- global stencil weights (same boundary PML on x1 and x2)
  Profile g;
  g.lo_on = g.hi_on = true;
  g.lo_edge = H.gamma * h;
  g.hi_edge = (n + 1 - H.gamma) * h;
  g.eta_lo = g.eta_hi = H.gamma * h;
  g.C = p->C;
  std::vector<double2> ca(n), cc(n), cd(n), s1v(n), s1i(n);
  for (int k = 0; k < n; ++k) {
    const double x = (k + 1) * h;
    const double2 sk = g.s(x, omega), sm = g.s(x - 0.5 * h, omega), sp = g.s(x + 0.5 * h, omega);
    s1v[k] = sk;
    const double d2 = sk.x * sk.x + sk.y * sk.y;
    s1i[k] = make_double2(sk.x / d2, -sk.y / d2);
    ca[k] = hscale(hmul(sk, sm), ih2);
    cc[k] = hscale(hmul(sk, sp), ih2);
    cd[k] = hscale(hadd(ca[k], cc[k]), -1.0);
  }
  // the longest run of nodes with real stencil coefficients (sigma = 0 there)
  {
    int best_lo = 0, best_len = 0;
    for (int k = 0; k < n;) {
      if (ca[k].y != 0.0 || cc[k].y != 0.0 || cd[k].y != 0.0) { ++k; continue; }
      int e = k;
      while (e < n && ca[e].y == 0.0 && cc[e].y == 0.0 && cd[e].y == 0.0) ++e;
      if (e - k > best_len) { best_len = e - k; best_lo = k; }
      k = e;
    }
    H.real_lo = best_lo;
    H.real_hi = best_lo + best_len;
  }
  std::vector<double> k2(N);
  for (long long i = 0; i < N; ++i) k2[i] = omega * omega / (ch[i] * ch[i]);

  // ---- subproblems (2D: strips of columns; 3D: slabs of planes) and their
  // sweep-axis profiles
  H.subM.assign(m + 1, -1); H.subR.assign(m + 1, -1); H.subL.assign(m + 1, -1);
  std::vector<double2> s2v, s2i;  // s and 1/s of every subproblem column, in SweepCoef order
  auto push_coef = [&](int lo, int w, const Profile& pr) {
    const int prof = (int)H.coef.size();
    for (int j = 0; j < w; ++j) {
      const double x = (lo + j) * h;
      const double2 sj = pr.s(x, omega), sm = pr.s(x - 0.5 * h, omega), sp = pr.s(x + 0.5 * h, omega);
      s2v.push_back(sj);
      const double d2 = sj.x * sj.x + sj.y * sj.y;
      s2i.push_back(make_double2(sj.x / d2, -sj.y / d2));
      SweepCoef cf;
      cf.up = hscale(hmul(sj, sp), ih2);
      cf.dn = hscale(hmul(sj, sm), ih2);
      cf.dg = hscale(hadd(cf.up, cf.dn), -1.0);
      H.coef.push_back(cf);
    }
    return prof;
  };
  long long woff = 0, aoff = 0, poff = 0, zoff = 0;
  auto add = [&](int kind, int q, int lo, int hi, const Profile& pr) {
    const int w = hi - lo + 1;
    H.wmax = std::max(H.wmax, w);
    if (kind != KIND_M) H.wmaxRL = std::max(H.wmaxRL, w);
    if (H.dim == 3) {
      Slab S{};
      S.kind = kind; S.p = q; S.lo = lo; S.w = w;
      S.xoff = H.x_lo[q] - lo;
      S.xw = H.x_hi[q] - H.x_lo[q] + 1;
      S.prof = push_coef(lo, w, pr);
      S.nb = n * w;
      S.ld = (S.nb + 3) & ~3;
      S.src_plane = 0;
      S.src_sweep = 0;
      if (kind == KIND_R) { S.src_plane = H.x_hi[q - 1] - 1; S.src_sweep = (q - 1 >= 2) ? 1 : 0; }
      if (kind == KIND_L) { S.src_plane = H.x_lo[q + 1] - 1; S.src_sweep = (q + 1 <= m - 1) ? 1 : 0; }
      S.woff = woff; woff += (long long)n * S.nb * S.ld;
      S.np = S.nb;
      S.aoff = aoff; aoff += slab_work_elems(S.nb, S.ld);
      S.zbo = 2LL * S.nb * S.ld;
      S.poff = poff; poff += 3LL * S.nb;
      S.zoff = zoff; zoff += (long long)n * S.nb * p->max_rhs;
      if (kind == KIND_M) H.nbmaxM = std::max(H.nbmaxM, S.nb);
      else H.nbmaxRL = std::max(H.nbmaxRL, S.nb);
      H.slabs.push_back(S);
      return (int)H.slabs.size() - 1;
    }
    SubDesc S{};
    S.kind = kind; S.p = q; S.lo = lo; S.w = w;
    S.wp = (H.prec == ASP_PREC_C64) ? ((S.w + 1) & ~1) : S.w;
    S.bs = H.packed ? packed_block_elems(S.w) : S.w * S.wp;
    S.xoff = H.x_lo[q] - lo;
    S.xw = H.x_hi[q] - H.x_lo[q] + 1;
    S.prof = push_coef(lo, w, pr);
    S.woff = woff;
    S.toff = -1;
    woff += (long long)n * S.bs;
    H.subs.push_back(S);
    return (int)H.subs.size() - 1;
  };
  const double eta = H.gamma * h, eta_a = H.gamma_a * h;
  for (int q = 1; q <= m; ++q) {
    Profile pr;  // sigma_q^M: zero on [alpha_q h, beta_q h]
    pr.C = p->C;
    pr.lo_on = pr.hi_on = true;
    pr.lo_edge = H.alpha[q] * h; pr.eta_lo = (q == 1) ? eta : eta_a;
    pr.hi_edge = H.beta[q] * h;  pr.eta_hi = (q == m) ? eta : eta_a;
    H.subM[q] = add(KIND_M, q, P.m_lo[q], P.m_hi[q], pr);
  }
  // s2(keep) / s2(in) of each sweep subproblem (the map's symmetry factor)
  std::vector<double2> rhoR(m + 1, make_double2(1, 0)), rhoL(m + 1, make_double2(1, 0));
  auto sratio = [&](const Profile& pr, int keep_g, int in_g) {
    const double2 a = pr.s(keep_g * h, omega), b = pr.s(in_g * h, omega);
    const double d2 = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d2, (a.y * b.x - a.x * b.y) / d2);
  };
  for (int q = 2; q <= m; ++q) {
    Profile pr;  // sigma_q^R: no layer on the left
    pr.C = p->C;
    pr.hi_on = true;
    pr.hi_edge = H.beta[q] * h; pr.eta_hi = (q == m) ? eta : eta_a;
    H.subR[q] = add(KIND_R, q, H.alpha[q], P.m_hi[q], pr);
    rhoR[q] = sratio(pr, H.x_hi[q], H.alpha[q]);
  }
  for (int q = 1; q <= m - 1; ++q) {
    Profile pr;  // sigma_q^L: no layer on the right
    pr.C = p->C;
    pr.lo_on = true;
    pr.lo_edge = H.alpha[q] * h; pr.eta_lo = (q == 1) ? eta : eta_a;
    H.subL[q] = add(KIND_L, q, P.m_lo[q], H.beta[q], pr);
    rhoL[q] = sratio(pr, H.x_lo[q], H.beta[q]);
  }
  H.W_elems = (size_t)woff;
  if (H.nd) {  // nd_setup plans and allocates the factors, work and pivots
    H.W_elems = 0;
    aoff = 0;
    poff = 0;
  }
  // transfer maps T_p^R, T_p^L for p = 2..m-1 (2D only)
  H.toffR.assign(m + 1, 0); H.toffL.assign(m + 1, 0);
  H.ldT = (n + 1) & ~1;
  long long toff = 0;
  if (H.dim == 2) {
    for (int q = 2; q <= m - 1; ++q) {
      H.toffR[q] = toff; H.subs[H.subR[q]].toff = toff; toff += (long long)n * H.ldT;
      H.toffL[q] = toff; H.subs[H.subL[q]].toff = toff; toff += (long long)n * H.ldT;
    }
  }
  H.tmap_elems = (size_t)toff;
  if (tc_maps(H.dim, H.prec, m, H.wmaxRL)) {
    long long goff = 0;
    for (int q = 2; q <= m - 1; ++q)
      for (int kind = 0; kind < 2; ++kind) {
        const SubDesc& S = H.subs[kind == 0 ? H.subR[q] : H.subL[q]];
        TmMap M{};
        M.woff = S.woff;
        M.toff = S.toff;
        M.goff = goff;
        goff += (long long)n * 2 * 32;
        M.w = S.w;
        M.wp = S.wp;
        M.bs = S.bs;
        M.prof = S.prof;
        M.jin = kind == 0 ? 0 : S.w - 1;
        M.keep = kind == 0 ? S.xoff + S.xw - 1 : S.xoff;
        const double2 rho = kind == 0 ? rhoR[q] : rhoL[q];
        M.rho = make_float2((float)rho.x, (float)rho.y);
        H.tm_host.push_back(M);
      }
  }

  // ---- device allocations (none when the footprint exceeds the free memory)
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && Z.bytes > free_b) {
      asp_destroy(hd);
      return fail(ASP_ERR_OOM, "footprint " + std::to_string(Z.bytes) + " bytes exceeds the free device memory (" +
                                   std::to_string(free_b) + " bytes)");
    }
  }
  const size_t esz = Z.esz;
  const int mr = p->max_rhs;
  bool ok = true;
  auto dal = [&](void** ptr, size_t bytes) {
    if (!ok) return;
    if (bytes == 0) bytes = 16;
    if (dev_malloc(ptr, bytes) != cudaSuccess) { ok = false; *ptr = nullptr; }
  };
  dal((void**)&H.k2, N * sizeof(double));
  if (H.dim == 2) dal((void**)&H.dgre, N * sizeof(double));
  dal((void**)&H.ca, n * sizeof(double2));
  dal((void**)&H.cc, n * sizeof(double2));
  dal((void**)&H.cd, n * sizeof(double2));
  dal((void**)&H.d_coef, H.coef.size() * sizeof(SweepCoef));
  dal(&H.W, H.W_elems * esz);
  if (H.dim == 2) {
    dal((void**)&H.d_subs, H.subs.size() * sizeof(SubDesc));
    dal(&H.tmap, H.tmap_elems * esz);
    dal((void**)&H.d_toffR, (m + 1) * sizeof(long long));
    dal((void**)&H.d_toffL, (m + 1) * sizeof(long long));
    dal(&H.accR, (size_t)(m + 1) * n * ((mr + 1) & ~1) * esz);
    dal(&H.accL, (size_t)(m + 1) * n * ((mr + 1) & ~1) * esz);
    H.zslots = Z.zslots;
    H.zslot = (long long)Z.zslot;
    dal(&H.zscr, (size_t)Z.zslots * Z.zslot * esz);
    if (!H.tm_host.empty()) {
      dal((void**)&H.d_tm, H.tm_host.size() * sizeof(TmMap));
      dal(&H.gdiag, H.tm_host.size() * (size_t)n * 2 * 32 * sizeof(float2));
    }
  } else {
    dal((void**)&H.d_slabs, H.slabs.size() * sizeof(Slab));
    dal((void**)&H.d_slab_lists, H.slabs.size() * sizeof(int));
    dal(&H.A3, (size_t)aoff * esz);
    dal((void**)&H.piv3, (size_t)poff * sizeof(int));
    dal(&H.z3, (size_t)zoff * esz);
    if (H.prec == ASP_PREC_C64 && !H.nd) dal((void**)&H.tc_area, Z.tc_floats * sizeof(float));
  }
  if (H.prec == ASP_PREC_C64) dal(&H.r_lo, (size_t)N * mr * esz);
  dal(&H.uM, (size_t)N * mr * esz);
  dal(&H.uR, (size_t)N * mr * esz);
  dal(&H.uL, (size_t)N * mr * esz);
  dal((void**)&H.bar, 64);
  const int R = p->restart;
  dal((void**)&H.V, (size_t)(R + 1) * N * mr * sizeof(double2));
  dal((void**)&H.Z, (size_t)R * N * mr * sizeof(double2));
  dal((void**)&H.wv, (size_t)N * mr * sizeof(double2));
  dal((void**)&H.red, (size_t)sms * 4 * 9 * mr * sizeof(double2));
  size_t n2, nd, ni;
  krylov_state_bytes(R, mr, &n2, &nd, &ni);
  dal((void**)&H.hess, n2 * sizeof(double2));
  dal((void**)&H.kstate, nd * sizeof(double));
  dal((void**)&H.kflags, ni * sizeof(int));
  dal((void**)&H.err, 2 * sizeof(int));
  if (ok && cudaMallocHost((void**)&H.h_flags, 64) != cudaSuccess) ok = false;
  if (ok && cudaStreamCreateWithFlags(&H.aux, cudaStreamNonBlocking) != cudaSuccess) ok = false;
  if (ok && cudaEventCreateWithFlags(&H.ev_fork, cudaEventDisableTiming) != cudaSuccess) ok = false;
  if (ok && cudaEventCreateWithFlags(&H.ev_join, cudaEventDisableTiming) != cudaSuccess) ok = false;
  if (!ok) {
    asp_destroy(hd);
    cudaGetLastError();
    return fail(ASP_ERR_OOM, "device allocation failed (footprint " + std::to_string(Z.bytes) + " bytes)");
  }
  bool up = true;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (up && bytes && cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) up = false;
  };
  cp(H.k2, k2.data(), N * sizeof(double));
  if (H.dim == 2) {
    // real part of the operator's diagonal, d_{i1} + d_{i2} + omega^2/c^2 (the matvec's)
    std::vector<double> dre(N);
    for (int i2 = 0; i2 < n; ++i2)
      for (int i1 = 0; i1 < n; ++i1)
        dre[(long long)i2 * n + i1] = cd[i1].x + cd[i2].x + k2[(long long)i2 * n + i1];
    cp(H.dgre, dre.data(), N * sizeof(double));
  }
  cp(H.ca, ca.data(), n * sizeof(double2));
  cp(H.cc, cc.data(), n * sizeof(double2));
  cp(H.cd, cd.data(), n * sizeof(double2));
  cp(H.d_coef, H.coef.data(), H.coef.size() * sizeof(SweepCoef));
  if (H.dim == 2) {
    cp(H.d_subs, H.subs.data(), H.subs.size() * sizeof(SubDesc));
    if (!H.tm_host.empty()) cp(H.d_tm, H.tm_host.data(), H.tm_host.size() * sizeof(TmMap));
    cp(H.d_toffR, H.toffR.data(), (m + 1) * sizeof(long long));
    cp(H.d_toffL, H.toffL.data(), (m + 1) * sizeof(long long));
  } else {
    std::vector<int> lists(H.slabs.size());
    for (size_t i = 0; i < lists.size(); ++i) lists[i] = (int)i;  // [M slabs | R slabs, L slabs]
    cp(H.d_slabs, H.slabs.data(), H.slabs.size() * sizeof(Slab));
    cp(H.d_slab_lists, lists.data(), lists.size() * sizeof(int));
    // factor groups: one per kind (the M slabs; the R and L slabs).  Finer
    // splits measured slower at n = 95: four streams took 3.88 s per factor
    // against 3.06 s for two.
    if (up) {
      auto add_group = [&](int first, int count) {
        if (count <= 0) return;
        Handle::FGroup g;
        g.first = first;
        g.count = count;
        for (int i = first; i < first + count; ++i) g.nbmax = std::max(g.nbmax, H.slabs[i].nb);
        H.fgroups.push_back(g);
      };
      add_group(0, m);
      add_group(m, (int)H.slabs.size() - m);
      for (size_t gi = 0; gi < H.fgroups.size() && up; ++gi) {
        Handle::FGroup& g = H.fgroups[gi];
        if (gi + 1 < H.fgroups.size() &&  // the last group runs on the caller's stream
            cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess)
          up = false;
        if (up && cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess) up = false;
      }
    }
    if (up && H.nd) {
      const int rc = nd_setup(H);
      if (rc != ASP_OK) {
        const std::string why = asp_last_error_detail();
        asp_destroy(hd);
        return fail(rc, why);
      }
    }
    if (up && H.prec == ASP_PREC_C64 && !H.nd) {
      // operand rows of the tensor-core update, per factor group in list order
      long long off = 0;
      int rc = ASP_OK;
      for (auto& g : H.fgroups) {
        std::vector<long long> rows;
        long long nrows = 0;
        for (int i = g.first; i < g.first + g.count; ++i) {
          rows.push_back(nrows);
          nrows += (H.slabs[i].nb + 127) / 128 * 128;
        }
        if (rc == ASP_OK) rc = tc_group_setup(g.tc, H.tc_area + off, rows, nrows);
        off += tc_group_floats(nrows);
      }
      if (rc != ASP_OK) {
        const std::string why = asp_last_error_detail();
        asp_destroy(hd);
        return fail(rc, why);
      }
    }
  }
  // factor-precision copies of the layer coefficients
  bool coef_oom = false;
  {
    const size_t nc = H.coef.size();
    std::vector<double2> upv(nc), dnv(nc), dgv(nc);
    for (size_t i = 0; i < nc; ++i) { upv[i] = H.coef[i].up; dnv[i] = H.coef[i].dn; dgv[i] = H.coef[i].dg; }
    auto put = [&](const void* hsrc, size_t bytes) -> void* {
      void* d = nullptr;
      if (!up) return nullptr;
      if (dev_malloc(&d, bytes ? bytes : 16) != cudaSuccess) {
        up = false;
        coef_oom = true;
        return nullptr;
      }
      H.coef_bufs.push_back(d);
      if (bytes && cudaMemcpy(d, hsrc, bytes, cudaMemcpyHostToDevice) != cudaSuccess) up = false;
      return d;
    };
    if (H.prec == ASP_PREC_C128) {
      H.fc64.s1 = (const double2*)put(s1v.data(), n * sizeof(double2));
      H.fc64.s1inv = (const double2*)put(s1i.data(), n * sizeof(double2));
      H.fc64.s2 = (const double2*)put(s2v.data(), nc * sizeof(double2));
      H.fc64.s2inv = (const double2*)put(s2i.data(), nc * sizeof(double2));
      H.fc64.ca = (const double2*)put(ca.data(), n * sizeof(double2));
      H.fc64.cc = (const double2*)put(cc.data(), n * sizeof(double2));
      H.fc64.cd = (const double2*)put(cd.data(), n * sizeof(double2));
      H.fc64.k2 = (const double*)put(k2.data(), N * sizeof(double));
      H.fc64.up = (const double2*)put(upv.data(), nc * sizeof(double2));
      H.fc64.dn = (const double2*)put(dnv.data(), nc * sizeof(double2));
      H.fc64.dg = (const double2*)put(dgv.data(), nc * sizeof(double2));
    } else {
      auto f2 = [](const std::vector<double2>& v) {
        std::vector<float2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
        return o;
      };
      std::vector<float> k2f(N);
      for (long long i = 0; i < N; ++i) k2f[i] = (float)k2[i];
      auto caf = f2(ca), ccf = f2(cc), cdf = f2(cd), upf = f2(upv), dnf = f2(dnv), dgf = f2(dgv);
      auto s1f = f2(s1v), s1if = f2(s1i), s2f = f2(s2v), s2if = f2(s2i);
      H.fc32.s1 = (const float2*)put(s1f.data(), n * sizeof(float2));
      H.fc32.s1inv = (const float2*)put(s1if.data(), n * sizeof(float2));
      H.fc32.s2 = (const float2*)put(s2f.data(), nc * sizeof(float2));
      H.fc32.s2inv = (const float2*)put(s2if.data(), nc * sizeof(float2));
      H.fc32.ca = (const float2*)put(caf.data(), n * sizeof(float2));
      H.fc32.cc = (const float2*)put(ccf.data(), n * sizeof(float2));
      H.fc32.cd = (const float2*)put(cdf.data(), n * sizeof(float2));
      H.fc32.k2 = (const float*)put(k2f.data(), N * sizeof(float));
      H.fc32.up = (const float2*)put(upf.data(), nc * sizeof(float2));
      H.fc32.dn = (const float2*)put(dnf.data(), nc * sizeof(float2));
      H.fc32.dg = (const float2*)put(dgf.data(), nc * sizeof(float2));
    }
  }
  if (up && cudaMemset(H.W, 0, H.W_elems * esz) != cudaSuccess) up = false;  // 3D: row padding stays zero
  if (up && H.piv3 && cudaMemset(H.piv3, 0, (size_t)poff * sizeof(int)) != cudaSuccess) up = false;
  if (up && cudaMemset(H.err, 0, 2 * sizeof(int)) != cudaSuccess) up = false;
  if (up && cudaDeviceSynchronize() != cudaSuccess) up = false;
  if (!up) {
    asp_destroy(hd);
    cudaGetLastError();
    if (coef_oom) return fail(ASP_ERR_OOM, "device allocation of the layer coefficients failed");
    return fail(ASP_ERR_CUDA, "uploading the setup data");
  }
  *out = hd;
  return ASP_OK;
}

int asp_factor(asp_handle* hd, void* stream) {
  if (!hd) return fail(ASP_ERR_INVALID, "null handle");
  Handle& H = hd->h;
  cudaStream_t s = (cudaStream_t)stream;
  if (H.dim == 3) {
    int rc3 = H.nd ? nd_factor(H, s) : factor3d(H, s);
    if (rc3 != ASP_OK) return rc3;
    rc3 = check_err(H, s, "factor");
    if (rc3 != ASP_OK) return rc3;
    H.factored = true;
    return ASP_OK;
  }
  // The M-subproblems (indices [0, m)) factor on the internal stream while the
  // R/L subproblems (indices [m, 3m-2)) factor on the caller's stream and their
  // transfer maps are built; the M factors are latency-bound and overlap well.
  const int m = H.m;
  if (cudaEventRecord(H.ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(H.aux, H.ev_fork, 0) != cudaSuccess)
    return fail(ASP_ERR_CUDA, "factor: stream fork");
  PhaseTok ta = phase_begin(H, PH_FACTOR, H.aux);
  cudaError_t ce = launch_factor(H, 0, m, H.aux);
  phase_end(H, ta, H.aux);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("factor launch: ") + cudaGetErrorString(ce));
  PhaseTok tb = phase_begin(H, PH_FACTOR, s);
  ce = launch_factor(H, m, (int)H.subs.size() - m, s);
  phase_end(H, tb, s);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("factor launch: ") + cudaGetErrorString(ce));
  // transfer maps: on the tensor cores from the diagonal blocks of the inverse
  // (complex64, widths <= 32), else columns of T_p^R and T_p^L in chunks of
  // right-hand sides (CLS_TMAP solves)
  if (!H.tm_host.empty()) {
    PhaseTok td = phase_begin(H, PH_TDIAG, s);
    ce = launch_tmap_diag(H, s);
    phase_end(H, td, s);
    if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("diagonal-block launch: ") + cudaGetErrorString(ce));
    PhaseTok tk = phase_begin(H, PH_TMAP, s);
    ce = launch_tmap_tc(H, s);
    phase_end(H, tk, s);
    if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("transfer-map launch: ") + cudaGetErrorString(ce));
  } else if (H.m >= 3) {
    const int cap = btsolve_rhs_capacity(H.n, H.wmaxRL, H.prec, true);
    JobCache& jc = cache_of(&H);
    if (!jc.have_tmap) {
      std::vector<Job> jobs;
      for (int r0 = 0; r0 < H.n; r0 += cap)
        for (int q = 2; q <= H.m - 1; ++q) {
          jobs.push_back({H.subR[q], MODE_TMAP_R, r0, std::min(cap, H.n - r0)});
          jobs.push_back({H.subL[q], MODE_TMAP_L, r0, std::min(cap, H.n - r0)});
        }
      int rc = upload_jobs(H, jobs, cap, H.wmaxRL, &jc.tmap);
      if (rc != ASP_OK) return rc;
      jc.have_tmap = true;
    }
    const JobList& L = jc.tmap;
    SolveParams P = base_params(H, 1);
    P.jobs = L.d;
    P.njobs = L.n;
    PhaseTok tk = phase_begin(H, PH_TMAP, s);
    ce = launch_btsolve_aux(H, P, CLS_TMAP, cap, H.wmaxRL, s);
    phase_end(H, tk, s);
    if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("transfer-map launch: ") + cudaGetErrorString(ce));
  }
  if (cudaEventRecord(H.ev_join, H.aux) != cudaSuccess || cudaStreamWaitEvent(s, H.ev_join, 0) != cudaSuccess)
    return fail(ASP_ERR_CUDA, "factor: stream join");
  int rc = check_err(H, s, "factor");
  if (rc != ASP_OK) return rc;
  H.factored = true;
  return ASP_OK;
}

int asp_apply_preconditioner(asp_handle* hd, const void* r, void* z, int nrhs, void* stream) {
  if (!hd || !r || !z) return fail(ASP_ERR_INVALID, "null argument");
  Handle& H = hd->h;
  if (nrhs < 1 || nrhs > H.prm.max_rhs) return fail(ASP_ERR_INVALID, "nrhs out of range");
  if (r == z) return fail(ASP_ERR_INVALID, "r and z alias");
  return apply_precond(H, (const double2*)r, (double2*)z, nrhs, (cudaStream_t)stream);
}

int asp_matvec(asp_handle* hd, const void* x, void* y, int nrhs, void* stream) {
  if (!hd || !x || !y) return fail(ASP_ERR_INVALID, "null argument");
  Handle& H = hd->h;
  if (nrhs < 1 || nrhs > H.prm.max_rhs) return fail(ASP_ERR_INVALID, "nrhs out of range");
  if (x == y) return fail(ASP_ERR_INVALID, "x and y alias");
  PhaseTok tk = phase_begin(H, PH_MATVEC, (cudaStream_t)stream);
  cudaError_t ce = launch_matvec(H, (const double2*)x, (double2*)y, nrhs, (cudaStream_t)stream);
  phase_end(H, tk, (cudaStream_t)stream);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("matvec launch: ") + cudaGetErrorString(ce));
  return ASP_OK;
}

int asp_subproblem_width(const asp_handle* hd, int kind, int p) {
  if (!hd) return ASP_ERR_INVALID;
  const Handle& H = hd->h;
  if (p < 1 || p > H.m) return ASP_ERR_INVALID;
  int idx = kind == KIND_M ? H.subM[p] : kind == KIND_R ? H.subR[p] : kind == KIND_L ? H.subL[p] : -1;
  if (idx < 0) return ASP_ERR_INVALID;
  return H.dim == 3 ? H.slabs[idx].w : H.subs[idx].w;
}

int asp_subproblem_solve(asp_handle* hd, int kind, int p, const void* g, void* v, int nrhs, void* stream) {
  if (!hd || !g || !v) return fail(ASP_ERR_INVALID, "null argument");
  Handle& H = hd->h;
  if (!H.factored) return fail(ASP_ERR_STATE, "subproblem solve before factor");
  if (nrhs < 1 || nrhs > H.prm.max_rhs) return fail(ASP_ERR_INVALID, "nrhs out of range");
  if (p < 1 || p > H.m) return fail(ASP_ERR_INVALID, "layer index out of range");
  int idx = kind == KIND_M ? H.subM[p] : kind == KIND_R ? H.subR[p] : kind == KIND_L ? H.subL[p] : -1;
  if (idx < 0) return fail(ASP_ERR_INVALID, "no such subproblem (H^R needs p >= 2, H^L needs p <= m-1)");
  cudaStream_t s = (cudaStream_t)stream;
  if (H.dim == 3) return subsolve3d(H, idx, (const double2*)g, (double2*)v, nrhs, s);
  const int w = H.subs[idx].w;
  const void* in = g;
  if (H.prec == ASP_PREC_C64) {
    if (launch_to_prec((const double2*)g, H.r_lo, (long long)w * H.n * nrhs, H.prec, s) != cudaSuccess)
      return fail(ASP_ERR_CUDA, "to_prec launch");
    in = H.r_lo;
  }
  const int cap = nrhs >= 4 ? 4 : 1;
  JobCache& jc = cache_of(&H);
  const long long key = (long long)idx * 1024 + nrhs;
  auto it = jc.sub.find(key);
  if (it == jc.sub.end()) {
    std::vector<Job> jobs;
    for (int r0 = 0; r0 < nrhs; r0 += cap) jobs.push_back({idx, MODE_SUB, r0, std::min(cap, nrhs - r0)});
    JobList L0;
    int rc = upload_jobs(H, jobs, cap, w, &L0);
    if (rc != ASP_OK) return rc;
    it = jc.sub.emplace(key, L0).first;
  }
  const JobList& L = it->second;
  SolveParams P = base_params(H, nrhs);
  P.in = in;
  P.outSub = v;
  P.jobs = L.d;
  P.njobs = L.n;
  cudaError_t ce = launch_btsolve_aux(H, P, CLS_SUB, cap, w, s);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("subproblem launch: ") + cudaGetErrorString(ce));
  return ASP_OK;
}

int asp_gmres_solve(asp_handle* hd, const void* f, void* u, int nrhs, double tol, int restart, int maxit,
                    asp_solve_info* info_host, void* stream) {
  if (!hd || !f || !u) return fail(ASP_ERR_INVALID, "null argument");
  Handle& H = hd->h;
  if (!H.factored) return fail(ASP_ERR_STATE, "solve before factor");
  if (nrhs < 1 || nrhs > H.prm.max_rhs) return fail(ASP_ERR_INVALID, "nrhs out of range");
  if (restart < 1 || restart > H.prm.restart) return fail(ASP_ERR_INVALID, "restart exceeds the setup value");
  if (maxit < 1 || !(tol >= 0)) return fail(ASP_ERR_INVALID, "maxit must be >= 1 and tol >= 0");
  if (f == u) return fail(ASP_ERR_INVALID, "f and u alias");
  int rc = gmres_run(H, (const double2*)f, (double2*)u, nrhs, tol, restart, maxit, info_host, (cudaStream_t)stream);
  if (rc != ASP_OK && rc != ASP_ERR_NOT_CONVERGED) return rc;
  int rc2 = check_err(H, (cudaStream_t)stream, "fgmres");
  return rc2 != ASP_OK ? rc2 : rc;
}

long long asp_take_launch_count(asp_handle* hd) {
  if (!hd) return 0;
  long long v = hd->h.launches;
  hd->h.launches = 0;
  return v;
}

int asp_testhook_fail_device_alloc(int after) {
  g_alloc_fail_after.store(after < 0 ? -1 : after);
  return ASP_OK;
}

int asp_selftest_bounded_wait(int polls, void* stream) {
  if (polls < 1 || polls > (int)(1u << 26)) return fail(ASP_ERR_INVALID, "polls out of range");
  cudaStream_t s = (cudaStream_t)stream;
  int* d_err = nullptr;
  if (cudaMalloc(&d_err, 2 * sizeof(int)) != cudaSuccess) return fail(ASP_ERR_OOM, "self-test error word");
  int e[2] = {0, 0};
  cudaError_t ce = cudaMemsetAsync(d_err, 0, 2 * sizeof(int), s);
  if (ce == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(d_err, (uint32_t)polls);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(e, d_err, sizeof(e), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("self-test: ") + cudaGetErrorString(ce));
  if (e[0] == ASP_ERR_TIMEOUT) return fail(ASP_ERR_TIMEOUT, "self-test: the bounded wait gave up, as designed");
  return e[0];
}

}  // extern "C"
