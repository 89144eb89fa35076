// noalloc.cu -- asp_residual_norms_noalloc: the residual check of the solver
// (rel_res[r] = ||f_r - A u_r|| / ||f_r||) for callers that cannot allocate
// device memory.
//
// Who needs it: a process whose device memory is owned by another allocator
// (a framework's caching pool or a fixed arena that must account for every
// byte), or a steady-state serving loop that is not allowed to allocate at
// all once it runs.  Such a caller owns f, u and the output and only needs to
// know how good a solution is; the handle-based path would have to allocate
// its coefficient arrays and reduction buffers in asp_setup.
//
// This entry point needs no handle: it recomputes the stencil weights of
// Eq. (4) on the device and keeps them, together with the per-block partial
// sums and a flag for an invalid velocity, in one file-scope device array of
// fixed size (kScratchBytes below, about 0.7 MB).  Every GPU that loads the
// library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it; that first call should therefore come before
// any stream capture.  All calls share the one array: calls that overlap on the
// GPU (different streams, or different host threads without ordering) race and
// may return wrong values.  Each call rewrites every scratch entry it reads and
// clears the velocity flag first, so nothing carries over from one call to the
// next.
#include <math.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kMaxN = ASP_NOALLOC_MAX_N;
constexpr int kMaxRhs = ASP_NOALLOC_MAX_RHS;
constexpr int kBlocks = 512;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

struct Scratch {
  double2 ca[kMaxN];                 // s_k s_{k-1/2} / h^2
  double2 cc[kMaxN];                 // s_k s_{k+1/2} / h^2
  double2 cd[kMaxN];                 // -(ca + cc)
  double2 partial[kBlocks][kMaxRhs];  // per block: (sum |r|^2, sum |f|^2)
  int bad_velocity;                   // set when some c is not positive and finite
};
constexpr size_t kScratchBytes = sizeof(Scratch);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
Scratch* g_addr[kMaxDevices] = {nullptr};

// s = 1 / (1 + i sigma/omega) with sigma = (C/eta)(d/eta)^2 at distance d past
// the physical interval [gamma h, (n+1-gamma) h] (the boundary PML of Section 2).
__device__ double2 pml_s(double x, int n, int gamma, double C, double omega) {
  const double h = 1.0 / (n + 1);
  const double eta = gamma * h, lo = gamma * h, hi = (n + 1 - gamma) * h;
  double d = 0.0;
  if (x < lo) d = lo - x;
  else if (x > hi) d = x - hi;
  const double sig = (C / eta) * (d / eta) * (d / eta);
  const double t = sig / omega;
  const double den = 1.0 + t * t;
  return make_double2(1.0 / den, -t / den);
}

__global__ void na_coef_kernel(int n, int gamma, double C, double omega, Scratch* S) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) S->bad_velocity = 0;  // this call's flag starts clear
  if (k >= n) return;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  const double x = (k + 1) * h;
  const double2 sk = pml_s(x, n, gamma, C, omega);
  const double2 sm = pml_s(x - 0.5 * h, n, gamma, C, omega);
  const double2 sp = pml_s(x + 0.5 * h, n, gamma, C, omega);
  double2 a = cmul(sk, sm), c = cmul(sk, sp);
  a.x *= ih2; a.y *= ih2;
  c.x *= ih2; c.y *= ih2;
  S->ca[k] = a;
  S->cc[k] = c;
  S->cd[k] = make_double2(-(a.x + c.x), -(a.y + c.y));
}

// Block sums of |f - A u|^2 and |f|^2 per right-hand side.  Threads keep one
// right-hand side r = tid % nrhs (block size and grid stride are multiples of
// nrhs).  A u is evaluated in the same operation order as the handle's
// matvec kernel.
__global__ void na_residual_kernel(const double* __restrict__ c, double omega, int n, int nrhs,
                                   const double2* __restrict__ f, const double2* __restrict__ u, Scratch* S) {
  __shared__ double2 red[kThreads];
  const int bt = blockDim.x, t = threadIdx.x;
  const long long total = (long long)n * n * nrhs;
  const long long rowst = (long long)n * nrhs;
  double rr = 0.0, ff = 0.0;
  for (long long e = (long long)blockIdx.x * bt + t; e < total; e += (long long)gridDim.x * bt) {
    const long long pt = e / nrhs;
    const int i1 = (int)(pt % n), i2 = (int)(pt / n);
    const double2 x = u[e];
    const double2 d1 = S->cd[i1], d2 = S->cd[i2];
    const double cv = c[pt];
    if (!(cv > 0.0) || !isfinite(cv)) S->bad_velocity = 1;
    const double k2 = omega * omega / (cv * cv);
    const double2 diag = make_double2(d1.x + d2.x + k2, d1.y + d2.y);
    double2 acc = cmul(diag, x);
    double2 acc2 = make_double2(0.0, 0.0);
    if (i1 > 0) cfma(acc, S->ca[i1], u[e - nrhs]);
    if (i2 > 0) cfma(acc2, S->ca[i2], u[e - rowst]);
    if (i1 < n - 1) cfma(acc, S->cc[i1], u[e + nrhs]);
    if (i2 < n - 1) cfma(acc2, S->cc[i2], u[e + rowst]);
    acc = make_double2(acc.x + acc2.x, acc.y + acc2.y);
    const double2 fe = f[e];
    const double2 r = make_double2(fe.x - acc.x, fe.y - acc.y);
    rr = fma(r.x, r.x, fma(r.y, r.y, rr));
    ff = fma(fe.x, fe.x, fma(fe.y, fe.y, ff));
  }
  red[t] = make_double2(rr, ff);
  __syncthreads();
  if (t < nrhs) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = t; q < bt; q += nrhs) { s.x += red[q].x; s.y += red[q].y; }
    S->partial[blockIdx.x][t] = s;
  }
}

__global__ void na_finish_kernel(int nblocks, int nrhs, const Scratch* S, double* rel) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double sr = 0.0, sf = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    sr += S->partial[b][r].x;
    sf += S->partial[b][r].y;
  }
  // a velocity that is not positive and finite has no operator: NaN for every right-hand side
  rel[r] = S->bad_velocity ? __longlong_as_double(0x7ff8000000000000LL) : (sf > 0.0 ? sqrt(sr / sf) : 0.0);
}

// Device address of g_scratch for the current device (looked up once per device).
int scratch_address(Scratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(ASP_ERR_UNSUPPORTED, "device index beyond the scratch table");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(ASP_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_addr[dev] = reinterpret_cast<Scratch*>(ptr);
  }
  *out = g_addr[dev];
  return ASP_OK;
}

}  // namespace

}  // namespace asp

using namespace asp;

extern "C" int asp_residual_norms_noalloc(const asp_params* p, const double* c, const void* f, const void* u,
                                          int nrhs, double* rel_res, void* stream) {
  if (!p || !c || !f || !u || !rel_res) return fail(ASP_ERR_INVALID, "null argument");
  if (p->dim != 2) return fail(ASP_ERR_UNSUPPORTED, "residual_norms_noalloc: dim must be 2");
  if (p->n < 3 || p->n > kMaxN)
    return fail(ASP_ERR_INVALID, "residual_norms_noalloc: n must be in [3, " + std::to_string(kMaxN) +
                                     "] (fixed scratch size)");
  if (nrhs < 1 || nrhs > kMaxRhs)
    return fail(ASP_ERR_INVALID, "residual_norms_noalloc: nrhs must be in [1, " + std::to_string(kMaxRhs) +
                                     "] (fixed scratch size)");
  if (!(p->omega > 0) || !isfinite(p->omega) || p->pml < 2 || 2 * p->pml > p->n + 1 || !(p->C > 0) ||
      !isfinite(p->C))
    return fail(ASP_ERR_INVALID, "residual_norms_noalloc: omega, pml or C out of range");
  Scratch* S = nullptr;
  int rc = scratch_address(&S);
  if (rc != ASP_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = p->n;
  na_coef_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, p->pml, p->C, p->omega, S);
  const int bt = nrhs * (kThreads / nrhs);
  na_residual_kernel<<<kBlocks, bt, 0, s>>>(c, p->omega, n, nrhs, (const double2*)f, (const double2*)u, S);
  na_finish_kernel<<<1, 64, 0, s>>>(kBlocks, nrhs, S, rel_res);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("residual_norms_noalloc launch: ") + cudaGetErrorString(e));
  return ASP_OK;
}
