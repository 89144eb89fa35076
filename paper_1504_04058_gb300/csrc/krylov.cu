// krylov.cu -- the FP64 outer solver: the 5-point PML operator A (Eq. (4) with
// the PML on all four sides, Section 3.2) and right-preconditioned flexible
// GMRES with restart (the Krylov solver of Section 3.2), with every vector
// operation on the device.
//
// Vectors are complex128 in the RHS-interleaved layout (element (point, r) at
// point*nrhs + r); each right-hand side has its own Krylov space.  Reductions
// are two-stage and in a fixed order, so results do not depend on scheduling.
// Arnoldi uses classical Gram-Schmidt (one pass, a second one on severe
// cancellation): equal to modified
// Gram-Schmidt in exact arithmetic and two passes over the basis instead of j;
// the second pass runs only on severe cancellation (reorth_check_kernel).
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asp {

int apply_precond(Handle& H, const double2* r, double2* z, int nrhs, cudaStream_t s);

namespace {

constexpr int kVecThreads = 256;
constexpr int kDotChunk = 8;

__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return cmul(a, b); }

// ------------------------------------------------------------------ matvec
// (Au)_{i1,i2} = a_{i1} u_{i1-1} + c_{i1} u_{i1+1} + a_{i2} u_{i2-1} + c_{i2} u_{i2+1}
//                + (d_{i1} + d_{i2} + omega^2/c^2) u,  zero outside the grid.
// One launch covers a region of the grid: rows r0 + blockIdx.y and columns
// c0 + (element / nrhs), each skipping a gap [skip_lo, skip_lo + skip_n) of
// indices, so that the interior box and the PML frame around it are separate
// launches.  REAL: every coefficient of the region is real (sigma = 0, outside
// the PML), and the products are real-by-complex, half the FP64 operations of
// the complex products and the same values (up to the sign of zero results).
// NRT is the number of right-hand sides when it is a compile-time constant
// (0: runtime `nrhs`), so that the point index needs no runtime division.
struct MvRegion {
  int r0, rskip_lo, rskip_n;  // rows: r0 + y, then + rskip_n from rskip_lo on
  int c0, ncols, cskip_lo, cskip_n;
};

template <int NRT, bool REAL>
__global__ void matvec_kernel(const double* __restrict__ dgre, const double2* __restrict__ ca,
                              const double2* __restrict__ cc, const double2* __restrict__ cd, int n,
                              int nrhs_rt, const double2* __restrict__ x, double2* __restrict__ y, MvRegion g) {
  const int nr = NRT > 0 ? NRT : nrhs_rt;
  const int er = blockIdx.x * blockDim.x + threadIdx.x;  // element within the region's row
  if (er >= g.ncols * nr) return;
  int i2 = g.r0 + (int)blockIdx.y;
  if (i2 >= g.rskip_lo) i2 += g.rskip_n;
  int i1 = g.c0 + er / nr;
  if (i1 >= g.cskip_lo) i1 += g.cskip_n;
  const int r = er - (er / nr) * nr;
  const long long rowst = (long long)n * nr;
  const long long e = (long long)i2 * rowst + (long long)i1 * nr + r;
  const double2 u = x[e];
  const double2 a1 = ca[i1], c1 = cc[i1], a2 = ca[i2], c2 = cc[i2];
  const double dg = dgre[(long long)i2 * n + i1];  // Re(d_{i1} + d_{i2}) + omega^2/c^2
  // one accumulator: the FP64 pipe, not the dependent chain, bounds this kernel
  double2 acc;
  if constexpr (REAL) {
    acc = make_double2(dg * u.x, dg * u.y);
    if (i1 > 0) { const double2 v = x[e - nr]; acc.x = fma(a1.x, v.x, acc.x); acc.y = fma(a1.x, v.y, acc.y); }
    if (i2 > 0) { const double2 v = x[e - rowst]; acc.x = fma(a2.x, v.x, acc.x); acc.y = fma(a2.x, v.y, acc.y); }
    if (i1 < n - 1) { const double2 v = x[e + nr]; acc.x = fma(c1.x, v.x, acc.x); acc.y = fma(c1.x, v.y, acc.y); }
    if (i2 < n - 1) { const double2 v = x[e + rowst]; acc.x = fma(c2.x, v.x, acc.x); acc.y = fma(c2.x, v.y, acc.y); }
  } else {
    const double2 diag = make_double2(dg, cd[i1].y + cd[i2].y);
    acc = dmul(diag, u);
    if (i1 > 0) cfma(acc, a1, x[e - nr]);
    if (i2 > 0) cfma(acc, a2, x[e - rowst]);
    if (i1 < n - 1) cfma(acc, c1, x[e + nr]);
    if (i2 < n - 1) cfma(acc, c2, x[e + rowst]);
  }
  y[e] = acc;
}

struct VecList {
  const double2* v[kDotChunk];
};

// Reductions over a vector of `count` = points*nrhs elements use blocks of
// bt = nrhs*floor(256/nrhs) threads and a grid stride that is a multiple of
// nrhs, so each thread always sees the same right-hand side r = tid % nrhs.
//
// partial[b][j][r] = this block's sum of conj(v_j) * w for j < J, and, when
// want_norm, partial[b][kDotChunk][r] = its sum of |w|^2.
// EU elements per thread and loop iteration: independent FP64 chains in flight
// (GB300 issues FP64 at 1/58 of the FP32 rate with a long result latency, so
// a single dependent chain per thread leaves the FP64 pipe idle).
// gate != nullptr: the launch does nothing when *gate == 0 (a pass that the
// device decided to skip, so the host need not wait for the decision).
template <int EU>
__global__ void gs_dot_kernel(VecList V, int J, int want_norm, const double2* __restrict__ w, long long count,
                              int nrhs, double2* __restrict__ partial, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ double2 red[kVecThreads];
  const int bt = blockDim.x;
  const int t = threadIdx.x;
  constexpr int JM = (EU >= 4) ? 2 : (EU == 2 ? 4 : kDotChunk);  // vectors handled per pass at this unroll
  double2 acc[EU][JM + 1];
#pragma unroll
  for (int u = 0; u < EU; ++u)
#pragma unroll
    for (int j = 0; j <= JM; ++j) acc[u][j] = make_double2(0, 0);
  const long long stride = (long long)gridDim.x * bt;
  for (long long e0 = (long long)blockIdx.x * bt + t; e0 < count; e0 += EU * stride) {
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long e = e0 + u * stride;
      if (e < count) {
        const double2 we = w[e];
#pragma unroll
        for (int j = 0; j < JM; ++j)
          if (j < J) {
            const double2 v = V.v[j][e];
            acc[u][j].x = fma(v.x, we.x, fma(v.y, we.y, acc[u][j].x));
            acc[u][j].y = fma(v.x, we.y, fma(-v.y, we.x, acc[u][j].y));
          }
        if (want_norm) acc[u][JM].x = fma(we.x, we.x, fma(we.y, we.y, acc[u][JM].x));
      }
    }
  }
#pragma unroll
  for (int j = 0; j <= JM; ++j) {
    if (j < J || (j == JM && want_norm)) {
      double2 sum = acc[0][j];
#pragma unroll
      for (int u = 1; u < EU; ++u) { sum.x += acc[u][j].x; sum.y += acc[u][j].y; }
      red[t] = sum;
      __syncthreads();
      if (t < nrhs) {
        double2 s = make_double2(0, 0);
        for (int q = t; q < bt; q += nrhs) { s.x += red[q].x; s.y += red[q].y; }
        partial[((long long)blockIdx.x * (kDotChunk + 1) + (j == JM ? kDotChunk : j)) * nrhs + t] = s;
      }
      __syncthreads();
    }
  }
}

// out[j0 + j][r] = sum_b partial[b][j][r] for j < J, and nrm[r] = sum_b
// partial[b][kDotChunk][r] when nrm != nullptr (fixed block order).
__global__ void dot_finish_kernel(const double2* __restrict__ partial, int nblocks, int J, int nrhs, int j0,
                                  double2* __restrict__ out, double2* __restrict__ nrm, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int slots = J + (nrm ? 1 : 0);
  if (idx >= slots * nrhs) return;
  const int jj = idx / nrhs, r = idx % nrhs;
  const int j = jj < J ? jj : kDotChunk;
  double2 s = make_double2(0, 0);
  for (int b = 0; b < nblocks; ++b) {
    const double2 v = partial[((long long)b * (kDotChunk + 1) + j) * nrhs + r];
    s.x += v.x; s.y += v.y;
  }
  if (jj < J) out[(long long)(j0 + jj) * nrhs + r] = s;
  else nrm[r] = s;
}

// w[e] += sgn * sum_j coef[(j0+j)][r] * v_j[e]; with want_norm also the block
// sums of |w_new|^2 in partial[b][kDotChunk][r].
// four elements per thread and iteration, and the J terms of each element in
// two independent partial sums, so several FP64 chains are in flight
__global__ void gs_axpy_kernel(VecList V, int J, const double2* __restrict__ coef, int j0, double sgn,
                               double2* __restrict__ w, long long count, int nrhs, int want_norm,
                               double2* __restrict__ partial, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  constexpr int EU = 4;
  __shared__ double2 red[kVecThreads];
  const int bt = blockDim.x;
  const int t = threadIdx.x;
  const int r = t % nrhs;
  double2 c[kDotChunk];
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) {
    c[j] = make_double2(0, 0);
    if (j < J) {
      const double2 cj = coef[(long long)(j0 + j) * nrhs + r];
      c[j] = make_double2(sgn * cj.x, sgn * cj.y);
    }
  }
  double nacc[EU] = {0.0};
  const long long stride = (long long)gridDim.x * bt;
  for (long long e0 = (long long)blockIdx.x * bt + t; e0 < count; e0 += EU * stride) {
    double2 a0[EU], a1[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) { a0[u] = make_double2(0, 0); a1[u] = make_double2(0, 0); }
#pragma unroll
    for (int j = 0; j < kDotChunk; j += 2) {
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const long long e = e0 + u * stride;
        if (e < count) {
          if (j < J) cfma(a0[u], c[j], V.v[j][e]);
          if (j + 1 < J) cfma(a1[u], c[j + 1], V.v[j + 1][e]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long e = e0 + u * stride;
      if (e < count) {
        double2 acc = w[e];
        acc.x += a0[u].x + a1[u].x;
        acc.y += a0[u].y + a1[u].y;
        w[e] = acc;
        if (want_norm) nacc[u] = fma(acc.x, acc.x, fma(acc.y, acc.y, nacc[u]));
      }
    }
  }
  if (want_norm) {
    double nsum = 0.0;
#pragma unroll
    for (int u = 0; u < EU; ++u) nsum += nacc[u];
    red[t] = make_double2(nsum, 0.0);
    __syncthreads();
    if (t < nrhs) {
      double2 s = make_double2(0, 0);
      for (int q = t; q < bt; q += nrhs) s.x += red[q].x;
      partial[((long long)blockIdx.x * (kDotChunk + 1) + kDotChunk) * nrhs + t] = s;
    }
  }
}

// dst[e] = src[e] * s[r]  (s real); same thread layout as the reductions
__global__ void scale_kernel(const double2* __restrict__ src, const double* __restrict__ sc,
                             double2* __restrict__ dst, long long count, int nrhs) {
  const int bt = blockDim.x;
  const double s = sc[threadIdx.x % nrhs];
  for (long long e = (long long)blockIdx.x * bt + threadIdx.x; e < count; e += (long long)gridDim.x * bt) {
    const double2 v = src[e];
    dst[e] = make_double2(v.x * s, v.y * s);
  }
}

// dst = a - b
__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ dst,
                           long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 x = a[e], y = b[e];
    dst[e] = make_double2(x.x - y.x, x.y - y.y);
  }
}

// Per-right-hand-side Krylov state (all arrays [...][nrhs]).
struct KState {
  double2* h1;    // [restart+1][nrhs]  first CGS pass
  double2* h2;    // [restart+1][nrhs]  second CGS pass
  double2* hn2;   // [1][nrhs]  ||w||^2 after orthogonalization (re)
  double2* nrm0;  // [1][nrhs]  ||w||^2 before orthogonalization (re)
  double2* Rm;    // [restart][restart+1][nrhs]  rotated Hessenberg columns
  double* cs;     // [restart][nrhs]
  double2* sn;    // [restart][nrhs]
  double2* g;     // [restart+1][nrhs]
  double2* y;     // [restart][nrhs]
  double* fnorm;  // [nrhs]
  double* est;    // [nrhs]
  double* inv;    // [nrhs] scale for the next basis vector
  int* done;      // [nrhs] 1 once converged (or broke down)
  int* kcur;      // [nrhs] columns in the current cycle
  int* its;       // [nrhs] iterations until done
  int* active;    // [1] number of right-hand sides still iterating
  int* need;      // [1] number of right-hand sides that need a second Gram-Schmidt pass
};

// Start of a restart cycle: beta = ||r||, g = [beta, 0..], inv = 1/beta.
// On the first cycle also records ||f|| (r = f there).
__global__ void cycle_start_kernel(KState K, int nrhs, int first, double tol) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double beta = sqrt(K.hn2[r].x);
  if (first) {
    K.fnorm[r] = beta;
    K.done[r] = (beta == 0.0);
    K.its[r] = 0;
    K.est[r] = beta == 0.0 ? 0.0 : 1.0;
  }
  K.kcur[r] = 0;
  K.g[r] = make_double2(K.done[r] ? 0.0 : beta, 0.0);
  K.inv[r] = (K.done[r] || beta == 0.0) ? 0.0 : 1.0 / beta;
}

// Column j of the Hessenberg matrix: h = h1 + h2 (rows 0..j), h_{j+1} = ||w||.
// Applies the previous Givens rotations, forms the new one, updates g and the
// residual estimate, and decides convergence.
__global__ void arnoldi_update_kernel(KState K, int nrhs, int j, int restart, double tol, int its_now) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double hn = sqrt(K.hn2[r].x);
  if (K.done[r]) {
    K.inv[r] = 0.0;
    return;
  }
  double2* col = K.Rm + (long long)j * (restart + 1) * nrhs;
  for (int i = 0; i <= j; ++i) {
    double2 a = K.h1[(long long)i * nrhs + r], b = K.h2[(long long)i * nrhs + r];
    col[(long long)i * nrhs + r] = make_double2(a.x + b.x, a.y + b.y);
  }
  double2 hj1 = make_double2(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const double c = K.cs[(long long)i * nrhs + r];
    const double2 s = K.sn[(long long)i * nrhs + r];
    const double2 hi = col[(long long)i * nrhs + r];
    const double2 hi1 = (i + 1 == j + 1) ? hj1 : col[(long long)(i + 1) * nrhs + r];
    // [c s; -conj(s) c] [hi; hi1]
    double2 t = make_double2(c * hi.x, c * hi.y);
    cfma(t, s, hi1);
    double2 u = make_double2(c * hi1.x, c * hi1.y);
    const double2 sc = make_double2(s.x, -s.y);
    cfms(u, sc, hi);
    col[(long long)i * nrhs + r] = t;
    col[(long long)(i + 1) * nrhs + r] = u;
  }
  const double2 a = col[(long long)j * nrhs + r];
  const double2 b = hj1;
  double c;
  double2 s;
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  if (bb == 0.0) {
    c = 1.0; s = make_double2(0, 0);
  } else if (aa == 0.0) {
    c = 0.0; s = make_double2(b.x / bb, -b.y / bb);
  } else {
    const double rho = hypot(aa, bb);
    c = aa / rho;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    const double2 cb = make_double2(b.x / rho, -b.y / rho);
    s = cmul(ph, cb);
  }
  // new diagonal: c a + s b
  double2 d = make_double2(c * a.x, c * a.y);
  cfma(d, s, b);
  col[(long long)j * nrhs + r] = d;
  col[(long long)(j + 1) * nrhs + r] = make_double2(0, 0);
  K.cs[(long long)j * nrhs + r] = c;
  K.sn[(long long)j * nrhs + r] = s;
  const double2 gj = K.g[(long long)j * nrhs + r];
  const double2 sc = make_double2(s.x, -s.y);
  double2 gj1 = cmul(sc, gj);
  gj1.x = -gj1.x; gj1.y = -gj1.y;
  K.g[(long long)(j + 1) * nrhs + r] = gj1;
  K.g[(long long)j * nrhs + r] = make_double2(c * gj.x, c * gj.y);
  K.kcur[r] = j + 1;
  const double est = hypot(gj1.x, gj1.y) / K.fnorm[r];
  K.est[r] = est;
  bool stop = (tol > 0.0 && est <= tol) || hn == 0.0;
  if (stop) {
    K.done[r] = 1;
    K.its[r] = its_now;
  }
  K.inv[r] = (stop || hn == 0.0) ? 0.0 : 1.0 / hn;
}

// A second Gram-Schmidt pass is needed only where the first one cancelled
// severely: ||w'|| < 1e-3 ||w||.  In FP64 a single classical pass leaves the
// new basis vector orthogonal to about eps ||w|| / ||w'||, i.e. 1e-13 or better
// under this threshold, far below the solver tolerances; with the preconditioner
// A M^-1 close to the identity, ||w'|| / ||w|| is the per-step residual
// reduction, so the classical 1/sqrt(2) threshold would fire every iteration.
// ||w||^2 is recovered as ||w'||^2 + sum_i |h_i|^2 (Pythagoras), so the first
// pass needs no extra norm.
__global__ void reorth_check_kernel(KState K, int nrhs, int j) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int c = 0;
    for (int r = 0; r < nrhs; ++r) {
      if (K.done[r]) continue;
      double sh = 0.0;
      for (int i = 0; i <= j; ++i) {
        const double2 h = K.h1[(long long)i * nrhs + r];
        sh += h.x * h.x + h.y * h.y;
      }
      const double w2 = K.hn2[r].x;
      if (w2 < 1e-6 * (w2 + sh)) ++c;
    }
    *K.need = c;
  }
}

__global__ void count_active_kernel(KState K, int nrhs) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int a = 0;
    for (int r = 0; r < nrhs; ++r) a += K.done[r] ? 0 : 1;
    *K.active = a;
  }
}

// y = R^{-1} g per right-hand side (k = kcur[r] columns); entries >= k are 0.
__global__ void ysolve_kernel(KState K, int nrhs, int restart) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int k = K.kcur[r];
  for (int i = restart - 1; i >= 0; --i) {
    if (i >= k) {
      K.y[(long long)i * nrhs + r] = make_double2(0, 0);
      continue;
    }
    double2 acc = K.g[(long long)i * nrhs + r];
    for (int l = i + 1; l < k; ++l) {
      const double2 Ril = K.Rm[((long long)l * (restart + 1) + i) * nrhs + r];
      cfms(acc, Ril, K.y[(long long)l * nrhs + r]);
    }
    const double2 Rii = K.Rm[((long long)i * (restart + 1) + i) * nrhs + r];
    K.y[(long long)i * nrhs + r] = cmul(acc, crecip(Rii));
  }
}

int grid_for(long long count, int threads, int sms) {
  long long g = (count + threads - 1) / threads;
  long long cap = (long long)sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <int NRT>
void matvec_regions(const Handle& H, const double2* x, double2* y, int nrhs, cudaStream_t s) {
  const int n = H.n;
  const int lo = H.real_lo, nb = H.real_hi - H.real_lo;
  auto go = [&](bool real, int nrows, const MvRegion& g) {
    const long long per_row = (long long)g.ncols * nrhs;
    if (nrows <= 0 || per_row <= 0) return;
    dim3 grid((unsigned)((per_row + kVecThreads - 1) / kVecThreads), (unsigned)nrows);
    if (real)
      matvec_kernel<NRT, true><<<grid, kVecThreads, 0, s>>>(H.dgre, H.ca, H.cc, H.cd, n, nrhs, x, y, g);
    else
      matvec_kernel<NRT, false><<<grid, kVecThreads, 0, s>>>(H.dgre, H.ca, H.cc, H.cd, n, nrhs, x, y, g);
    const_cast<Handle&>(H).launches += 1;
  };
  const int kNone = 1 << 30;
  if (nb <= 0) {
    go(false, n, MvRegion{0, kNone, 0, 0, n, kNone, 0});
    return;
  }
  go(true, nb, MvRegion{lo, kNone, 0, lo, nb, kNone, 0});          // interior box, real coefficients
  go(false, n - nb, MvRegion{0, lo, nb, 0, n, kNone, 0});           // rows outside the box
  go(false, nb, MvRegion{lo, kNone, 0, 0, n - nb, lo, nb});         // the box rows' PML columns
}

cudaError_t launch_matvec(const Handle& H, const double2* x, double2* y, int nrhs, cudaStream_t s) {
  if (H.dim == 3) return launch_matvec3d(H, x, y, nrhs, s);
  switch (nrhs) {
    case 1: matvec_regions<1>(H, x, y, nrhs, s); break;
    case 2: matvec_regions<2>(H, x, y, nrhs, s); break;
    case 4: matvec_regions<4>(H, x, y, nrhs, s); break;
    case 8: matvec_regions<8>(H, x, y, nrhs, s); break;
    case 16: matvec_regions<16>(H, x, y, nrhs, s); break;
    case 32: matvec_regions<32>(H, x, y, nrhs, s); break;
    default: matvec_regions<0>(H, x, y, nrhs, s); break;
  }
  return cudaGetLastError();
}

namespace {

struct Krylov {
  Handle& H;
  int nrhs, restart;
  long long count;
  cudaStream_t s;
  KState K;
  int red_blocks, red_threads;
  double2* partial;

  double2* Vv(int i) const { return H.V + (long long)i * count; }
  double2* Zv(int i) const { return H.Z + (long long)i * count; }

  // out[j][r] = conj(V_j)^T w for j < J (chunks of kDotChunk); nrm[r] = ||w||^2
  // when nrm != nullptr (computed with the first chunk, or alone when J == 0).
  // gate: see gs_dot_kernel.
  cudaError_t dots(const double2* const* vs, int J, const double2* w, double2* out, double2* nrm,
                   const int* gate = nullptr) {
    // small J: more elements per thread; chunks of at most JM vectors per pass
    const int JM = J <= 2 ? 2 : (J <= 4 ? 4 : kDotChunk);
    for (int j0 = 0; j0 < J || (J == 0 && j0 == 0); j0 += JM) {
      VecList L{};
      const int Jc = std::max(0, std::min(JM, J - j0));
      for (int j = 0; j < Jc; ++j) L.v[j] = vs[j0 + j];
      for (int j = Jc; j < kDotChunk; ++j) L.v[j] = w;
      double2* nr = (j0 == 0) ? nrm : nullptr;
      if (JM == 2)
        gs_dot_kernel<4><<<red_blocks, red_threads, 0, s>>>(L, Jc, nr ? 1 : 0, w, count, nrhs, partial, gate);
      else if (JM == 4)
        gs_dot_kernel<2><<<red_blocks, red_threads, 0, s>>>(L, Jc, nr ? 1 : 0, w, count, nrhs, partial, gate);
      else
        gs_dot_kernel<1><<<red_blocks, red_threads, 0, s>>>(L, Jc, nr ? 1 : 0, w, count, nrhs, partial, gate);
      const int slots = Jc + (nr ? 1 : 0);
      dot_finish_kernel<<<(slots * nrhs + 127) / 128, 128, 0, s>>>(partial, red_blocks, Jc, nrhs, j0, out, nr, gate);
      H.launches += 2;
      if (J == 0) break;
    }
    return cudaGetLastError();
  }
  // w += sgn * sum_j coef[j] V_j; nrm[r] = ||w_new||^2 when nrm != nullptr
  cudaError_t axpys(const double2* const* vs, int J, const double2* coef, double sgn, double2* w, double2* nrm,
                    const int* gate = nullptr) {
    for (int j0 = 0; j0 < J; j0 += kDotChunk) {
      VecList L{};
      const int Jc = std::min(kDotChunk, J - j0);
      for (int j = 0; j < Jc; ++j) L.v[j] = vs[j0 + j];
      for (int j = Jc; j < kDotChunk; ++j) L.v[j] = vs[j0];
      const bool last = j0 + kDotChunk >= J;
      const bool want = last && nrm;
      gs_axpy_kernel<<<red_blocks, red_threads, 0, s>>>(L, Jc, coef, j0, sgn, w, count, nrhs, want ? 1 : 0, partial,
                                                        gate);
      H.launches += 1;
      if (want) {
        dot_finish_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(partial, red_blocks, 0, nrhs, 0, nullptr, nrm, gate);
        H.launches += 1;
      }
    }
    return cudaGetLastError();
  }
  cudaError_t scale(const double2* src, const double* sc, double2* dst) {
    scale_kernel<<<red_blocks, red_threads, 0, s>>>(src, sc, dst, count, nrhs);
    H.launches += 1;
    return cudaGetLastError();
  }
};

}  // namespace

int gmres_run(Handle& H, const double2* f, double2* u, int nrhs, double tol, int restart, int maxit,
              asp_solve_info* info, cudaStream_t s) {
  Krylov G{H, nrhs, restart, H.N * nrhs, s, {}, 0, 0, nullptr};
  // carve the Krylov state out of the handle's blob
  {
    const int R = H.prm.restart;
    double2* p2 = H.hess;
    auto take2 = [&](long long cnt) { double2* q = p2; p2 += cnt; return q; };
    G.K.h1 = take2((long long)(R + 1) * nrhs);
    G.K.h2 = take2((long long)(R + 1) * nrhs);
    G.K.hn2 = take2(nrhs);
    G.K.nrm0 = take2(nrhs);
    G.K.Rm = take2((long long)R * (R + 1) * nrhs);
    G.K.sn = take2((long long)R * nrhs);
    G.K.g = take2((long long)(R + 1) * nrhs);
    G.K.y = take2((long long)R * nrhs);
    double* pd = H.kstate;
    G.K.cs = pd; pd += (long long)R * nrhs;
    G.K.fnorm = pd; pd += nrhs;
    G.K.est = pd; pd += nrhs;
    G.K.inv = pd; pd += nrhs;
    int* pi = H.kflags;
    G.K.done = pi; pi += nrhs;
    G.K.kcur = pi; pi += nrhs;
    G.K.its = pi; pi += nrhs;
    G.K.active = pi; pi += 1;
    G.K.need = pi;
  }
  G.red_threads = nrhs * std::max(1, kVecThreads / nrhs);
  G.red_blocks = H.num_sms * 2;
  G.partial = reinterpret_cast<double2*>(H.red);
  const long long count = G.count;
  const int gv = grid_for(count, kVecThreads, H.num_sms);
  const int gr = (nrhs + 127) / 128;
  cudaError_t ce = cudaSuccess;
#define CK(x)                                                                              \
  do {                                                                                     \
    ce = (x);                                                                              \
    if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("fgmres: ") + cudaGetErrorString(ce)); \
  } while (0)

  CK(cudaMemsetAsync(u, 0, sizeof(double2) * count, s));
  int its = 0;
  bool first = true;
  std::vector<const double2*> vl(restart + 1);
  int rc = ASP_OK;
  int active = nrhs;
  while (true) {
    // r = f - A u (u = 0 on the first cycle, so r = f)
    const double2* rvec = f;
    if (!first) {
      CK(launch_matvec(H, u, H.wv, nrhs, s));
      sub_kernel<<<gv, kVecThreads, 0, s>>>(f, H.wv, H.wv, count);
      H.launches += 1;
      rvec = H.wv;
    }
    CK(G.dots(nullptr, 0, rvec, nullptr, G.K.hn2));
    cycle_start_kernel<<<gr, 128, 0, s>>>(G.K, nrhs, first ? 1 : 0, tol);
    H.launches += 1;
    CK(G.scale(rvec, G.K.inv, G.Vv(0)));
    first = false;
    int jrun = 0;  // Arnoldi steps of this cycle: no right-hand side has more columns
    for (int j = 0; j < restart && its < maxit; ++j) {
      rc = apply_precond(H, G.Vv(j), G.Zv(j), nrhs, s);
      if (rc != ASP_OK) return rc;
      double2* w = G.Vv(j + 1);
      PhaseTok tmv = phase_begin(H, PH_MATVEC, s);
      CK(launch_matvec(H, G.Zv(j), w, nrhs, s));
      phase_end(H, tmv, s);
      PhaseTok tkr = phase_begin(H, PH_KRYLOV, s);
      for (int i = 0; i <= j; ++i) vl[i] = G.Vv(i);
      // classical Gram-Schmidt, a second pass only where cancellation demands it
      CK(G.dots(vl.data(), j + 1, w, G.K.h1, nullptr));
      CK(G.axpys(vl.data(), j + 1, G.K.h1, -1.0, w, G.K.hn2));
      reorth_check_kernel<<<1, 32, 0, s>>>(G.K, nrhs, j);
      H.launches += 1;
      // the second pass is enqueued always and runs only where the device found
      // that some right-hand side needs it (K.need > 0); skipped, h2 stays 0 and
      // w and ||w||^2 keep the first pass's values
      CK(cudaMemsetAsync(G.K.h2, 0, sizeof(double2) * (j + 1) * nrhs, s));
      CK(G.dots(vl.data(), j + 1, w, G.K.h2, nullptr, G.K.need));
      CK(G.axpys(vl.data(), j + 1, G.K.h2, -1.0, w, G.K.hn2, G.K.need));
      ++its;
      jrun = j + 1;
      arnoldi_update_kernel<<<gr, 128, 0, s>>>(G.K, nrhs, j, H.prm.restart, tol, its);
      H.launches += 1;
      CK(G.scale(w, G.K.inv, w));
      count_active_kernel<<<1, 32, 0, s>>>(G.K, nrhs);
      H.launches += 1;
      phase_end(H, tkr, s);
      CK(cudaMemcpyAsync(H.h_flags, G.K.active, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      active = H.h_flags[0];
      if (active == 0) break;
    }
    // u += Z y  (per right-hand side, its own number of columns; y is zero
    // past them, so only the cycle's jrun basis vectors are read)
    ysolve_kernel<<<gr, 128, 0, s>>>(G.K, nrhs, H.prm.restart);
    H.launches += 1;
    std::vector<const double2*> zl(std::max(jrun, 1));
    for (int i = 0; i < jrun; ++i) zl[i] = G.Zv(i);
    if (jrun > 0) CK(G.axpys(zl.data(), jrun, G.K.y, 1.0, u, nullptr));
    if (active == 0 || its >= maxit) break;
  }
  // true residual ||f - A u|| / ||f||
  CK(launch_matvec(H, u, H.wv, nrhs, s));
  sub_kernel<<<gv, kVecThreads, 0, s>>>(f, H.wv, H.wv, count);
  H.launches += 1;
  CK(G.dots(nullptr, 0, H.wv, nullptr, G.K.hn2));
  std::vector<double2> hn2(nrhs);
  std::vector<double> fn(nrhs), est(nrhs);
  std::vector<int> done(nrhs), itv(nrhs);
  CK(cudaMemcpyAsync(hn2.data(), G.K.hn2, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(fn.data(), G.K.fnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(est.data(), G.K.est, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(done.data(), G.K.done, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(itv.data(), G.K.its, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
#undef CK
  bool all = true;
  for (int r = 0; r < nrhs; ++r) {
    const double rel = fn[r] > 0 ? sqrt(hn2[r].x) / fn[r] : 0.0;
    const bool conv = tol > 0.0 ? (rel <= tol * 1.0000001 || fn[r] == 0.0) : true;
    if (!conv) all = false;
    if (info) {
      info[r].iterations = done[r] ? itv[r] : its;
      info[r].converged = conv ? 1 : 0;
      info[r].rel_res_est = est[r];
      info[r].rel_res_true = rel;
    }
  }
  if (tol > 0.0 && !all) return fail(ASP_ERR_NOT_CONVERGED, "fgmres: tolerance not reached within maxit");
  return ASP_OK;
}

size_t krylov_state_bytes(int restart, int nrhs, size_t* n2, size_t* nd, size_t* ni) {
  const long long R = restart;
  *n2 = (size_t)((R + 1) * nrhs * 2 + 2 * nrhs + R * (R + 1) * nrhs + R * nrhs + (R + 1) * nrhs + R * nrhs);
  *nd = (size_t)(R * nrhs + 3 * nrhs);
  *ni = (size_t)(3 * nrhs + 2);
  return *n2 * sizeof(double2) + *nd * sizeof(double) + *ni * sizeof(int);
}

}  // namespace asp
