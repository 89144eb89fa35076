// factor3d.cu -- Algorithm 1 for the 3D slab subproblems (Section 4: the
// layers are slabs of planes and the auxiliary problems H_q^M, H_p^R, H_p^L
// are the quasi-2D problems of each slab).
//
// Ordered with x2 as the block index (local index j = i3l*n + i1 inside a
// block), a slab of padded width w is block tridiagonal with n dense blocks of
// size nb = n*w coupled by the x2 stencil weights times the identity, so block
// elimination needs only the inverses of the Schur complements:
//     S_0 = T_0,   S_k = T_k - a_k c_{k-1} W_{k-1},   W_k = S_k^-1,
// the solver then runs z_k = W_k (g_k - a_k z_{k-1}) and x_k = z_k - c_k W_k x_{k+1}.
// W_k is dense; each inversion is blocked Gauss-Jordan with partial pivoting
// inside the block, done for every slab of a group at once:
//   * form/store: W_{k-1} is un-permuted out of the work matrix into the
//     factor storage, and S_k = T_k - beta_k W_{k-1} is written into the other
//     work matrix;
//   * per outer block of kSlabOuter columns, per inner panel of kSlabPanel
//     columns inside it:
//       panel  -- Gauss-Jordan steps restricted to the panel columns, all rows;
//                 the panel is split over a thread-block cluster (rows across
//                 CTAs, in shared memory); the pivot search and the pivot row
//                 travel through distributed shared memory; at the end the
//                 panel's pivot rows inside the outer block are copied aside;
//       inner update -- the other columns of the outer block take the panel's
//                 steps (a rank-kSlabPanel product);
//   * then every column outside the outer block takes all of its steps at
//     once: with R the block's pivot rows and P the block's columns after its
//     panels, A[:, j] <- A[:, j] (rows R cleared) + P * A_old[R, j]; the rows
//     R are copied aside first (gather), so one complex rank-kSlabOuter
//     product updates pivot and non-pivot rows alike (big update).
// Composing Gauss-Jordan steps this way is exact: a column outside a block of
// steps changes only through the block's pivot rows.  After the last block the
// work matrix holds the inverse with rows and columns permuted:
// W[i][j] = B[piv_row[i]][col_of_row[j]], with piv_row[c] the pivot row of
// column c and col_of_row its inverse.  Zero or non-finite pivots record
// ASP_ERR_SMALL_PIVOT with the slab index.
#include <cooperative_groups.h>
#include <limits.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace asp {

namespace {

constexpr int kPW = kSlabPanel;  // panel width
constexpr int kKO = kSlabOuter;  // outer block width
constexpr int kLDP = kPW + 1;
constexpr int kPanelThreads = 512;
constexpr int kPanelWarps = kPanelThreads / 32;
constexpr int kBM = 128, kBN = 64;  // update tile: 16 x 16 threads, 8 x 4 complex each (strided by 16)
constexpr int kUpdThreads = 256;

template <typename R> __device__ __forceinline__ Cx<R>* work(const Slab3Params& P, const Slab& S, int buf) {
  return reinterpret_cast<Cx<R>*>(P.A) + S.aoff + (long long)buf * S.nb * S.ld;
}
// outer block's pivot rows, kKO x ld
template <typename R> __device__ __forceinline__ Cx<R>* zbig(const Slab3Params& P, const Slab& S) {
  return reinterpret_cast<Cx<R>*>(P.A) + S.aoff + S.zbo;
}
// inner panel's pivot rows inside the outer block, kPW x kKO
template <typename R> __device__ __forceinline__ Cx<R>* zpan(const Slab3Params& P, const Slab& S) {
  return reinterpret_cast<Cx<R>*>(P.A) + S.aoff + S.zbo + (long long)kKO * S.ld;
}

// ------------------------------------------------------------ form / store
// Row i = blockIdx.x of slab list[blockIdx.y].
template <typename R>
__global__ void __launch_bounds__(256) form_store_kernel(Slab3Params P, FactorCoefs<R> F, int k, int src_buf,
                                                         int store, int form) {
  using C = Cx<R>;
  const Slab S = P.slabs[P.list[blockIdx.y]];
  const int i = blockIdx.x;
  if (i >= S.nb) return;
  const int nb = S.nb, ld = S.ld, n = P.n;
  const C* src = work<R>(P, S, src_buf);
  C* dst = work<R>(P, S, src_buf ^ 1);
  int* piv_row = P.piv + S.poff;
  const int* col_of_row = piv_row + nb;
  int* row_step = piv_row + 2 * nb;
  C* Wk = reinterpret_cast<C*>(P.W) + S.woff + (long long)(k - 1) * nb * ld;
  // the pivot tables are complete unless a pivot search failed (recorded as
  // ASP_ERR_SMALL_PIVOT); clamping keeps every access inside the block anyway
  const int pr = store ? min(max(piv_row[i], 0), nb - 1) : 0;
  const int i3l = i / n, i1 = i - i3l * n;
  C diag = czero<R>(), beta = czero<R>(), xm = czero<R>(), xp = czero<R>(), zm = czero<R>(), zp = czero<R>();
  if (form) {
    diag = cadd(cadd(F.dg[S.prof + i3l], F.cd[i1]), F.cd[k]);
    diag.x += F.k2[((long long)(S.lo - 1 + i3l) * n + k) * n + i1];
    if (k > 0) beta = cmul(F.ca[k], F.cc[k - 1]);
    if (i1 > 0) xm = F.ca[i1];
    if (i1 < n - 1) xp = F.cc[i1];
    zm = F.dn[S.prof + i3l];
    zp = F.up[S.prof + i3l];
  }
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    C wv = czero<R>();
    if (store) {
      wv = src[(long long)pr * ld + min(max(col_of_row[j], 0), nb - 1)];
      Wk[(long long)i * ld + j] = wv;
    }
    if (form) {
      C t = czero<R>();
      if (j == i) t = diag;
      else if (j == i - 1) t = xm;
      else if (j == i + 1) t = xp;
      else if (j == i - n) t = zm;
      else if (j == i + n) t = zp;
      if (store) cfms(t, beta, wv);
      dst[(long long)i * ld + j] = t;
    }
  }
  if (form && threadIdx.x == 0) row_step[i] = -1;
}

// ------------------------------------------------------------------- panel
// Grid (CL, nlist) with clusters of CL CTAs along x: CTA rank q holds rows
// [q*rpc, (q+1)*rpc) of the panel in shared memory; warp w owns the contiguous
// local rows [w*R, (w+1)*R) for both the pivot search and the updates, so within
// a step only the CTA-wide candidate reduction needs a block barrier (and the
// search, one row per lane, reads rows kLDP apart: no bank conflicts).  Per step
// every CTA pushes its pivot candidate (|value|^2, row, and the row's kPW
// entries) into a slot of every CTA of the cluster (distributed shared memory,
// slots double-buffered by step parity); after one cluster barrier each CTA
// picks the same winner from its own slots and applies the step to its rows,
// two rows per warp instruction (a half-warp per row, columns c and c + 16 per lane).
constexpr int kMaxCluster = 8;

template <typename R>
__global__ void __launch_bounds__(kPanelThreads, 1) panel_kernel(Slab3Params P, int c0, int C0, int buf) {
  using C = Cx<R>;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int sidx = P.list[blockIdx.y];
  const Slab S = P.slabs[sidx];
  const int nb = S.nb, ld = S.ld, np = S.np;
  if (c0 >= np) return;  // the whole cluster leaves together
  const int pw = min(kPW, np - c0);
  const int rpc = (nb + CL - 1) / CL;
  const int row0 = q * rpc;
  const int nrows = max(0, min(nb, row0 + rpc) - row0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Ps = reinterpret_cast<C*>(smem_raw);                        // [rpc][kLDP]
  int* rstep = reinterpret_cast<int*>(Ps + (size_t)rpc * kLDP);  // [rpc]
  __shared__ C slot_row[2][kMaxCluster][kPW];
  __shared__ R slot_val[2][kMaxCluster];
  __shared__ int slot_idx[2][kMaxCluster];
  __shared__ R wbest[kPanelWarps];
  __shared__ int wrow[kPanelWarps];
  __shared__ int pivs[kPW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rpw = (nrows + kPanelWarps - 1) / kPanelWarps;  // rows per warp
  const int wlo = min(warp * rpw, nrows), whi = min(wlo + rpw, nrows);
  C* A = work<R>(P, S, buf);
  int* piv_row = P.piv + S.poff;
  int* col_of_row = piv_row + nb;
  int* row_step = piv_row + 2 * nb;

  for (int e = tid; e < nrows * kPW; e += kPanelThreads) {
    const int l = e / kPW, t = e - l * kPW;
    Ps[l * kLDP + t] = (t < pw) ? A[(long long)(row0 + l) * ld + c0 + t] : czero<R>();
  }
  for (int l = tid; l < nrows; l += kPanelThreads) rstep[l] = row_step[row0 + l];
  __syncthreads();

  bool bad = false;
  for (int t = 0; t < pw; ++t) {
    const int c = c0 + t;
    const int par = t & 1;
    // ---- candidate of this warp's rows: largest |A[i][c]| over rows not yet pivots
    R best = R(-1);
    int bi = INT_MAX;
    for (int l = wlo + lane; l < whi; l += 32) {
      if (rstep[l] < 0 && row0 + l < np) {  // pivots come from the first np rows only
        const C v = Ps[l * kLDP + t];
        const R a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bi = row0 + l; }  // rows ascend along a lane: ties keep the first
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const R ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { wbest[warp] = best; wrow[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < kPanelWarps ? wbest[lane] : R(-1);
      bi = lane < kPanelWarps ? wrow[lane] : INT_MAX;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const bool have = bi >= row0 && bi < row0 + nrows;
      const C rv = (have && lane < pw) ? Ps[(bi - row0) * kLDP + lane] : czero<R>();
      for (int d = 0; d < CL; ++d) {
        cluster.map_shared_rank(&slot_row[par][q][0], d)[lane] = rv;
        if (lane == 0) {
          *cluster.map_shared_rank(&slot_val[par][q], d) = best;
          *cluster.map_shared_rank(&slot_idx[par][q], d) = bi;
        }
      }
    }
    cluster.sync();
    // ---- the cluster's pivot, from this CTA's own slots (same choice everywhere)
    R gb = R(-1);
    int gr = INT_MAX, gq = 0;
    for (int r = 0; r < CL; ++r) {
      const R a = slot_val[par][r];
      const int ri = slot_idx[par][r];
      if (a > gb || (a == gb && ri < gr)) { gb = a; gr = ri; gq = r; }
    }
    const bool okp = gr >= 0 && gr < nb;
    if (!(gb > R(0)) || !isfinite(gb)) bad = true;
    if (okp) {
      // lane: half-warp hw takes rows wlo + hw, wlo + hw + 2, ...; columns cj and cj + 16
      // (unit stride across the half-warp: no bank conflicts)
      const int hw = lane >> 4, cj = lane & 15, cj1 = cj + 16;
      const C* prow = slot_row[par][gq];
      const C inv = crecip(prow[t]);
      const C pl0 = prow[cj], pl1 = prow[cj1];
      // the pivot row's new entries
      const C ps0 = (cj == t) ? inv : cmul(pl0, inv);
      const C ps1 = (cj1 == t) ? inv : cmul(pl1, inv);
      const int lg = gr - row0;  // local index of the pivot row (if here)
      // four row pairs per pass: all reads, one warp barrier, then all writes
      // (the lanes of column t overwrite the entry the other lanes read)
      for (int l0 = wlo; l0 < whi; l0 += 8) {  // warp-uniform bound (the barriers below)
        C v0[4], v1[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int l = l0 + 2 * a + hw;
          if (l < whi) {
            const C* rowp = Ps + l * kLDP;
            const C f = cmul(rowp[t], inv);
            C x0 = rowp[cj], x1 = rowp[cj1];
            cfms(x0, f, pl0);
            cfms(x1, f, pl1);
            if (cj == t) { x0.x = -f.x; x0.y = -f.y; }
            if (cj1 == t) { x1.x = -f.x; x1.y = -f.y; }
            v0[a] = (l == lg) ? ps0 : x0;
            v1[a] = (l == lg) ? ps1 : x1;
          }
        }
        __syncwarp();
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int l = l0 + 2 * a + hw;
          if (l < whi) {
            if (cj < pw) Ps[l * kLDP + cj] = v0[a];
            if (cj1 < pw) Ps[l * kLDP + cj1] = v1[a];
          }
        }
        __syncwarp();
      }
      if (lg >= wlo && lg < whi && lane == 0) rstep[lg] = c;
      if (tid == 0 && q == 0) {
        piv_row[c] = gr;
        col_of_row[gr] = c;
      }
    }
    if (tid == 0) pivs[t] = okp ? gr : 0;
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < nrows * pw; e += kPanelThreads) {
    const int l = e / pw, t = e - l * pw;
    A[(long long)(row0 + l) * ld + c0 + t] = Ps[l * kLDP + t];
  }
  for (int l = tid; l < nrows; l += kPanelThreads) row_step[row0 + l] = rstep[l];
  // pivot rows inside the outer block, outside the panel (untouched here), for
  // the inner update; rows t = q, q + CL, ... on this CTA
  {
    const int C1 = min(C0 + kKO, np);
    Cx<R>* zp = zpan<R>(P, S);
    for (int t = q; t < pw; t += CL) {
      const Cx<R>* src = A + (long long)pivs[t] * ld;
      for (int j = C0 + tid; j < C1; j += kPanelThreads)
        zp[t * kKO + (j - C0)] = (j >= c0 && j < c0 + pw) ? czero<R>() : src[j];
    }
  }
  if (bad && tid == 0 && q == 0) record_error(P.err, ASP_ERR_SMALL_PIVOT, sidx);
}

// ------------------------------------------------------------------ gather
// zbig[t][j] = A[piv_row[C0 + t]][j] for the outer block's pivots.  Grid
// (row t, nlist).
template <typename R>
__global__ void __launch_bounds__(256) gather_kernel(Slab3Params P, int C0, int buf) {
  const Slab S = P.slabs[P.list[blockIdx.y]];
  const int nb = S.nb, ld = S.ld;
  const int t = blockIdx.x;
  if (C0 >= S.np || t >= min(kKO, S.np - C0)) return;
  const int* piv_row = P.piv + S.poff;
  const int r = min(max(piv_row[C0 + t], 0), nb - 1);
  const Cx<R>* src = work<R>(P, S, buf) + (long long)r * ld;
  Cx<R>* dst = zbig<R>(P, S) + (long long)t * ld;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) dst[j] = src[j];
}

// ------------------------------------------------------------------ update
// For every row i and every column j in the update range outside [a0, a0+K):
//     A[i][j] = (i a pivot of columns [a0, a0+K) ? 0 : A[i][j]) + sum_u A[i][a0+u] Z[u][j]
// inner (big == 0): a0 = c0, K = the panel width, columns [C0, C0 + kKO), Z = zpan;
// big   (big == 1): a0 = C0, K = the outer block width, all columns, Z = zbig.
// Grid (column tiles, row tiles, nlist); K is consumed in chunks of kPW.
template <typename R>
__global__ void __launch_bounds__(kUpdThreads) update_kernel(Slab3Params P, int C0, int c0, int buf, int big) {
  using C = Cx<R>;
  const Slab S = P.slabs[P.list[blockIdx.z]];
  const int nb = S.nb, ld = S.ld, np = S.np;
  const int a0 = big ? C0 : c0;
  if (a0 >= np) return;
  const int K = big ? min(kKO, np - C0) : min(kPW, np - c0);
  const int jlo = big ? 0 : C0;
  const int jhi = big ? nb : min(C0 + kKO, np);
  const int j0 = jlo + blockIdx.x * kBN, i0 = blockIdx.y * kBM;
  if (j0 >= jhi || i0 >= nb) return;
  if (j0 >= a0 && j0 + kBN <= a0 + K) return;  // the tile lies inside the eliminated columns
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* As = reinterpret_cast<C*>(smem_raw);  // [kBM][kLDP]   eliminated columns, chunk
  C* Bs = As + kBM * kLDP;                 // [kPW][kBN]    old pivot rows, chunk
  C* A = work<R>(P, S, buf);
  const C* Z = big ? zbig<R>(P, S) : zpan<R>(P, S);
  const long long ldz = big ? ld : kKO;
  const int zc0 = big ? 0 : C0;
  const int* row_step = P.piv + S.poff + 2 * nb;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  // The accumulators start from this thread's entries of the tile, loaded before
  // the staging below so that their latency overlaps it and the products:
  // A[i][j] for the other rows, zero for the pivot rows of the step block (their
  // old values leave through Z).  The epilogue then only stores.
  C acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = i0 + ty + 16 * a;
    const int st = i < nb ? row_step[i] : -1;
    const bool piv = st >= a0 && st < a0 + K;
    const C* rowp = A + (long long)min(i, nb - 1) * ld;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      const bool in = i < nb && j < jhi && !(j >= a0 && j < a0 + K);
      acc[a][b] = (in && !piv) ? rowp[j] : czero<R>();
    }
  }
  for (int kc = 0; kc < K; kc += kPW) {
    const int kw = min(kPW, K - kc);
    __syncthreads();
    for (int e = tid; e < kBM * kPW; e += kUpdThreads) {
      const int ii = e / kPW, t = e - ii * kPW;
      const int i = i0 + ii;
      As[ii * kLDP + t] = (t < kw && i < nb) ? A[(long long)i * ld + a0 + kc + t] : czero<R>();
    }
    for (int e = tid; e < kPW * kBN; e += kUpdThreads) {
      const int t = e / kBN, jj = e - t * kBN;
      const int j = j0 + jj;
      Bs[t * kBN + jj] = (t < kw && j < jhi) ? Z[(long long)(kc + t) * ldz + (j - zc0)] : czero<R>();
    }
    __syncthreads();
    for (int t = 0; t < kw; ++t) {
      C av[8], bv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) av[a] = As[(ty + 16 * a) * kLDP + t];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[t * kBN + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= nb) continue;
    C* rowp = A + (long long)i * ld;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j >= jhi || (j >= a0 && j < a0 + K)) continue;
      rowp[j] = acc[a][b];
    }
  }
}

// ------------------------------------------------------------------ driver
// The Gauss-Jordan steps on columns [0, np) of every matrix of one list (slabs
// of one factor group, or nested-dissection fronts of one level): setup()
// sizes the launches once, run(buf) enqueues the panels and updates.
template <typename R> struct GjRun {
  Slab3Params P{};
  cudaLaunchConfig_t pc{};
  cudaLaunchAttribute pattr[1];
  dim3 igrid, bgrid;
  size_t usmem = 0;
  int nbmax = 0, npmax = 0, nlist = 0;
  const TcGroup* tc = nullptr;
  cudaStream_t s = nullptr;

  cudaError_t setup(const Slab3Params& base, int nbmax_, int npmax_, const TcGroup* tc_, int num_sms,
                    cudaStream_t s_) {
    P = base;
    nlist = base.nlist;
    nbmax = nbmax_;
    npmax = npmax_;
    tc = tc_;
    s = s_;
    if (nlist <= 0) return cudaSuccess;
    const size_t esz = sizeof(Cx<R>);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t static_bytes = 12288;  // the kernel's static shared arrays, with room
    const int rows_cap = (int)(((size_t)optin - static_bytes) / (kLDP * esz + sizeof(int)));
    // about 512 rows per CTA (the per-step row updates are issue-bound) while
    // all clusters of the list fit in one wave (one CTA per SM), and at least
    // as many CTAs as shared memory requires
    const int by_rows = std::min(kMaxCluster, (nbmax + 511) / 512);
    const int by_sms = std::max(1, num_sms / std::max(nlist, 1));
    int CL = std::max((nbmax + rows_cap - 1) / rows_cap, std::min(by_rows, by_sms));
    if (CL < 1) CL = 1;
    if (CL > kMaxCluster) return cudaErrorInvalidValue;
    const int rpc = (nbmax + CL - 1) / CL;
    const size_t psmem = (size_t)rpc * (kLDP * esz + sizeof(int));
    cudaError_t e = ensure_dyn_smem((const void*)panel_kernel<R>, psmem);
    if (e != cudaSuccess) return e;
    if (CL > 1) {
      e = cudaFuncSetAttribute(panel_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
      if (e != cudaSuccess) return e;
    }
    usmem = (size_t)(kBM * kLDP + kPW * kBN) * esz;
    e = ensure_dyn_smem((const void*)update_kernel<R>, usmem);
    if (e != cudaSuccess) return e;
    pattr[0].id = cudaLaunchAttributeClusterDimension;
    pattr[0].val.clusterDim.x = CL;
    pattr[0].val.clusterDim.y = 1;
    pattr[0].val.clusterDim.z = 1;
    pc.gridDim = dim3(CL, nlist);
    pc.blockDim = dim3(kPanelThreads);
    pc.dynamicSmemBytes = psmem;
    pc.stream = s;
    pc.numAttrs = 1;
    igrid = dim3(kKO / kBN, (nbmax + kBM - 1) / kBM, nlist);
    bgrid = dim3((nbmax + kBN - 1) / kBN, (nbmax + kBM - 1) / kBM, nlist);
    return cudaSuccess;
  }

  cudaError_t run(Handle& H, int buf) {
    if (nlist <= 0) return cudaSuccess;
    pc.attrs = pattr;  // the struct may have moved since setup
    cudaError_t e;
    for (int C0 = 0; C0 < npmax; C0 += kKO) {
      for (int c0 = C0; c0 < std::min(C0 + kKO, npmax); c0 += kPW) {
        e = cudaLaunchKernelEx(&pc, panel_kernel<R>, P, c0, C0, buf);
        if (e != cudaSuccess) return e;
        update_kernel<R><<<igrid, kUpdThreads, usmem, s>>>(P, C0, c0, buf, 0);
        H.launches += 2;
      }
      if (tc) {  // complex64: split-precision TF32 product on the tensor cores
        PhaseTok ts = phase_begin(H, PH_SCHUR, s);
        e = launch_tc_update(*tc, P, nbmax, C0, buf, s);
        phase_end(H, ts, s);
        if (e != cudaSuccess) return e;
      } else {
        gather_kernel<R><<<dim3(kKO, nlist), 256, 0, s>>>(P, C0, buf);
        update_kernel<R><<<bgrid, kUpdThreads, usmem, s>>>(P, C0, 0, buf, 1);
      }
      H.launches += 2;
    }
    return cudaGetLastError();
  }
};

// One factor group (slabs of one kind of subproblem sharing a stream).
// block(k) enqueues the store of W_{k-1} and, for k < n, the inversion of S_k.
// The groups' blocks are enqueued alternately, so that each stream always has
// queued work and the groups overlap on the GPU (enqueued one group after the
// other, the host would block on the full launch queue of the first group
// until that group was nearly done).
template <typename R> struct Factor3Group {
  GjRun<R> gj;
  int nbmax = 0, nlist = 0;
  cudaStream_t s = nullptr;

  cudaError_t setup(Handle& H, const int* d_list, int nlist_, int nbmax_, const TcGroup* tc_, cudaStream_t s_) {
    nlist = nlist_;
    nbmax = nbmax_;
    s = s_;
    Slab3Params P{};
    P.slabs = H.d_slabs;
    P.list = d_list;
    P.nlist = nlist;
    P.n = H.n;
    P.W = H.W;
    P.A = H.A3;
    P.piv = H.piv3;
    P.err = H.err;
    return gj.setup(P, nbmax, nbmax, tc_, H.num_sms, s);
  }

  cudaError_t block(Handle& H, const FactorCoefs<R>& F, int k) {
    if (nlist <= 0) return cudaSuccess;
    const int n = H.n;
    const int store = k > 0, form = k < n;
    form_store_kernel<R><<<dim3(nbmax, nlist), 256, 0, s>>>(gj.P, F, k, (k + 1) & 1, store, form);
    H.launches += 1;
    if (!form) return cudaGetLastError();
    return gj.run(H, k & 1);
  }
};

template <typename R> cudaError_t factor_groups(Handle& H, const FactorCoefs<R>& F, cudaStream_t s) {
  std::vector<Factor3Group<R>> runs(H.fgroups.size());
  std::vector<PhaseTok> toks(H.fgroups.size());
  cudaError_t e = cudaSuccess;
  for (size_t g = 0; g < H.fgroups.size(); ++g) {
    auto& G = H.fgroups[g];
    cudaStream_t gs = G.stream ? G.stream : s;
    const TcGroup* tc = std::is_same<R, float>::value ? &G.tc : nullptr;
    if ((e = runs[g].setup(H, H.d_slab_lists + G.first, G.count, G.nbmax, tc, gs)) != cudaSuccess) return e;
  }
  for (size_t g = 0; g < runs.size(); ++g) toks[g] = phase_begin(H, PH_FACTOR, runs[g].s);
  for (int k = 0; k <= H.n && e == cudaSuccess; ++k)
    for (auto& r : runs)
      if ((e = r.block(H, F, k)) != cudaSuccess) break;
  for (size_t g = 0; g < runs.size(); ++g) phase_end(H, toks[g], runs[g].s);
  return e;
}

}  // namespace

cudaError_t gj_partial(Handle& H, const Slab3Params& P, int nbmax, int npmax, const TcGroup* tc, cudaStream_t s) {
  if (H.prec == ASP_PREC_C128) {
    GjRun<double> g;
    cudaError_t e = g.setup(P, nbmax, npmax, nullptr, H.num_sms, s);
    return e != cudaSuccess ? e : g.run(H, 0);
  }
  GjRun<float> g;
  cudaError_t e = g.setup(P, nbmax, npmax, tc, H.num_sms, s);
  return e != cudaSuccess ? e : g.run(H, 0);
}

// Factors every slab: each factor group (the M slabs; the R and L slabs) on its
// own stream, forked from and joined back into the caller's.
int factor3d(Handle& H, cudaStream_t s) {
  auto cuda_fail = [](const char* what, cudaError_t e) {
    return fail(ASP_ERR_CUDA, std::string("3D factor: ") + what + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaEventRecord(H.ev_fork, s);
  if (e != cudaSuccess) return cuda_fail("fork record", e);
  for (auto& g : H.fgroups)
    if (g.stream && (e = cudaStreamWaitEvent(g.stream, H.ev_fork, 0)) != cudaSuccess) return cuda_fail("fork wait", e);
  const cudaError_t launch_err =
      H.prec == ASP_PREC_C128 ? factor_groups<double>(H, H.fc64, s) : factor_groups<float>(H, H.fc32, s);
  for (auto& g : H.fgroups) {
    if (!g.stream) continue;
    if ((e = cudaEventRecord(g.done, g.stream)) != cudaSuccess) return cuda_fail("join record", e);
    if ((e = cudaStreamWaitEvent(s, g.done, 0)) != cudaSuccess) return cuda_fail("join wait", e);
  }
  if (launch_err != cudaSuccess) return cuda_fail("launch", launch_err);
  return ASP_OK;
}

}  // namespace asp
