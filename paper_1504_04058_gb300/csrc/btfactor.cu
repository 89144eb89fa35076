// btfactor.cu -- Algorithm 1 on the GPU: factor every layer subproblem
// H_q^M, H_p^R, H_p^L (Section 3.1) in one launch.
//
// Ordered x2-fastest (the quasi-1D ordering of Section 3.1), a subproblem on an
// n x w grid is block tridiagonal: n diagonal blocks T_k (w x w, tridiagonal in
// x2 plus the x1 and omega^2/c^2 diagonal terms) coupled to their neighbours
// by scalar multiples of the identity, a_k I (to block k-1) and c_k I (to
// block k+1), because the x1 stencil weights s_k s_{k+-1/2}/h^2 do not depend
// on x2.  Block elimination gives
//     S_0 = T_0,   S_k = T_k - a_k c_{k-1} S_{k-1}^{-1},
// and the solver needs only W_k = S_k^{-1}: the forward pass is
// z_k = W_k (g_k - a_k z_{k-1}) and the backward pass x_k = z_k - c_k W_k x_{k+1}.
// With ASP_PREC_C64_SYM the factors are stored as the upper triangle of the
// symmetric W_k Delta (internal.h, packed_index), half the bytes.
// This is the banded LU of Section 3.1 with the fill of each w x w pivot block
// kept as an explicit inverse, which turns every solve step into a dense
// matrix product.
//
// One CTA of 4 ROWS threads factors one subproblem; the n block inversions
// are sequential.  Thread t owns row i = t mod ROWS and every fourth column
// (j = t/ROWS, t/ROWS + 4, ...) of the block, so no index arithmetic divides.
// A launch takes the smallest ROWS of 32, 48, 64 that covers its widest block,
// so that few threads own no row (the pivot search runs in every warp).
// Each inversion is Gauss-Jordan with partial pivoting inside the block, in
// shared memory with implicit row exchanges and two ping-pong buffers: step c
// picks the largest unused entry of column c as pivot (row r_c, found by every
// warp redundantly so the step needs a single barrier; complex64 by one warp
// max-reduction of a packed magnitude-and-row key), and after w steps the
// inverse is W[i][j] = B[r_i][col(j)] with col(r) the column whose pivot row
// was r.  Zero or non-finite pivots are reported as ASP_ERR_SMALL_PIVOT with the
// subproblem index.  All arithmetic is in the factor precision R (the FP64
// coefficients are converted once on the host for complex64).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kColGroups = 4;  // threads sharing a row

template <typename R, int ROWS>
__global__ void __launch_bounds__(ROWS * kColGroups)
    btfactor_kernel(const SubDesc* __restrict__ subs, int first, FactorCoefs<R> F, int n,
                    Cx<R>* __restrict__ Wout, int* err, int packed) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int sub = first + blockIdx.x;
  const SubDesc S = subs[sub];
  const int w = S.w, wp = S.wp;
  const int ld = w | 1;  // odd row stride: column accesses spread over the banks
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + w * ld;
  __shared__ int piv_row[64];
  __shared__ int col_of_row[64];
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int kCols = ROWS / kColGroups;  // most columns a thread owns (w <= ROWS)
  const int i = tid % ROWS;  // my row
  const int jh = tid / ROWS; // my first column (then every kColGroups-th)
  const bool row_ok = i < w;
  const Cx<R>* up = F.up + S.prof;
  const Cx<R>* dn = F.dn + S.prof;
  const Cx<R>* dg = F.dg + S.prof;
  const Cx<R>* s2 = F.s2 + S.prof;
  C* Wsub = Wout + S.woff;
  bool bad = false;
  C* prev = buf1;  // holds the permuted inverse of the previous block

  for (int k = 0; k < n; ++k) {
    C* src = (prev == buf0) ? buf1 : buf0;  // S_k is formed here
    // ---- S_k = T_k - a_k c_{k-1} W_{k-1}
    C beta = czero<R>();
    if (k > 0) beta = cmul(F.ca[k], F.cc[k - 1]);
    if (row_ok) {
      const C diag = cadd(cadd(dg[i], F.cd[k]), cmake<R>(F.k2[(long long)(S.lo - 1 + i) * n + k], R(0)));
      const int pr = (k > 0) ? piv_row[i] : 0;
#pragma unroll
      for (int u = 0; u < kCols; ++u) {
        const int j = jh + u * kColGroups;
        if (j >= w) break;
        C t = czero<R>();
        if (j == i) t = diag;
        else if (j == i + 1) t = up[i];
        else if (j == i - 1) t = dn[i];
        if (k > 0) cfms(t, beta, prev[pr * ld + col_of_row[j]]);
        src[i * ld + j] = t;
      }
    }
    __syncthreads();

    // ---- Gauss-Jordan, w exchange steps src -> dst -> src ...
    C* dst = prev;
    uint64_t used = 0;
    for (int c = 0; c < w; ++c) {
      int r;
      R best;
      if constexpr (std::is_same<R, float>::value) {
        // one warp reduction: key = |entry|^2 (its bits order like the value)
        // with the low 6 bits replaced by 63 - row, so ties (and values that
        // differ in those bits only, 2^-17 relative) go to the lower row
        unsigned key = 0u;
        for (int q = lane; q < w; q += 32) {
          if (!((used >> q) & 1ull)) {
            const C v = src[q * ld + c];
            const unsigned k = (__float_as_uint(v.x * v.x + v.y * v.y) & ~63u) | (unsigned)(63 - q);
            key = key > k ? key : k;
          }
        }
        key = __reduce_max_sync(0xffffffffu, key);
        r = 63 - (int)(key & 63u);
        best = __uint_as_float(key & ~63u);
      } else {
        best = R(-1);
        int bi = 0x7fffffff;
        for (int q = lane; q < w; q += 32) {
          if (!((used >> q) & 1ull)) {
            const C v = src[q * ld + c];
            const R a = v.x * v.x + v.y * v.y;
            if (a > best || (a == best && q < bi)) { best = a; bi = q; }
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const R ob = __shfl_xor_sync(0xffffffffu, best, off);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        r = bi;
      }
      if (!(best > R(0)) || !isfinite(best)) bad = true;
      r = min(max(r, 0), w - 1);  // a failed search is recorded above; stay inside the block
      used |= 1ull << r;
      if (tid == 0) { piv_row[c] = r; col_of_row[r] = c; }
      const C* prow = src + r * ld;
      const C inv = crecip(prow[c]);
      if (row_ok) {
        // the general update on every entry of the row, then the pivot row and
        // column take their own values (same thread, so program order)
        const C* srow = src + i * ld;
        C* drow = dst + i * ld;
        const C f = cmul(srow[c], inv);
        // fully unrolled over the thread's (at most ROWS / 4) columns, so that
        // every load of the row update can be issued before its products
        if (i != r) {
#pragma unroll
          for (int u = 0; u < kCols; ++u) {
            const int j = jh + u * kColGroups;
            if (j < w) {
              C v = srow[j];
              cfms(v, f, prow[j]);
              drow[j] = v;
            }
          }
          if (jh == (c & (kColGroups - 1))) drow[c] = cmake<R>(-f.x, -f.y);
        } else {
#pragma unroll
          for (int u = 0; u < kCols; ++u) {
            const int j = jh + u * kColGroups;
            if (j < w) drow[j] = cmul(prow[j], inv);
          }
          if (jh == (c & (kColGroups - 1))) drow[c] = inv;
        }
      }
      __syncthreads();
      C* t = src; src = dst; dst = t;
    }
    // src holds the permuted inverse of S_k; store W_k (column-major, ld wp),
    // or (packed factors) the upper triangle of the symmetric W_k Delta
    if (row_ok) {
      C* Wk = Wsub + (long long)k * S.bs;
      const int pr = piv_row[i];
      if (packed) {
        for (int j = jh; j < w; j += kColGroups)
          if (i <= j) Wk[packed_index(i, j)] = cmul(src[pr * ld + col_of_row[j]], s2[j]);
      } else {
        for (int j = jh; j < w; j += kColGroups) Wk[j * wp + i] = src[pr * ld + col_of_row[j]];
      }
    }
    prev = src;
    // the next formation reads prev and piv/col tables; the barrier after it
    // orders those reads before the next Gauss-Jordan overwrites them
  }
  if (bad && tid == 0) record_error(err, ASP_ERR_SMALL_PIVOT, sub);
}

}  // namespace

cudaError_t launch_factor(Handle& H, int first, int count, cudaStream_t s) {
  const int nsub = count;
  if (nsub <= 0) return cudaSuccess;
  int wmax = 0;  // the launch's widest block sets its shared memory and row count
  for (int q = first; q < first + count; ++q) wmax = std::max(wmax, H.subs[q].w);
  const size_t esz = H.prec == ASP_PREC_C128 ? sizeof(double2) : sizeof(float2);
  const size_t smem = 2 * (size_t)wmax * (wmax | 1) * esz;
  auto go = [&](auto kern, int rows, auto* W, const auto& F, int packed) -> cudaError_t {
    cudaError_t e = ensure_dyn_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<nsub, rows * kColGroups, smem, s>>>(H.d_subs, first, F, H.n, W, H.err, packed);
    return cudaSuccess;
  };
  cudaError_t e;
  if (H.prec == ASP_PREC_C128)
    e = wmax <= 32   ? go(btfactor_kernel<double, 32>, 32, (double2*)H.W, H.fc64, 0)
        : wmax <= 48 ? go(btfactor_kernel<double, 48>, 48, (double2*)H.W, H.fc64, 0)
                     : go(btfactor_kernel<double, 64>, 64, (double2*)H.W, H.fc64, 0);
  else
    e = wmax <= 32   ? go(btfactor_kernel<float, 32>, 32, (float2*)H.W, H.fc32, H.packed ? 1 : 0)
        : wmax <= 48 ? go(btfactor_kernel<float, 48>, 48, (float2*)H.W, H.fc32, H.packed ? 1 : 0)
                     : go(btfactor_kernel<float, 64>, 64, (float2*)H.W, H.fc32, H.packed ? 1 : 0);
  if (e != cudaSuccess) return e;
  H.launches += 1;
  return cudaGetLastError();
}

}  // namespace asp
