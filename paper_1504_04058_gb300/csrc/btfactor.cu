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
// This is the banded LU of Section 3.1 with the fill of each w x w pivot block
// kept as an explicit inverse, which turns every solve step into a dense
// matrix-vector product.
//
// One CTA factors one subproblem; the n block inversions are sequential.  Each
// inversion is Gauss-Jordan with partial pivoting inside the block, done in
// shared memory with implicit row exchanges: step c picks the largest unused
// entry of column c as pivot (row r_c), and after w steps the inverse is
// W[i][j] = B[r_i][col(j)] where col(r) is the column whose pivot row was r.
// Pivots that are zero or non-finite are reported as ASP_ERR_SMALL_PIVOT with
// the subproblem index.
#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kFactorThreads = 128;

template <typename R>
__global__ void __launch_bounds__(kFactorThreads)
    btfactor_kernel(const SubDesc* __restrict__ subs, const SweepCoef* __restrict__ coef,
                    const double* __restrict__ k2, const double2* __restrict__ ca,
                    const double2* __restrict__ cc, const double2* __restrict__ cd, int n,
                    Cx<R>* __restrict__ Wout, int* err) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubDesc S = subs[blockIdx.x];
  const int w = S.w, wp = S.wp, ld = w + 1;
  C* A = reinterpret_cast<C*>(smem_raw);  // current matrix (row-major, ld)
  C* B = A + w * ld;                      // Gauss-Jordan target
  __shared__ int piv_row[64];
  __shared__ int col_of_row[64];
  const SweepCoef* cf = coef + S.prof;
  const int tid = threadIdx.x, lane = tid & 31;
  C* Wsub = Wout + S.woff;
  bool bad = false;

  for (int k = 0; k < n; ++k) {
    // ---- form S_k in A: T_k - a_k c_{k-1} W_{k-1} (W_{k-1} read from B with the
    //      pivot permutation of the previous inversion)
    const double2 dk = cd[k];
    C beta = czero<R>();
    if (k > 0) {
      double2 a = ca[k], c = cc[k - 1];
      beta = cmake<R>(R(a.x * c.x - a.y * c.y), R(a.x * c.y + a.y * c.x));
    }
    for (int e = tid; e < w * w; e += kFactorThreads) {
      const int i = e % w, j = e / w;
      C t = czero<R>();
      if (i == j) {
        double kk = k2[(long long)(S.lo - 1 + i) * n + k];
        t = cmake<R>(R(cf[i].dg.x + dk.x + kk), R(cf[i].dg.y + dk.y));
      } else if (j == i + 1) {
        t = cmake<R>(R(cf[i].up.x), R(cf[i].up.y));
      } else if (j == i - 1) {
        t = cmake<R>(R(cf[i].dn.x), R(cf[i].dn.y));
      }
      if (k > 0) {
        C wprev = B[piv_row[i] * ld + col_of_row[j]];
        cfms(t, beta, wprev);
      }
      A[i * ld + j] = t;
    }
    __syncthreads();

    // ---- Gauss-Jordan: w exchange steps A -> B -> A ...
    uint64_t used = 0;
    C* src = A;
    C* dst = B;
    for (int c = 0; c < w; ++c) {
      // every warp finds the pivot redundantly (no extra barrier needed)
      R best = R(-1);
      int bi = 0x7fffffff;
      for (int i = lane; i < w; i += 32) {
        if (!((used >> i) & 1ull)) {
          C v = src[i * ld + c];
          R a = v.x * v.x + v.y * v.y;
          if (a > best || (a == best && i < bi)) { best = a; bi = i; }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        R ob = __shfl_xor_sync(0xffffffffu, best, off);
        int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const int r = bi;
      used |= 1ull << r;
      if (tid == 0) { piv_row[c] = r; col_of_row[r] = c; }
      const C p = src[r * ld + c];
      if (!(best > R(0)) || !isfinite(best)) bad = true;
      const C inv = crecip(p);
      for (int e = tid; e < w * w; e += kFactorThreads) {
        const int i = e / w, j = e % w;
        C v;
        if (i == r) {
          v = (j == c) ? inv : cmul(src[r * ld + j], inv);
        } else if (j == c) {
          C aic = src[i * ld + c];
          v = cmul(aic, inv);
          v.x = -v.x; v.y = -v.y;
        } else {
          v = src[i * ld + j];
          cfms(v, src[i * ld + c], cmul(src[r * ld + j], inv));
        }
        dst[i * ld + j] = v;
      }
      __syncthreads();
      C* t = src; src = dst; dst = t;
    }
    // src now holds the permuted inverse; make it "B" for the next block
    if (src != B) {
      for (int e = tid; e < w * w; e += kFactorThreads) B[e / w * ld + e % w] = src[e / w * ld + e % w];
      __syncthreads();
    }
    // ---- store W_k (column-major, leading dimension wp)
    C* Wk = Wsub + (long long)k * w * wp;
    for (int e = tid; e < w * w; e += kFactorThreads) {
      const int i = e % w, j = e / w;
      Wk[j * wp + i] = B[piv_row[i] * ld + col_of_row[j]];
    }
    __syncthreads();
  }
  if (bad && tid == 0) record_error(err, ASP_ERR_SMALL_PIVOT, blockIdx.x);
}

}  // namespace

cudaError_t launch_factor(Handle& H, cudaStream_t s) {
  const int nsub = (int)H.subs.size();
  if (nsub == 0) return cudaSuccess;
  const size_t esz = H.prec == ASP_PREC_C128 ? sizeof(double2) : sizeof(float2);
  const size_t smem = 2 * (size_t)H.wmax * (H.wmax + 1) * esz;
  cudaError_t e;
  if (H.prec == ASP_PREC_C128) {
    e = cudaFuncSetAttribute(btfactor_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    btfactor_kernel<double><<<nsub, kFactorThreads, smem, s>>>(H.d_subs, H.d_coef, H.k2, H.ca, H.cc, H.cd, H.n,
                                                               (double2*)H.W, H.err);
  } else {
    e = cudaFuncSetAttribute(btfactor_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    btfactor_kernel<float><<<nsub, kFactorThreads, smem, s>>>(H.d_subs, H.d_coef, H.k2, H.ca, H.cc, H.cd, H.n,
                                                              (float2*)H.W, H.err);
  }
  H.launches += 1;
  return cudaGetLastError();
}

}  // namespace asp
