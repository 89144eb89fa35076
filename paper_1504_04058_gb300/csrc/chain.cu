// chain.cu -- the sequential part of Algorithm 2: accumulation of the boundary
// traces along the right-going and left-going sweeps (Section 2.2 and Section
// 3.1 "Putting together"):
//     (u~_{p,1:p})^R = (G~_p^R (u~_{p-1,1:p-1})^R)^R + (u~_{p,p})^R,   p = 2..m-1
//     (u~_{p,p:m})^L = (u~_{p,p})^L + (G~_p^L (u~_{p+1,p+1:m})^L)^L,   p = m-1..2
// Only the traces travel from layer to layer, so the map w -> (G~_p^R w)^R is
// applied as a dense n x n matrix T_p^R built once at factor time (btsolve.cu,
// MODE_TMAP_R); the full layer fields G~_p^R w are then computed for all p at
// once afterwards.  This turns a chain of 2(m-1) dependent banded solves, each
// n block-steps long, into 2(m-2) dependent dense products that spread over
// the whole GPU.
//
// accR[p] holds (u~_{p,p})^R on entry and (u~_{p,1:p})^R on exit; accL likewise.
// One cooperative launch runs both sweeps: the first half of the CTAs the R
// chain, the second half the L chain, each with its own grid barrier between
// layers.  Barrier waits are bounded; a timeout records ASP_ERR_TIMEOUT.
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kChainThreads = 256;
constexpr int kChunk = 64;     // k-extent of one shared-memory tile
constexpr int kMaxItems = 16;  // (output, k-slice) items per thread

template <typename R>
__global__ void __launch_bounds__(kChainThreads) chain_kernel(ChainParams P) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int half = gridDim.x / 2;
  const bool isR = (int)blockIdx.x < half;
  const int cta = isR ? blockIdx.x : blockIdx.x - half;
  const int nct = isR ? half : (int)gridDim.x - half;
  const int n = P.n, m = P.m, ldv = P.ldv, nrhs = P.nrhs;
  unsigned int* bar = P.bar + (isR ? 0 : 1);
  C* acc = reinterpret_cast<C*>(isR ? P.accR : P.accL);
  const C* tm = reinterpret_cast<const C*>(P.tmap);

  const int row0 = (int)((long long)cta * n / nct);
  const int row1 = (int)((long long)(cta + 1) * n / nct);
  const int rows = row1 - row0;
  const int O = rows * nrhs;  // outputs of this CTA
  int KS = O > 0 ? kChainThreads / O : 1;
  if (KS < 1) KS = 1;
  if (KS > kChunk) KS = kChunk;
  const int items = O * KS;

  C* s_src = reinterpret_cast<C*>(smem_raw);       // [kChunk][nrhs]
  C* s_T = s_src + (size_t)kChunk * nrhs;          // [rows][kChunk]
  C* s_red = s_T + (size_t)rows * kChunk;          // [kChainThreads] for the K-split reduction
  if (tid == 0) s_abort = 0;

  for (int t = 0; t < m - 2; ++t) {
    const int p = isR ? 2 + t : m - 1 - t;
    const C* src = acc + (long long)(isR ? p - 1 : p + 1) * n * ldv;
    C* dst = acc + (long long)p * n * ldv;
    const C* T = tm + (isR ? P.toffR[p] : P.toffL[p]);

    C part[kMaxItems];
#pragma unroll
    for (int u = 0; u < kMaxItems; ++u) part[u] = czero<R>();

    for (int kc = 0; kc < n; kc += kChunk) {
      const int kn = (n - kc) < kChunk ? (n - kc) : kChunk;
      __syncthreads();
      for (int e = tid; e < kn * nrhs; e += kChainThreads) {
        const int kk = e / nrhs, r = e % nrhs;
        s_src[kk * nrhs + r] = __ldcg(src + (long long)(kc + kk) * ldv + r);  // L2: written by other CTAs
      }
      for (int e = tid; e < rows * kn; e += kChainThreads) {
        const int rr = e / kn, kk = e % kn;
        s_T[rr * kChunk + kk] = T[(long long)(row0 + rr) * n + kc + kk];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kMaxItems; ++u) {
        const int it = tid + u * kChainThreads;
        if (it < items) {
          const int o = it / KS, ks = it % KS;
          const int rr = o / nrhs, r = o % nrhs;
          C a = part[u];
          for (int kk = ks; kk < kn; kk += KS) cfma(a, s_T[rr * kChunk + kk], s_src[kk * nrhs + r]);
          part[u] = a;
        }
      }
    }
    // reduce K-slices and accumulate into dst
    if (KS > 1) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kMaxItems; ++u) {
        const int it = tid + u * kChainThreads;
        if (it < items) s_red[it] = part[u];
      }
      __syncthreads();
      for (int o = tid; o < O; o += kChainThreads) {
        C s = czero<R>();
        for (int ks = 0; ks < KS; ++ks) s = cadd(s, s_red[o * KS + ks]);
        const int rr = o / nrhs, r = o % nrhs;
        C* d = dst + (long long)(row0 + rr) * ldv + r;
        *d = cadd(__ldcg(d), s);
      }
    } else {
#pragma unroll
      for (int u = 0; u < kMaxItems; ++u) {
        const int it = tid + u * kChainThreads;
        if (it < items) {
          const int rr = it / nrhs, r = it % nrhs;
          C* d = dst + (long long)(row0 + rr) * ldv + r;
          *d = cadd(__ldcg(d), part[u]);
        }
      }
    }
    // ---- grid barrier of this chain (bounded)
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(bar, 1u);
      const unsigned target = (unsigned)(t + 1) * (unsigned)nct;
      uint32_t spins = 0;
      while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) break;
        if (++spins > kSpinLimit) {
          record_error(P.err, ASP_ERR_TIMEOUT, 1000000 + (int)blockIdx.x);
          s_abort = 1;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_abort) return;
  }
}

}  // namespace

cudaError_t launch_chain(Handle& H, const ChainParams& P, cudaStream_t s) {
  if (P.m < 3) return cudaSuccess;
  int half = H.num_sms / 2;
  if (half > P.n) half = P.n;
  if (half < 1) half = 1;
  // every CTA must own few enough outputs for its register items
  const int rows_max = (P.n + half - 1) / half;
  if ((long long)rows_max * P.nrhs > (long long)kChainThreads * kMaxItems || P.nrhs > 64)
    return cudaErrorInvalidValue;
  const size_t esz = H.prec == ASP_PREC_C128 ? sizeof(double2) : sizeof(float2);
  const size_t smem = esz * ((size_t)kChunk * P.nrhs + (size_t)rows_max * kChunk + (size_t)kChainThreads);
  cudaError_t e = cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  ChainParams Q = P;
  void* args[] = {&Q};
  dim3 grid(2 * half), block(kChainThreads);
  if (H.prec == ASP_PREC_C128) {
    e = cudaFuncSetAttribute(chain_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel((void*)chain_kernel<double>, grid, block, args, smem, s);
  } else {
    e = cudaFuncSetAttribute(chain_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel((void*)chain_kernel<float>, grid, block, args, smem, s);
  }
  H.launches += 1;
  return e;
}

}  // namespace asp
