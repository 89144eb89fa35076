// chain.cu -- the sequential part of Algorithm 2: accumulation of the boundary
// traces along the right-going and left-going sweeps (Section 2.2 and Section
// 3.1 "Putting together"):
//     (u~_{p,1:p})^R = (G~_p^R (u~_{p-1,1:p-1})^R)^R + (u~_{p,p})^R,   p = 2..m-1
//     (u~_{p,p:m})^L = (u~_{p,p})^L + (G~_p^L (u~_{p+1,p+1:m})^L)^L,   p = m-1..2
// Only the traces travel from layer to layer, so the map w -> (G~_p^R w)^R is
// applied as a dense n x n matrix T_p^R built once at factor time (btsolve.cu,
// MODE_TMAP_R); the full layer fields G~_p^R w are then computed for all p at
// once afterwards.  This turns a chain of 2(m-1) dependent banded solves, each
// n block-steps long, into 2(m-2) dependent dense products spread over the
// whole GPU.
//
// accR[p] holds (u~_{p,p})^R on entry and (u~_{p,1:p})^R on exit; accL likewise.
// One cooperative launch runs both sweeps: the first half of the CTAs the R
// chain, the second half the L chain, each with its own grid barrier between
// layers.  Per layer a CTA owns RC <= 16 rows of the product; its 16 warps split
// the k-range (each chunk of KC columns is staged in shared memory by cp.async,
// double-buffered), each lane holds an 8-row x 2-right-hand-side tile, and the
// warps' partial sums are reduced through shared memory.  Barrier waits are
// bounded; a timeout records ASP_ERR_TIMEOUT.
#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kChainThreads = 512;
constexpr int kWarps = kChainThreads / 32;
constexpr int kMaxRows = 16;  // rows of the product per CTA
constexpr int kRhs = 32;      // right-hand sides per launch (two per lane, 16 lanes)

template <typename R> struct ChainKC;
template <> struct ChainKC<float> { static constexpr int v = 256; };
template <> struct ChainKC<double> { static constexpr int v = 128; };

template <typename R> __host__ __device__ constexpr size_t chain_smem() {
  // s_T[2][KC][kMaxRows] + s_src[2][KC][kRhs]; the cross-warp reduction buffer
  // red[kWarps][kMaxRows][kRhs] reuses s_src once the last chunk is consumed
  static_assert(2 * ChainKC<R>::v >= kWarps * kMaxRows, "reduction buffer must fit in the staging area");
  return sizeof(Cx<R>) * ((size_t)2 * kMaxRows * ChainKC<R>::v + (size_t)2 * ChainKC<R>::v * kRhs);
}

__device__ __forceinline__ void pair_ld(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void pair_ld(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }

template <typename R>
__global__ void __launch_bounds__(kChainThreads, 1) chain_kernel(ChainParams P) {
  using C = Cx<R>;
  constexpr int KC = ChainKC<R>::v;
  constexpr int CB = (int)sizeof(C);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s_T = reinterpret_cast<C*>(smem_raw);                // [2][KC][kMaxRows] (rows fastest)
  C* s_src = s_T + (size_t)2 * kMaxRows * KC;             // [2][KC][kRhs]
  C* red = s_src;                                         // [kWarps][kMaxRows][kRhs], after the chunks
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = gridDim.x / 2;
  const bool isR = (int)blockIdx.x < half;
  const int cta = isR ? blockIdx.x : blockIdx.x - half;
  const int nct = isR ? half : (int)gridDim.x - half;
  const int n = P.n, m = P.m, lda = P.ldacc, nrhs = P.nrhs, ldT = P.ldT;
  unsigned int* bar = P.bar + (isR ? 0 : 1);
  C* acc = reinterpret_cast<C*>(isR ? P.accR : P.accL);
  const C* tm = reinterpret_cast<const C*>(P.tmap);

  const int row0 = (int)((long long)cta * n / nct);
  const int rows = (int)((long long)(cta + 1) * n / nct) - row0;  // <= kMaxRows (checked on the host)
  const int rp = lane & 15;        // right-hand-side pair of this lane
  const int rh = lane >> 4;        // row half: rows rh*8 .. rh*8+7
  const int nch = (n + KC - 1) / KC;
  if (tid == 0) s_abort = 0;

  for (int t = 0; t < m - 2; ++t) {
    const int p = isR ? 2 + t : m - 1 - t;
    const C* src = acc + (long long)(isR ? p - 1 : p + 1) * n * lda;
    C* dst = acc + (long long)p * n * lda;
    const C* T = tm + (isR ? P.toffR[p] : P.toffL[p]);

    // stage chunk ch into buffer b: T[row0 .. row0+rows)[kc .. kc+KC) and src[kc .. kc+KC)[0 .. nrhs)
    auto stage = [&](int ch, int b) {
      const int kc = ch * KC;
      const int kn = min(KC, n - kc);
      C* dT = s_T + (size_t)b * kMaxRows * KC;
      C* dS = s_src + (size_t)b * KC * kRhs;
      // T chunk, transposed so that a lane's 8 rows at one k are contiguous;
      // consecutive threads take consecutive rows (contiguous shared stores)
      {
        const int rr = tid & (kMaxRows - 1);
        if (rr < rows)
          for (int kk = tid / kMaxRows; kk < kn; kk += kChainThreads / kMaxRows)
            cp_async<CB>(dT + kk * kMaxRows + rr, T + (long long)(row0 + rr) * ldT + kc + kk);
      }
      if constexpr (CB == 16) {
        for (int e = tid; e < kn * nrhs; e += kChainThreads) {
          const int kk = e / nrhs, r = e % nrhs;
          cp_async<16>(dS + kk * kRhs + r, src + (long long)(kc + kk) * lda + r);
        }
      } else {  // complex64 traces: pairs of elements (16 bytes, L2 only); lda is even
        const int nr2 = (nrhs + 1) / 2;
        for (int e = tid; e < kn * nr2; e += kChainThreads) {
          const int kk = e / nr2, r = 2 * (e % nr2);
          cp_async<16>(dS + kk * kRhs + r, src + (long long)(kc + kk) * lda + r);
        }
      }
      cp_async_commit();
    };

    C a[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i][0] = a[i][1] = czero<R>();

    __syncthreads();  // previous layer's users of the staging buffers are done
    stage(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
      if (ch + 1 < nch) stage(ch + 1, (ch + 1) & 1);
      else cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      const int kn = min(KC, n - ch * KC);
      const C* bT = s_T + (size_t)(ch & 1) * kMaxRows * KC;
      const C* bS = s_src + (size_t)(ch & 1) * KC * kRhs;
#pragma unroll 2
      for (int kk = warp; kk < kn; kk += kWarps) {
        C s0, s1;
        pair_ld(bS + kk * kRhs + 2 * rp, s0, s1);
        C tv[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) pair_ld(bT + kk * kMaxRows + rh * 8 + i, tv[i], tv[i + 1]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          cfma(a[i][0], tv[i], s0);
          cfma(a[i][1], tv[i], s1);
        }
      }
      __syncthreads();  // buffer (ch & 1) is refilled two chunks later (and red reuses s_src)
    }
    // cross-warp reduction and accumulation into dst
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      C* rw = red + ((size_t)warp * kMaxRows + rh * 8 + i) * kRhs + 2 * rp;
      rw[0] = a[i][0];
      rw[1] = a[i][1];
    }
    __syncthreads();
    for (int o = tid; o < rows * nrhs; o += kChainThreads) {
      const int rr = o / nrhs, r = o % nrhs;
      C s = czero<R>();
#pragma unroll
      for (int wv = 0; wv < kWarps; ++wv) s = cadd(s, red[((size_t)wv * kMaxRows + rr) * kRhs + r]);
      C* d = dst + (long long)(row0 + rr) * lda + r;
      *d = cadd(__ldcg(d), s);
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
        __nanosleep(32);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_abort) {
      cp_async_wait<0>();
      return;
    }
  }
  cp_async_wait<0>();
}

}  // namespace

cudaError_t launch_chain(Handle& H, const ChainParams& P, cudaStream_t s) {
  if (P.m < 3) return cudaSuccess;
  if (P.nrhs < 1 || P.nrhs > kRhs) return cudaErrorInvalidValue;
  int half = H.num_sms / 2;
  if (half > P.n) half = P.n;
  if (half < 1) half = 1;
  while ((P.n + half - 1) / half > kMaxRows) ++half;  // rows per CTA must fit the tile
  if (2 * half > H.num_sms) return cudaErrorInvalidValue;  // cooperative: one CTA per SM
  cudaError_t e = cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  ChainParams Q = P;
  void* args[] = {&Q};
  dim3 grid(2 * half), block(kChainThreads);
  if (H.prec == ASP_PREC_C128) {
    const size_t smem = chain_smem<double>();
    e = ensure_dyn_smem((const void*)chain_kernel<double>, smem);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel((void*)chain_kernel<double>, grid, block, args, smem, s);
  } else {
    const size_t smem = chain_smem<float>();
    e = ensure_dyn_smem((const void*)chain_kernel<float>, smem);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel((void*)chain_kernel<float>, grid, block, args, smem, s);
  }
  H.launches += 1;
  return e;
}

}  // namespace asp
