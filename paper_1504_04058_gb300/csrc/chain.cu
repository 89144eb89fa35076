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
// layers.  Per layer a CTA owns up to 2*RPL rows of the product.  The CTA is
// warp-specialised:
//   * a producer warp moves both operands into shared memory by bulk (TMA)
//     copies that complete on mbarriers: map rows, KC columns per chunk, in a
//     kTStages-deep ring (the maps do not depend on the sweep, so this ring runs
//     ahead across layer boundaries), and trace chunks (KC rows of the previous
//     layer's trace, one contiguous block since its rows are lda apart) in a
//     kSStages-deep ring.  It also waits at the grid barrier, and issues a
//     layer's trace chunks only once the barrier shows every CTA's part of the
//     previous layer written;
//   * 8 consumer warps wait on the full barriers, split each chunk's columns in
//     pairs (each lane holds an RPL-row x 2-right-hand-side tile, reads the
//     two columns of a map row with one 16-byte load, and loads the next pair
//     while the current one's products issue), release the stages on
//     the empty barriers, reduce their partial sums through shared memory (the
//     idle trace ring) into the layer's trace, and arrive at the grid barrier.
// Every wait is bounded and also gives up when another warp has aborted; a
// timeout records ASP_ERR_TIMEOUT, and the producer drains the copies it
// issued before the CTA exits.
#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kWarps = 8;                       // consumer warps
constexpr int kConsumers = kWarps * 32;
constexpr int kChainThreads = kConsumers + 32;  // + the producer warp
constexpr int kRhs = 32;     // right-hand sides per launch (two per lane, 16 lanes)
// chunk width and ring depths (fewer, larger chunks: each handoff costs about a microsecond)
// (the widest complex64 tile takes narrower chunks so that everything fits the 227 KB)
template <typename R, int RPL> struct ChainKC { static constexpr int v = 64, ts = 6, ss = 3; };
template <int RPL> struct ChainKC<float, RPL> {
  static constexpr int v = RPL <= 7 ? 256 : 128, ts = RPL <= 7 ? 3 : 6, ss = RPL <= 7 ? 2 : 3;
};

template <typename R, int RPL> struct ChainLayout {
  using C = Cx<R>;
  static constexpr int KC = ChainKC<R, RPL>::v;
  static constexpr int kTStages = ChainKC<R, RPL>::ts;  // map-chunk ring depth
  static constexpr int kSStages = ChainKC<R, RPL>::ss;  // trace-chunk ring depth
  static constexpr int KCP = KC + 2;  // padded map row: rows RPL apart fall in different banks
  static constexpr int MR = 2 * RPL;  // rows per CTA
  static constexpr size_t bar_bytes = 256;
  static constexpr size_t t_elems = (size_t)kTStages * MR * KCP;
  static constexpr size_t s_stage = (size_t)KC * kRhs;  // a trace chunk, rows lda <= kRhs apart
  static constexpr size_t s_elems = (size_t)kSStages * s_stage;
  static constexpr size_t d_elems = (size_t)MR * kRhs;  // the layer's own trace rows (u~_{p,p} on entry)
  // the cross-warp reduction reuses the trace ring, in passes over row halves if needed
  static constexpr int NPASS = ((size_t)kWarps * MR * kRhs <= s_elems) ? 1 : 2;
  static constexpr int RPP = NPASS == 1 ? MR : RPL;  // rows per reduction pass
  static_assert((size_t)kWarps * RPP * kRhs <= s_elems, "reduction buffer must fit in the trace ring");
  static_assert((2 * (kTStages + kSStages) + 1) * 8 <= bar_bytes, "mbarrier area");
  static constexpr size_t bytes() { return bar_bytes + (t_elems + s_elems + d_elems) * sizeof(C); }
  static_assert(bar_bytes + (t_elems + s_elems + d_elems) * sizeof(C) + 64 <= 232448, "shared memory per CTA");
};

__device__ __forceinline__ void pair_ld(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void pair_ld(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }

// Bounded wait for an mbarrier phase that also returns (false) once *abort is set.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const uint32_t addr = smem_addr(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort) return false;
  }
  return false;
}
// The consumers' wait: test_wait does not suspend the thread, so a consumer
// resumes as soon as its chunk lands.
__device__ __forceinline__ bool spin_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const uint32_t addr = smem_addr(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

template <typename R, int RPL>
__global__ void __launch_bounds__(kChainThreads, 1) chain_kernel(ChainParams P) {
  using C = Cx<R>;
  using Lay = ChainLayout<R, RPL>;
  constexpr int KC = Lay::KC, KCP = Lay::KCP, MR = Lay::MR;
  constexpr int kTStages = Lay::kTStages, kSStages = Lay::kSStages;
  constexpr int CB = (int)sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* fullT = reinterpret_cast<uint64_t*>(smem_raw);  // [kTStages], one arrival + bytes
  uint64_t* emptyT = fullT + kTStages;                      // [kTStages], one arrival per consumer warp
  uint64_t* fullS = emptyT + kTStages;                      // [kSStages]
  uint64_t* emptyS = fullS + kSStages;                      // [kSStages]
  uint64_t* fullD = emptyS + kSStages;                       // the layer's own trace rows
  C* s_T = reinterpret_cast<C*>(smem_raw + Lay::bar_bytes);  // [kTStages][MR][KCP]
  C* s_S = s_T + Lay::t_elems;                               // [kSStages][KC][lda]
  C* s_D = s_S + Lay::s_elems;                               // [rows][lda]
  C* red = s_S;                                              // [kWarps][RPP][kRhs]
  __shared__ int s_abort;
  volatile int* abort = &s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = gridDim.x / 2;
  const bool isR = (int)blockIdx.x < half;
  const int cta = isR ? blockIdx.x : blockIdx.x - half;
  const int nct = isR ? half : (int)gridDim.x - half;
  const int n = P.n, m = P.m, lda = P.ldacc, nrhs = P.nrhs, ldT = P.ldT;
  unsigned int* bar = P.bar + (isR ? 0 : 1);
  C* acc = reinterpret_cast<C*>(isR ? P.accR : P.accL);

  const int row0 = (int)((long long)cta * n / nct);
  const int rows = (int)((long long)(cta + 1) * n / nct) - row0;  // <= MR (checked on the host)
  const int nch = (n + KC - 1) / KC;
  const int layers = m - 2;
  const int total = layers * nch;  // chunks of each kind this CTA consumes
  auto layer_p = [&](int t) { return isR ? 2 + t : m - 1 - t; };

  if (tid == 0) {
    for (int s = 0; s < kTStages; ++s) { mbar_init(&fullT[s], 1); mbar_init(&emptyT[s], kWarps); }
    for (int s = 0; s < kSStages; ++s) { mbar_init(&fullS[s], 1); mbar_init(&emptyS[s], kWarps); }
    mbar_init(fullD, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kWarps) {
    // ================================================================ producer
    const C* tm = reinterpret_cast<const C*>(P.tmap);
    auto issue_T = [&](int g) {  // map chunk g (layer g / nch, columns (g % nch) * KC ..); whole warp
      const int t = g / nch, kc = (g - t * nch) * KC;
      const int kn = min(KC, n - kc);
      const int kcopy = (CB == 8) ? ((kn + 1) & ~1) : kn;  // 16-byte multiple; the padded row holds it
      const uint32_t rbytes = (uint32_t)(kcopy * CB);
      const int pp = layer_p(t);
      const C* T = tm + (isR ? P.toffR[pp] : P.toffL[pp]) + (long long)row0 * ldT + kc;
      const int st = g % kTStages;
      if (lane == 0) mbar_arrive_expect_tx(&fullT[st], rbytes * (uint32_t)rows);
      __syncwarp();
      for (int r = lane; r < rows; r += 32)
        bulk_g2s(s_T + ((size_t)st * MR + r) * KCP, T + (long long)r * ldT, rbytes, &fullT[st]);
    };
    auto issue_S = [&](int g) {  // trace chunk g: rows kc .. kc+kn of the previous layer's trace; lane 0
      const int t = g / nch, kc = (g - t * nch) * KC;
      const int kn = min(KC, n - kc);
      const int pp = layer_p(t);
      if (kc == 0) {  // with a layer's first chunk: the CTA's rows of that layer's own trace
        const uint32_t dbytes = (uint32_t)((long long)rows * lda * CB);
        mbar_arrive_expect_tx(fullD, dbytes);
        bulk_g2s(s_D, acc + (long long)pp * n * lda + (long long)row0 * lda, dbytes, fullD);
      }
      const C* src = acc + (long long)(isR ? pp - 1 : pp + 1) * n * lda + (long long)kc * lda;
      const uint32_t bytes = (uint32_t)((long long)kn * lda * CB);  // lda even: a 16-byte multiple
      const int ss = g % kSStages;
      mbar_arrive_expect_tx(&fullS[ss], bytes);
      bulk_g2s(s_S + (size_t)ss * Lay::s_stage, src, bytes, &fullS[ss]);
    };
    // the producer's own bounded wait for every CTA's rows of layers < t (lane 0)
    auto grid_wait = [&](int t) {
      const unsigned target = (unsigned)t * (unsigned)nct;
      for (uint32_t spins = 0;; ++spins) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) break;
        if (*abort) return false;
        if (spins > kSpinLimit) {
          record_error(P.err, ASP_ERR_TIMEOUT, 1000000 + (int)blockIdx.x);
          *abort = 1;
          return false;
        }
      }
      // the trace written by the other CTAs is read through the async proxy
      asm volatile("fence.proxy.async.global;" ::: "memory");
      return true;
    };
    int gT = 0, gS = 0;  // next map / trace chunk to issue
    for (; gT < kTStages && gT < total; ++gT) issue_T(gT);
    if (lane == 0)
      for (; gS < kSStages && gS < nch; ++gS) issue_S(gS);
    gS = __shfl_sync(0xffffffffu, gS, 0);
    bool ok = true;
    // each chunk the consumers release frees one stage of each ring
    for (int c = 0; c < total && ok; ++c) {
      if (gT < total) {  // gT == c + kTStages: its stage held chunk c
        int freed = 0;
        if (lane == 0) freed = wait_or_abort(&emptyT[c % kTStages], (uint32_t)((c / kTStages) & 1), abort) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, freed, 0)) { ok = false; break; }
        issue_T(gT++);
      }
      if (lane == 0) {
        // trace chunks whose stage is free (held chunk <= c); a layer's first
        // chunk only once every CTA has written the previous layer
        for (; ok && gS < total && gS <= c + kSStages; ++gS) {
          const int prev = gS - kSStages;  // the chunk this stage held
          if (prev >= 0 && !wait_or_abort(&emptyS[prev % kSStages], (uint32_t)((prev / kSStages) & 1), abort)) {
            ok = false;
            break;
          }
          if (gS % nch == 0 && !grid_wait(gS / nch)) { ok = false; break; }
          issue_S(gS);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      gS = __shfl_sync(0xffffffffu, gS, 0);
    }
    // drain: the last chunk issued into each stage has landed (bounded)
    if (lane == 0) {
      for (int g = max(0, gT - kTStages); g < gT; ++g) mbar_wait(&fullT[g % kTStages], (uint32_t)((g / kTStages) & 1));
      for (int g = max(0, gS - kSStages); g < gS; ++g) mbar_wait(&fullS[g % kSStages], (uint32_t)((g / kSStages) & 1));
      if (gS > 0) mbar_wait(fullD, (uint32_t)(((gS - 1) / nch) & 1));
    }
    return;
  }

  // ================================================================ consumers
  // After an abort the consumers still pass every consumer barrier and arrive at
  // the grid barrier (so that no warp or CTA waits on them), doing no work.
  const int rp = lane & 15;  // right-hand-side pair of this lane
  const int rh = lane >> 4;  // row half: rows rh*RPL .. rh*RPL+RPL-1
  bool live = true;
  for (int t = 0; t < layers; ++t) {
    C* dst = acc + (long long)layer_p(t) * n * lda;
    C a[RPL][2];
#pragma unroll
    for (int i = 0; i < RPL; ++i) a[i][0] = a[i][1] = czero<R>();

    for (int ch = 0; ch < nch && live; ++ch) {
      const int g = t * nch + ch;
      const int st = g % kTStages, ss = g % kSStages;
      const bool landed = spin_or_abort(&fullT[st], (uint32_t)((g / kTStages) & 1), abort) &&
                          spin_or_abort(&fullS[ss], (uint32_t)((g / kSStages) & 1), abort);
      if (!__all_sync(0xffffffffu, landed)) {  // warp-uniform
        if (lane == 0 && !*abort) {
          record_error(P.err, ASP_ERR_TIMEOUT, 2000000 + (int)blockIdx.x);
          *abort = 1;
        }
        live = false;
        break;
      }
      const int kn = min(KC, n - ch * KC);
      const C* bT = s_T + (size_t)st * MR * KCP + (size_t)rh * RPL * KCP;
      const C* bS = s_S + (size_t)ss * Lay::s_stage + 2 * rp;
      const int npair = kn >> 1;
      // column pairs warp, warp + kWarps, ...; the next pair's operands are
      // loaded into the other register set while this pair's products issue
      C sv[sizeof(R) == 4 ? 2 : 1][4], tv[sizeof(R) == 4 ? 2 : 1][RPL][2];
      auto ld = [&](int b, int kp) {
        const int kk = 2 * kp;
        pair_ld(bS + kk * lda, sv[b][0], sv[b][1]);
        pair_ld(bS + (kk + 1) * lda, sv[b][2], sv[b][3]);
#pragma unroll
        for (int i = 0; i < RPL; ++i) pair_ld(bT + i * KCP + kk, tv[b][i][0], tv[b][i][1]);
      };
      auto mac = [&](int b) {
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          cfma(a[i][0], tv[b][i][0], sv[b][0]);
          cfma(a[i][1], tv[b][i][0], sv[b][1]);
          cfma(a[i][0], tv[b][i][1], sv[b][2]);
          cfma(a[i][1], tv[b][i][1], sv[b][3]);
        }
      };
      if constexpr (sizeof(R) == 4) {
        if (warp < npair) ld(0, warp);
        for (int kp = warp; kp < npair; kp += 2 * kWarps) {
          if (kp + kWarps < npair) ld(1, kp + kWarps);
          mac(0);
          if (kp + kWarps >= npair) break;
          if (kp + 2 * kWarps < npair) ld(0, kp + 2 * kWarps);
          mac(1);
        }
      } else {  // complex128 (checking path): one register set
        for (int kp = warp; kp < npair; kp += kWarps) {
          ld(0, kp);
          mac(0);
        }
      }
      if ((kn & 1) && warp == npair % kWarps) {  // odd last column
        const int kk = kn - 1;
        C s0, s1;
        pair_ld(bS + kk * lda, s0, s1);
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const C tv = bT[i * KCP + kk];
          cfma(a[i][0], tv, s0);
          cfma(a[i][1], tv, s1);
        }
      }
      __syncwarp();
      if (lane == 0) {  // this warp is done with both stages
        mbar_arrive1(&emptyT[st]);
        mbar_arrive1(&emptyS[ss]);
      }
    }
    // cross-warp reduction into dst through the trace ring: every consumer warp
    // is past its last read of this layer's traces, and the producer issues the
    // next layer's only after this CTA has arrived at the grid barrier below
    consumer_sync();
    live = live && !*abort;
    if (live && !spin_or_abort(fullD, (uint32_t)(t & 1), abort)) {  // the CTA-uniform abort flag decides below
      if (!*abort) {
        record_error(P.err, ASP_ERR_TIMEOUT, 3000000 + (int)blockIdx.x);
        *abort = 1;
      }
    }
    consumer_sync();
    live = live && !*abort;
#pragma unroll
    for (int h = 0; h < Lay::NPASS; ++h) {
      if (live && (Lay::NPASS == 1 || rh == h)) {
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int rr = (Lay::NPASS == 1 ? rh * RPL : 0) + i;
          C* rw = red + ((size_t)warp * Lay::RPP + rr) * kRhs + 2 * rp;
          rw[0] = a[i][0];
          rw[1] = a[i][1];
        }
      }
      consumer_sync();
      for (int o = tid; live && o < Lay::RPP * nrhs; o += kConsumers) {
        const int rr = o / nrhs, r = o - rr * nrhs;
        const int row = (Lay::NPASS == 1 ? 0 : h * RPL) + rr;
        if (row >= rows) continue;
        C s = czero<R>();
#pragma unroll
        for (int wv = 0; wv < kWarps; ++wv) s = cadd(s, red[((size_t)wv * Lay::RPP + rr) * kRhs + r]);
        dst[(long long)(row0 + row) * lda + r] = cadd(s_D[row * lda + r], s);
      }
      // red (shared) and the trace (global) are next written or read by bulk copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      consumer_sync();
    }
    if (tid == 0) {  // this CTA's rows of layer t are written
      __threadfence();
      atomicAdd(bar, 1u);
    }
  }
}

template <typename R, int RPL> cudaError_t launch_rpl(const ChainParams& P, int grid, cudaStream_t s) {
  const size_t smem = ChainLayout<R, RPL>::bytes();
  cudaError_t e = ensure_dyn_smem((const void*)chain_kernel<R, RPL>, smem);
  if (e != cudaSuccess) return e;
  ChainParams Q = P;
  void* args[] = {&Q};
  return cudaLaunchCooperativeKernel((void*)chain_kernel<R, RPL>, dim3(grid), dim3(kChainThreads), args, smem, s);
}

template <typename R> cudaError_t launch_prec(const ChainParams& P, int grid, int maxrows, cudaStream_t s) {
  if (maxrows <= 8) return launch_rpl<R, 4>(P, grid, s);
  if (maxrows <= 14) return launch_rpl<R, 7>(P, grid, s);
  return launch_rpl<R, 8>(P, grid, s);
}

}  // namespace

cudaError_t launch_chain(Handle& H, const ChainParams& P, cudaStream_t s) {
  if (P.m < 3) return cudaSuccess;
  if (P.nrhs < 1 || P.nrhs > kRhs) return cudaErrorInvalidValue;
  int half = H.num_sms / 2;
  if (half > P.n) half = P.n;
  if (half < 1) half = 1;
  while ((P.n + half - 1) / half > 16) ++half;  // rows per CTA must fit the largest tile
  if (2 * half > H.num_sms) return cudaErrorInvalidValue;  // cooperative: one CTA per SM
  const int maxrows = (P.n + half - 1) / half;
  cudaError_t e = cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  e = H.prec == ASP_PREC_C128 ? launch_prec<double>(P, 2 * half, maxrows, s)
                              : launch_prec<float>(P, 2 * half, maxrows, s);
  H.launches += 1;
  return e;
}

}  // namespace asp
