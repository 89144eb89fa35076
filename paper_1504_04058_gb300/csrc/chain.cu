// chain.cu -- the sequential part of Algorithm 2: accumulation of the boundary
// traces along the right-going and left-going sweeps (Section 2.2 and Section
// 3.1 "Putting together"):
//     (u~_{p,1:p})^R = (G~_p^R (u~_{p-1,1:p-1})^R)^R + (u~_{p,p})^R,   p = 2..m-1
//     (u~_{p,p:m})^L = (u~_{p,p})^L + (G~_p^L (u~_{p+1,p+1:m})^L)^L,   p = m-1..2
// Only the traces travel from layer to layer, so the map w -> (G~_p^R w)^R is
// applied as a dense n x n matrix T_p^R built once at factor time (btsolve.cuh,
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
//     ahead across layer boundaries), and trace chunks (the launch's columns of
//     KC rows of the previous layer's trace, packed) in a kSStages-deep ring,
//     with a layer's first chunk also the CTA's rows of that layer's own trace.
//     It also waits at the grid barrier, and issues a layer's trace chunks only
//     once the barrier shows every CTA's part of the previous layer written;
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
constexpr int kRhs = 32;     // most right-hand sides per launch
// Chunk width and ring depths: fewer, larger chunks (each handoff costs about
// a microsecond) as far as shared memory allows.  MRT: map rows a CTA holds
// (the launcher gives a CTA at most kChainMaxRows = 16 rows, and asp_setup
// refuses 2D grids that would need more).
template <typename R, int MRT, int NR> struct ChainKC { static constexpr int v = 64, ts = 6, ss = 3; };
template <int MRT, int NR> struct ChainKC<float, MRT, NR> {
  static constexpr bool wide = MRT <= 14 || NR <= 8;
  static constexpr int v = wide ? 256 : 128, ts = wide ? (NR <= 8 ? 4 : 3) : 6, ss = wide ? 2 : 3;
};

// Lane layout: RP right-hand-side pairs across a warp row, RH = 32 / RP row
// groups of RPL rows each.  RP = 16 serves up to 32 right-hand sides, RP = 4
// up to 8, RP = 1 up to 2 (fewer right-hand sides do proportionally less work);
// lanes whose rows lie past MRT repeat row group 0 and their results are dropped.
template <typename R, int RPL, int RP> struct ChainLayout {
  using C = Cx<R>;
  static constexpr int RH = 32 / RP;
  static constexpr int MR = RH * RPL;              // rows the lane layout covers
  static_assert(kChainMaxRows == 16, "the lane layouts and ring sizes are chosen for 16 rows per CTA");
  static constexpr int MRT = MR < kChainMaxRows ? MR : kChainMaxRows;  // rows a CTA holds
  static constexpr int NR = 2 * RP;                // right-hand sides per launch
  static constexpr int KC = ChainKC<R, MRT, NR>::v;
  static constexpr int kTStages = ChainKC<R, MRT, NR>::ts;  // map-chunk ring depth
  static constexpr int kSStages = ChainKC<R, MRT, NR>::ss;  // trace-chunk ring depth
  static constexpr int KCP = KC + 2;  // padded map row: neighbouring row groups fall in different banks
  static constexpr size_t bar_bytes = 256;
  static constexpr size_t t_elems = (size_t)kTStages * MRT * KCP;
  static constexpr size_t s_stage = (size_t)KC * NR;  // a trace chunk, rows nr2 <= NR apart
  static constexpr size_t s_elems = (size_t)kSStages * s_stage;
  static constexpr size_t d_elems = (size_t)MRT * NR;  // the layer's own trace rows (u~_{p,p} on entry)
  // the cross-warp reduction reuses the trace ring, in passes over halves of the rows if needed
  static constexpr int NPASS = ((size_t)kWarps * MRT * NR <= s_elems) ? 1 : 2;
  static constexpr int RPP = (MRT + NPASS - 1) / NPASS;  // rows per reduction pass
  static_assert((size_t)kWarps * RPP * NR <= s_elems, "reduction buffer must fit in the trace ring");
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

template <typename R, int RPL, int RP>
__global__ void __launch_bounds__(kChainThreads, 1) chain_kernel(ChainParams P) {
  using C = Cx<R>;
  using Lay = ChainLayout<R, RPL, RP>;
  constexpr int KC = Lay::KC, KCP = Lay::KCP, MRT = Lay::MRT, NR = Lay::NR;
  constexpr int kTStages = Lay::kTStages, kSStages = Lay::kSStages;
  constexpr int CB = (int)sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* fullT = reinterpret_cast<uint64_t*>(smem_raw);  // [kTStages], one arrival + bytes
  uint64_t* emptyT = fullT + kTStages;                      // [kTStages], one arrival per consumer warp
  uint64_t* fullS = emptyT + kTStages;                      // [kSStages]
  uint64_t* emptyS = fullS + kSStages;                      // [kSStages]
  uint64_t* fullD = emptyS + kSStages;                       // the layer's own trace rows
  C* s_T = reinterpret_cast<C*>(smem_raw + Lay::bar_bytes);  // [kTStages][MRT][KCP]
  C* s_S = s_T + Lay::t_elems;                               // [kSStages][KC][lda]
  C* s_D = s_S + Lay::s_elems;                               // [rows][lda]
  C* red = s_S;                                              // [kWarps][RPP][NR]
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

  // this launch's columns of a trace row, rounded up to even (16 bytes for
  // complex64; lda is even, so the padded row holds the extra column)
  const int nr2 = (nrhs + 1) & ~1;
  const uint32_t rb = (uint32_t)(nr2 * CB);
  const bool whole = lda == nr2;
  const int row0 = (int)((long long)cta * n / nct);
  const int rows = (int)((long long)(cta + 1) * n / nct) - row0;  // <= MRT (checked on the host)
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
        bulk_g2s(s_T + ((size_t)st * MRT + r) * KCP, T + (long long)r * ldT, rbytes, &fullT[st]);
    };
    // trace chunk g: rows kc .. kc+kn of the previous layer's trace, this
    // launch's nr2 columns of each, packed nr2 apart in shared memory; with a
    // layer's first chunk also the CTA's rows of that layer's own trace.  When
    // the launch covers whole trace rows (lda == nr2, every handle with at most
    // 32 right-hand sides) each is one contiguous bulk copy; otherwise one copy
    // per row across the warp (small copies are slow, but only handles with
    // more than 32 right-hand sides take this path)
    auto issue_S = [&](int g) {  // whole warp
      const int t = g / nch, kc = (g - t * nch) * KC;
      const int kn = min(KC, n - kc);
      const int pp = layer_p(t);
      const int ss = g % kSStages;
      if (lane == 0) {
        if (kc == 0) mbar_arrive_expect_tx(fullD, rb * (uint32_t)rows);
        mbar_arrive_expect_tx(&fullS[ss], rb * (uint32_t)kn);
      }
      __syncwarp();
      asm volatile("fence.proxy.async.global;" ::: "memory");  // traces written by other CTAs
      const C* own = acc + (long long)pp * n * lda + (long long)row0 * lda;
      const C* src = acc + (long long)(isR ? pp - 1 : pp + 1) * n * lda + (long long)kc * lda;
      C* dS = s_S + (size_t)ss * Lay::s_stage;
      if (whole) {
        if (lane == 0) {
          if (kc == 0) bulk_g2s(s_D, own, rb * (uint32_t)rows, fullD);
          bulk_g2s(dS, src, rb * (uint32_t)kn, &fullS[ss]);
        }
      } else {
        if (kc == 0)
          for (int r = lane; r < rows; r += 32) bulk_g2s(s_D + (size_t)r * nr2, own + (long long)r * lda, rb, fullD);
        for (int kk = lane; kk < kn; kk += 32) bulk_g2s(dS + (size_t)kk * nr2, src + (long long)kk * lda, rb, &fullS[ss]);
      }
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
    int gT = 0, gS = 0;  // next map / trace chunk to issue (warp-uniform)
    for (; gT < kTStages && gT < total; ++gT) issue_T(gT);
    for (; gS < kSStages && gS < nch; ++gS) issue_S(gS);
    bool ok = true;
    // each chunk the consumers release frees one stage of each ring
    for (int c = 0; c < total && ok; ++c) {
      if (gT < total) {  // gT == c + kTStages: its stage held chunk c
        int freed = 0;
        if (lane == 0) freed = wait_or_abort(&emptyT[c % kTStages], (uint32_t)((c / kTStages) & 1), abort) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, freed, 0)) { ok = false; break; }
        issue_T(gT++);
      }
      // trace chunks whose stage is free (held chunk <= c); a layer's first
      // chunk only once every CTA has written the previous layer
      for (; ok && gS < total && gS <= c + kSStages; ++gS) {
        int go = 1;
        if (lane == 0) {
          const int prev = gS - kSStages;  // the chunk this stage held
          if (prev >= 0 && !wait_or_abort(&emptyS[prev % kSStages], (uint32_t)((prev / kSStages) & 1), abort)) go = 0;
          else if (gS % nch == 0 && !grid_wait(gS / nch)) go = 0;
        }
        if (!__shfl_sync(0xffffffffu, go, 0)) { ok = false; break; }
        issue_S(gS);
      }
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
  const int rp = lane % RP;  // right-hand-side pair of this lane
  const int rh = lane / RP;  // row group: rows rh*RPL .. rh*RPL+RPL-1
  const bool active = rh * RPL + RPL <= MRT;  // this lane's rows are held (MRT is a multiple of RPL)
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
      const C* bT = s_T + (size_t)st * MRT * KCP + (size_t)(active ? rh * RPL : 0) * KCP;
      const C* bS = s_S + (size_t)ss * Lay::s_stage + 2 * rp;
      const int npair = kn >> 1;
      // column pairs warp, warp + kWarps, ...; the next pair's operands are
      // loaded into the other register set while this pair's products issue
      C sv[sizeof(R) == 4 ? 2 : 1][4], tv[sizeof(R) == 4 ? 2 : 1][RPL][2];
      auto ld = [&](int b, int kp) {
        const int kk = 2 * kp;
        pair_ld(bS + kk * nr2, sv[b][0], sv[b][1]);
        pair_ld(bS + (kk + 1) * nr2, sv[b][2], sv[b][3]);
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
        pair_ld(bS + kk * nr2, s0, s1);
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
      constexpr int RPP = Lay::RPP;
      if (live && active) {
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int rr = rh * RPL + i - h * RPP;  // this lane's row within the pass
          if (rr >= 0 && rr < RPP) {
            C* rw = red + ((size_t)warp * RPP + rr) * NR + 2 * rp;
            rw[0] = a[i][0];
            rw[1] = a[i][1];
          }
        }
      }
      consumer_sync();
      for (int o = tid; live && o < RPP * nrhs; o += kConsumers) {
        const int rr = o / nrhs, r = o - rr * nrhs;
        const int row = h * RPP + rr;
        if (row >= rows) continue;
        C s = czero<R>();
#pragma unroll
        for (int wv = 0; wv < kWarps; ++wv) s = cadd(s, red[((size_t)wv * RPP + rr) * NR + r]);
        dst[(long long)(row0 + row) * lda + r] = cadd(s_D[row * nr2 + r], s);
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

template <typename R, int RPL, int RP> cudaError_t launch_rpl(const ChainParams& P, int grid, cudaStream_t s) {
  const size_t smem = ChainLayout<R, RPL, RP>::bytes();
  cudaError_t e = ensure_dyn_smem((const void*)chain_kernel<R, RPL, RP>, smem);
  if (e != cudaSuccess) return e;
  ChainParams Q = P;
  void* args[] = {&Q};
  return cudaLaunchCooperativeKernel((void*)chain_kernel<R, RPL, RP>, dim3(grid), dim3(kChainThreads), args, smem, s);
}

// maxrows <= 16 (the launcher sizes the grid so)
template <typename R> cudaError_t launch_prec(const ChainParams& P, int grid, int maxrows, cudaStream_t s) {
  if (P.nrhs <= 2) return launch_rpl<R, 1, 1>(P, grid, s);   // 32 rows per CTA at most
  if (P.nrhs <= 8) return launch_rpl<R, 2, 4>(P, grid, s);   // 16 rows
  if (maxrows <= 8) return launch_rpl<R, 4, 16>(P, grid, s);
  if (maxrows <= 14) return launch_rpl<R, 7, 16>(P, grid, s);
  return launch_rpl<R, 8, 16>(P, grid, s);
}

}  // namespace

cudaError_t launch_chain(Handle& H, const ChainParams& P, cudaStream_t s) {
  if (P.m < 3) return cudaSuccess;
  if (P.nrhs < 1 || P.nrhs > kRhs) return cudaErrorInvalidValue;
  int half = H.num_sms / 2;
  if (half > P.n) half = P.n;
  if (half < 1) half = 1;
  while ((P.n + half - 1) / half > kChainMaxRows) ++half;  // rows per CTA must fit the largest tile
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
