// btsolve.cuh -- batched solves with the layer factors: the G~ operators of
// Section 3.1 ("Auxiliary Green's operators") for many subproblems and
// right-hand sides in one launch.  Included by btsolve_apply.cu (M-solves and
// sweep fills) and btsolve_aux.cu (transfer maps and single solves), which
// instantiate it.
//
// A job is (subproblem, block of right-hand sides, mode).  For one job the CTA
// runs the two passes of the block-tridiagonal solve with the factors of
// btfactor.cu (W_k = S_k^{-1}):
//     forward   z_k = W_k (g_k - a_k z_{k-1}),           k = k0 .. n-1
//     backward  x_{n-1} = z_{n-1},  x_k = z_k - c_k W_k x_{k+1},   k = n-2 .. 0
// Each step multiplies the dense w x w block W_k by a w x NR panel of
// right-hand sides.  Work split: every thread owns a TR-row x TC-column tile of
// the panel for the whole job, so the recurrences (z_{k-1} -> y_k,
// x_{k+1} -> x_k) stay in its registers; a warp covers (32/(LC*KS))*TR rows x
// LC*TC right-hand sides, the CTA stacks warps over rows (and NCW column
// blocks).  The inner product loads TR rows of W_k (16-byte shared loads of row
// pairs) and TC panel entries per column j and issues 4*TR*TC FMAs.  A
// thread's TC columns come in pairs 2*LC apart so that lanes sharing a row
// touch one contiguous span (no shared-memory bank conflicts).  With KS > 1
// (one or two right-hand sides, where a step is a short dependent chain) KS
// lanes share each tile, each takes every KS-th column j, and a butterfly of
// shuffles sums their partial products; one lane of the group stores.
//
// Data movement: the W_k blocks stream from HBM through an STG-stage
// shared-memory ring (3; 6 for few right-hand sides; 2 where a block near 64
// columns would overflow shared memory with more) filled by 1D bulk (TMA)
// copies that complete on mbarriers.  Complex64 factors are stored as the
// packed upper triangle of the symmetric W'_k = W_k Delta (internal.h): four
// extra producer warps issue the bulk copies of the packed blocks into a
// 3-stage landing ring and expand each into the ring of STG full blocks the
// compute warps read (ready / empty mbarriers), ahead of them, so the
// expansion stays off the steps' dependent chain; the panel rows are scaled by
// Delta^-1 when they are stored (W_k y = W'_k Delta^-1 y), and the compute
// warps synchronise on a named barrier of their own (blocks of 60 or more
// columns with many right-hand sides fall back to one landing stage and one
// full block); the per-step right-hand-side entries
// (and, in the backward pass, the z_k saved by the forward pass in a per-CTA
// scratch slot) stream through a per-thread cp.async ring.  One __syncthreads per step publishes the panel.
//
// Mode classes (compile time) and modes (per job):
//   CLS_EMBED  EMBED   G~_q^M f_q: g = input on the rows of X_q; writes x on X_q
//                      to outM and its first / last X_q column to the trace buffers.
//   CLS_FILL   FILL_R  G~_p^R w: g = -(1/h^2) accR[p-1] on local column 0; x on X_p -> outR.
//              FILL_L  G~_p^L w: g = -(1/h^2) accL[p+1] on local column w-1; -> outL.
//   CLS_TMAP   TMAP_R  columns r of the dense map w -> (G~_p^R w)^R: g = -(1/h^2) e_r on
//                      column 0; keeps the last column of X_p.  The forward pass starts
//                      at block k0 = the job's first r (earlier blocks are zero).
//              TMAP_L  same for G~_p^L: g on column w-1, keeps the first column of X_p.
//   CLS_SUB    SUB     v = H^-1 g on the whole padded grid (checking entry point).
// Per job every thread resolves, for its two rows, whether the row takes
// input, where its input and outputs live, and the per-step strides, so the
// step loop does only pointer increments.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace asp {

enum ModeClass : int { CLS_EMBED = 0, CLS_FILL = 1, CLS_TMAP = 2, CLS_SUB = 3 };

namespace bts {

constexpr int kMaxStages = 8;  // W-block ring depth: 3 by default, deeper for few right-hand sides
constexpr int kRing = 3;    // per-thread input ring depth

struct Geometry {
  int wcap;    // largest w in the launch
  int wstage;  // elements of one W stage (largest w*wp, plus slack for the row tiles)
  int pstage;  // packed factors: elements of one landing stage (largest packed block)
  int packed;  // 1: blocks stored as packed symmetric triangles (ASP_PREC_C64_SYM)
};

__host__ __device__ inline size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

template <typename R, int TR_, int TC, int LC, int NCW, int STG = 3, int KS = 1, bool PKT = false>
struct Tiling {
  static_assert(STG >= (PKT ? 1 : 2) && STG <= kMaxStages, "W-block ring depth");
  static constexpr bool PK = PKT;
  using C = Cx<R>;
  static constexpr int TR = TR_;                   // rows per thread (2 or 4)
  static constexpr int WR = (32 / (LC * KS)) * TR;  // rows per warp
  static constexpr int WC = LC * TC;           // right-hand sides per warp
  static constexpr int NR = WC * NCW;          // right-hand sides per CTA
  static constexpr int E = TR * TC;            // panel entries per thread
  // packed factors (symmetric W_k Delta, internal.h): producer warps land them
  // in an LS-stage ring and expand them into STG full blocks
  static constexpr int LS = STG == 1 ? 1 : 3;  // one landing stage only in the widest fallback
  static constexpr int kProdWarps = 4;           // producer warps of packed factors
  __host__ __device__ static size_t bars() { return 256; }
  __host__ __device__ static size_t wst(const Geometry& g) {
    return PK ? ((size_t)LS * g.pstage + (size_t)STG * g.wstage) * sizeof(C) : (size_t)STG * g.wstage * sizeof(C);
  }
  __host__ __device__ static size_t ybuf(const Geometry& g) { return (size_t)2 * g.wcap * NR * sizeof(C); }
  __host__ __device__ static size_t ring(int nt) { return (size_t)kRing * E * nt * sizeof(C); }
  __host__ __device__ static size_t total(const Geometry& g, int nt) {
    return align128(bars()) + align128(wst(g)) + align128(ybuf(g)) + align128(ring(nt));
  }
};

__device__ __forceinline__ void mbar_arrive1(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

template <typename C> struct Vec2;
template <> struct Vec2<float2> {
  __device__ static void ld(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  }
  __device__ static void st(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  }
};
template <> struct Vec2<double2> {
  __device__ static void ld(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }
  __device__ static void st(double2* p, double2 a, double2 b) { p[0] = a; p[1] = b; }
};

template <typename C, int TC, int PS> __device__ __forceinline__ void ld_cols(const C* p, C (&v)[TC]) {
  if constexpr (TC == 1) {
    v[0] = p[0];
  } else {
#pragma unroll
    for (int c = 0; c < TC; c += 2) Vec2<C>::ld(p + (c / 2) * PS, v[c], v[c + 1]);
  }
}
template <typename C, int TC, int PS> __device__ __forceinline__ void st_cols(C* p, const C (&v)[TC]) {
  if constexpr (TC == 1) {
    p[0] = v[0];
  } else {
#pragma unroll
    for (int c = 0; c < TC; c += 2) Vec2<C>::st(p + (c / 2) * PS, v[c], v[c + 1]);
  }
}

template <typename R, int TRT, int TC, int LC, int NCW, int MAXT, int MINB, int CLS, int STG, int KS, bool PKT>
__global__ void __launch_bounds__(MAXT, MINB) btsolve_kernel(SolveParams P, Geometry G) {
  using C = Cx<R>;
  using T = Tiling<R, TRT, TC, LC, NCW, STG, KS, PKT>;
  constexpr int kStages = STG;
  constexpr bool PK = T::PK;
  constexpr int TR = T::TR, WR = T::WR, WC = T::WC, NR = T::NR, E = T::E;
  constexpr int CB = (int)sizeof(C);
  constexpr int PS = 2 * LC;  // column distance between a thread's pairs
  constexpr int LS = T::LS;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kProd = T::kProdWarps;
  const int NT = PK ? (int)blockDim.x - 32 * kProd : (int)blockDim.x;  // compute threads (PK: + producer warps)
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  // PK barriers: bar[0, LS) landing copies, then ready[kStages], empty[kStages]
  uint64_t* ready = bar + LS;
  uint64_t* empty = bar + LS + kStages;
  C* Wst = reinterpret_cast<C*>(smem + align128(T::bars()));  // !PK: the W ring; PK: the landing ring
  C* Wfull = Wst + (size_t)LS * G.pstage;                      // PK: the full blocks
  C* ybuf = reinterpret_cast<C*>(smem + align128(T::bars()) + align128(T::wst(G)));
  C* ring = reinterpret_cast<C*>(smem + align128(T::bars()) + align128(T::wst(G)) + align128(T::ybuf(G)));
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wr = warp / NCW, wc = warp % NCW;
  // lane = (row group * LC + column lane) * KS + column slice: with KS > 1 the
  // KS lanes of a group share the tile and split the block's columns j
  const int js = lane % KS;
  const bool wlane = js == 0;  // the lane of a group that stores the tile's results
  const int cl = (lane / KS) % LC;
  const int i0 = wr * WR + (lane / (LC * KS)) * TR;             // first row of the tile
  const int r0 = wc * WC + (TC == 1 ? cl : 2 * cl);            // first column of the tile
  auto rhs_of = [&](int c) { return TC == 1 ? r0 : r0 + (c & 1) + (c >> 1) * PS; };
  const int n = P.n, ldv = P.ldv, lda = P.ldacc, ldT = P.ldT;
  const C* __restrict__ Wg = reinterpret_cast<const C*>(P.W);
  C* zslot = reinterpret_cast<C*>(P.zscr) + (long long)blockIdx.x * P.zslot;
  const C neg_ih2 = cmake<R>(R(-P.inv_h2), R(0));
  const C* cap = reinterpret_cast<const C*>(P.ca);
  const C* ccp = reinterpret_cast<const C*>(P.cc);

  if (tid == 0) {
    if constexpr (PK) {
      for (int s = 0; s < LS; ++s) mbar_init(&bar[s], 1);
      for (int s = 0; s < kStages; ++s) {
        mbar_init(&ready[s], 1);
        mbar_init(&empty[s], NT / 32);
      }
    } else {
      for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  // bounded wait that also gives up once another warp has aborted
  auto wait_or_abort = [&](uint64_t* b, uint32_t parity) -> bool {
    const uint32_t addr = smem_addr(b);
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
      if ((it & 1023u) == 1023u && *(volatile int*)&s_abort) return false;
    }
    return false;
  };
  // compute threads: all of the CTA, or (PK) all but the producer warp
  auto sync_compute = [&]() {
    if constexpr (PK) asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
    else __syncthreads();
  };
  // the same barrier, returning whether any warp has aborted; with a producer
  // warp that may set the flag at any time, the compute threads take one
  // common decision (an OR over their reads at the barrier)
  auto sync_compute_aborted = [&]() -> bool {
    if constexpr (PK) {
      const uint32_t mine = *(volatile int*)&s_abort ? 1u : 0u;
      uint32_t any;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\t"
          "setp.ne.u32 p, %1, 0;\n\t"
          "bar.red.or.pred q, 1, %2, p;\n\t"
          "selp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(any)
          : "r"(mine), "r"(NT)
          : "memory");
      return any != 0;
    } else {
      __syncthreads();
      return s_abort != 0;
    }
  };

  if constexpr (PK) {
    if (warp >= NT / 32) {
      // ---- producer warps: packed blocks in, full blocks out.  Thread pt of
      // the kProd*32 takes an even share of the packed entries; entry (r, c),
      // r <= c, goes to (r, c) and (c, r) of the full block.
      const int pt = tid - NT, PT = 32 * kProd;
      const bool lead = pt == 0;
      uint32_t gi = 0, ge = 0;  // copies issued, blocks expanded (across jobs)
      bool stop = false;
      for (int job = blockIdx.x; job < P.njobs && !stop; job += gridDim.x) {
        const Job J = P.jobs[job];
        const SubDesc S = P.subs[J.sub];
        const int w = S.w, wp = S.wp;
        const int k0 = (CLS == CLS_TMAP) ? J.rhs0 : 0;
        const int nf = n - k0;
        const int L = nf + (n - 1);
        const uint32_t bbytes = (uint32_t)(S.bs * CB);
        const C* Wsub = Wg + S.woff;
        auto blk = [&](int q) { return q < nf ? k0 + q : n - 2 - (q - nf); };
        // this thread's share of the packed entries and its first (r, c)
        const int np = w * (w + 1) / 2;
        const int e0 = (int)(((long long)np * pt) / PT), e1 = (int)(((long long)np * (pt + 1)) / PT);
        int c0 = (int)((sqrtf(8.f * e0 + 1.f) - 1.f) * 0.5f);
        while (c0 * (c0 + 1) / 2 > e0) --c0;
        while ((c0 + 1) * (c0 + 2) / 2 <= e0) ++c0;
        const int r0e = e0 - c0 * (c0 + 1) / 2;
        int issued = 0;
        for (int t = 0; t < L; ++t) {
          while (issued < L && issued < t + LS) {  // LS copies in flight
            if (lead) {
              const uint32_t st = gi % LS;
              mbar_arrive_expect_tx(&bar[st], bbytes);
              bulk_g2s(Wst + (size_t)st * G.pstage, Wsub + (long long)blk(issued) * S.bs, bbytes, &bar[st]);
            }
            ++gi;
            ++issued;
          }
          const uint32_t sl = ge % LS, fs = ge % kStages;
          const bool ok = wait_or_abort(&bar[sl], (ge / LS) & 1u) &&
                          (ge < (uint32_t)kStages || wait_or_abort(&empty[fs], ((ge / kStages) - 1) & 1u));
          // one common decision of the producer threads (they meet at barrier 2 below)
          uint32_t failed;
          asm volatile(
              "{\n\t.reg .pred p, q;\n\t"
              "setp.eq.u32 p, %1, 0;\n\t"
              "bar.red.or.pred q, 2, %2, p;\n\t"
              "selp.u32 %0, 1, 0, q;\n\t}"
              : "=r"(failed)
              : "r"(ok ? 1u : 0u), "r"(PT)
              : "memory");
          if (failed) {
            if (lead && !*(volatile int*)&s_abort) record_error(P.err, ASP_ERR_TIMEOUT, blockIdx.x);
            s_abort = 1;
            stop = true;
            break;
          }
          // full block (column-major, ld wp) from the packed upper triangle
          const C* pk = Wst + (size_t)sl * G.pstage;
          C* full = Wfull + (size_t)fs * G.wstage;
          int r = r0e, c = c0;
#pragma unroll 4
          for (int e = e0; e < e1; ++e) {
            const C v = pk[e];
            full[c * wp + r] = v;
            full[r * wp + c] = v;
            if (++r > c) { r = 0; ++c; }
          }
          // every producer thread's entries are in place before the block is published
          asm volatile("bar.sync 2, %0;" ::"r"(PT) : "memory");
          if (lead) mbar_arrive1(&ready[fs]);
          ++ge;
        }
      }
      if (stop && lead) {  // copies still in flight complete on their landing barrier
        for (uint32_t q = gi >= (uint32_t)LS ? gi - LS : 0; q < gi; ++q) mbar_wait(&bar[q % LS], (q / LS) & 1u);
      }
      return;
    }
  }
  uint32_t wuse = 0;  // W stages consumed so far (identical in every compute thread)

  for (int job = blockIdx.x; job < P.njobs; job += gridDim.x) {
    const Job J = P.jobs[job];
    const SubDesc S = P.subs[J.sub];
    const int w = S.w, wp = S.wp, xoff = S.xoff, xw = S.xw, lo = S.lo, p = S.p;
    const int rhs0 = J.rhs0, nr = J.nr;
    const bool right = (J.mode == MODE_FILL_R || J.mode == MODE_TMAP_R);
    const int k0 = (CLS == CLS_TMAP) ? rhs0 : 0;
    const int nf = n - k0;
    const int L = nf + (n - 1);
    const uint32_t bbytes = (uint32_t)(S.bs * CB);
    const C* Wsub = Wg + S.woff;
    auto blk = [&](int q) { return q < nf ? k0 + q : n - 2 - (q - nf); };

    // ---- per-job, per-row resolution of inputs and outputs
    const int bnd = right ? 0 : w - 1;                 // boundary-data row (FILL, TMAP)
    const int keep = right ? xoff + xw - 1 : xoff;     // kept column (TMAP)
    bool row_ok[TR], has_in[TR], out_row[TR], trR[TR], trL[TR];
    const C* in_base[TR];
    C* out_base[TR];
    long long in_step = 0, out_step = 0;
#pragma unroll
    for (int a = 0; a < TR; ++a) {
      const int i = i0 + a;
      row_ok[a] = i < w;
      const bool inx = i >= xoff && i < xoff + xw;
      has_in[a] = false; out_row[a] = false; trR[a] = false; trL[a] = false;
      in_base[a] = nullptr; out_base[a] = nullptr;
      if (CLS == CLS_EMBED) {
        has_in[a] = row_ok[a] && inx;
        in_base[a] = reinterpret_cast<const C*>(P.in) + (long long)(lo - 1 + i) * n * ldv + rhs0;
        in_step = ldv;
        out_row[a] = has_in[a];
        out_base[a] = reinterpret_cast<C*>(P.outM) + (long long)(lo - 1 + i) * n * ldv + rhs0;
        out_step = ldv;
        trR[a] = row_ok[a] && i == xoff + xw - 1;
        trL[a] = row_ok[a] && i == xoff;
      } else if (CLS == CLS_FILL) {
        has_in[a] = row_ok[a] && i == bnd;
        in_base[a] = reinterpret_cast<const C*>(right ? P.accR : P.accL) +
                     (long long)(right ? p - 1 : p + 1) * n * lda + rhs0;
        in_step = lda;
        out_row[a] = row_ok[a] && inx;
        out_base[a] = reinterpret_cast<C*>(right ? P.outR : P.outL) + (long long)(lo - 1 + i) * n * ldv + rhs0;
        out_step = ldv;
      } else if (CLS == CLS_TMAP) {
        has_in[a] = row_ok[a] && i == bnd;  // computed, not loaded
        out_row[a] = row_ok[a] && i == keep;
        out_base[a] = reinterpret_cast<C*>(P.tmap) + S.toff + rhs0;
        out_step = ldT;
      } else {  // CLS_SUB
        has_in[a] = row_ok[a];
        in_base[a] = reinterpret_cast<const C*>(P.in) + (long long)i * n * ldv + rhs0;
        in_step = ldv;
        out_row[a] = row_ok[a];
        out_step = ldv;
      }
    }
    C* zrow[TR];
#pragma unroll
    for (int a = 0; a < TR; ++a) zrow[a] = zslot + (long long)(i0 + a) * NR;
    C dr[TR];  // PK: 1/s2 of the thread's rows (panel rows are stored as Delta^-1 y)
#pragma unroll
    for (int a = 0; a < TR; ++a)
      dr[a] = (PK && row_ok[a]) ? reinterpret_cast<const C*>(P.s2inv)[S.prof + i0 + a] : cmake<R>(R(1), R(0));
    const long long zstep = (long long)w * NR;
    C* accRp = reinterpret_cast<C*>(P.accR) + (long long)p * n * lda + rhs0;
    C* accLp = reinterpret_cast<C*>(P.accL) + (long long)p * n * lda + rhs0;

    sync_compute();  // the previous job's last reads of the W ring and panels are done
    if (!PK && tid == 0) {
      for (int t = 0; t < kStages && t < L; ++t) {
        const int st = (wuse + t) % kStages;
        mbar_arrive_expect_tx(&bar[st], bbytes);
        bulk_g2s(Wst + (size_t)st * G.wstage, Wsub + (long long)blk(t) * S.bs, bbytes, &bar[st]);
      }
    }

    // per-thread ring slot of tile entry (a, c): the TC columns in adjacent
    // pairs, so that one 16-byte copy fills both entries of a pair
    auto sidx = [&](int a, int c) -> size_t {
      if constexpr (TC == 1) return (size_t)a * NT + tid;
      else return ((size_t)(a * (TC / 2) + (c >> 1)) * NT + tid) * 2 + (c & 1);
    };
    auto load_step = [&](int q2) {
      if (q2 < L) {
        const int kk = blk(q2);
        C* slot = ring + (size_t)(q2 % kRing) * E * NT;
        if (q2 < nf) {
          if (CLS != CLS_TMAP) {
#pragma unroll
            for (int a = 0; a < TR; ++a) {
              if (!has_in[a]) continue;
              const C* src = in_base[a] + (long long)kk * in_step;
#pragma unroll
              for (int c = 0; c < TC; ++c)
                if (rhs_of(c) < nr) cp_async<CB>(slot + sidx(a, c), src + rhs_of(c));
            }
          }
        } else if (kk >= k0 && kk <= n - 3) {
#pragma unroll
          for (int a = 0; a < TR; ++a) {
            if (!row_ok[a]) continue;
            const C* src = zrow[a] + (long long)kk * zstep;
            if constexpr (TC >= 2 && CB == 8) {
              // a pair's two columns are adjacent in the scratch slot (16-byte
              // aligned: the slot, the row stride NR and the pair's first column
              // are even), so half the copies
#pragma unroll
              for (int c = 0; c < TC; c += 2) cp_async<16>(slot + sidx(a, c), src + rhs_of(c));
            } else {
#pragma unroll
              for (int c = 0; c < TC; ++c) cp_async<CB>(slot + sidx(a, c), src + rhs_of(c));
            }
          }
        }
      }
      cp_async_commit();
    };
    for (int t = 0; t < kRing - 1; ++t) load_step(t);

    // carry: z_{k-1} in the forward pass, x_{k+1} in the backward pass
    C carry[TR][TC], zkeep[TR][TC];
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
      for (int c = 0; c < TC; ++c) carry[a][c] = zkeep[a][c] = czero<R>();

    C ak_next = cap[blk(0)], ck_next = ccp[blk(0)];
    for (int q = 0; q < L; ++q) {
      const int k = blk(q);
      const bool fwd = q < nf;
      const C a_k = ak_next;
      const C c_k = ck_next;
      if (q + 1 < L) {  // prefetch next step's coupling coefficients
        const int kn = blk(q + 1);
        ak_next = cap[kn];
        ck_next = ccp[kn];
      }
      load_step(q + kRing - 1);
      cp_async_wait<kRing - 1>();
      const C* slot = ring + (size_t)(q % kRing) * E * NT;
      C* yb = ybuf + (size_t)(q & 1) * G.wcap * NR;

      // ---- this step's panel rows of the thread's tile
#pragma unroll
      for (int a = 0; a < TR; ++a) {
        if (!row_ok[a]) continue;
        C y[TC];
        if (fwd) {
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            C g = czero<R>();
            if (has_in[a] && rhs_of(c) < nr) {
              if (CLS == CLS_TMAP) {
                if (k == rhs0 + rhs_of(c)) g = neg_ih2;
              } else {
                g = slot[sidx(a, c)];
                if (CLS == CLS_FILL) g = cmul(neg_ih2, g);
              }
            }
            y[c] = g;
            cfms(y[c], a_k, carry[a][c]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < TC; ++c) y[c] = carry[a][c];
        }
        if constexpr (PK) {
#pragma unroll
          for (int c = 0; c < TC; ++c) y[c] = cmul(y[c], dr[a]);
        }
        if (wlane) st_cols<C, TC, PS>(yb + (size_t)(i0 + a) * NR + r0, y);
      }
      if (sync_compute_aborted()) return;
      if (!PK && tid == 0 && q >= 1 && q - 1 + kStages < L) {
        const int st = (wuse + q - 1) % kStages;
        mbar_arrive_expect_tx(&bar[st], bbytes);
        bulk_g2s(Wst + (size_t)st * G.wstage, Wsub + (long long)blk(q - 1 + kStages) * S.bs, bbytes, &bar[st]);
      }
      const C* Wk;
      const uint32_t fs = (wuse + q) % kStages;
      if constexpr (PK) {  // the producer warp's full block
        if (!wait_or_abort(&ready[fs], ((wuse + q) / kStages) & 1u)) {
          if (!*(volatile int*)&s_abort) record_error(P.err, ASP_ERR_TIMEOUT, blockIdx.x);
          s_abort = 1;
        }
        Wk = Wfull + (size_t)fs * G.wstage;
      } else {
        const uint32_t st = (wuse + q) % kStages;
        const uint32_t par = ((wuse + q) / kStages) & 1u;
        if (!mbar_wait(&bar[st], par)) {
          record_error(P.err, ASP_ERR_TIMEOUT, blockIdx.x);
          s_abort = 1;
        }
        Wk = Wst + (size_t)st * G.wstage;
      }

      // ---- acc = W_k * panel on the thread's 2 x TC tile
      C acc[TR][TC];
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int c = 0; c < TC; ++c) acc[a][c] = czero<R>();
      if (row_ok[0]) {
        const C* yj = yb + r0 + (size_t)js * NR;
        const C* wj = Wk + i0 + (size_t)js * wp;
#pragma unroll 2
        for (int j = js; j < w; j += KS) {
          C yv[TC];
          ld_cols<C, TC, PS>(yj, yv);
          C wv[TR];
#pragma unroll
          for (int a = 0; a < TR; a += 2) Vec2<C>::ld(wj + a, wv[a], wv[a + 1]);
#pragma unroll
          for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c) cfma(acc[a][c], wv[a], yv[c]);
          yj += KS * NR;
          wj += KS * wp;
        }
      }
      if constexpr (KS > 1) {  // every lane of the group ends with the full sums
#pragma unroll
        for (int off = 1; off < KS; off <<= 1)
#pragma unroll
          for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
              acc[a][c].x += __shfl_xor_sync(0xffffffffu, acc[a][c].x, off);
              acc[a][c].y += __shfl_xor_sync(0xffffffffu, acc[a][c].y, off);
            }
      }

      if constexpr (PK) {  // this warp is done with the full block
        __syncwarp();
        if (lane == 0) mbar_arrive1(&empty[fs]);
      }

      // ---- epilogue
#pragma unroll
      for (int a = 0; a < TR; ++a) {
        if (!row_ok[a]) continue;
        C x[TC];
        if (fwd) {
          if (k <= n - 3 && wlane) st_cols<C, TC, PS>(zrow[a] + (long long)k * zstep + r0, acc[a]);
          if (k != n - 1) {
#pragma unroll
            for (int c = 0; c < TC; ++c) carry[a][c] = acc[a][c];
            continue;
          }
#pragma unroll
          for (int c = 0; c < TC; ++c) { zkeep[a][c] = carry[a][c]; x[c] = acc[a][c]; }
        } else {
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            C z = czero<R>();
            if (k >= k0) z = (k == n - 2) ? zkeep[a][c] : slot[sidx(a, c)];
            x[c] = z;
            cfms(x[c], c_k, acc[a][c]);
          }
        }
#pragma unroll
        for (int c = 0; c < TC; ++c) carry[a][c] = x[c];
        if (out_row[a] && wlane) {
          C* o = out_base[a] + (long long)k * out_step;
#pragma unroll
          for (int c = 0; c < TC; ++c)
            if (rhs_of(c) < nr) {
              if (CLS == CLS_SUB)
                reinterpret_cast<double2*>(P.outSub)[((long long)(i0 + a) * n + k) * ldv + rhs0 + rhs_of(c)] =
                    make_double2((double)x[c].x, (double)x[c].y);
              else
                o[rhs_of(c)] = x[c];
            }
        }
        if (CLS == CLS_EMBED && wlane) {
          if (trR[a]) {
#pragma unroll
            for (int c = 0; c < TC; ++c)
              if (rhs_of(c) < nr) accRp[(long long)k * lda + rhs_of(c)] = x[c];
          }
          if (trL[a]) {
#pragma unroll
            for (int c = 0; c < TC; ++c)
              if (rhs_of(c) < nr) accLp[(long long)k * lda + rhs_of(c)] = x[c];
          }
        }
      }
    }
    wuse += (uint32_t)L;
    cp_async_wait<0>();
  }
  sync_compute();
  if (tid == 0) {
    if constexpr (PK) {
      for (int s = 0; s < LS + 2 * kStages; ++s) mbar_inval(&bar[s]);
    } else {
      for (int s = 0; s < kStages; ++s) mbar_inval(&bar[s]);
    }
  }
}

// TRT: rows per thread.  MAXT / MINB: largest CTA the instance is compiled for
// and the number of such CTAs per SM its register budget is sized for.  STG:
// W-block ring depth (few right-hand sides do little work per block, so they
// need more blocks in flight to keep HBM busy).
template <typename R, int TRT, int TC, int LC, int NCW, int CLS, int MAXT = 512, int MINB = 1, int STG = 3,
          int KS = 1, bool PKT = false>
cudaError_t run(Handle& H, const SolveParams& P, int wcap, cudaStream_t s) {
  using T = Tiling<R, TRT, TC, LC, NCW, STG, KS, PKT>;
  if (H.packed != PKT) return cudaErrorInvalidValue;  // the instance must match the factor storage
  const int nrw = (wcap + T::WR - 1) / T::WR;
  const int nt = 32 * nrw * NCW;                 // compute threads
  constexpr bool packed = PKT;
  const int nlaunch = nt + (packed ? 32 * T::kProdWarps : 0);  // + the producer warps of packed factors
  if (nlaunch > MAXT) return cudaErrorInvalidValue;
  Geometry G;
  G.wcap = wcap;
  const int wpc = (sizeof(R) == 4) ? ((wcap + 1) & ~1) : wcap;
  // slack: the 2-row tiles of the last row block may read up to WR rows past
  // column w-1 of a stage (their results are discarded)
  G.wstage = wcap * wpc + T::WR * nrw + 2;
  if (sizeof(R) == 4) G.wstage = (G.wstage + 1) & ~1;
  G.pstage = packed_block_elems(wcap);
  G.packed = packed ? 1 : 0;
  const size_t smem = T::total(G, nt);
  auto kern = btsolve_kernel<R, TRT, TC, LC, NCW, MAXT, MINB, CLS, STG, KS, PKT>;
  if constexpr (STG > 2 || (PKT && STG > 1)) {
    // Wide blocks (w near 64 with many right-hand sides) can need more than
    // the opt-in shared memory with a deep W ring; they run with two stages
    // (packed factors: then one full block).
    // The limit is the device's opt-in size less the kernel's static shared
    // bytes, read once per instance (thread-safe static initialisation).
    static const size_t dyn_limit = [kern]() -> size_t {
      int dev = 0, optin = 0;
      cudaFuncAttributes fa{};
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, (const void*)kern) != cudaSuccess)
        return 0;
      return (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    }();
    // (packed factors may go on to one full block; the plain ring keeps two)
    if (smem > dyn_limit) return run<R, TRT, TC, LC, NCW, CLS, MAXT, MINB, (STG > 2 ? 2 : 1), KS, PKT>(H, P, wcap, s);
  }
  cudaError_t e = ensure_dyn_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  int grid = P.njobs < P.zslots ? P.njobs : P.zslots;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, nlaunch, smem, s>>>(P, G);
  H.launches += 1;
  return cudaGetLastError();
}

}  // namespace bts

}  // namespace asp
