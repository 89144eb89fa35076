// tmap_tc.cu -- the dense trace-transfer maps of the two sweeps (Section 3.1,
// "Putting together") for complex64 factors, built on the tcgen05 tensor cores
// from the diagonal blocks of the subproblem inverse.
//
// A map is an n x n block of the inverse of one layer subproblem H = H_p^R (or
// H_p^L):  T[k][r] = -(1/h^2) G_{(k,keep),(r,in)}, G = H^-1, where `in` is the
// boundary-data column (local 0 for H^R, w-1 for H^L) and `keep` the traced
// column of X_p (its last column for R, its first for L).  Ordered x2-fastest,
// H is block tridiagonal: n diagonal blocks T_k (w x w), couplings a_k I to
// block k-1 and c_k I to block k+1, factored by btfactor.cu into
// W_k = S_k^-1 (S_0 = T_0, S_k = T_k - a_k c_{k-1} W_{k-1}).  Three identities
// give every entry of the map with one chain per column and no stored
// intermediate vectors:
//   * up-chain: for k < r, G_{k,r} = -c_k W_k G_{k+1,r} (the forward pass of a
//     solve with data in block r is zero above block r, so its backward pass
//     is this chain);
//   * diagonal blocks: Gamma_{n-1} = W_{n-1},
//     Gamma_k = W_k + c_k a_{k+1} W_k Gamma_{k+1} W_k  (Gamma_k = G_{k,k});
//   * symmetry: D^-1 H is complex symmetric for D = diag(s1_k s2_j) (the PML
//     weights of the x1 node and of the sweep column; Section 3.1, practical
//     remark 4), so G_{(k,keep),(r,in)} = G_{(r,in),(k,keep)} s1_k s2_keep /
//     (s1_r s2_in).
// So the upper triangle and diagonal (k <= r) come from the columns
// x^(r)_r = Gamma_r e_in, x^(r)_k = -c_k W_k x^(r)_{k+1}, T[k][r] = -(1/h^2) x^(r)_k[keep]
// ("family A"), and the lower triangle (k > r) from the columns with data in
// `keep`: y^(k)_k = Gamma_k e_keep, y^(k)_j = -c_j W_j y^(k)_{j+1},
// T[k][j] = -(1/h^2) rho s1_k / s1_j y^(k)_j[in] with rho = s2_keep / s2_in
// ("family B").  Both families advance with the same -c_k W_k at step k, so
// one CTA runs a 128-column tile of each over the same steps and stages each
// W_k once.  Per map this is n(n-1) w^2 complex multiply-adds against
// 1.5 n^2 w^2 for building the columns by forward and backward solves, and it
// needs no forward-pass scratch.
//
// With packed factors (ASP_PREC_C64_SYM) the blocks arrive as the upper
// triangle of the symmetric W'_k = W_k Delta (internal.h), and both kernels
// read W_k[i][j] = W'_k(i, j) / s2_j; otherwise full blocks (ld wp).
//
// gdiag_kernel runs the Gamma recursion (one CTA per map, n dependent steps of
// two w x w x w complex products in shared memory) and stores Gamma_k e_in and
// Gamma_k e_keep for every k.
//
// tmap_tc_kernel runs the chains on the tensor cores.  A tile's state (128
// columns x w complex) is the real matrix A (128 x 2w, re and im interleaved
// along K) and lives in tensor memory, one column per row: the MMAs read it
// from there and the epilogue writes the next state back with tcgen05.st, so
// shared memory carries only the small W operand.  -c_k W_k becomes the real
// matrix B_k^T (2w x 2w) with the 2 x 2 block [[re v, -im v], [im v, re v]] per
// complex entry, so D = A B_k^T is the next state in the same layout.  Split precision as in the
// 3D Schur update: x_hi = x with its 13 low mantissa bits cleared, x_lo =
// x - x_hi, D = A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (kind::tf32, M = 128,
// N = 2w rounded up to 16, K = 8 per instruction), which keeps the maps within
// a small factor of complex64 accuracy.  Persistent CTAs walk the jobs
// (map, 128-column tile), longest first.  Warp roles:
//   warp 0      TMA producer: W_k and the step's two diagonal-block columns by
//               1D bulk copies into a ring of W stages (and the TMEM allocation);
//   warp 1      MMA issuer: per step, both tiles' products into their TMEM
//               accumulators once B_k is in shared memory and the tile's state
//               in tensor memory;
//   warps 2-5   converter: -c_k W_k into the split B_k^T stage (128-byte
//               swizzled, as the MMA descriptors read it), and the step's
//               injected columns and output scale into a small ring;
//   warps 6-9   epilogue of the family-A tile, warps 10-13 of the family-B
//               tile: one thread per column reads its accumulator row
//               (tcgen05.ld), injects Gamma_k e at r = k, writes the map
//               entries, and stores the split state back (tcgen05.st) for the
//               next step.
// Every wait is bounded; a timeout records ASP_ERR_TIMEOUT and makes every role
// stop; the issuer then waits (bounded) for its products and the producer for
// its copies before the tensor memory is freed.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kTT = 128;       // columns per tile (the MMA's M)
constexpr int kGS = 32;        // complex entries per stored diagonal-block column (>= w)
constexpr int kThreadsTm = 14 * 32;
constexpr int kInjRing = 4;    // steps of injected columns held by the converter ring
// tensor memory per tile: the accumulator D, then the state A_hi and A_lo (up
// to 64 columns each), tiles 256 columns apart
constexpr uint32_t kTmemColsTm = 512;
constexpr uint32_t kTileCols = 256, kAhiCol = 64, kAloCol = 128;

struct TmParams {
  const TmMap* maps;
  int nmaps, ntiles;  // ntiles: 128-column tiles per family (ceil(n / 128))
  int n, ldT;
  int wcap, K8, N16, natoms, wstages;
  uint32_t b_half, w_stage;  // bytes: one stage's B_hi, one W stage
  uint32_t idesc;
  int packed;  // blocks stored as packed symmetric triangles (else full, ld wp)
  float inv_h2;
  const float2* W;
  const float2* cc;
  const float2* ca;
  const float2* s1;
  const float2* s1inv;
  const float2* s2inv;
  const float2* gd;
  float2* T;
  int* err;
};

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Byte offset of float f (0..31) of row `row` inside one 128-byte-swizzled
// atom: 8-row groups 1024 bytes apart, 16-byte chunk c of row r at c ^ (r % 8).
__device__ __forceinline__ uint32_t swz(int row, int f) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((f >> 2) ^ (row & 7)) & 7) << 4) + (f & 3) * 4);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle
// layout (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// D (tensor memory) (+)= A (tensor memory, row m in lane m) B (shared memory).
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit_tm(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void arrive_tm(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- jobs
struct TmJob {
  int mi, t, kmax;
};

__device__ __forceinline__ TmJob tm_job(const TmParams& P, int j) {
  TmJob J;
  J.t = P.ntiles - 1 - j / P.nmaps;  // longest tiles first
  J.mi = j % P.nmaps;
  J.kmax = min(P.n - 1, J.t * kTT + kTT - 1);
  return J;
}

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool tm_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
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
    if ((it & 1023u) == 1023u && *abort_flag) return false;
  }
  return false;
}

// The step's data a converter hands to the epilogues: the two injected
// diagonal-block columns (Gamma_k e_in for family A, Gamma_k e_keep for B) and
// family B's output scale -(1/h^2) rho / s1_k.
struct InjSlot {
  float2 col[2][kGS];
  float2 scaleB;
  float2 pad;
};

// At most 80 registers a thread (35,840 a CTA), so that a CTA fits on an SM
// beside two CTAs of the M-subproblem factor that runs concurrently.
__global__ void __maxnreg__(80) tmap_tc_kernel(const __grid_constant__ TmParams P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t sraw = smem_addr(smem_raw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* sgen = smem_raw + (sbase - sraw);
  // layout: B stages [2][hi, lo], W stages, then the injection ring
  const uint32_t offB = 0;
  const uint32_t offW = offB + 4 * P.b_half;
  const uint32_t offI = offW + (uint32_t)P.wstages * P.w_stage;
  InjSlot* inj = reinterpret_cast<InjSlot*>(sgen + offI);
  __shared__ __align__(8) uint64_t wfull[8], wempty[8], bfull[2], bempty[2], afull[2], dfull[2], last;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int njobs = P.nmaps * P.ntiles;
  const int WS = P.wstages;

  if (tid == 0) {
    for (int s = 0; s < WS; ++s) {
      mbar_init(&wfull[s], 1);
      mbar_init(&wempty[s], 128);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bfull[s], 128);
      mbar_init(&bempty[s], 1);
      mbar_init(&afull[s], 128);
      mbar_init(&dfull[s], 1);
    }
    mbar_init(&last, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTmemColsTm)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // B stages start at zero: rows and floats past 2w are never written again
  for (uint32_t o = (uint32_t)tid * 16; o < 4 * P.b_half; o += kThreadsTm * 16)
    *reinterpret_cast<float4*>(sgen + offB + o) = make_float4(0.f, 0.f, 0.f, 0.f);
  fence_async_smem();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int* abort_flag = &s_abort;
  auto timeout = [&](int where) {
    record_error(P.err, ASP_ERR_TIMEOUT, where + blockIdx.x);
    atomicExch(&s_abort, 1);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: W_k and the step's diagonal-block columns
      uint32_t wc = 0;
      bool stop = false;
      for (int j = blockIdx.x; j < njobs && !stop; j += gridDim.x) {
        const TmJob J = tm_job(P, j);
        const TmMap M = P.maps[J.mi];
        const uint32_t wbytes = (uint32_t)(M.bs * 8);
        for (int k = J.kmax; k >= 0; --k, ++wc) {
          const int s = (int)(wc % WS);
          if (wc >= (uint32_t)WS && !tm_wait(&wempty[s], ((wc / WS) - 1) & 1u, abort_flag)) {
            if (!*abort_flag) timeout(4100000);
            stop = true;
            break;
          }
          unsigned char* dst = sgen + offW + (uint32_t)s * P.w_stage;
          mbar_arrive_expect_tx(&wfull[s], wbytes + 2 * kGS * 8);
          bulk_g2s(dst, P.W + M.woff + (long long)k * M.bs, wbytes, &wfull[s]);
          bulk_g2s(dst + P.w_stage - 2 * kGS * 8, P.gd + M.goff + (long long)k * 2 * kGS, 2 * kGS * 8, &wfull[s]);
        }
      }
      // copies in flight complete on their stage's full barrier
      const uint32_t lo = wc >= (uint32_t)WS ? wc - WS : 0;
      for (uint32_t q = lo; q < wc; ++q) tm_wait(&wfull[q % WS], (q / WS) & 1u, abort_flag);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      uint32_t bc = 0;
      bool stop = false, issued = false;
      for (int j = blockIdx.x; j < njobs && !stop; j += gridDim.x) {
        const TmJob J = tm_job(P, j);
        for (int k = J.kmax; k >= 0 && !stop; --k, ++bc) {
          const int sb = (int)(bc & 1u);
          if (!tm_wait(&bfull[sb], (bc >> 1) & 1u, abort_flag)) {
            if (!*abort_flag) timeout(4200000);
            stop = true;
            break;
          }
          for (int tau = 0; tau < 2; ++tau) {
            if (!tm_wait(&afull[tau], bc & 1u, abort_flag)) {
              if (!*abort_flag) timeout(4300000);
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)tau * kTileCols;
            const uint32_t ah = d + kAhiCol, al = d + kAloCol;
            // the descriptors differ only in their start-address field (bits 0-13,
            // address / 16): step them by offset / 16
            const uint64_t dbh = sw128(sbase + offB + (uint32_t)(2 * sb) * P.b_half);
            const uint64_t dbl = dbh + (uint64_t)(P.b_half >> 4);
            const uint32_t atom16 = (uint32_t)(P.N16 * 128) >> 4;
            for (int kk = 0; kk < P.K8 / 8; ++kk) {
              const uint64_t boff = (uint64_t)((uint32_t)(kk >> 2) * atom16 + (uint32_t)(kk & 3) * 2);
              const uint32_t ac = (uint32_t)(kk * 8);  // 8 K columns per instruction
              mma_tf32_ta(d, ah + ac, dbh + boff, P.idesc, kk > 0 ? 1u : 0u);
              mma_tf32_ta(d, ah + ac, dbl + boff, P.idesc, 1u);
              mma_tf32_ta(d, al + ac, dbh + boff, P.idesc, 1u);
            }
            issued = true;
            commit_tm(&dfull[tau]);
          }
          if (stop) break;
          commit_tm(&bempty[sb]);
        }
      }
      if (issued) {
        commit_tm(&last);
        tm_wait(&last, 0u, abort_flag);
      }
    }
  } else if (warp < 6) {
    // ---- converter: B_k^T = real form of -c_k W_k, split; the injection ring
    const int ct = tid - 64;
    uint32_t wc = 0, bc = 0;
    bool stop = false;
    for (int j = blockIdx.x; j < njobs && !stop; j += gridDim.x) {
      const TmJob J = tm_job(P, j);
      const TmMap M = P.maps[J.mi];
      const int w = M.w, wcap = P.wcap;
      const float2* dinv = P.s2inv + M.prof;  // W_k[i][j] = W'_k(i, j) / s2_j
      for (int k = J.kmax; k >= 0; --k, ++wc, ++bc) {
        const int sw = (int)(wc % WS), sb = (int)(bc & 1u);
        const float2 nc = make_float2(-P.cc[k].x, -P.cc[k].y);
        float2 sB = make_float2(0.f, 0.f);
        if (ct == 0) {
          const float2 si = P.s1inv[k];
          const float2 rs = make_float2(M.rho.x * si.x - M.rho.y * si.y, M.rho.x * si.y + M.rho.y * si.x);
          sB = make_float2(-P.inv_h2 * rs.x, -P.inv_h2 * rs.y);
        }
        if (!tm_wait(&wfull[sw], (wc / WS) & 1u, abort_flag) ||
            (bc >= 2 && !tm_wait(&bempty[sb], ((bc >> 1) - 1) & 1u, abort_flag))) {
          if (!*abort_flag && ct == 0) timeout(4400000);
          stop = true;
          break;
        }
        const float2* Wk = reinterpret_cast<const float2*>(sgen + offW + (uint32_t)sw * P.w_stage);
        const float2* gk = reinterpret_cast<const float2*>(sgen + offW + (uint32_t)sw * P.w_stage + P.w_stage -
                                                           2 * kGS * 8);
        unsigned char* bhi = sgen + offB + (uint32_t)(2 * sb) * P.b_half;
        unsigned char* blo = bhi + P.b_half;
        // a warp converts 4 x 8 entries (i, jj) at a time: its 32 float2 stores
        // fall on distinct 8-byte bank pairs of the swizzled rows 2i, 2i+1
        const int nti = (wcap + 3) >> 2, ntj = (wcap + 7) >> 3;
        for (int tt = ct >> 5; tt < nti * ntj; tt += 4) {
          const int i = (tt / ntj) * 4 + (lane >> 3), jj = (tt % ntj) * 8 + (lane & 7);
          if (i >= wcap || jj >= wcap) continue;
          float2 v = make_float2(0.f, 0.f);
          if (i < w && jj < w) {
            const float2 wv = P.packed ? cmul(Wk[packed_index(i, jj)], __ldg(dinv + jj)) : Wk[jj * M.wp + i];
            v = make_float2(nc.x * wv.x - nc.y * wv.y, nc.x * wv.y + nc.y * wv.x);
          }
          // rows 2i (re output) and 2i+1 (im output), floats 2jj, 2jj+1
          const int f = 2 * jj, atom = f >> 5, fa = f & 31;
          const uint32_t o0 = (uint32_t)atom * (uint32_t)(P.N16 * 128) + swz(2 * i, fa);
          const uint32_t o1 = (uint32_t)atom * (uint32_t)(P.N16 * 128) + swz(2 * i + 1, fa);
          const float r0 = v.x, r1 = -v.y, q0 = v.y, q1 = v.x;
          const float h0 = tf32_hi(r0), h1 = tf32_hi(r1), g0 = tf32_hi(q0), g1 = tf32_hi(q1);
          *reinterpret_cast<float2*>(bhi + o0) = make_float2(h0, h1);
          *reinterpret_cast<float2*>(blo + o0) = make_float2(r0 - h0, r1 - h1);
          *reinterpret_cast<float2*>(bhi + o1) = make_float2(g0, g1);
          *reinterpret_cast<float2*>(blo + o1) = make_float2(q0 - g0, q1 - g1);
        }
        InjSlot& S = inj[bc % kInjRing];
        if (ct < 2 * kGS) S.col[ct / kGS][ct % kGS] = gk[ct];
        if (ct == 0) S.scaleB = sB;
        fence_async_smem();
        arrive_tm(&bfull[sb]);
        arrive_tm(&wempty[sw]);
      }
    }
  } else {
    // ---- epilogues: warps 6-9 family A (tile 0), warps 10-13 family B (tile 1)
    const int tau = (warp - 6) >> 2;
    const int q = warp & 3;
    const int m = q * 32 + lane;
    const uint32_t dcol = tmem + (uint32_t)tau * kTileCols + ((uint32_t)(q * 32) << 16);
    const uint32_t ahi = dcol + kAhiCol, alo = dcol + kAloCol;
    uint32_t dc = 0;
    bool stop = false;
    for (int j = blockIdx.x; j < njobs && !stop; j += gridDim.x) {
      const TmJob J = tm_job(P, j);
      const TmMap M = P.maps[J.mi];
      const int r = J.t * kTT + m;
      const bool valid = r < P.n;
      const int sel = tau == 0 ? M.keep : M.jin;  // the row this family writes out
      float2 s1r = make_float2(0.f, 0.f);
      if (tau == 1 && valid) s1r = P.s1[r];
      float2* Tm = P.T + M.toff;
      // the state before the first step is zero
      {
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < P.K8; c += 8) {
          tmem_st8(ahi + (uint32_t)c, z);
          tmem_st8(alo + (uint32_t)c, z);
        }
        tmem_wait_st();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      arrive_tm(&afull[tau]);
      for (int k = J.kmax; k >= 0; --k, ++dc) {
        if (!tm_wait(&dfull[tau], dc & 1u, abort_flag)) {
          if (!*abort_flag && lane == 0) timeout(4500000 + 100000 * tau);
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the written-out entry first, read on its own (no runtime index into
        // a register array), with the first 16 accumulator columns
        float sre = tmem_ld1(dcol + (uint32_t)(2 * sel));
        float sim = tmem_ld1(dcol + (uint32_t)(2 * sel + 1));
        float da[16], db[16];
        tmem_ld16(dcol, da);
        tmem_wait_ld();
        // tie the loaded registers to the wait, so that no use moves above it
#pragma unroll
        for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(da[i]));
        asm volatile("" : "+f"(sre), "+f"(sim));
        const InjSlot& S = inj[dc % kInjRing];
        const bool injecting = valid && r == k;
        const float2 out = injecting ? S.col[tau][sel] : make_float2(sre, sim);
        if (valid) {
          if (tau == 0 && r >= k) {
            Tm[(long long)k * P.ldT + r] = make_float2(-P.inv_h2 * out.x, -P.inv_h2 * out.y);
          } else if (tau == 1 && r > k) {
            const float2 sc = S.scaleB;
            const float2 f = make_float2(sc.x * s1r.x - sc.y * s1r.y, sc.x * s1r.y + sc.y * s1r.x);
            Tm[(long long)r * P.ldT + k] = make_float2(f.x * out.x - f.y * out.y, f.x * out.y + f.y * out.x);
          }
        }
        if (k > 0) {
          // the next step's state, split, one tensor-memory column per float,
          // 16 columns at a time: the next chunk's load is in flight while
          // this one is split and stored
          const int K2 = 2 * M.w;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c * 16 >= P.K8) break;
            float* cur = (c & 1) ? db : da;
            float* nxt = (c & 1) ? da : db;
            const bool more = (c + 1) * 16 < P.K8;
            if (more) tmem_ld16(dcol + (uint32_t)((c + 1) * 16), nxt);
            if (injecting) {
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const float2 g = S.col[tau][c * 8 + e];
                cur[2 * e] = g.x;
                cur[2 * e + 1] = g.y;
              }
            }
#pragma unroll
            for (int h8 = 0; h8 < 2; ++h8) {
              if (c * 16 + h8 * 8 >= P.K8) break;
              float hv[8], lv[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int f = c * 16 + h8 * 8 + e;
                const float x = f < K2 ? cur[h8 * 8 + e] : 0.f;
                hv[e] = tf32_hi(x);
                lv[e] = x - hv[e];
              }
              tmem_st8(ahi + (uint32_t)(c * 16 + h8 * 8), hv);
              tmem_st8(alo + (uint32_t)(c * 16 + h8 * 8), lv);
            }
            if (more) {
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(nxt[i]));
            }
          }
          tmem_wait_st();
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          arrive_tm(&afull[tau]);
        }
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemColsTm) : "memory");
}

// ---------------------------------------------------------------- Gamma
// Diagonal blocks of the subproblem inverse, Gamma_{n-1} = W_{n-1},
// Gamma_k = W_k + (c_k a_{k+1}) W_k Gamma_{k+1} W_k, one CTA per map, in shared
// memory; stores Gamma_k e_in and Gamma_k e_keep at gd[goff + (2k + f) kGS + i].
// NU columns per thread: thread t owns row i = t / 8 and columns j = t % 8 + 8u
// (u < NU) of the (8 NU) x (8 NU) working blocks, so a launch for blocks of at
// most 24 columns (NU = 3, 192 threads) spends no lanes on padding; W_{k-1} is
// fetched into registers during step k.
template <int NU>
__global__ void __launch_bounds__(64 * NU) gdiag_kernel(const TmMap* __restrict__ maps, int n,
                                                       const float2* __restrict__ W,
                                                       const float2* __restrict__ ca,
                                                       const float2* __restrict__ cc,
                                                       const float2* __restrict__ s2inv, float2* __restrict__ gd,
                                                       int packed) {
  __shared__ float2 sW[32][33], sG[32][33], sP[32][33];
  const TmMap M = maps[blockIdx.x];
  const int w = M.w;
  const int tid = threadIdx.x, i = tid >> 3, j0 = tid & 7;
  const float2* Wsub = W + M.woff;
  float2* g = gd + M.goff;
  // W_k[i][j] = W'_k(i, j) / s2_j from the packed symmetric factor
  float2 dinv[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u) dinv[u] = (j0 + 8 * u < w) ? s2inv[M.prof + j0 + 8 * u] : make_float2(0.f, 0.f);
  auto fetch = [&](int k, float2 (&v)[NU]) {
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int jj = j0 + 8 * u;
      v[u] = (i >= w || jj >= w) ? make_float2(0.f, 0.f)
             : packed ? cmul(Wsub[(long long)k * M.bs + packed_index(i, jj)], dinv[u])
                      : Wsub[(long long)k * M.bs + (long long)jj * M.wp + i];
    }
  };
  float2 wr[NU];
  fetch(n - 1, wr);
#pragma unroll
  for (int u = 0; u < NU; ++u) { sG[i][j0 + 8 * u] = wr[u]; }
  if (n >= 2) fetch(n - 2, wr);
  __syncthreads();
  auto emit = [&](int k) {
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int jj = j0 + 8 * u;
      if (i < w && jj == M.jin) g[(long long)(2 * k) * kGS + i] = sG[i][jj];
      if (i < w && jj == M.keep) g[(long long)(2 * k + 1) * kGS + i] = sG[i][jj];
    }
  };
  emit(n - 1);
  float2 beta_next = n >= 2 ? cmul(cc[n - 2], ca[n - 1]) : make_float2(0.f, 0.f);
  for (int k = n - 2; k >= 0; --k) {
#pragma unroll
    for (int u = 0; u < NU; ++u) sW[i][j0 + 8 * u] = wr[u];
    __syncthreads();
    if (k >= 1) fetch(k - 1, wr);  // in flight during this step
    // P = W_k Gamma_{k+1}
    float2 acc[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int l = 0; l < w; ++l) {
      const float2 a = sW[i][l];
#pragma unroll
      for (int u = 0; u < NU; ++u) cfma(acc[u], a, sG[l][j0 + 8 * u]);
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) sP[i][j0 + 8 * u] = acc[u];
    __syncthreads();
    // Gamma_k = W_k + beta P W_k
    const float2 beta = beta_next;
    if (k >= 1) beta_next = cmul(cc[k - 1], ca[k]);  // in flight during this step
#pragma unroll
    for (int u = 0; u < NU; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int l = 0; l < w; ++l) {
      const float2 a = sP[i][l];
#pragma unroll
      for (int u = 0; u < NU; ++u) cfma(acc[u], a, sW[l][j0 + 8 * u]);
    }
    __syncthreads();  // every read of sG (previous block) is done
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      float2 v = sW[i][j0 + 8 * u];
      cfma(v, beta, acc[u]);
      sG[i][j0 + 8 * u] = v;
    }
    __syncthreads();
    emit(k);
  }
}

}  // namespace

// Launches for the handle's maps (complex64, padded widths <= 32): the Gamma
// recursion, then the chains.  The map table and the Gamma columns live in the
// handle (d_tm, gdiag).
cudaError_t launch_tmap_diag(Handle& H, cudaStream_t s) {
  const int nmaps = (int)H.tm_host.size();
  if (nmaps == 0) return cudaSuccess;
  int wcap = 0;
  for (const TmMap& M : H.tm_host) {
    if (M.w > kTmapTcMaxW) return cudaErrorInvalidValue;
    wcap = std::max(wcap, M.w);
  }
  if (wcap <= 24)
    gdiag_kernel<3><<<nmaps, 64 * 3, 0, s>>>(H.d_tm, H.n, (const float2*)H.W, H.fc32.ca, H.fc32.cc, H.fc32.s2inv,
                                             (float2*)H.gdiag, H.packed ? 1 : 0);
  else
    gdiag_kernel<4><<<nmaps, 64 * 4, 0, s>>>(H.d_tm, H.n, (const float2*)H.W, H.fc32.ca, H.fc32.cc, H.fc32.s2inv,
                                             (float2*)H.gdiag, H.packed ? 1 : 0);
  H.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_tmap_tc(Handle& H, cudaStream_t s) {
  const int nmaps = (int)H.tm_host.size();
  if (nmaps == 0) return cudaSuccess;
  int wcap = 0;
  for (const TmMap& M : H.tm_host) wcap = std::max(wcap, M.w);
  if (wcap > kTmapTcMaxW) return cudaErrorInvalidValue;
  cudaError_t e;
  TmParams P{};
  P.maps = H.d_tm;
  P.nmaps = nmaps;
  P.ntiles = (H.n + kTT - 1) / kTT;
  P.n = H.n;
  P.ldT = H.ldT;
  P.wcap = wcap;
  P.K8 = (2 * wcap + 7) / 8 * 8;
  P.N16 = (2 * wcap + 15) / 16 * 16;
  P.natoms = (P.K8 + 31) / 32;
  P.b_half = (uint32_t)P.natoms * (uint32_t)P.N16 * 128;
  int wpc = 0;
  for (const TmMap& M : H.tm_host) wpc = std::max(wpc, M.bs * 8);
  P.w_stage = (uint32_t)((wpc + 2 * kGS * 8 + 127) / 128 * 128);
  P.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(P.N16 >> 3) << 17) | ((uint32_t)(kTT >> 4) << 24);
  P.inv_h2 = (float)H.inv_h2;
  P.W = (const float2*)H.W;
  P.cc = H.fc32.cc;
  P.ca = H.fc32.ca;
  P.s1 = H.fc32.s1;
  P.s1inv = H.fc32.s1inv;
  P.s2inv = H.fc32.s2inv;
  P.packed = H.packed ? 1 : 0;
  P.gd = (const float2*)H.gdiag;
  P.T = (float2*)H.tmap;
  P.err = H.err;
  int dev = 0, optin = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const size_t fixed = 1024 + 4 * (size_t)P.b_half + kInjRing * sizeof(InjSlot);
  cudaFuncAttributes fa{};
  if ((e = cudaFuncGetAttributes(&fa, (const void*)tmap_tc_kernel)) != cudaSuccess) return e;
  const size_t limit = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  P.wstages = 4;
  while (P.wstages > 2 && fixed + (size_t)P.wstages * P.w_stage > limit) --P.wstages;
  const size_t smem = fixed + (size_t)P.wstages * P.w_stage;
  if (smem > limit) return cudaErrorInvalidValue;
  if ((e = ensure_dyn_smem((const void*)tmap_tc_kernel, smem)) != cudaSuccess) return e;
  const int njobs = nmaps * P.ntiles;
  const int grid = std::max(1, std::min(njobs, sms));
  tmap_tc_kernel<<<grid, kThreadsTm, smem, s>>>(P);
  H.launches += 1;
  return cudaGetLastError();
}

}  // namespace asp
