// btsolve.cu -- batched solves with the layer factors: the G~ operators of
// Section 3.1 ("Auxiliary Green's operators") for many subproblems and
// right-hand sides in one launch.
//
// A job is (subproblem, block of right-hand sides, mode).  For one job the CTA
// runs the two passes of the block-tridiagonal solve with the factors of
// btfactor.cu (W_k = S_k^{-1}):
//     forward   z_k = W_k (g_k - a_k z_{k-1}),           k = k0 .. n-1
//     backward  x_{n-1} = z_{n-1},  x_k = z_k - c_k W_k x_{k+1},   k = n-2 .. 0
// Each step is a dense w x w block times a w x nr panel of right-hand sides.
// The W_k blocks stream from HBM through a 3-stage shared-memory ring filled by
// 1D bulk (TMA) copies that complete on mbarriers; the per-step right-hand
// side entries (and, in the backward pass, the z_k saved by the forward pass)
// stream through a per-thread cp.async ring.  One __syncthreads per step
// publishes the new w x nr panel.
//
// Modes (what g_k is and what is written):
//   EMBED   G~_q^M f_q: g = input on the rows of X_q;  writes x on X_q to outM,
//           its first / last X_q column to the left / right trace buffers.
//   FILL_R  G~_p^R w: g = -(1/h^2) accR[p-1] on local column 0; writes x on X_p to outR.
//   FILL_L  G~_p^L w: g = -(1/h^2) accL[p+1] on local column w-1; writes outL.
//   TMAP_R  columns r of the dense map w -> (G~_p^R w)^R: g = -(1/h^2) e_r on column 0;
//           keeps the last column of X_p.  The forward pass starts at block k0 = first r
//           of the job (earlier blocks are zero).
//   TMAP_L  same for G~_p^L, g on column w-1, keeps the first column of X_p.
//   SUB     v = H^-1 g on the whole padded grid (checking entry point).
#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kStages = 3;  // W-block ring depth
constexpr int kRing = 3;    // per-thread input ring depth

struct Geometry {
  int wcap;    // largest w in the launch
  int wstage;  // elements of one W stage (largest w*wp)
};

template <typename R, int NT, int RL, int RQ, int RS>
struct Layout {
  using C = Cx<R>;
  static constexpr int NR = RL * RQ;
  __host__ __device__ static size_t bars() { return 64; }
  __host__ __device__ static size_t wst(const Geometry& g) { return (size_t)kStages * g.wstage * sizeof(C); }
  __host__ __device__ static size_t ybuf(const Geometry& g) { return (size_t)2 * g.wcap * NR * sizeof(C); }
  __host__ __device__ static size_t ring() { return (size_t)kRing * RS * RQ * NT * sizeof(C); }
  __host__ __device__ static size_t total(const Geometry& g) {
    auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
    return al(bars()) + al(wst(g)) + al(ybuf(g)) + al(ring());
  }
};

template <typename R, int NT, int RL, int RQ, int RS>
__global__ void __launch_bounds__(NT) btsolve_kernel(SolveParams P, Geometry G) {
  using C = Cx<R>;
  using LY = Layout<R, NT, RL, RQ, RS>;
  constexpr int RG = NT / RL;
  constexpr int NR = RL * RQ;
  constexpr int RSQ = RS * RQ;
  extern __shared__ __align__(128) unsigned char smem[];
  auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  C* Wst = reinterpret_cast<C*>(smem + al(LY::bars()));
  C* ybuf = reinterpret_cast<C*>(smem + al(LY::bars()) + al(LY::wst(G)));
  C* ring = reinterpret_cast<C*>(smem + al(LY::bars()) + al(LY::wst(G)) + al(LY::ybuf(G)));
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int tr = tid % RL, ti = tid / RL;
  const int n = P.n, ldv = P.ldv;
  const C* __restrict__ Wg = reinterpret_cast<const C*>(P.W);
  C* zslot = reinterpret_cast<C*>(P.zscr) + (long long)blockIdx.x * P.zslot;
  const C neg_ih2 = cmake<R>(R(-P.inv_h2), R(0));

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t wuse = 0;  // W stages consumed so far (all threads track it identically)

  for (int job = blockIdx.x; job < P.njobs; job += gridDim.x) {
    const Job J = P.jobs[job];
    const SubDesc S = P.subs[J.sub];
    const int w = S.w, wp = S.wp, xoff = S.xoff, xw = S.xw, lo = S.lo, p = S.p;
    const int mode = J.mode, rhs0 = J.rhs0, nr = J.nr;
    const bool tmap = (mode == MODE_TMAP_R || mode == MODE_TMAP_L);
    const int k0 = tmap ? rhs0 : 0;
    const int nf = n - k0;
    const int L = nf + (n - 1);
    const uint32_t bbytes = (uint32_t)(w * wp * sizeof(C));
    const C* Wsub = Wg + S.woff;
    auto blk = [&](int q) { return q < nf ? k0 + q : n - 2 - (q - nf); };

    __syncthreads();  // previous job's last reads of the W ring and ybuf are done
    if (tid == 0) {
      for (int t = 0; t < kStages && t < L; ++t) {
        const int st = (wuse + t) % kStages;
        mbar_arrive_expect_tx(&bar[st], bbytes);
        bulk_g2s(Wst + (size_t)st * G.wstage, Wsub + (long long)blk(t) * w * wp, bbytes, &bar[st]);
      }
    }

    // ---- per-thread input ring
    const C* inM = reinterpret_cast<const C*>(P.in);
    const C* accRp = reinterpret_cast<const C*>(P.accR);
    const C* accLp = reinterpret_cast<const C*>(P.accL);
    auto load_step = [&](int q2) {
      if (q2 < L) {
        const int kk = blk(q2);
        C* slot = ring + (size_t)(q2 % kRing) * RSQ * NT;
        if (q2 < nf) {
          if (mode == MODE_EMBED || mode == MODE_FILL_R || mode == MODE_FILL_L || mode == MODE_SUB) {
#pragma unroll
            for (int s = 0; s < RS; ++s) {
              const int i = ti + RG * s;
              if (i >= w) continue;
#pragma unroll
              for (int qq = 0; qq < RQ; ++qq) {
                const int r = tr + RL * qq;
                if (r >= nr) continue;
                const C* src = nullptr;
                if (mode == MODE_EMBED) {
                  if (i >= xoff && i < xoff + xw) src = inM + ((long long)(lo - 1 + i) * n + kk) * ldv + rhs0 + r;
                } else if (mode == MODE_FILL_R) {
                  if (i == 0) src = accRp + ((long long)(p - 1) * n + kk) * ldv + rhs0 + r;
                } else if (mode == MODE_FILL_L) {
                  if (i == w - 1) src = accLp + ((long long)(p + 1) * n + kk) * ldv + rhs0 + r;
                } else {
                  src = inM + ((long long)i * n + kk) * ldv + rhs0 + r;
                }
                if (src) cp_async<sizeof(C)>(slot + (size_t)(s * RQ + qq) * NT + tid, src);
              }
            }
          }
        } else if (kk >= k0 && kk <= n - 3) {
#pragma unroll
          for (int s = 0; s < RS; ++s) {
            const int i = ti + RG * s;
            if (i >= w) continue;
#pragma unroll
            for (int qq = 0; qq < RQ; ++qq) {
              const int r = tr + RL * qq;
              cp_async<sizeof(C)>(slot + (size_t)(s * RQ + qq) * NT + tid,
                                  zslot + ((long long)kk * w + i) * NR + r);
            }
          }
        }
      }
      cp_async_commit();
    };
    for (int t = 0; t < kRing - 1; ++t) load_step(t);

    C zprev[RS][RQ], zkeep[RS][RQ], xprev[RS][RQ];
#pragma unroll
    for (int s = 0; s < RS; ++s)
#pragma unroll
      for (int qq = 0; qq < RQ; ++qq) zprev[s][qq] = zkeep[s][qq] = xprev[s][qq] = czero<R>();

    for (int q = 0; q < L; ++q) {
      const int k = blk(q);
      const bool fwd = q < nf;
      load_step(q + kRing - 1);
      cp_async_wait<kRing - 1>();
      const C* slot = ring + (size_t)(q % kRing) * RSQ * NT;
      C* yb = ybuf + (size_t)(q & 1) * G.wcap * NR;

      // ---- right-hand panel of this step
      const double2 ak = P.ca[k];
      const C a_k = cmake<R>(R(ak.x), R(ak.y));
#pragma unroll
      for (int s = 0; s < RS; ++s) {
        const int i = ti + RG * s;
        if (i >= w) continue;
#pragma unroll
        for (int qq = 0; qq < RQ; ++qq) {
          const int r = tr + RL * qq;
          C y;
          if (fwd) {
            C g = czero<R>();
            if (mode == MODE_EMBED) {
              if (i >= xoff && i < xoff + xw && r < nr) g = slot[(size_t)(s * RQ + qq) * NT + tid];
            } else if (mode == MODE_FILL_R) {
              if (i == 0 && r < nr) g = cmul(neg_ih2, slot[(size_t)(s * RQ + qq) * NT + tid]);
            } else if (mode == MODE_FILL_L) {
              if (i == w - 1 && r < nr) g = cmul(neg_ih2, slot[(size_t)(s * RQ + qq) * NT + tid]);
            } else if (mode == MODE_SUB) {
              if (r < nr) g = slot[(size_t)(s * RQ + qq) * NT + tid];
            } else if (mode == MODE_TMAP_R) {
              if (i == 0 && r < nr && k == rhs0 + r) g = neg_ih2;
            } else {  // MODE_TMAP_L
              if (i == w - 1 && r < nr && k == rhs0 + r) g = neg_ih2;
            }
            y = g;
            cfms(y, a_k, zprev[s][qq]);
          } else {
            y = xprev[s][qq];
          }
          yb[i * NR + r] = y;
        }
      }
      __syncthreads();
      if (s_abort) return;
      if (tid == 0 && q >= 1 && q - 1 + kStages < L) {
        const int st = (wuse + q - 1) % kStages;
        mbar_arrive_expect_tx(&bar[st], bbytes);
        bulk_g2s(Wst + (size_t)st * G.wstage, Wsub + (long long)blk(q - 1 + kStages) * w * wp, bbytes, &bar[st]);
      }
      const uint32_t st = (wuse + q) % kStages;
      const uint32_t par = ((wuse + q) / kStages) & 1u;
      if (!mbar_wait(&bar[st], par)) {
        record_error(P.err, ASP_ERR_TIMEOUT, blockIdx.x);
        s_abort = 1;
      }
      const C* Wk = Wst + (size_t)st * G.wstage;

      // ---- acc = W_k * panel
      C acc[RS][RQ];
#pragma unroll
      for (int s = 0; s < RS; ++s)
#pragma unroll
        for (int qq = 0; qq < RQ; ++qq) acc[s][qq] = czero<R>();
#pragma unroll 2
      for (int j = 0; j < w; ++j) {
        C yv[RQ];
#pragma unroll
        for (int qq = 0; qq < RQ; ++qq) yv[qq] = yb[j * NR + tr + RL * qq];
        const C* Wc = Wk + j * wp;
#pragma unroll
        for (int s = 0; s < RS; ++s) {
          const int i = ti + RG * s;
          if (i < w) {
            const C wv = Wc[i];
#pragma unroll
            for (int qq = 0; qq < RQ; ++qq) cfma(acc[s][qq], wv, yv[qq]);
          }
        }
      }

      // ---- epilogue
      const double2 ck = P.cc[k];
      const C c_k = cmake<R>(R(ck.x), R(ck.y));
#pragma unroll
      for (int s = 0; s < RS; ++s) {
        const int i = ti + RG * s;
        if (i >= w) continue;
#pragma unroll
        for (int qq = 0; qq < RQ; ++qq) {
          const int r = tr + RL * qq;
          C x;
          bool have_x = false;
          if (fwd) {
            const C z = acc[s][qq];
            if (k <= n - 3) zslot[((long long)k * w + i) * NR + r] = z;
            if (k == n - 1) {
              zkeep[s][qq] = zprev[s][qq];
              x = z;
              have_x = true;
            }
            zprev[s][qq] = z;
          } else {
            C z = czero<R>();
            if (k >= k0) z = (k == n - 2) ? zkeep[s][qq] : slot[(size_t)(s * RQ + qq) * NT + tid];
            x = z;
            cfms(x, c_k, acc[s][qq]);
            have_x = true;
          }
          if (have_x) {
            xprev[s][qq] = x;
            if (r < nr) {
              const long long gi = ((long long)(lo - 1 + i) * n + k) * ldv + rhs0 + r;
              if (mode == MODE_EMBED) {
                if (i >= xoff && i < xoff + xw) reinterpret_cast<C*>(P.outM)[gi] = x;
                if (i == xoff + xw - 1) reinterpret_cast<C*>(P.accR)[((long long)p * n + k) * ldv + rhs0 + r] = x;
                if (i == xoff) reinterpret_cast<C*>(P.accL)[((long long)p * n + k) * ldv + rhs0 + r] = x;
              } else if (mode == MODE_FILL_R) {
                if (i >= xoff && i < xoff + xw) reinterpret_cast<C*>(P.outR)[gi] = x;
              } else if (mode == MODE_FILL_L) {
                if (i >= xoff && i < xoff + xw) reinterpret_cast<C*>(P.outL)[gi] = x;
              } else if (mode == MODE_TMAP_R) {
                if (i == xoff + xw - 1) reinterpret_cast<C*>(P.tmap)[S.toff + (long long)k * n + rhs0 + r] = x;
              } else if (mode == MODE_TMAP_L) {
                if (i == xoff) reinterpret_cast<C*>(P.tmap)[S.toff + (long long)k * n + rhs0 + r] = x;
              } else {
                reinterpret_cast<double2*>(P.outSub)[((long long)i * n + k) * ldv + rhs0 + r] =
                    make_double2((double)x.x, (double)x.y);
              }
            }
          }
        }
      }
    }
    wuse += (uint32_t)L;
    cp_async_wait<0>();
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < kStages; ++s) mbar_inval(&bar[s]);
}

template <typename R, int NT, int RL, int RQ, int RS>
cudaError_t run(Handle& H, const SolveParams& P, int wcap, cudaStream_t s) {
  Geometry G;
  G.wcap = wcap;
  int wpc = (sizeof(R) == 4) ? ((wcap + 1) & ~1) : wcap;
  G.wstage = wcap * wpc;
  const size_t smem = Layout<R, NT, RL, RQ, RS>::total(G);
  auto kern = btsolve_kernel<R, NT, RL, RQ, RS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = P.njobs < H.zslots ? P.njobs : H.zslots;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, NT, smem, s>>>(P, G);
  H.launches += 1;
  return cudaGetLastError();
}

}  // namespace

// Right-hand sides one CTA handles for a launch whose jobs have at most
// `nrhs` right-hand sides and width <= wmax.  Returns 0 if no instance fits.
int btsolve_rhs_capacity(int nrhs, int wmax, int prec, bool tmap) {
  if (wmax > 64) return 0;
  if (tmap && prec == ASP_PREC_C64 && wmax <= 32) return 64;
  if (nrhs >= 32 || tmap) {
    if (prec == ASP_PREC_C64 && wmax <= 64) return 32;
    if (prec == ASP_PREC_C128 && wmax <= 64) return 16;
  }
  if (nrhs >= 16) return 16;
  if (nrhs >= 8) return 8;
  if (nrhs >= 4) return 4;
  if (nrhs >= 2) return 2;
  return 1;
}

cudaError_t launch_btsolve(Handle& H, const SolveParams& P, int cap, int wmax, cudaStream_t s) {
  if (H.prec == ASP_PREC_C64) {
    switch (cap) {
      case 64: return run<float, 128, 32, 2, 8>(H, P, wmax, s);
      case 32: return run<float, 128, 32, 1, 16>(H, P, wmax, s);
      case 16: return run<float, 128, 16, 1, 8>(H, P, wmax, s);
      case 8: return run<float, 128, 8, 1, 4>(H, P, wmax, s);
      case 4: return run<float, 128, 4, 1, 2>(H, P, wmax, s);
      case 2: return run<float, 128, 2, 1, 1>(H, P, wmax, s);
      case 1: return run<float, 64, 1, 1, 1>(H, P, wmax, s);
    }
  } else {
    switch (cap) {
      case 16: return run<double, 128, 16, 1, 8>(H, P, wmax, s);
      case 8: return run<double, 128, 8, 1, 4>(H, P, wmax, s);
      case 4: return run<double, 128, 4, 1, 2>(H, P, wmax, s);
      case 2: return run<double, 128, 2, 1, 1>(H, P, wmax, s);
      case 1: return run<double, 64, 1, 1, 1>(H, P, wmax, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace asp
