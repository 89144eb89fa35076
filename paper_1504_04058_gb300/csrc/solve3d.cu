// solve3d.cu -- Algorithm 2 for 3D (Section 4) and the 7-point matvec.
//
// Every slab solve is block substitution with the stored inverses:
//     forward   z_k = W_k (g_k - a_k z_{k-1}),          k = 0 .. n-1
//     backward  x_k = z_k - c_k W_k x_{k+1},             k = n-2 .. 0
// (a_k, c_k the x2 stencil weights, blocks = x2 planes).  One cooperative
// launch runs a batch of independent slab solves ("jobs") through all 2n-1
// block steps, with a bounded grid barrier between steps: per step the rows of
// every job's W_k are cut into work items of kRowsPerItem rows, a CTA stages
// the input vector of its item's job in shared memory once and its warps
// stream the W_k rows (one warp per row, lanes along the row) from HBM.
//
// The apply follows Algorithm 2 literally:
//   1. one launch solves every H_q^M with f restricted to X_q (u~_{q,q});
//   2. m-1 launches run the two sweeps in step: launch t solves H_p^R for
//      p = 2+t with -(1/h^2) times the accumulated right trace
//      (u~_{p-1,1:p-2} + u~_{p-1,p-1}) on its first plane, and H_p^L for
//      p = m-1-t with the accumulated left trace on its last plane; each
//      solution restricted to X_p is written where the next step reads it;
//   3. u~_p = u~_{p,1:p-1} + u~_{p,p} + u~_{p,p+1:m}.
// Unlike the 2D path there are no trace-transfer maps: a trace is a whole
// n x n plane, so a dense map would cost n^4 entries per layer.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr int kRowsPerWarp = 2;
constexpr int kRowsPerItem = kSolveWarps * kRowsPerWarp;

__host__ __device__ inline int stage_len(int nb) { return (nb + 63) & ~63; }

// Loads two consecutive complex entries of a W row (c64: one 16-byte load).
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  a = __ldcs(p);
  b = __ldcs(p + 1);
}

template <typename R>
__device__ __forceinline__ Cx<R> ld_vec(const void* base, long long idx) {
  return reinterpret_cast<const Cx<R>*>(base)[idx];
}

__device__ __forceinline__ int find_job(const Solve3Job* jobs, int njobs, int it) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item0 <= it) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Bounded grid barrier; returns false (after recording ASP_ERR_TIMEOUT) if the
// wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int target, int* err, int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    uint32_t spins = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (++spins > kSpinLimit) {
        record_error(err, ASP_ERR_TIMEOUT, 2000000 + (int)blockIdx.x);
        *s_abort = 1;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return *s_abort == 0;
}

template <typename R, int NR>
__global__ void __launch_bounds__(kSolveThreads) slab_solve_kernel(Solve3Params P) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* vec = reinterpret_cast<C*>(smem_raw);  // [stage_len(nb)][NR]
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_abort = 0;
  __syncthreads();
  const int n = P.n, ldv = P.ldv;
  const C* ca = reinterpret_cast<const C*>(P.ca);
  const C* cc = reinterpret_cast<const C*>(P.cc);
  C* zb = reinterpret_cast<C*>(P.z);
  const int G = gridDim.x;
  const int it_begin = (int)(((long long)P.nitems * blockIdx.x) / G);
  const int it_end = (int)(((long long)P.nitems * (blockIdx.x + 1)) / G);
  unsigned int step = 0;

  // stage the vector of job jb for block k: forward (g_k - a_k z_{k-1}) or
  // backward (x_{k+1})
  auto stage = [&](int jb, int k, bool fwd) {
    const Solve3Job J = P.jobs[jb];
    const Slab S = P.slabs[J.slab];
    const int nb = S.nb, L = stage_len(nb);
    const C* zs = zb + S.zoff;
    for (int e = tid; e < L * NR; e += kSolveThreads) {
      const int j = e / NR, r = e - j * NR;
      C v = czero<R>();
      if (j < nb && r < J.nr) {
        const int col = J.rhs0 + r;
        if (fwd) {
          const int i3l = j / n, i1 = j - i3l * n;
          if (J.mode == MODE_EMBED) {
            if (i3l >= S.xoff && i3l < S.xoff + S.xw)
              v = ld_vec<R>(P.in, ((long long)((S.lo - 1 + i3l) * n + k) * n + i1) * ldv + col);
          } else if (J.mode == MODE_FILL_R || J.mode == MODE_FILL_L) {
            const bool edge = (J.mode == MODE_FILL_R) ? (i3l == 0) : (i3l == S.w - 1);
            if (edge) {
              const long long idx = ((long long)(S.src_plane * n + k) * n + i1) * ldv + col;
              v = ld_vec<R>(P.outM, idx);
              if (S.src_sweep) v = cadd(v, ld_vec<R>(J.mode == MODE_FILL_R ? P.outR : P.outL, idx));
              v.x *= (R)(-P.inv_h2);
              v.y *= (R)(-P.inv_h2);
            }
          } else {  // MODE_SUB
            v = ld_vec<R>(P.in, ((long long)(i3l * n + k) * n + i1) * ldv + col);
          }
          if (k > 0) cfms(v, ca[k], zs[((long long)(k - 1) * nb + j) * ldv + col]);
        } else {
          v = zs[((long long)(k + 1) * nb + j) * ldv + col];
        }
      }
      vec[e] = v;
    }
  };

  // y[rr][r] = W_k[row_rr] . vec for the warp's rows
  auto rows_product = [&](const Slab& S, int k, int rowa, C (&y)[kRowsPerWarp][NR]) {
    const int nb = S.nb, ld = S.ld;
    const C* Wk = reinterpret_cast<const C*>(P.W) + S.woff + (long long)k * nb * ld;
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr)
#pragma unroll
      for (int r = 0; r < NR; ++r) y[rr][r] = czero<R>();
    const C* w0 = Wk + (long long)min(rowa, nb - 1) * ld;
    const C* w1 = Wk + (long long)min(rowa + 1, nb - 1) * ld;
#pragma unroll 4
    for (int j = 2 * lane; j < nb; j += 64) {
      C a0, a1, b0, b1;
      ld_pair(w0 + j, a0, a1);
      ld_pair(w1 + j, b0, b1);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const C v0 = vec[j * NR + r], v1 = vec[(j + 1) * NR + r];
        cfma(y[0][r], a0, v0);
        cfma(y[0][r], a1, v1);
        cfma(y[1][r], b0, v0);
        cfma(y[1][r], b1, v1);
      }
    }
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr)
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          y[rr][r].x += __shfl_xor_sync(0xffffffffu, y[rr][r].x, off);
          y[rr][r].y += __shfl_xor_sync(0xffffffffu, y[rr][r].y, off);
        }
  };

  // ---------------------------------------------------------------- forward
  for (int k = 0; k < n; ++k) {
    int cur = -1;
    for (int it = it_begin; it < it_end; ++it) {
      const int jb = find_job(P.jobs, P.njobs, it);
      if (jb != cur) {
        __syncthreads();
        stage(jb, k, true);
        __syncthreads();
        cur = jb;
      }
      const Solve3Job J = P.jobs[jb];
      const Slab S = P.slabs[J.slab];
      const int rowa = (it - J.item0) * kRowsPerItem + warp * kRowsPerWarp;
      if (rowa >= S.nb) continue;
      C y[kRowsPerWarp][NR];
      rows_product(S, k, rowa, y);
      if (lane == 0) {
        C* zk = zb + S.zoff + (long long)k * S.nb * ldv;
#pragma unroll
        for (int rr = 0; rr < kRowsPerWarp; ++rr) {
          const int row = rowa + rr;
          if (row >= S.nb) break;
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (r < J.nr) zk[(long long)row * ldv + J.rhs0 + r] = y[rr][r];
        }
      }
    }
    ++step;
    if (!grid_barrier(P.bar, step * (unsigned)G, P.err, &s_abort)) return;
  }

  // --------------------------------------------------------------- backward
  for (int k = n - 1; k >= 0; --k) {
    int cur = -1;
    for (int it = it_begin; it < it_end; ++it) {
      const int jb = find_job(P.jobs, P.njobs, it);
      const Solve3Job J = P.jobs[jb];
      const Slab S = P.slabs[J.slab];
      if (k < n - 1 && jb != cur) {
        __syncthreads();
        stage(jb, k, false);
        __syncthreads();
        cur = jb;
      }
      const int rowa = (it - J.item0) * kRowsPerItem + warp * kRowsPerWarp;
      if (rowa >= S.nb) continue;
      C y[kRowsPerWarp][NR];
      if (k < n - 1) rows_product(S, k, rowa, y);
      if (lane == 0) {
        C* zk = zb + S.zoff + (long long)k * S.nb * ldv;
        const C ck = cc[k];
#pragma unroll
        for (int rr = 0; rr < kRowsPerWarp; ++rr) {
          const int row = rowa + rr;
          if (row >= S.nb) break;
          const int i3l = row / n, i1 = row - i3l * n;
          const bool keep = i3l >= S.xoff && i3l < S.xoff + S.xw;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            if (r >= J.nr) continue;
            const int col = J.rhs0 + r;
            C x = zk[(long long)row * ldv + col];
            if (k < n - 1) {
              cfms(x, ck, y[rr][r]);
              zk[(long long)row * ldv + col] = x;
            }
            if (J.mode == MODE_SUB) {
              reinterpret_cast<double2*>(P.outSub)[((long long)(i3l * n + k) * n + i1) * ldv + col] =
                  make_double2((double)x.x, (double)x.y);
            } else if (keep) {
              const long long idx = ((long long)((S.lo - 1 + i3l) * n + k) * n + i1) * ldv + col;
              C* out = reinterpret_cast<C*>(J.mode == MODE_EMBED ? P.outM : J.mode == MODE_FILL_R ? P.outR : P.outL);
              out[idx] = x;
            }
          }
        }
      }
    }
    if (k > 0 && k < n - 1) {
      ++step;
      if (!grid_barrier(P.bar, step * (unsigned)G, P.err, &s_abort)) return;
    }
  }
}

// 7-point FP64 matvec: y = A x with A the 3D analogue of Eq. (4) (boundary PML on
// all three axes, the same profile on each).
__global__ void matvec3d_kernel(const double* __restrict__ k2, const double2* __restrict__ ca,
                                const double2* __restrict__ cc, const double2* __restrict__ cd, int n, int nrhs,
                                const double2* __restrict__ x, double2* __restrict__ y) {
  const long long nn = (long long)n * n;
  const long long total = nn * n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long pt = e / nrhs;
    const int i1 = (int)(pt % n);
    const int i2 = (int)((pt / n) % n);
    const int i3 = (int)(pt / nn);
    const double2 d1 = cd[i1], d2 = cd[i2], d3 = cd[i3];
    const double2 diag = make_double2(d1.x + d2.x + d3.x + k2[pt], d1.y + d2.y + d3.y);
    double2 acc = cmul(diag, x[e]);
    const long long s2 = (long long)n * nrhs, s3 = nn * nrhs;
    if (i1 > 0) cfma(acc, ca[i1], x[e - nrhs]);
    if (i1 < n - 1) cfma(acc, cc[i1], x[e + nrhs]);
    if (i2 > 0) cfma(acc, ca[i2], x[e - s2]);
    if (i2 < n - 1) cfma(acc, cc[i2], x[e + s2]);
    if (i3 > 0) cfma(acc, ca[i3], x[e - s3]);
    if (i3 < n - 1) cfma(acc, cc[i3], x[e + s3]);
    y[e] = acc;
  }
}

// ------------------------------------------------------------------ host
struct Launch3 {
  int first = 0, count = 0, nitems = 0;
};

struct Jobs3 {
  Solve3Job* d = nullptr;
  int NR = 1;
  std::vector<Launch3> launches;
};

std::mutex& jobs3_mu() {
  static std::mutex mu;
  return mu;
}
std::map<const Handle*, std::map<long long, Jobs3>>& jobs3() {
  static std::map<const Handle*, std::map<long long, Jobs3>> m;
  return m;
}

int pick_nr(int nrhs) { return nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1; }

// Appends the jobs of one slab for all right-hand sides, in chunks of NR.
void add_jobs(const Handle& H, std::vector<Solve3Job>& v, int slab, int mode, int nrhs, int NR, int* items) {
  const int per = (H.slabs[slab].nb + kRowsPerItem - 1) / kRowsPerItem;
  for (int r0 = 0; r0 < nrhs; r0 += NR) {
    Solve3Job J{slab, mode, r0, std::min(NR, nrhs - r0), *items};
    v.push_back(J);
    *items += per;
  }
}

int get_jobs(Handle& H, long long key, int nrhs, int sub_slab, Jobs3** out) {
  std::lock_guard<std::mutex> lock(jobs3_mu());
  auto& mp = jobs3()[&H];
  auto it = mp.find(key);
  if (it != mp.end()) {
    *out = &it->second;
    return ASP_OK;
  }
  Jobs3 J;
  J.NR = pick_nr(nrhs);
  std::vector<Solve3Job> v;
  auto open = [&]() { Launch3 L; L.first = (int)v.size(); return L; };
  if (sub_slab >= 0) {
    Launch3 L = open();
    int items = 0;
    add_jobs(H, v, sub_slab, MODE_SUB, nrhs, J.NR, &items);
    L.count = (int)v.size() - L.first;
    L.nitems = items;
    J.launches.push_back(L);
  } else {
    Launch3 L = open();
    int items = 0;
    for (int q = 1; q <= H.m; ++q) add_jobs(H, v, H.subM[q], MODE_EMBED, nrhs, J.NR, &items);
    L.count = (int)v.size() - L.first;
    L.nitems = items;
    J.launches.push_back(L);
    for (int t = 0; t + 2 <= H.m; ++t) {
      Launch3 S = open();
      int it2 = 0;
      add_jobs(H, v, H.subR[2 + t], MODE_FILL_R, nrhs, J.NR, &it2);
      add_jobs(H, v, H.subL[H.m - 1 - t], MODE_FILL_L, nrhs, J.NR, &it2);
      S.count = (int)v.size() - S.first;
      S.nitems = it2;
      J.launches.push_back(S);
    }
  }
  if (cudaMalloc(&J.d, v.size() * sizeof(Solve3Job)) != cudaSuccess) return fail(ASP_ERR_OOM, "3D job list");
  if (cudaMemcpy(J.d, v.data(), v.size() * sizeof(Solve3Job), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(J.d);
    return fail(ASP_ERR_CUDA, "3D job list upload");
  }
  it = mp.emplace(key, J).first;
  *out = &it->second;
  return ASP_OK;
}

template <typename R, int NR>
cudaError_t launch_solve_t(Handle& H, Solve3Params P, int nbmax, cudaStream_t s) {
  const size_t smem = (size_t)stage_len(nbmax) * NR * sizeof(Cx<R>);
  cudaError_t e = ensure_dyn_smem((const void*)slab_solve_kernel<R, NR>, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slab_solve_kernel<R, NR>, kSolveThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(P.nitems, per_sm * H.num_sms));
  e = cudaMemsetAsync(P.bar, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&P};
  e = cudaLaunchCooperativeKernel((void*)slab_solve_kernel<R, NR>, dim3(grid), dim3(kSolveThreads), args, smem, s);
  H.launches += 1;
  return e;
}

cudaError_t launch_solve(Handle& H, const Solve3Params& P, int NR, int nbmax, cudaStream_t s) {
  if (H.prec == ASP_PREC_C128) {
    if (NR == 4) return launch_solve_t<double, 4>(H, P, nbmax, s);
    if (NR == 2) return launch_solve_t<double, 2>(H, P, nbmax, s);
    return launch_solve_t<double, 1>(H, P, nbmax, s);
  }
  if (NR == 4) return launch_solve_t<float, 4>(H, P, nbmax, s);
  if (NR == 2) return launch_solve_t<float, 2>(H, P, nbmax, s);
  return launch_solve_t<float, 1>(H, P, nbmax, s);
}

Solve3Params base3(Handle& H, int ldv) {
  Solve3Params P{};
  P.slabs = H.d_slabs;
  P.n = H.n;
  P.ldv = ldv;
  P.inv_h2 = H.inv_h2;
  P.W = H.W;
  P.ca = H.prec == ASP_PREC_C64 ? (const void*)H.fc32.ca : (const void*)H.fc64.ca;
  P.cc = H.prec == ASP_PREC_C64 ? (const void*)H.fc32.cc : (const void*)H.fc64.cc;
  P.outM = H.uM;
  P.outR = H.uR;
  P.outL = H.uL;
  P.z = H.z3;
  P.bar = H.bar;
  P.err = H.err;
  return P;
}

}  // namespace

void release_jobs3(const Handle* H) {
  std::lock_guard<std::mutex> lock(jobs3_mu());
  auto it = jobs3().find(H);
  if (it == jobs3().end()) return;
  for (auto& kv : it->second)
    if (kv.second.d) cudaFree(kv.second.d);
  jobs3().erase(it);
}

cudaError_t launch_matvec3d(const Handle& H, const double2* x, double2* y, int nrhs, cudaStream_t s) {
  const long long total = H.N * nrhs;
  long long g = (total + 255) / 256;
  g = std::min<long long>(g, (long long)std::max(H.num_sms, 1) * 16);
  matvec3d_kernel<<<(int)std::max<long long>(g, 1), 256, 0, s>>>(H.k2, H.ca, H.cc, H.cd, H.n, nrhs, x, y);
  return cudaGetLastError();
}

int apply3d(Handle& H, const double2* r, double2* z, int nrhs, cudaStream_t s) {
  if (!H.factored) return fail(ASP_ERR_STATE, "apply before factor");
  const long long count = H.N * nrhs;
  const void* in = r;
  if (H.prec == ASP_PREC_C64) {
    PhaseTok tk = phase_begin(H, PH_SUM, s);
    if (launch_to_prec(r, H.r_lo, count, H.prec, s) != cudaSuccess) return fail(ASP_ERR_CUDA, "to_prec launch");
    phase_end(H, tk, s);
    H.launches += 1;
    in = H.r_lo;
  }
  Jobs3* J = nullptr;
  int rc = get_jobs(H, nrhs, nrhs, -1, &J);
  if (rc != ASP_OK) return rc;
  for (size_t l = 0; l < J->launches.size(); ++l) {
    const Launch3& L = J->launches[l];
    Solve3Params P = base3(H, nrhs);
    P.in = in;
    P.jobs = J->d + L.first;
    P.njobs = L.count;
    P.nitems = L.nitems;
    const bool first = l == 0;
    PhaseTok tk = phase_begin(H, first ? PH_EMBED : PH_FILL, s);
    const int nbmax = first ? H.nbmaxM : H.nbmaxRL;
    cudaError_t ce = H.nd ? nd_solve(H, P, J->NR, nbmax, s) : launch_solve(H, P, J->NR, nbmax, s);
    phase_end(H, tk, s);
    if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("3D slab-solve launch: ") + cudaGetErrorString(ce));
  }
  PhaseTok tk = phase_begin(H, PH_SUM, s);
  cudaError_t ce = launch_sum3(H.uM, H.uR, H.uL, z, (long long)H.n * H.n * nrhs, H.n, H.x_hi[1], H.x_lo[H.m] - 1,
                               H.prec, s);
  phase_end(H, tk, s);
  H.launches += 1;
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("sum launch: ") + cudaGetErrorString(ce));
  return ASP_OK;
}

int subsolve3d(Handle& H, int slab, const double2* g, double2* v, int nrhs, cudaStream_t s) {
  const Slab& S = H.slabs[slab];
  const void* in = g;
  if (H.prec == ASP_PREC_C64) {
    if (launch_to_prec(g, H.r_lo, (long long)S.w * H.n * H.n * nrhs, H.prec, s) != cudaSuccess)
      return fail(ASP_ERR_CUDA, "to_prec launch");
    H.launches += 1;
    in = H.r_lo;
  }
  Jobs3* J = nullptr;
  int rc = get_jobs(H, -(1000LL * (slab + 1) + nrhs), nrhs, slab, &J);
  if (rc != ASP_OK) return rc;
  const Launch3& L = J->launches[0];
  Solve3Params P = base3(H, nrhs);
  P.in = in;
  P.outSub = v;
  P.jobs = J->d + L.first;
  P.njobs = L.count;
  P.nitems = L.nitems;
  cudaError_t ce = H.nd ? nd_solve(H, P, J->NR, S.nb, s) : launch_solve(H, P, J->NR, S.nb, s);
  if (ce != cudaSuccess) return fail(ASP_ERR_CUDA, std::string("3D subproblem launch: ") + cudaGetErrorString(ce));
  return ASP_OK;
}

}  // namespace asp
