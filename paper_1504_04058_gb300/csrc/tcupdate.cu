// tcupdate.cu -- the rank-kSlabOuter update of the 3D slab factor (factor3d.cu,
// "big update") on the tcgen05 tensor cores, for complex64 factors.
//
// Per slab and outer block [C0, C0+K) the update is
//     C[i][j] = (i a pivot of the block ? 0 : C[i][j]) + sum_u P[i][u] Z[u][j]
// for every column j outside the block, with P the block's columns after its
// panels and Z the block's pivot rows before the update.  It is a complex
// product of inner dimension K <= 256, written here as one real product:
//   * A' = P read as a real nb x 2K matrix (re, im interleaved along K) -- the
//     complex row-major layout already is K-major;
//   * B' (2K x 2nb) holds for every complex entry z = Z[u][j] the real 2 x 2
//     block [[re z, im z], [-im z, re z]] (rows 2u, 2u+1; columns 2j, 2j+1), so
//     the product's columns 2j, 2j+1 are re and im of the complex result and
//     the accumulator rows are complex64 rows of C;
//   * split precision: each operand x is split into x_hi = x with its 13 low
//     mantissa bits cleared (exact in TF32) and x_lo = x - x_hi, and the
//     product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32
//     (the dropped A_lo B_lo term is 2^-22 relative).
// A prep kernel writes A_hi, A_lo (rows of 2*kSlabOuter floats) and B'^T_hi,
// B'^T_lo (2nb rows of 2*kSlabOuter floats, K-major) for every slab of the
// launch.  The update kernel computes 128 x 128 complex tiles of C:
//   * one thread issues TMA 2D tiled loads (128-byte swizzle) of 32-float K
//     chunks of the four operands into a two-stage shared-memory ring, tracked
//     by mbarriers;
//   * one thread issues tcgen05.mma (kind::tf32, M = 128, N = 256, K = 8 per
//     instruction, both operands K-major from shared-memory descriptors) into
//     a 128 x 256 FP32 accumulator in tensor memory; tcgen05.commit releases
//     each ring stage and finally signals the epilogue;
//   * eight epilogue warps (two per TMEM lane quarter, each taking half of the
//     columns) read the accumulator with tcgen05.ld and add it into (or, for
//     pivot rows, store it as) C.
// Every wait is bounded; a timeout records ASP_ERR_TIMEOUT, and the CTA still
// waits (bounded) for its copies and products in flight and frees its tensor
// memory before it returns.
#include <cuda.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asp {

namespace {

constexpr int kTM = 128;            // tile rows (complex rows of C)
constexpr int kTNc = 128;           // tile columns (complex)
constexpr int kTN = 2 * kTNc;       // MMA N (real columns)
constexpr int kKC = 32;             // floats per K chunk (one 128-byte swizzle row)
constexpr int kStages = 2;
constexpr int kRowF = 2 * kSlabOuter;  // floats per operand row (K' capacity)
constexpr uint32_t kABytes = kTM * kKC * 4;  // 16 KB
constexpr uint32_t kBBytes = kTN * kKC * 4;  // 32 KB
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr uint32_t kTmemCols = 256;
constexpr size_t kTcSmem = (size_t)kStages * kStageBytes + 1024;

struct TcMaps {
  CUtensorMap ahi, alo, bhi, blo;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout written by the TMA (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
  d |= (uint64_t)1u << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;                   // descriptor version
  d |= (uint64_t)2u << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major,
// M = kTM, N = kTN.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// ------------------------------------------------------------------- prep
// A_hi/A_lo row i (of slab s) = P[i][0..K) as 2K floats; B^T row 2j+c, float
// 2u+d = the (d, c) entry of the 2 x 2 block of Z[u][j].  Rows past nb and
// floats past 2K are zero.  Grid (tiles of 32 x 32 complex (u, j), slab);
// block (32, 8).
__global__ void __launch_bounds__(256) tc_prep_kernel(Slab3Params P, const long long* rowA, int C0, int buf,
                                                      float* ahi, float* alo, float* bhi, float* blo) {
  const Slab S = P.slabs[P.list[blockIdx.y]];
  const int nb = S.nb, ld = S.ld;
  if (C0 >= S.np) return;
  const int K = min(kSlabOuter, S.np - C0);
  const int nbpad = (nb + kTM - 1) / kTM * kTM;
  const int tiles_j = nbpad / 32;  // this slab's tiles; grid.x covers the largest slab's
  const int tu = blockIdx.x / tiles_j, tj = blockIdx.x - tu * tiles_j;  // tu < kSlabOuter / 32
  const int u0 = tu * 32, jt0 = tj * 32;
  if (tu >= kSlabOuter / 32) return;  // the grid is sized for the group's largest slab
  const float2* Aw = reinterpret_cast<const float2*>(P.A) + S.aoff + (long long)buf * nb * ld;
  const int* piv_row = P.piv + S.poff;
  const long long ra = rowA[blockIdx.y];
  __shared__ float2 tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  // A operand: rows i = jt0 + r (the j tile doubles as the row tile), complex u
  for (int r = ty; r < 32; r += 8) {
    const int i = jt0 + r, u = u0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (i < nb && u < K) v = Aw[(long long)i * ld + C0 + u];
    const long long o = (ra + i) * kRowF + 2 * u;
    const float hx = tf32_hi(v.x), hy = tf32_hi(v.y);
    ahi[o] = hx;
    ahi[o + 1] = hy;
    alo[o] = v.x - hx;
    alo[o + 1] = v.y - hy;
  }
  // B operand: Z[u][j] = A[piv_row[C0+u]][j], transposed through shared memory
  for (int r = ty; r < 32; r += 8) {
    const int u = u0 + r, j = jt0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (u < K && j < nb) {
      const int pr = min(max(piv_row[C0 + u], 0), nb - 1);
      v = Aw[(long long)pr * ld + j];
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = jt0 + r, u = u0 + tx;
    const float2 z = tile[tx][r];
    const long long o0 = (2 * ra + 2LL * j) * kRowF + 2 * u;  // row 2j   (re column)
    const long long o1 = o0 + kRowF;                           // row 2j+1 (im column)
    const float re = z.x, im = z.y;
    const float hre = tf32_hi(re), him = tf32_hi(im), hnim = tf32_hi(-im);
    bhi[o0] = hre;      blo[o0] = re - hre;
    bhi[o0 + 1] = hnim; blo[o0 + 1] = -im - hnim;
    bhi[o1] = him;      blo[o1] = im - him;
    bhi[o1 + 1] = hre;  blo[o1 + 1] = re - hre;
  }
}

// ------------------------------------------------------ persistent update
// The same tiles, with one CTA per SM walking them (tile t = blockIdx.x,
// blockIdx.x + gridDim.x, ... over (column tile, row tile, slab), skipping
// tiles that lie inside the eliminated block).  Warp roles:
//   warp 0 lane 0  TMA producer for every K chunk of every tile, into the
//                  two-stage ring (counters run on across tiles);
//   warp 1 lane 0  MMA issuer; tile it accumulates into tensor-memory buffer
//                  it & 1 (two 256-column accumulators), once the epilogue has
//                  released that buffer;
//   warps 2..      epilogue of tile it while the MMAs of tile it+1 run; warp w
//                  reads accumulator lanes 32*(w%4) .. +31, its share of the
//                  columns, and releases the buffer with one arrival per warp.
// Every wait is bounded; on a timeout the role records ASP_ERR_TIMEOUT and
// stops, the others time out in turn, and before the tensor memory is freed the
// issuer waits (bounded) for its last products and the producer for its last
// copies.
constexpr int kEpiWarps = 8;  // kEpiWarps / 4 per accumulator lane quarter, splitting the columns (4 and 16 measured slower)
constexpr int kPersistThreads = 64 + 32 * kEpiWarps;

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

struct TcTile {
  int valid, z, i0, j0, K, nb, ld;
  long long ra, aoff;
  int poff;
};

__device__ __forceinline__ TcTile tc_tile(const Slab3Params& P, const long long* rowA, int C0, int ncx, int ncy,
                                          int t) {
  TcTile T;
  const int bx = t % ncx, by = (t / ncx) % ncy, z = t / (ncx * ncy);
  const Slab S = P.slabs[P.list[z]];
  T.z = z;
  T.nb = S.nb;
  T.ld = S.ld;
  T.i0 = by * kTM;
  T.j0 = bx * kTNc;
  T.K = min(kSlabOuter, S.np - C0);
  T.ra = rowA[z];
  T.aoff = S.aoff;
  T.poff = (int)S.poff;
  T.valid = C0 < S.np && T.j0 < S.nb && T.i0 < S.nb && !(T.j0 >= C0 && T.j0 + kTNc <= C0 + T.K);
  return T;
}

__global__ void __launch_bounds__(kPersistThreads, 1)
    tc_update_persistent_kernel(const __grid_constant__ TcMaps maps, Slab3Params P, const long long* rowA, int C0,
                                int buf, int ncx, int ncy) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t sbase = (smem_addr(smem_raw) + 1023u) & ~1023u;
  unsigned char* sgen = smem_raw + (sbase - smem_addr(smem_raw));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2], last;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = ncx * ncy * P.nlist;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kEpiWarps);
    }
    mbar_init(&last, 1);
    s_err = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  auto stage_ptr = [&](int s, int which) -> unsigned char* {
    const uint32_t off = (uint32_t)s * kStageBytes +
                         (which < 2 ? which * kABytes : 2 * kABytes + (which - 2) * kBBytes);
    return sgen + off;
  };
  auto timeout = [&](int where) {
    record_error(P.err, ASP_ERR_TIMEOUT, where + blockIdx.x);
    atomicExch(&s_err, 1);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer
      long long g = 0;  // chunks issued by this CTA
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const TcTile T = tc_tile(P, rowA, C0, ncx, ncy, t);
        if (!T.valid) continue;
        const int nch = (2 * T.K + kKC - 1) / kKC;
        for (int ch = 0; ch < nch; ++ch, ++g) {
          const int s = (int)(g % kStages);
          const long long u = g / kStages;
          if (u >= 1 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) {
            timeout(3300000);
            stop = true;
            break;
          }
          if (s_err) { stop = true; break; }
          mbar_arrive_expect_tx(&full[s], kStageBytes);
          const int x = ch * kKC;
          tma_load_2d(stage_ptr(s, 0), &maps.ahi, x, (int)(T.ra + T.i0), &full[s]);
          tma_load_2d(stage_ptr(s, 1), &maps.alo, x, (int)(T.ra + T.i0), &full[s]);
          tma_load_2d(stage_ptr(s, 2), &maps.bhi, x, (int)(2 * T.ra + 2 * T.j0), &full[s]);
          tma_load_2d(stage_ptr(s, 3), &maps.blo, x, (int)(2 * T.ra + 2 * T.j0), &full[s]);
        }
      }
      if (stop) {
        // copies still in flight complete on their stage's full barrier
        for (int s = 0; s < kStages; ++s) {
          long long lastg = -1;
          for (long long q = g - 1; q >= 0 && q >= g - kStages; --q)
            if (q % kStages == s) lastg = q;
          if (lastg >= 0) mbar_wait(&full[s], (uint32_t)((lastg / kStages) & 1));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      long long g = 0;
      int it = 0;
      bool stop = false;
      bool issued_any = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const TcTile T = tc_tile(P, rowA, C0, ncx, ncy, t);
        if (!T.valid) continue;
        const int a = it & 1, ua = it >> 1;
        if (ua >= 1 && !mbar_wait(&acc_empty[a], (uint32_t)((ua - 1) & 1))) {
          timeout(3400000);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(a * kTmemCols);
        const int nch = (2 * T.K + kKC - 1) / kKC;
        for (int ch = 0; ch < nch; ++ch, ++g) {
          const int s = (int)(g % kStages);
          if (!mbar_wait(&full[s], (uint32_t)((g / kStages) & 1)) || s_err) {
            if (!s_err) timeout(3500000);
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = smem_addr(stage_ptr(s, 0)), al = smem_addr(stage_ptr(s, 1));
          const uint32_t bh = smem_addr(stage_ptr(s, 2)), bl = smem_addr(stage_ptr(s, 3));
#pragma unroll
          for (int kk = 0; kk < kKC / 8; ++kk) {
            const uint32_t ko = kk * 32;
            const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
            mma_tf32(dacc, sw128_desc(ah + ko), sw128_desc(bh + ko), acc);
            mma_tf32(dacc, sw128_desc(ah + ko), sw128_desc(bl + ko), 1u);
            mma_tf32(dacc, sw128_desc(al + ko), sw128_desc(bh + ko), 1u);
          }
          issued_any = true;
          mma_commit(&empty[s]);
        }
        if (stop) break;
        mma_commit(&acc_full[a]);
        ++it;
      }
      // every product issued by this thread has completed once `last` fires
      if (issued_any) {
        mma_commit(&last);
        mbar_wait(&last, 0u);
      }
    }
  } else {
    // ---- epilogue warps 2..9
    const int q = warp & 3;  // accumulator lane quarter this warp may read
    const int part = (warp - 2) >> 2;
    constexpr int kChunksPerWarp = (kTN / 32) / (kEpiWarps / 4);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const TcTile T = tc_tile(P, rowA, C0, ncx, ncy, t);
      if (!T.valid) continue;
      const int a = it & 1, ua = it >> 1;
      const bool ok = mbar_wait(&acc_full[a], (uint32_t)(ua & 1));
      if (!ok) {
        if (lane == 0) timeout(3600000);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int i = T.i0 + q * 32 + lane;
      const int* row_step = P.piv + T.poff + 2 * T.nb;
      const int st = i < T.nb ? row_step[i] : -1;
      const bool piv = st >= C0 && st < C0 + T.K;
      float2* crow = reinterpret_cast<float2*>(P.A) + T.aoff + (long long)buf * T.nb * T.ld +
                     (long long)min(i, T.nb - 1) * T.ld;
      const bool write = s_err == 0 && i < T.nb;
#pragma unroll 1
      for (int cc = part * kChunksPerWarp; cc < (part + 1) * kChunksPerWarp; ++cc) {
        float v[32];
        tmem_ld32(tmem + (uint32_t)(a * kTmemCols) + ((uint32_t)(q * 32) << 16) + (uint32_t)(cc * 32), v);
        if (write) {
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) {
            const int j = T.j0 + cc * 16 + qq;
            if (j < T.nb && !(j >= C0 && j < C0 + T.K)) {
              const float2 av = make_float2(v[2 * qq], v[2 * qq + 1]);
              if (piv) {
                crow[j] = av;
              } else {
                const float2 c = crow[j];
                crow[j] = make_float2(c.x + av.x, c.y + av.y);
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive1(&acc_empty[a]);
      ++it;
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Looked up once; the static's initialisation is thread-safe, so handles
// factored from several host threads at once all see the same result.
EncodeTiled encoder() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiled>(p);
    return nullptr;
  }();
  return fn;
}

bool make_map(CUtensorMap* m, float* base, long long rows, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kRowF, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kRowF * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Floats of one group's operand area: A_hi, A_lo (rows sum nbpad) and B_hi,
// B_lo (2 * rows) of kRowF floats.
long long tc_group_floats(long long rows) { return 6LL * rows * kRowF; }

int tc_group_setup(TcGroup& G, float* area, const std::vector<long long>& rowA_host, long long rows) {
  G.ahi = area;
  G.alo = G.ahi + rows * kRowF;
  G.bhi = G.alo + rows * kRowF;
  G.blo = G.bhi + 2 * rows * kRowF;
  TcMaps* maps = new TcMaps();
  bool ok = make_map(&maps->ahi, G.ahi, rows, kTM) && make_map(&maps->alo, G.alo, rows, kTM) &&
            make_map(&maps->bhi, G.bhi, 2 * rows, kTN) && make_map(&maps->blo, G.blo, 2 * rows, kTN);
  if (!ok) {
    delete maps;
    return fail(ASP_ERR_UNSUPPORTED, "tensor-map encoding for the tensor-core update failed");
  }
  G.maps = maps;
  if (dev_malloc((void**)&G.rowA, rowA_host.size() * sizeof(long long)) != cudaSuccess)
    return fail(ASP_ERR_OOM, "tensor-core update row table");
  if (cudaMemcpy(G.rowA, rowA_host.data(), rowA_host.size() * sizeof(long long), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return fail(ASP_ERR_CUDA, "tensor-core update row table upload");
  return ASP_OK;
}

void tc_group_release(TcGroup& G) {
  delete reinterpret_cast<TcMaps*>(G.maps);
  G.maps = nullptr;
  if (G.rowA) cudaFree(G.rowA);
  G.rowA = nullptr;
}

cudaError_t launch_tc_update(const TcGroup& G, const Slab3Params& P, int nbmax, int C0, int buf, cudaStream_t s) {
  const int nbpad = (nbmax + kTM - 1) / kTM * kTM;
  const dim3 pgrid((kSlabOuter / 32) * (nbpad / 32), P.nlist);
  tc_prep_kernel<<<pgrid, dim3(32, 8), 0, s>>>(P, G.rowA, C0, buf, G.ahi, G.alo, G.bhi, G.blo);
  cudaError_t e = ensure_dyn_smem((const void*)tc_update_persistent_kernel, kTcSmem);
  if (e != cudaSuccess) return e;
  const int ncx = (nbmax + kTNc - 1) / kTNc, ncy = (nbmax + kTM - 1) / kTM;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = std::max(1, std::min(ncx * ncy * P.nlist, sms));
  tc_update_persistent_kernel<<<grid, kPersistThreads, kTcSmem, s>>>(*reinterpret_cast<const TcMaps*>(G.maps), P,
                                                                     G.rowA, C0, buf, ncx, ncy);
  return cudaGetLastError();
}

}  // namespace asp
