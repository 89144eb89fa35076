// common.cuh -- device helpers shared by the libasp kernels (sm_103a).
//
// Complex arithmetic on interleaved (re, im) pairs, the inline-PTX wrappers for
// mbarriers, 1D bulk (TMA) copies and cp.async, and the bounded-wait / error-flag
// conventions: no kernel in this library traps or spins without a limit; a wait
// that runs out records ASP_ERR_TIMEOUT in the handle's device error word and
// the kernel returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "asp.h"

namespace asp {

// ------------------------------------------------------------------ complex
template <typename R> struct CxT;
template <> struct CxT<float> { using T = float2; };
template <> struct CxT<double> { using T = double2; };
template <typename R> using Cx = typename CxT<R>::T;

template <typename R> __host__ __device__ __forceinline__ Cx<R> cmake(R re, R im) {
  Cx<R> c; c.x = re; c.y = im; return c;
}
template <typename R> __host__ __device__ __forceinline__ Cx<R> czero() { return cmake<R>(R(0), R(0)); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename C> __device__ __forceinline__ void cfms(C& acc, C a, C b) {
  acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ C cconjmul(C a, C b) {  // conj(a) * b
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename R> __device__ __forceinline__ Cx<R> cvt(double2 a) { return cmake<R>(R(a.x), R(a.y)); }
template <typename R> __device__ __forceinline__ Cx<R> cvt(float2 a) { return cmake<R>(R(a.x), R(a.y)); }

// 1/z for complex z (used for pivots; z != 0 checked by the caller)
template <typename C> __device__ __forceinline__ C crecip(C z) {
  auto d = z.x * z.x + z.y * z.y;
  C r;
  if constexpr (sizeof(z.x) == 4) {
    // complex64: one correctly rounded reciprocal of |z|^2 and two products
    // (within an ulp of the two divisions, and off the dependent chain of a
    // Gauss-Jordan step's pivot for most of their latency)
    const float rd = __frcp_rn(d);
    r.x = z.x * rd; r.y = -z.y * rd;
  } else {
    r.x = z.x / d; r.y = -z.y / d;
  }
  return r;
}

// ------------------------------------------------------------- error word
// err[0]: first error code recorded (ASP_OK = 0 means none), err[1]: detail
// (e.g. the subproblem index with a bad pivot).
__device__ __forceinline__ void record_error(int* err, int code, int detail) {
  if (err && atomicCAS(err, 0, code) == 0) atomicExch(err + 1, detail);
}

// Iteration limit of every device spin-wait (each try_wait may itself block for
// a hardware-chosen time slice); far above any legitimate wait in this library.
constexpr uint32_t kSpinLimit = 1u << 26;

// ------------------------------------------------------------ mbarrier PTX
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Returns true once the phase with the given parity has completed; false if the
// bounded spin (limit polls) ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  uint32_t addr = smem_addr(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 1D bulk copy global -> shared (the TMA's non-tensor form).  dst, src 16-byte
// aligned, bytes a multiple of 16.  Completion is signalled on `bar` as
// transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------------------- cp.async
template <int BYTES> __device__ __forceinline__ void cp_async(void* dst, const void* src) {
  static_assert(BYTES == 8 || BYTES == 16, "cp.async size");
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace asp
