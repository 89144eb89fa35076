// btsolve_apply.cu -- instances of the batched layer solve used by every
// preconditioner apply: the M-solves (CLS_EMBED) and the sweep fills (CLS_FILL).
#include "btsolve.cuh"

namespace asp {

// Complex64 instances for full (PKT false) or packed symmetric factor blocks
// (PKT true, ASP_PREC_C64_SYM: four producer warps more, so the thread bounds
// grow by 128 and the register bounds are relaxed).  Variant 0 is each
// capacity's default tile; variant 1 the alternative the autotuner also times
// (asp_autotune): other rows per thread at 32 right-hand sides, eight lanes
// instead of four splitting each block's columns at 1 (shorter inner loops,
// one more shuffle round).
template <bool PKT>
cudaError_t apply_c64(Handle& H, const SolveParams& P, int cls, int cap, int variant, int wmax, cudaStream_t s) {
  using namespace bts;
  constexpr int X = PKT ? 128 : 0;
  if (variant == 1) {
    if (cls == CLS_EMBED) {
      if (cap == 32) return run<float, 2, 2, 8, 2, CLS_EMBED, 512 + X, 1, 3, 1, PKT>(H, P, wmax, s);
      if (cap == 1) return run<float, 2, 1, 1, 1, CLS_EMBED, 512, 1, 6, 8, PKT>(H, P, wmax, s);
    } else {
      if (cap == 32) return run<float, 4, 2, 8, 2, CLS_FILL, 256 + X, PKT ? 1 : 2, 3, 1, PKT>(H, P, wmax, s);
      if (cap == 1) return run<float, 2, 1, 1, 1, CLS_FILL, 512, 1, 6, 8, PKT>(H, P, wmax, s);
    }
    return cudaErrorInvalidValue;
  }
  if (variant != 0) return cudaErrorInvalidValue;
  if (cls == CLS_EMBED) {
    switch (cap) {
      case 32: return run<float, 4, 2, 8, 2, CLS_EMBED, 256 + X, PKT ? 1 : 2, 3, 1, PKT>(H, P, wmax, s);
      case 16: return run<float, 2, 2, 8, 1, CLS_EMBED, 512, 1, 3, 1, PKT>(H, P, wmax, s);
      case 8: return run<float, 2, 2, 4, 1, CLS_EMBED, 512, 1, 3, 1, PKT>(H, P, wmax, s);
      case 4: return run<float, 2, 2, 2, 1, CLS_EMBED, 512, 1, 6, 1, PKT>(H, P, wmax, s);
      case 2: return run<float, 2, 2, 1, 1, CLS_EMBED, 512, 1, 6, 4, PKT>(H, P, wmax, s);
      case 1: return run<float, 2, 1, 1, 1, CLS_EMBED, 512, 1, 6, 4, PKT>(H, P, wmax, s);
    }
  } else {
    switch (cap) {
      case 32:  // blocks wider than 48 need 8 row warps per column half (512 threads)
        if (wmax > 48) return run<float, 2, 2, 8, 2, CLS_FILL, 512 + X, 1, 3, 1, PKT>(H, P, wmax, s);
        return run<float, 2, 2, 8, 2, CLS_FILL, 384 + X, PKT ? 1 : 2, 3, 1, PKT>(H, P, wmax, s);
      case 16: return run<float, 2, 2, 8, 1, CLS_FILL, 512, 1, 3, 1, PKT>(H, P, wmax, s);
      case 8: return run<float, 2, 2, 4, 1, CLS_FILL, 512, 1, 3, 1, PKT>(H, P, wmax, s);
      case 4: return run<float, 2, 2, 2, 1, CLS_FILL, 512, 1, 6, 1, PKT>(H, P, wmax, s);
      case 2: return run<float, 2, 2, 1, 1, CLS_FILL, 512, 1, 6, 4, PKT>(H, P, wmax, s);
      case 1: return run<float, 2, 1, 1, 1, CLS_FILL, 512, 1, 6, 4, PKT>(H, P, wmax, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_btsolve_apply(Handle& H, const SolveParams& P, int cls, int cap, int variant, int wmax,
                                 cudaStream_t s) {
  using namespace bts;
  if (H.prec == ASP_PREC_C64)
    return H.packed ? apply_c64<true>(H, P, cls, cap, variant, wmax, s)
                    : apply_c64<false>(H, P, cls, cap, variant, wmax, s);
  if (variant != 0) return cudaErrorInvalidValue;
  if (cls == CLS_EMBED) {
    switch (cap) {
      case 16: return run<double, 2, 2, 8, 1, CLS_EMBED>(H, P, wmax, s);
      case 8: return run<double, 2, 2, 4, 1, CLS_EMBED>(H, P, wmax, s);
      case 4: return run<double, 2, 2, 2, 1, CLS_EMBED>(H, P, wmax, s);
      case 2: return run<double, 2, 2, 1, 1, CLS_EMBED>(H, P, wmax, s);
      case 1: return run<double, 2, 1, 1, 1, CLS_EMBED>(H, P, wmax, s);
    }
  } else {
    switch (cap) {
      case 16: return run<double, 2, 2, 8, 1, CLS_FILL>(H, P, wmax, s);
      case 8: return run<double, 2, 2, 4, 1, CLS_FILL>(H, P, wmax, s);
      case 4: return run<double, 2, 2, 2, 1, CLS_FILL>(H, P, wmax, s);
      case 2: return run<double, 2, 2, 1, 1, CLS_FILL>(H, P, wmax, s);
      case 1: return run<double, 2, 1, 1, 1, CLS_FILL>(H, P, wmax, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace asp
