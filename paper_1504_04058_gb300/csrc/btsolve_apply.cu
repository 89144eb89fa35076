// btsolve_apply.cu -- instances of the batched layer solve used by every
// preconditioner apply: the M-solves (CLS_EMBED) and the sweep fills (CLS_FILL).
#include "btsolve.cuh"

namespace asp {

cudaError_t launch_btsolve_apply(Handle& H, const SolveParams& P, int cls, int cap, int wmax, cudaStream_t s) {
  using namespace bts;
  if (H.prec == ASP_PREC_C64) {
    if (cls == CLS_EMBED) {
      switch (cap) {
        case 32: return run<float, 4, 2, 8, 2, CLS_EMBED, 256, 2>(H, P, wmax, s);
        case 16: return run<float, 2, 2, 8, 1, CLS_EMBED>(H, P, wmax, s);
        case 8: return run<float, 2, 2, 4, 1, CLS_EMBED>(H, P, wmax, s);
        case 4: return run<float, 2, 2, 2, 1, CLS_EMBED, 512, 1, 6>(H, P, wmax, s);
        case 2: return run<float, 2, 2, 1, 1, CLS_EMBED, 512, 1, 6, 4>(H, P, wmax, s);
        case 1: return run<float, 2, 1, 1, 1, CLS_EMBED, 512, 1, 6, 4>(H, P, wmax, s);
      }
    } else {
      switch (cap) {
        case 32:  // blocks wider than 48 need 8 row warps per column half (512 threads)
          if (wmax > 48) return run<float, 2, 2, 8, 2, CLS_FILL, 512, 1>(H, P, wmax, s);
          return run<float, 2, 2, 8, 2, CLS_FILL, 384, 2>(H, P, wmax, s);
        case 16: return run<float, 2, 2, 8, 1, CLS_FILL>(H, P, wmax, s);
        case 8: return run<float, 2, 2, 4, 1, CLS_FILL>(H, P, wmax, s);
        case 4: return run<float, 2, 2, 2, 1, CLS_FILL, 512, 1, 6>(H, P, wmax, s);
        case 2: return run<float, 2, 2, 1, 1, CLS_FILL, 512, 1, 6, 4>(H, P, wmax, s);
        case 1: return run<float, 2, 1, 1, 1, CLS_FILL, 512, 1, 6, 4>(H, P, wmax, s);
      }
    }
  } else {
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
  }
  return cudaErrorInvalidValue;
}

}  // namespace asp
