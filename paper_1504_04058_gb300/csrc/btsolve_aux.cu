// btsolve_aux.cu -- instances of the batched layer solve used at factor time
// (the transfer maps, CLS_TMAP) and by the single-subproblem checking entry
// point (CLS_SUB).
#include "btsolve.cuh"

namespace asp {

template <bool PKT>
cudaError_t aux_c64(Handle& H, const SolveParams& P, int cls, int cap, int wmax, cudaStream_t s) {
  using namespace bts;
  constexpr int X = PKT ? 128 : 0;  // producer warps of packed factors
  if (cls == CLS_TMAP) {
    if (cap == 64 && wmax <= 24) return run<float, 2, 4, 8, 2, CLS_TMAP, 192 + X, PKT ? 2 : 3, 3, 1, PKT>(H, P, wmax, s);
    if (cap == 64) return run<float, 2, 4, 8, 2, CLS_TMAP, 512 + X, 1, 3, 1, PKT>(H, P, wmax, s);
  } else {
    if (cap == 4) return run<float, 2, 2, 2, 1, CLS_SUB, 512, 1, 3, 1, PKT>(H, P, wmax, s);
    if (cap == 1) return run<float, 2, 1, 1, 1, CLS_SUB, 512, 1, 3, 1, PKT>(H, P, wmax, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_btsolve_aux(Handle& H, const SolveParams& P, int cls, int cap, int wmax, cudaStream_t s) {
  using namespace bts;
  if (H.prec == ASP_PREC_C64)
    return H.packed ? aux_c64<true>(H, P, cls, cap, wmax, s) : aux_c64<false>(H, P, cls, cap, wmax, s);
  if (cls == CLS_TMAP) {
    if (cap == 16) return run<double, 2, 2, 8, 1, CLS_TMAP>(H, P, wmax, s);
  } else {
    if (cap == 4) return run<double, 2, 2, 2, 1, CLS_SUB>(H, P, wmax, s);
    if (cap == 1) return run<double, 2, 1, 1, 1, CLS_SUB>(H, P, wmax, s);
  }
  return cudaErrorInvalidValue;
}

// Right-hand sides one CTA handles, for jobs with at most `nrhs` right-hand
// sides (`tmap`: the transfer-map construction, whose n columns are the
// right-hand sides).  Returns 0 if no instance fits (w > 64).
int btsolve_rhs_capacity(int nrhs, int wmax, int prec, bool tmap) {
  if (wmax > 64) return 0;
  if (tmap) return prec == ASP_PREC_C64 ? 64 : 16;
  if (nrhs >= 32) return prec == ASP_PREC_C64 ? 32 : 16;
  if (nrhs >= 16) return 16;
  if (nrhs >= 8) return 8;
  if (nrhs >= 4) return 4;
  if (nrhs >= 2) return 2;
  return 1;
}

}  // namespace asp
