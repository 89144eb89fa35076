// chain_bench.cu -- standalone timing of the sweep-chain launch (chain.cu) at
// the shape of a 2D problem with n points per side and m layers, 32 right-hand
// sides, on synthetic maps and traces.  It holds only the 2(m-2) transfer maps
// and the trace buffers (4.1 GB at n = 1023, m = 246), not the factors or the
// Krylov space of a full solve, so a profiler can capture the launch on its own.
// Not part of libasp.so; build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -lineinfo -Iinclude \
//        -Ipaper_1504_04058_gb300/csrc -o chain_bench paper_1504_04058_gb300/csrc/chain_bench.cu
//   ./chain_bench [n] [m] [launches]
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "chain.cu"

namespace asp {
cudaError_t ensure_dyn_smem(const void* func, size_t bytes) {
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
}  // namespace asp

using namespace asp;

// deterministic pseudo-random fill, values in [-scale/2, scale/2)
__global__ void fill_kernel(float2* p, long long count, unsigned seed, float scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 13;
    h *= 0x5bd1e995u;
    h ^= h >> 15;
    p[i] = make_float2(scale * ((h & 0xffff) / 65536.f - 0.5f), scale * ((h >> 16) / 65536.f - 0.5f));
  }
}

#define CHECK(x)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) {                                                               \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                        \
      return 1;                                                                            \
    }                                                                                      \
  } while (0)

int main(int argc, char** argv) {
  const int n = argc > 1 ? std::atoi(argv[1]) : 1023;
  const int m = argc > 2 ? std::atoi(argv[2]) : 246;
  const int reps = argc > 3 ? std::atoi(argv[3]) : 10;
  const int nrhs = 32, lda = 32, ldT = (n + 1) & ~1;
  if (n < 2 || m < 3 || reps < 1) {
    std::fprintf(stderr, "usage: chain_bench [n >= 2] [m >= 3] [launches >= 1]\n");
    return 2;
  }
  Handle H;
  CHECK(cudaDeviceGetAttribute(&H.num_sms, cudaDevAttrMultiProcessorCount, 0));
  H.prec = ASP_PREC_C64;
  const long long tm_elems = 2LL * (m - 2) * n * ldT, acc_elems = (long long)(m + 1) * n * lda;
  float2 *tm = nullptr, *accR = nullptr, *accL = nullptr;
  unsigned* bar = nullptr;
  int* err = nullptr;
  long long *toffR = nullptr, *toffL = nullptr;
  CHECK(cudaMalloc(&tm, tm_elems * sizeof(float2)));
  CHECK(cudaMalloc(&accR, acc_elems * sizeof(float2)));
  CHECK(cudaMalloc(&accL, acc_elems * sizeof(float2)));
  CHECK(cudaMalloc(&bar, 2 * sizeof(unsigned)));
  CHECK(cudaMalloc(&err, 2 * sizeof(int)));
  CHECK(cudaMemset(err, 0, 2 * sizeof(int)));
  std::vector<long long> tr(m + 1, 0), tl(m + 1, 0);
  long long off = 0;
  for (int q = 2; q <= m - 1; ++q) {
    tr[q] = off;
    off += (long long)n * ldT;
    tl[q] = off;
    off += (long long)n * ldT;
  }
  CHECK(cudaMalloc(&toffR, (m + 1) * sizeof(long long)));
  CHECK(cudaMalloc(&toffL, (m + 1) * sizeof(long long)));
  CHECK(cudaMemcpy(toffR, tr.data(), (m + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(toffL, tl.data(), (m + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  // maps of norm about 1/2 keep the traces bounded over the chain
  fill_kernel<<<1024, 256>>>(tm, tm_elems, 1u, 1.0f / n);
  fill_kernel<<<1024, 256>>>(accR, acc_elems, 2u, 1.0f);
  fill_kernel<<<1024, 256>>>(accL, acc_elems, 3u, 1.0f);
  CHECK(cudaDeviceSynchronize());

  ChainParams C{};
  C.n = n; C.m = m; C.ldacc = lda; C.ldT = ldT; C.nrhs = nrhs;
  C.tmap = tm; C.toffR = toffR; C.toffL = toffL; C.accR = accR; C.accL = accL; C.bar = bar; C.err = err;
  cudaEvent_t a, b;
  CHECK(cudaEventCreate(&a));
  CHECK(cudaEventCreate(&b));
  for (int i = 0; i < 3; ++i) CHECK(launch_chain(H, C, 0));
  CHECK(cudaEventRecord(a, 0));
  for (int i = 0; i < reps; ++i) CHECK(launch_chain(H, C, 0));
  CHECK(cudaEventRecord(b, 0));
  CHECK(cudaEventSynchronize(b));
  float ms = 0.f;
  CHECK(cudaEventElapsedTime(&ms, a, b));
  int herr[2] = {0, 0};
  CHECK(cudaMemcpy(herr, err, sizeof(herr), cudaMemcpyDeviceToHost));
  const double per = ms / reps;
  const double bytes = 2.0 * (m - 2) * (double)n * n * sizeof(float2);
  const double flops = 8.0 * nrhs * 2.0 * (m - 2) * (double)n * n;
  std::printf("n %d m %d SMs %d: %.3f ms per launch, %.2f us per layer, maps %.1f GB/s, %.2f TFLOP/s, error word %d %d\n",
              n, m, H.num_sms, per, 1e3 * per / (m - 2), bytes / (per * 1e-3) / 1e9, flops / (per * 1e-3) / 1e12,
              herr[0], herr[1]);
  return herr[0] == 0 ? 0 : 3;
}
