// bench_peaks.cu -- FP32 and FP64 fused multiply-add peaks of the GPU, the
// denominators of the benchmark's ALU rooflines (bench.py loads it as
// _build/libbenchpeaks.so; __graft_entry__.build() compiles it).
//
// Each thread runs 8 independent FMA chains a = a * b + c for `iters` steps
// (8 chains hide the FMA latency at any occupancy above a quarter), on a grid
// of blocks_per_sm x SM-count blocks of 256 threads.  b slightly below 1 and a
// small c keep every value finite and normal.  One FMA = 2 flops.  The kernel
// is timed with CUDA events on its stream after one untimed launch; the best
// of `repeats` launches is returned.
#include <cuda_runtime.h>

#include <cstdio>

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ sink, long long iters, T b, T c) {
  T a0 = (T)(threadIdx.x + 1) * (T)1e-3, a1 = a0 + (T)0.1, a2 = a0 + (T)0.2, a3 = a0 + (T)0.3;
  T a4 = a0 + (T)0.4, a5 = a0 + (T)0.5, a6 = a0 + (T)0.6, a7 = a0 + (T)0.7;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u) {
      a0 = fma(a0, b, c);
      a1 = fma(a1, b, c);
      a2 = fma(a2, b, c);
      a3 = fma(a3, b, c);
      a4 = fma(a4, b, c);
      a5 = fma(a5, b, c);
      a6 = fma(a6, b, c);
      a7 = fma(a7, b, c);
    }
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  // never true for these inputs; keeps the chains live
  if (s == (T)-1.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int run(long long iters, int blocks_per_sm, int repeats, float* best_ms, double* flops) {
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int blocks = n_sm * blocks_per_sm, threads = 256;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -2;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T b = (T)0.99999, c = (T)1e-4;
  k_fma_chains<T><<<blocks, threads, 0, st>>>(sink, iters, b, c);
  float best = 1e30f;
  for (int r = 0; r < repeats; ++r) {
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, threads, 0, st>>>(sink, iters, b, c);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(sink);
  if (err != cudaSuccess) return -3;
  *best_ms = best;
  *flops = 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * threads;
  return 0;
}

}  // namespace

extern "C" int bp_fma(int fp64, long long iters, int blocks_per_sm, int repeats, float* best_ms, double* flops) {
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || repeats < 1 || !best_ms || !flops) return -1;
  return fp64 ? run<double>(iters, blocks_per_sm, repeats, best_ms, flops)
              : run<float>(iters, blocks_per_sm, repeats, best_ms, flops);
}
