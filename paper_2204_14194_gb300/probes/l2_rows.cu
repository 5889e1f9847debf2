// l2_rows.cu -- L2 -> SM read bandwidth on the iteration kernel's access pattern:
// each warp streams pseudo-random 8 KiB rows of an L2-resident 16 MiB table
// (the rows of C for K = 2048), and plain coalesced streaming for comparison.
// Prints GB/s per resident-warp count; used to place the iteration kernel.
#include <cstdio>
#include <cuda_runtime.h>
__global__ void rows_kernel(const float4* __restrict__ T, int K, int rows_per_warp, float* out, int salt) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  unsigned h = warp * 2654435761u + salt;
  float acc = 0.f;
  for (int i = 0; i < rows_per_warp; ++i) {
    h = h * 1664525u + 1013904223u;
    int u = (h >> 8) % K;
    const float4* row = T + (size_t)u * (K / 4);
    #pragma unroll
    for (int ch = 0; ch < 16; ++ch) { float4 v = __ldg(row + ch * 32 + lane); acc += v.x + v.y + v.z + v.w; }
    acc = __shfl_xor_sync(0xffffffffu, acc, 1) * 0.5f + acc * 0.5f;   // dependency like a reduction
  }
  if (acc == 12345.f) out[0] = acc;
}
__global__ void stream_kernel(const float4* __restrict__ T, size_t n4, int reps, float* out) {
  float acc = 0.f;
  for (int r = 0; r < reps; ++r)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
      float4 v = __ldg(T + i); acc += v.x + v.y + v.z + v.w; }
  if (acc == 12345.f) out[0] = acc;
}
int main() {
  const int K = 2048; size_t n = (size_t)K * K;
  float4* T; float* out; cudaMalloc(&T, n * 4); cudaMalloc(&out, 4); cudaMemset(T, 0, n * 4);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  for (int wps : {8, 16, 24, 32, 48}) {
    int threads = 128, ctas = sms * wps / 4, rows = 200;
    rows_kernel<<<ctas, threads>>>(T, K, rows, out, 1);
    cudaEventRecord(a);
    for (int r = 0; r < 5; ++r) rows_kernel<<<ctas, threads>>>(T, K, rows, out, r);
    cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    double bytes = 5.0 * ctas * 4 * rows * 8192.0;
    printf("rows  warps/SM=%2d  %.1f GB/s  (%.3f ms)\n", wps, bytes / ms / 1e6, ms / 5);
  }
  for (int mult : {4, 8, 16}) {
    int ctas = sms * mult, reps = 20;
    stream_kernel<<<ctas, 256>>>(T, n / 4, 1, out);
    cudaEventRecord(a); stream_kernel<<<ctas, 256>>>(T, n / 4, reps, out); cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    printf("stream ctas=%d  %.1f GB/s\n", ctas, reps * (double)n * 4 / ms / 1e6);
  }
  cudaError_t e = cudaGetLastError(); printf("err=%s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}
