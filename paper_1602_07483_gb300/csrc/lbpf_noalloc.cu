// lbpf_noalloc.cu -- allocation-free FP64 field sums for callers that cannot
// allocate device memory.
//
// lbpf_sums reduces into a partials buffer that lbpf_create allocated.  Some
// callers have device fields but may not allocate: latency-critical loops that
// must avoid the implicit device synchronisation of cudaMalloc and cudaFree, and
// hosts whose device memory is entirely reserved by another allocator (a memory
// pool sized to the whole device) so that a fresh cudaMalloc would fail.
// lbpf_field_sums_noalloc serves them: its scratch is the file-scope array below,
// which exists once per device for as long as the library is loaded.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/lbpf.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerBlock = kThreads * 16;  // one partial per 4096 sites
constexpr int kMaxPartials = 65536;            // 2 MiB of partials + 4 results

// Scratch of every call on this device: [kMaxPartials][4] partials, then 4 results.
// In host code `g_scratch` is only a stand-in for the symbol; kernels get its
// device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_scratch[4 * kMaxPartials + 4];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

template <typename T>
__global__ void k_sums_blocks(const T* __restrict__ phi, const T* __restrict__ U, const T* __restrict__ th,
                              double theta0, double k, long long n, double* __restrict__ part) {
  const long long base = (long long)blockIdx.x * kSitesPerBlock;
  double a = 0, b = 0, c = 0, d = 0;
  for (int j = threadIdx.x; j < kSitesPerBlock; j += kThreads) {
    const long long s = base + j;
    if (s >= n) break;
    const double p = (double)phi[s], u = (double)U[s];
    a += p;
    b += u;
    c += th ? (double)th[s] : theta0;
    d += 0.5 * ((1.0 + k) - (1.0 - k) * p) * (1.0 + (1.0 - k) * u);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
    d += __shfl_down_sync(0xffffffffu, d, o);
  }
  __shared__ double red[kThreads / 32][4];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w][0] = a; red[w][1] = b; red[w][2] = c; red[w][3] = d;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q][threadIdx.x];
    part[4 * blockIdx.x + threadIdx.x] = t;
  }
}

// Fixed-order sum of the partials: thread t adds partials t, t+256, ..., then a
// fixed tree; the result lands after the partials.
__global__ void k_sums_total(double* __restrict__ part, int nblk) {
  __shared__ double acc[kThreads][4];
  double v[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += kThreads)
    for (int c = 0; c < 4; ++c) v[c] += part[4 * b + c];
  for (int c = 0; c < 4; ++c) acc[threadIdx.x][c] = v[c];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 4; ++c) acc[threadIdx.x][c] += acc[threadIdx.x + s][c];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[4 * kMaxPartials + threadIdx.x] = acc[0][threadIdx.x];
}

// Device address of the scratch on the current device, looked up once per device (the
// first call on a device does this set-up).  The address belongs to that device's primary
// context: after cudaDeviceReset the module is loaded again and the cached address is
// stale, so a process that resets a device must not call this entry point on it again.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBPF_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBPF_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return LBPF_OK;
}

}  // namespace

extern "C" int lbpf_field_sums_noalloc(const void* phi, const void* U, const void* theta, int32_t storage,
                                       int64_t n_sites, double k, double theta0, double out[4], void* cuda_stream) {
  if (!phi || !U || !out || n_sites < 1) return LBPF_EINVAL;
  if (storage < LBPF_F64 || storage > LBPF_BF16) return LBPF_EINVAL;
  if (n_sites > LBPF_NOALLOC_MAX_SITES) return LBPF_EINVAL;  // more partials than the scratch holds
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the result is copied to host memory and the stream synchronised, which a stream under
  // capture does not allow: refuse such a stream before enqueueing anything on it
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    fprintf(stderr, "lbpf_field_sums_noalloc: the stream is being captured; call it outside stream capture\n");
    return LBPF_EINVAL;
  }
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != LBPF_OK) return rc;
  const int nblk = (int)((n_sites + kSitesPerBlock - 1) / kSitesPerBlock);
  if (storage == LBPF_F64)
    k_sums_blocks<double><<<nblk, kThreads, 0, st>>>((const double*)phi, (const double*)U, (const double*)theta,
                                                     theta0, k, (long long)n_sites, scratch);
  else
    k_sums_blocks<float><<<nblk, kThreads, 0, st>>>((const float*)phi, (const float*)U, (const float*)theta, theta0,
                                                    k, (long long)n_sites, scratch);
  if (cudaGetLastError() != cudaSuccess) return LBPF_ECUDA;
  k_sums_total<<<1, kThreads, 0, st>>>(scratch, nblk);
  if (cudaGetLastError() != cudaSuccess) return LBPF_ECUDA;
  if (cudaMemcpyAsync(out, scratch + 4 * kMaxPartials, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LBPF_ECUDA;
  for (int c = 0; c < 4; ++c)
    if (!isfinite(out[c])) return LBPF_ENAN;
  return LBPF_OK;
}
