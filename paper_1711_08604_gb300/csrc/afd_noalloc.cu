// afd_inner_products_noalloc: the FP64 rectangle-rule inner product
// <G, e_a>~ = sqrt(1-|a|^2)/N * sum_m G(z_m) / (1 - a conj(z_m)) at arbitrary
// points a of the disc, computed without allocating any memory.
//
// Who needs this: code that must not call cudaMalloc -- work recorded into a
// CUDA graph or issued from a latency-critical loop (an allocation can
// synchronise the device and is not allowed while a stream is being
// captured), and hosts that hand a library a fixed, pre-reserved memory pool
// and forbid it from growing device memory on its own.  Such callers pass
// device-resident inputs and outputs; the scratch this kernel needs (one
// partial sum per point and sample chunk, plus a completion counter) lives in
// a file-scope static device array that every GPU loading the library keeps
// until the process exits.
//
// The array is shared by every call: calls that overlap on the GPU (on
// different streams, or from different host threads) race on it.  Its counter
// is cleared with a memset at the start of each call; the partial sums are
// fully rewritten before they are read.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/afd.h"
#include "afd_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 512;                                   // samples per CTA
constexpr int kMaxChunks = AFD_NOALLOC_MAX_N / kChunk;        // 128
constexpr size_t kPartialBytes = sizeof(double2) * AFD_NOALLOC_MAX_POINTS * kMaxChunks;  // 128 KiB
constexpr size_t kScratchBytes = kPartialBytes + 256;        // + completion counter

// The scratch array.  In host code its name is only a stand-in: the device
// address comes from cudaGetSymbolAddress (see scratch_for_current_device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

__global__ void __launch_bounds__(kThreads)
k_inner_noalloc(const double2* __restrict__ G, int N, const double2* __restrict__ a, int n_points,
                double2* __restrict__ out, unsigned char* scratch, int chunks) {
  __shared__ double red_re[kThreads / 32], red_im[kThreads / 32];
  __shared__ int s_last;
  double2* part = reinterpret_cast<double2*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kPartialBytes);
  const int point = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
  const double2 ap = a[point];
  const int m0 = chunk * kChunk, m1 = min(N, m0 + kChunk);
  double sr = 0.0, si = 0.0;
  for (int m = m0 + threadIdx.x; m < m1; m += kThreads) {
    double zs, zc;
    sincospi(2.0 * (double)m / (double)N, &zs, &zc);
    // d = 1 - a conj(z_m);  G / d = G conj(d) / |d|^2
    const double dr = 1.0 - (ap.x * zc + ap.y * zs);
    const double di = ap.x * zs - ap.y * zc;
    const double inv = 1.0 / fma(dr, dr, di * di);
    const double2 g = G[m];
    sr += (g.x * dr + g.y * di) * inv;
    si += (g.y * dr - g.x * di) * inv;
  }
  // fixed-order block reduction
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, off);
    si += __shfl_xor_sync(0xffffffffu, si, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red_re[threadIdx.x >> 5] = sr;
    red_im[threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      tr += red_re[w];
      ti += red_im[w];
    }
    part[point * chunks + chunk] = make_double2(tr, ti);
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: sum each point's chunks in order
  for (int p = threadIdx.x; p < n_points; p += kThreads) {
    double tr = 0.0, ti = 0.0;
    for (int c = 0; c < chunks; ++c) {
      const double2 v = __ldcg(&part[p * chunks + c]);
      tr += v.x;
      ti += v.y;
    }
    const double2 q = a[p];
    const double sc = sqrt(1.0 - (q.x * q.x + q.y * q.y)) / (double)N;
    out[p] = make_double2(sc * tr, sc * ti);
  }
}

// Device address of g_scratch for each device, looked up once per device with
// that device current.
std::mutex g_mu;
void* g_scratch_ptr[64] = {};

afd_status scratch_for_current_device(void** ptr, char* err, size_t errlen) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    snprintf(err, errlen, "cudaGetDevice: %s", cudaGetErrorString(e));
    return AFD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(err, errlen, "cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
      return AFD_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return AFD_OK;
}

// True if the current device (dev) can read and write p directly: device or
// managed memory of that device, or host memory mapped for the device.
// Device memory of another GPU is refused: the kernel runs on the current one.
bool device_accessible(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == dev;
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr);
}

thread_local char g_noalloc_err[256];

afd_status fail(afd_status st) {
  afd::set_last_error_text(g_noalloc_err);
  return st;
}

}  // namespace

extern "C" afd_status afd_inner_products_noalloc(const double* G, int N, const double* points,
                                                 int n_points, double* out, void* stream) {
  g_noalloc_err[0] = 0;
  afd::set_last_error_text("");
  if (!G || !points || !out) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "G, points and out must be non-NULL");
    return fail(AFD_ERR_INVALID);
  }
  if (N < 1 || N > AFD_NOALLOC_MAX_N) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "N = %d outside 1..%d (the static scratch limit)", N,
             AFD_NOALLOC_MAX_N);
    return fail(AFD_ERR_INVALID);
  }
  if (n_points < 1 || n_points > AFD_NOALLOC_MAX_POINTS) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "n_points = %d outside 1..%d (the static scratch limit)",
             n_points, AFD_NOALLOC_MAX_POINTS);
    return fail(AFD_ERR_INVALID);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "no current CUDA device");
    return fail(AFD_ERR_CUDA);
  }
  if (!device_accessible(G, dev) || !device_accessible(points, dev) || !device_accessible(out, dev)) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err),
             "G, points and out must be memory of the current device %d (or host memory mapped for it)", dev);
    return fail(AFD_ERR_INVALID);
  }
  void* scratch = nullptr;
  afd_status st = scratch_for_current_device(&scratch, g_noalloc_err, sizeof(g_noalloc_err));
  if (st != AFD_OK) return fail(st);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int chunks = (N + kChunk - 1) / kChunk;
  cudaError_t e = cudaMemsetAsync(static_cast<unsigned char*>(scratch) + kPartialBytes, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    k_inner_noalloc<<<n_points * chunks, kThreads, 0, s>>>(
        reinterpret_cast<const double2*>(G), N, reinterpret_cast<const double2*>(points), n_points,
        reinterpret_cast<double2*>(out), static_cast<unsigned char*>(scratch), chunks);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "launch failed: %s", cudaGetErrorString(e));
    return fail(AFD_ERR_CUDA);
  }
  return AFD_OK;
}
