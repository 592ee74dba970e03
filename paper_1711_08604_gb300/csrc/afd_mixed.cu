// Grid and forward kernels for N = 2^a 3^b 5^c 7^d 11^e 13^f that is not a
// power of two.
//
// The paper's fast route (Eq. (rcl), Theorem 2.1, Sec. 3.1) splits the sum
// over l by the factors of N; the remark after Table 9 (Sec. 4.2) notes that
// the algorithm stays valid for N = p^K, p prime.  Here the transform is a
// mixed-radix Stockham FFT with radices 16, 8, 4, 2 and the odd primes 3, 5,
// 7, 11, 13 (mixed_schedule): pass p of
// radix R over sub-transforms of length Ns reads x[b + q N/R] (q < R) for
// butterfly b, multiplies input q by w^(dir q (b mod Ns) N/(Ns R)) with
// w = exp(2 pi i / N), does an R-point DFT and writes output q to
// ((b - b mod Ns) R + b mod Ns + q Ns); after the last pass the values are in
// natural order.  Pass 0 reads its inputs straight from global memory and the
// last pass hands its outputs to the caller from registers; the passes in
// between ping-pong between two shared-memory buffers of N points.
//
// k_grid_mixed  one CTA per (radius, signal): f(l) = r_s^l c_l / N, inverse
//               transform, objective w_s^2 |F_s(j)|^2, the per-radius best
//               pair(s) and, in the last CTA of the signal, the selection of
//               Step 2 -- the same contract as k_grid.
// k_forward_mixed  one CTA per signal: c_l / N = (1/N) sum_m G(z_m) w^{-ml};
//               k_forward_mixed_split the same over S CTAs per signal when N
//               has a factor 2 (mx_split).
// The FP64 guard and update kernels are shared with the power-of-two path
// (they index the sample points modulo N).  The transforms and the kernels'
// bodies live in afd_mixed.cuh, which the multi-signal persistent kernel
// shares.
#include <climits>
#include <cstdint>

#include "../../include/afd.h"
#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_internal.h"
#include "afd_mixed.cuh"

namespace afd {

namespace {

template <typename T>
__global__ void __launch_bounds__(MX_THREADS)
k_grid_mixed(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  pdl_launch_dependents();
  if constexpr (sizeof(T) == 4) {
    __shared__ SelectScratch scr;
    grid_mixed_body<T>(slots, ids, blockIdx.x, blockIdx.y, gridDim.x, &scr);
  } else {
    grid_mixed_body<T>(slots, ids, blockIdx.x, blockIdx.y, gridDim.x, nullptr);
  }
}

template <typename T>
__global__ void __launch_bounds__(MX_THREADS)
k_forward_mixed(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  pdl_launch_dependents();
  forward_mixed_body<T>(slots, ids, blockIdx.x);
}

// The forward transform over S = gridDim.x CTAs per signal (mx_split).
template <typename T>
__global__ void __launch_bounds__(MX_THREADS)
k_forward_mixed_split(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  pdl_launch_dependents();
  forward_mixed_split_body<T>(slots, ids, blockIdx.x, blockIdx.y, gridDim.x);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_mx(void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(MX_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

size_t mixed_smem_bytes(int N, int prec) { return 2 * (size_t)N * (prec == AFD_FP32_GUARDED ? 8 : 16); }

cudaError_t launch_grid_mixed(const SlotDev* slots, const int* ids, int n, int N, int prec, int Mmax,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid(Mmax, n);
  const size_t smem = mixed_launch_smem(N, prec);
  if (prec == AFD_FP32_GUARDED) return launch_pdl_mx(k_grid_mixed<float>, grid, smem, st, slots, ids);
  return launch_pdl_mx(k_grid_mixed<double>, grid, smem, st, slots, ids);
}

cudaError_t launch_forward_mixed(const SlotDev* slots, const int* ids, int n, int N, int prec, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int S = mx_split(N);
  if (S > 1) {
    const size_t sm = mixed_split_smem(N, prec);
    if (prec == AFD_FP32_GUARDED) return launch_pdl_mx(k_forward_mixed_split<float>, dim3(S, n), sm, st, slots, ids);
    return launch_pdl_mx(k_forward_mixed_split<double>, dim3(S, n), sm, st, slots, ids);
  }
  const size_t smem = mixed_launch_smem(N, prec);
  if (prec == AFD_FP32_GUARDED) return launch_pdl_mx(k_forward_mixed<float>, dim3(n), smem, st, slots, ids);
  return launch_pdl_mx(k_forward_mixed<double>, dim3(n), smem, st, slots, ids);
}

cudaError_t mixed_configure() {
  cudaError_t e;
  const int smem = MIXED_MAX_SMEM;
  if ((e = cudaFuncSetAttribute(k_grid_mixed<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_grid_mixed<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_forward_mixed<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_forward_mixed_split<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_forward_mixed_split<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  return cudaFuncSetAttribute(k_forward_mixed<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace afd

