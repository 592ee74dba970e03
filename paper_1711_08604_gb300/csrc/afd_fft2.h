// Two-pass TMA-staged FFT path for N = 65536 (afd_fft2.cu).  Internal.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "afd_internal.h"

namespace afd {

constexpr int FFT2_LOGN = 16;  // the one size that takes the two-pass path

// TMA descriptors of one signal's buffers, all viewed as 256 x 256 (x M for
// X) arrays of 8-byte complex64 elements.
struct Fft2Maps {
  CUtensorMap c;   // spectrum c32 [256 rows][256], box {16, 256}, 128B swizzle
  CUtensorMap g;   // G / N in FP32, g32 [256][256], box {16, 256}, 128B swizzle
  CUtensorMap xs;  // X [M * 256][256], box {16, 256}, 128B swizzle (pass-1 stores)
  CUtensorMap xl;  // X [M * 256][256], box {256, 16}, no swizzle (pass-2 loads)
};

cudaError_t fft2_configure();
// grid of one step (pass 1 and pass 2 over M radii), then the selection
cudaError_t launch_grid2(const SlotDev* slots, const Fft2Maps& maps, int M, cudaStream_t st);
// forward transform c = DFT(G) / N
cudaError_t launch_forward2(const SlotDev* slots, const Fft2Maps& maps, cudaStream_t st);
// Encodes the four maps (host).  Returns 0, or a nonzero driver status.
int fft2_make_maps(Fft2Maps* maps, void* c32, void* g32, void* X, int M);

}  // namespace afd
