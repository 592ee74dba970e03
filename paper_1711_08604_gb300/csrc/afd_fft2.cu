// Two-pass (four-step) FFT path for N = 65536 = 256 x 256, sm_103a, with the
// intermediate array staged through HBM by the Tensor Memory Accelerator.
//
// With l = l1 + 256 l2 and j = j2 + 256 j1 (all indices < 256),
//   F(j) = sum_l f(l) w^{jl} = sum_{l1} w256^{j1 l1} [ w^{j2 l1} sum_{l2} f(l1 + 256 l2) w256^{j2 l2} ],
// w = exp(DIR 2 pi i / N).  This is the splitting of Theorem 2.1 (Sec. 3.1)
// taken with a radix of 256 instead of 2: pass 1 does the 256 inner sums
// (length-256 transforms over l2) and the twiddle w^{j2 l1}; pass 2 the outer
// length-256 transforms over l1.
//
// Pass 1: a CTA takes 16 consecutive columns l1 of f (one radius s): a TMA
// load of a {16 l1 x 256 l2} tile (128-byte rows, 128B swizzle), the spectrum
// times r_s^l = r_s^{l1} r_s^{256 l2} in registers, 16 transforms of 256
// points, the twiddle, and a TMA store of the tile X_s[j2][l1] (X is stored
// transposed so that pass 2 reads whole rows).
// Pass 2: a CTA takes 16 rows j2 of X_s: a TMA load of {256 l1 x 16 j2}, 16
// transforms of 256 points, then either the objective w_s^2 |F_s(j)|^2 with
// the CTA's best two (grid mode) or, for the forward transform of G, a TMA
// store of c_j (forward mode).  X holds 512 KiB per radius: 2 x 512 KiB of
// HBM traffic per radius per step, the dominant memory stream.
//
// mbarrier waits are bounded: a load that does not arrive within the limit
// sets error bit 2 of the signal (AFD_ERR_TIMEOUT at the host) and stops it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_fft2.h"
#include "afd_internal.h"

namespace afd {

namespace {

constexpr int L8 = 8;                  // log2 of the 256-point sub-transforms
using S8 = FftShape<float, L8>;        // 16 threads x 16 points per transform
constexpr int kThreads = 256;          // 16 transforms per CTA
constexpr int kTileElems = 16 * 256;   // one TMA tile of float2
constexpr int kTileBytes = kTileElems * 8;
constexpr size_t kSmemBytes = 1024 + kTileBytes + sizeof(float2) * 16 * S8::SMEM;
constexpr long kWaitLimit = 1L << 22;  // mbarrier polls before giving up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(map), "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Element (row y, column x) of a {16 x 256} tile with 128-byte rows under the
// 128B swizzle: the 16-byte chunk index is XOR-ed with (y mod 8).
__device__ __forceinline__ int swz16(int y, int x) { return y * 16 + ((((x >> 1) ^ (y & 7))) << 1) + (x & 1); }

__device__ __forceinline__ float2* align1024(unsigned char* p) {
  const unsigned a = smem_u32(p);
  return reinterpret_cast<float2*>(p + ((1024u - (a & 1023u)) & 1023u));
}

// The tile's TMA load, with a bounded wait; false (after flagging the signal)
// when it did not arrive.
__device__ bool load_tile(float2* tile, const CUtensorMap* map, int x, int y, uint64_t* bar, SlotCtl* ctl) {
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, kTileBytes);
    tma_load_2d(tile, map, x, y, bar);
  }
  if (mbar_wait_bounded(bar, 0)) return true;
  if (threadIdx.x == 0) {
    atomicOr(&ctl->err, 4);
    ctl->done = 1;
  }
  mbar_wait_bounded(bar, 0);  // give a late copy a last chance to land before the CTA exits
  return false;
}

__device__ __forceinline__ bool better2(float va, int ja, float vb, int jb) {
  return va > vb || (va == vb && ja < jb);
}

}  // namespace

// MODE 0: grid (inverse transform of r_s^l c_l, one radius per blockIdx.y);
// MODE 1: forward transform of G / N.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_fft2_pass1(const SlotDev* __restrict__ slots, const __grid_constant__ Fft2Maps maps) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ alignas(8) uint64_t bar;
  pdl_launch_dependents();
  const SlotDev& sd = slots[0];
  float2* tile = align1024(smem_raw);
  float2* fbuf = tile + kTileElems;
  const int a = blockIdx.x, s = blockIdx.y;
  const int g = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int l1 = 16 * a + g;
  float lo = 1.f, h[16];
  if constexpr (MODE == 0) {
    lo = __ldg(&sd.p.rlo32[s * 256 + l1]);
#pragma unroll
    for (int q = 0; q < 16; ++q) h[q] = __ldg(&sd.p.rhi32[s * 256 + t + 16 * q]);
  }
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  if (!load_tile(tile, MODE == 0 ? &maps.c : &maps.g, 16 * a, 0, &bar, sd.ctl)) return;

  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float2 x = tile[swz16(t + 16 * q, g)];  // l2 = t + 16 q
    if constexpr (MODE == 0) {
      const float rp = lo * h[q];
      v[q] = make_float2(x.x * rp, x.y * rp);
    } else {
      v[q] = x;
    }
  }
  fft_run<float, L8, MODE == 0 ? 1 : -1>(v, t, fbuf + g * S8::SMEM, sd.p.st32);
  // twiddle w^{j2 l1} and the transposed tile X[j2][l1]
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int j2 = fft_out_index<float, L8>(t, e);
    const float2 w = __ldg(&sd.p.tw32n[j2 * l1]);
    tile[swz16(j2, g)] = MODE == 0 ? cmul<float>(v[e], w) : cmulc<float>(v[e], w);
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) tma_store_2d(&maps.xs, 16 * a, MODE == 0 ? s * 256 : 0, tile);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_fft2_pass2(const SlotDev* __restrict__ slots, const __grid_constant__ Fft2Maps maps) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ alignas(8) uint64_t bar;
  __shared__ float rv1[16], rv2[16];
  __shared__ int rj1[16], rj2[16];
  __shared__ int s_last;
  pdl_launch_dependents();
  const SlotDev& sd = slots[0];
  float2* tile = align1024(smem_raw);
  float2* fbuf = tile + kTileElems;
  const int b = blockIdx.x, s = blockIdx.y;
  const int g = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int j2 = 16 * b + g;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  if (!load_tile(tile, &maps.xl, 0, (MODE == 0 ? s * 256 : 0) + 16 * b, &bar, sd.ctl)) return;

  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = tile[g * 256 + t + 16 * q];  // row j2, l1 = t + 16 q
  fft_run<float, L8, MODE == 0 ? 1 : -1>(v, t, fbuf + g * S8::SMEM, sd.p.st32);

  if constexpr (MODE == 1) {
    // c_j for j = j2 + 256 j1, through a {16 j2 x 256 j1} tile
#pragma unroll
    for (int e = 0; e < 16; ++e) tile[swz16(fft_out_index<float, L8>(t, e), g)] = v[e];
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) tma_store_2d(&maps.c, 16 * b, 0, tile);
  } else {
    // best two of the CTA's 4096 grid points (j = j2 + 256 j1)
    float v1 = -1.f, v2 = -1.f;
    int i1 = INT_MAX, i2 = INT_MAX;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float o = v[e].x * v[e].x + v[e].y * v[e].y;
      const int j = j2 + 256 * fft_out_index<float, L8>(t, e);
      if (better2(o, j, v1, i1)) { v2 = v1; i2 = i1; v1 = o; i1 = j; }
      else if (better2(o, j, v2, i2)) { v2 = o; i2 = j; }
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      const float ov1 = __shfl_xor_sync(0xffffffffu, v1, off), ov2 = __shfl_xor_sync(0xffffffffu, v2, off);
      const int oi1 = __shfl_xor_sync(0xffffffffu, i1, off), oi2 = __shfl_xor_sync(0xffffffffu, i2, off);
      if (better2(ov1, oi1, v1, i1)) {
        if (better2(v1, i1, ov2, oi2)) { v2 = v1; i2 = i1; } else { v2 = ov2; i2 = oi2; }
        v1 = ov1; i1 = oi1;
      } else if (better2(ov1, oi1, v2, i2)) {
        v2 = ov1; i2 = oi1;
      }
    }
    if (t == 0) { rv1[g] = v1; rv2[g] = v2; rj1[g] = i1; rj2[g] = i2; }
    __syncthreads();
    if (threadIdx.x == 0) {
      float b1 = -1.f, b2 = -1.f;
      int k1 = INT_MAX, k2 = INT_MAX;
      for (int q = 0; q < 16; ++q) {
        const float cand[2] = {rv1[q], rv2[q]};
        const int cj[2] = {rj1[q], rj2[q]};
        for (int u = 0; u < 2; ++u) {
          if (better2(cand[u], cj[u], b1, k1)) { b2 = b1; k2 = k1; b1 = cand[u]; k1 = cj[u]; }
          else if (better2(cand[u], cj[u], b2, k2)) { b2 = cand[u]; k2 = cj[u]; }
        }
      }
      const float w2 = sd.p.wsq32[s];
      Top2F o;
      o.v1 = b1 * w2;
      o.v2 = b2 * w2;
      o.j1 = k1;
      o.j2 = k2;
      reinterpret_cast<Top2F*>(sd.top2)[s * 16 + b] = o;
      if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(o.v1));
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x * gridDim.y, &s_last)) return;
    select_candidates_f32<kThreads>(sd, sd.ctl->k, 16);
  }
}

cudaError_t fft2_configure() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_fft2_pass1<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes)))
    return e;
  if ((e = cudaFuncSetAttribute(k_fft2_pass1<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes)))
    return e;
  if ((e = cudaFuncSetAttribute(k_fft2_pass2<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes)))
    return e;
  return cudaFuncSetAttribute(k_fft2_pass2<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

namespace {
template <typename K>
cudaError_t launch2(K kernel, dim3 grid, const SlotDev* slots, const Fft2Maps& maps, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, slots, maps);
}
}  // namespace

cudaError_t launch_grid2(const SlotDev* slots, const Fft2Maps& maps, int M, cudaStream_t st) {
  cudaError_t e = launch2(k_fft2_pass1<0>, dim3(16, M), slots, maps, st);
  if (e != cudaSuccess) return e;
  return launch2(k_fft2_pass2<0>, dim3(16, M), slots, maps, st);
}

cudaError_t launch_forward2(const SlotDev* slots, const Fft2Maps& maps, cudaStream_t st) {
  cudaError_t e = launch2(k_fft2_pass1<1>, dim3(16, 1), slots, maps, st);
  if (e != cudaSuccess) return e;
  return launch2(k_fft2_pass2<1>, dim3(16, 1), slots, maps, st);
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int encode(CUtensorMap* m, void* base, cuuint64_t inner, cuuint64_t outer, cuuint32_t box_inner,
           cuuint32_t box_outer, bool swizzle) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return -1;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {inner * 8};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  return (int)fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}
}  // namespace

int fft2_make_maps(Fft2Maps* maps, void* c32, void* g32, void* X, int M) {
  int r;
  if ((r = encode(&maps->c, c32, 256, 256, 16, 256, true))) return r;
  if ((r = encode(&maps->g, g32, 256, 256, 16, 256, true))) return r;
  if ((r = encode(&maps->xs, X, 256, (cuuint64_t)M * 256, 16, 256, true))) return r;
  return encode(&maps->xl, X, 256, (cuuint64_t)M * 256, 256, 16, false);
}

}  // namespace afd
