// Two-pass (four-step) FFT path for N = 65536 = 256 x 256, sm_103a, with the
// intermediate array staged through HBM by the Tensor Memory Accelerator.
//
// With l = l1 + 256 l2 and j = j2 + 256 j1 (all indices < 256),
//   F(j) = sum_l f(l) w^{jl} = sum_{l1} w256^{j1 l1} [ w^{j2 l1} sum_{l2} f(l1 + 256 l2) w256^{j2 l2} ],
// w = exp(DIR 2 pi i / N).  This is the splitting of Theorem 2.1 (Sec. 3.1)
// taken with a radix of 256 instead of 2: pass 1 does the 256 inner sums
// (length-256 transforms over l2) and the twiddle w^{j2 l1}; pass 2 the outer
// length-256 transforms over l1.  X holds 512 KiB per radius: 2 x 512 KiB of
// HBM traffic per radius per step, the dominant memory stream.
//
// Grid step (inverse transforms of r_s^l c_l, all radii), two persistent,
// pipelined kernels:
//   k_grid2_pass1  CTA = (column block a of 16 columns l1, a set of radii).  One
//                  TMA load of the spectrum tile {16 l1 x 256 l2} (128-byte
//                  rows, 128B swizzle), kept for all its radii; per radius the
//                  tile times r_s^l = r_s^{l1} r_s^{256 l2}, 16 transforms of
//                  256 points, the twiddle (held in registers: it does not
//                  depend on the radius), and an asynchronous TMA store of
//                  X_s[j2][l1] (X is stored transposed so that pass 2 reads
//                  whole rows) from one of two buffers, so that the store of
//                  one radius overlaps the transforms of the next.
//   k_grid2_pass2  CTA = a strided set of (radius, block of 16 rows j2) items;
//                  a two-stage ring of TMA loads {256 l1 x 16 j2} keeps the
//                  next item's load in flight during the current item's 16
//                  transforms of 256 points, objective w_s^2 |F_s(j)|^2 and
//                  best two.  The last CTA selects the candidates.
// Forward transform of G (one per step, 16 CTAs): k_fwd2_pass1/2, one tile per
// CTA, ending with a TMA store of c_j.
//
// mbarrier waits are bounded: a load that does not arrive within the limit
// sets error bit 2 of the signal (AFD_ERR_TIMEOUT at the host) and stops it;
// the CTA waits (bounded) for its other copies before it leaves.
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
// grid passes: an FFT exchange buffer of 16 padded transforms, also used as
// pass 1's output tile (1 KiB multiple, for the 128B-swizzled TMA store)
constexpr int kScratchBytes = 35 * 1024;
static_assert(sizeof(float2) * 16 * S8::SMEM <= (size_t)kScratchBytes && kTileBytes <= kScratchBytes,
              "scratch holds the transforms and the tile");
constexpr size_t kP1Smem = 1024 + kTileBytes + 2 * (size_t)kScratchBytes;
// pass 2: the two ring slots only (each transform exchanges in its own row of
// the slot it read), so that three CTAs fit on an SM
constexpr size_t kP2Smem = 1024 + 2 * (size_t)kTileBytes;
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

// Asynchronous TMA store, committed as its own bulk group (thread 0 only).
__device__ __forceinline__ void tma_store_2d_async(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(map), "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// None of this thread's bulk stores still reading shared memory.
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// All of this thread's bulk stores complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Element (row y, column x) of a {16 x 256} tile with 128-byte rows under the
// 128B swizzle: the 16-byte chunk index is XOR-ed with (y mod 8).
__device__ __forceinline__ int swz16(int y, int x) { return y * 16 + ((((x >> 1) ^ (y & 7))) << 1) + (x & 1); }

__device__ __forceinline__ float2* align1024(unsigned char* p) {
  const unsigned a = smem_u32(p);
  return reinterpret_cast<float2*>(p + ((1024u - (a & 1023u)) & 1023u));
}

// Bounded wait of the whole CTA for phase `parity` of bar: thread 0 polls and
// the outcome is shared, so every thread takes the same branch; the others
// then observe the completed phase themselves (it is already complete).
__device__ bool cta_wait(uint64_t* bar, unsigned parity, int* s_flag) {
  if (threadIdx.x == 0) *s_flag = mbar_wait_bounded(bar, parity) ? 1 : 0;
  __syncthreads();
  const bool ok = *s_flag != 0;
  if (ok) mbar_wait_bounded(bar, parity);
  return ok;
}

// The tile's TMA load, with a bounded wait; false in every thread (after
// flagging the signal) when it did not arrive.
__device__ bool load_tile(float2* tile, const CUtensorMap* map, int x, int y, uint64_t* bar, SlotCtl* ctl) {
  __shared__ int s_flag;
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, kTileBytes);
    tma_load_2d(tile, map, x, y, bar);
  }
  if (cta_wait(bar, 0, &s_flag)) return true;
  if (threadIdx.x == 0) {
    atomicOr(&ctl->err, 4);
    ctl->done = 1;
    mbar_wait_bounded(bar, 0);  // give a late copy a last chance to land before the CTA exits
  }
  return false;
}



// A 256-point transform of one 16-thread group (half a warp) in registers,
// exchanging through x (256 float2) with an XOR swizzle instead of padding:
// element e = 16 a + b sits at 16 a + (b ^ a), so both exchange patterns are
// free of bank conflicts and the exchange needs no more room than the data.
// The arithmetic is that of fft_run<float, 8> (two radix-16 Stockham passes,
// stage twiddles tw from global memory), so the values are bitwise the same.
// In: v[q] = x_{t + 16 q}; out: v[k] = X_{t + 16 k}.  The whole warp calls it
// (it synchronises with __syncwarp); x may hold the inputs being read, once
// the warp is past its reads of them.
template <int DIR>
__device__ __forceinline__ void fft256_swz(float2* v, int t, float2* x, const float2* __restrict__ tw) {
  dft<16, DIR, float>(v);
#pragma unroll
  for (int k = 0; k < 16; ++k) x[16 * t + (k ^ t)] = v[k];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = x[16 * q + (t ^ q)];
#pragma unroll
  for (int q = 1; q < 16; ++q) {
    const float2 w = __ldg(&tw[(q - 1) * 16 + t]);
    v[q] = DIR > 0 ? cmul<float>(v[q], w) : cmulc<float>(v[q], w);
  }
  dft<16, DIR, float>(v);
}

}  // namespace

// Forward transform of G / N, pass 1: one tile of 16 columns per CTA.
__global__ void __launch_bounds__(kThreads)
k_fwd2_pass1(const SlotDev* __restrict__ slots, const __grid_constant__ Fft2Maps maps) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ alignas(8) uint64_t bar;
  pdl_launch_dependents();
  const SlotDev& sd = slots[0];
  float2* tile = align1024(smem_raw);
  float2* fbuf = tile + kTileElems;
  const int a = blockIdx.x;
  const int g = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int l1 = 16 * a + g;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  if (!load_tile(tile, &maps.g, 16 * a, 0, &bar, sd.ctl)) return;

  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = tile[swz16(t + 16 * q, g)];  // l2 = t + 16 q
  fft_run<float, L8, -1>(v, t, fbuf + g * S8::SMEM, sd.p.st32);
  __syncthreads();  // every warp has read its inputs from the tile
  // twiddle w^{-j2 l1} and the transposed tile X[j2][l1]
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int j2 = fft_out_index<float, L8>(t, e);
    const float2 w = __ldg(&sd.p.tw32n[j2 * l1]);
    tile[swz16(j2, g)] = cmulc<float>(v[e], w);
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) tma_store_2d(&maps.xs, 16 * a, 0, tile);
}

// Forward transform, pass 2: 16 rows j2 per CTA, c_j (j = j2 + 256 j1) stored
// through a {16 j2 x 256 j1} tile.
__global__ void __launch_bounds__(kThreads)
k_fwd2_pass2(const SlotDev* __restrict__ slots, const __grid_constant__ Fft2Maps maps) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ alignas(8) uint64_t bar;
  pdl_launch_dependents();
  const SlotDev& sd = slots[0];
  float2* tile = align1024(smem_raw);
  float2* fbuf = tile + kTileElems;
  const int b = blockIdx.x;
  const int g = threadIdx.x >> 4, t = threadIdx.x & 15;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  if (!load_tile(tile, &maps.xl, 0, 16 * b, &bar, sd.ctl)) return;

  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = tile[g * 256 + t + 16 * q];  // row j2, l1 = t + 16 q
  fft_run<float, L8, -1>(v, t, fbuf + g * S8::SMEM, sd.p.st32);
  __syncthreads();  // every warp has read its inputs from the tile
#pragma unroll
  for (int e = 0; e < 16; ++e) tile[swz16(fft_out_index<float, L8>(t, e), g)] = v[e];
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) tma_store_2d(&maps.c, 16 * b, 0, tile);
}

// Grid pass 1 (see the file comment).  gridDim.x = 16 R: CTA (a, r) takes
// column block a and radii r, r + R, ...
__global__ void __launch_bounds__(kThreads)
k_grid2_pass1(const SlotDev* __restrict__ slots, const __grid_constant__ Fft2Maps maps) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ alignas(8) uint64_t bar;
  pdl_launch_dependents();
  const SlotDev& sd = slots[0];
  float2* ctile = align1024(smem_raw);
  float2* obuf = ctile + kTileElems;
  const int R = gridDim.x / 16;
  const int a = blockIdx.x % 16, r0 = blockIdx.x / 16;
  const int g = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int l1 = 16 * a + g;
  // w^{j2 l1} for this thread's outputs j2 = t + 16 e, as w^{t l1} w^{16 e l1}
  // (the second from the 4096-entry table after w^k): the same for all radii
  float2 tw[16];
  {
    const float2 base = __ldg(&sd.p.tw32n[t * l1]);
    const float2* t4k = sd.p.tw32n + 65536;
#pragma unroll
    for (int e = 0; e < 16; ++e) tw[e] = cmul<float>(base, __ldg(&t4k[(e * l1) & 4095]));
  }
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  if (!load_tile(ctile, &maps.c, 16 * a, 0, &bar, sd.ctl)) return;
  const int M = sd.p.M;
  // r_s^l = lo[l1] hi[l2] of the next radius, fetched one radius ahead
  float lo_n = 0.f, h_n[16];
  auto fetch = [&](int s) {
    if (s >= M) return;
    lo_n = __ldg(&sd.p.rlo32[s * 256 + l1]);
#pragma unroll
    for (int q = 0; q < 16; ++q) h_n[q] = __ldg(&sd.p.rhi32[s * 256 + t + 16 * q]);
  };
  fetch(r0);
  int it = 0;
  for (int s = r0; s < M; s += R, ++it) {
    // (the store issued from this buffer two radii ago had read it before
    // the previous radius's last barrier)
    float2* ob = obuf + (it & 1) * (kScratchBytes / 8);
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float rp = lo_n * h_n[q];
      const float2 x = ctile[swz16(t + 16 * q, g)];  // l2 = t + 16 q
      v[q] = make_float2(x.x * rp, x.y * rp);
    }
    fetch(s + R);
    fft_run<float, L8, 1>(v, t, ob + g * S8::SMEM, sd.p.st32);
    __syncthreads();  // the tile below overlaps other transforms' exchange space
#pragma unroll
    for (int e = 0; e < 16; ++e) ob[swz16(fft_out_index<float, L8>(t, e), g)] = cmul<float>(v[e], tw[e]);
    fence_proxy_async();
    // the store issued from the other buffer one radius ago has read it (the
    // next radius transforms there), before the barrier that releases it
    if (threadIdx.x == 0) bulk_wait_read0();
    __syncthreads();
    if (threadIdx.x == 0) tma_store_2d_async(&maps.xs, 16 * a, s * 256, ob);
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// Grid pass 2 (see the file comment): items (s, b) = (i / 16, i mod 16), i =
// blockIdx.x, + gridDim.x, ...  The warps go through the items on their own,
// without CTA barriers: each warp waits for the item's slot itself, does its
// two rows, and the last warp of the CTA to finish an item merges the eight
// warps' best pairs and refills the slot with the item two ahead (a smem
// arrival counter per slot; the refill waits for every warp, since no warp
// can need the slot's next contents before all of them are done with it).
__global__ void __launch_bounds__(kThreads)
k_grid2_pass2(const SlotDev* __restrict__ slots, const __grid_constant__ Fft2Maps maps) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ alignas(8) uint64_t bars[2];
  __shared__ float rv1[2][kThreads / 32], rv2[2][kThreads / 32];
  __shared__ int rj1[2][kThreads / 32], rj2[2][kThreads / 32];
  __shared__ unsigned s_arrive[2], s_issued[2];
  __shared__ int s_last, s_fail;
  pdl_launch_dependents();
  const SlotDev& sd = slots[0];
  float2* in = align1024(smem_raw);
  const int g = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  static_assert(FftSchedule::npass(L8) == 2 && FftSchedule::tw_off(L8, 1) == 0, "fft256_swz: 16 x 16");
  if (threadIdx.x == 0) {
    mbar_init(&bars[0]);
    mbar_init(&bars[1]);
    s_arrive[0] = s_arrive[1] = 0u;
    s_issued[0] = s_issued[1] = 0u;
    s_fail = 0;
  }
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  const int items = 16 * sd.p.M;
  // the TMA load of this CTA's item number i into ring slot i mod 2 (one thread)
  auto issue = [&](int i) {
    const int item = (int)blockIdx.x + i * (int)gridDim.x;
    if (item >= items) return;
    ++s_issued[i & 1];
    mbar_expect_tx(&bars[i & 1], kTileBytes);
    tma_load_2d(in + (i & 1) * kTileElems, &maps.xl, 0, (item >> 4) * 256 + 16 * (item & 15), &bars[i & 1]);
  };
  if (threadIdx.x == 0) {
    issue(0);
    issue(1);
  }
  int i = 0;
  for (;; ++i) {
    const int item = (int)blockIdx.x + i * (int)gridDim.x;
    if (item >= items) break;
    const int s = item >> 4, b = item & 15;
    const int j2 = 16 * b + g;
    float2* tile = in + (i & 1) * kTileElems;
    // every lane polls the slot's barrier (bounded); a warp that gives up, or
    // sees that another did, leaves the loop
    if (*((volatile int*)&s_fail) || !mbar_wait_bounded(&bars[i & 1], (i >> 1) & 1)) {
      if (lane == 0) atomicOr(&s_fail, 1);
      break;
    }
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = tile[g * 256 + t + 16 * q];  // row j2, l1 = t + 16 q
    __syncwarp();  // the warp's two rows are read: they become its exchange space
    fft256_swz<1>(v, t, tile + g * 256, sd.p.st32);
    // the slot's generic writes before the TMA load that refills it
    fence_proxy_async();
    // best two of the warp's 512 grid points (j = j2 + 256 j1); a thread's
    // outputs come in increasing j1 = t + 16 e
    Best2F bb;
    bb.init();
#pragma unroll
    for (int e = 0; e < 16; ++e) bb.push_ascending(norm2<float>(v[e]), j2 + 256 * (t + 16 * e));
    warp_top2(bb);
    unsigned last = 0;
    __syncwarp();  // the warp's reads and writes of the slot come before its arrival
    if (lane == 0) {
      rv1[i & 1][warp] = bb.v1;
      rv2[i & 1][warp] = bb.v2;
      rj1[i & 1][warp] = bb.j1;
      rj2[i & 1][warp] = bb.j2;
      __threadfence_block();
      last = atomicAdd(&s_arrive[i & 1], 1u) == kThreads / 32 - 1;
      if (last) __threadfence_block();
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      // every warp is done with the slot and has posted its pair: read the
      // item's eight pairs (their buffer is rewritten for item i + 2, which
      // the refill lets other warps start), then refill the slot
      Best2F o;
      o.init();
      if (lane < kThreads / 32) {
        o.v1 = rv1[i & 1][lane];
        o.v2 = rv2[i & 1][lane];
        o.j1 = rj1[i & 1][lane];
        o.j2 = rj2[i & 1][lane];
      }
      __syncwarp();
      if (lane == 0) {
        s_arrive[i & 1] = 0u;
        issue(i + 2);
      }
      warp_top2(o);  // the eight pairs (the other lanes hold empty ones)
      if (lane == 0) {
        const float w2 = obj_w32(sd, s);
        Top2F r;
        r.v1 = o.v1 * w2;
        r.v2 = o.v2 * w2;
        r.j1 = o.j1;
        r.j2 = o.j2;
        reinterpret_cast<Top2F*>(sd.top2)[s * 16 + b] = r;
        if (r.v1 >= 0.0f && r.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(r.v1));
      }
    }
  }
  __syncthreads();
  if (s_fail) {
    // a load did not arrive: flag the signal and leave once the copies this
    // CTA started have landed (bounded)
    if (threadIdx.x == 0) {
      atomicOr(&sd.ctl->err, 4);
      sd.ctl->done = 1;
      // the last load issued into each slot completes that slot's phase
      // s_issued - 1
      for (int k = 0; k < 2; ++k)
        if (s_issued[k]) mbar_wait_bounded(&bars[k], (s_issued[k] - 1) & 1);
    }
    return;
  }
  __threadfence();  // the Top2F pairs and vmax before the last CTA reads them
  if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x, &s_last)) return;
  __shared__ SelectScratch scr;
  select_candidates_f32<kThreads>(sd, sd.ctl->k, 16, scr);
}

// Self-test of the mbarrier wait's bound (failure detection without a
// fault): the phase expects 16 bytes that no copy delivers (none is issued),
// so cta_wait polls kWaitLimit times and returns false; the kernel flags the
// timeout (error bit 2 of ctl->err) as the TMA-staged passes do.
__global__ void k_selftest_mbarrier(SlotCtl* ctl, unsigned long long* elapsed_ns) {
  __shared__ alignas(8) uint64_t bar;
  __shared__ int s_flag;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  const unsigned long long t0 = globaltimer_ns();
  if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
  const bool ok = cta_wait(&bar, 0, &s_flag);
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(&ctl->err, 4);
    *elapsed_ns = globaltimer_ns() - t0;
  }
}

cudaError_t launch_selftest_mbarrier(SlotCtl* ctl, unsigned long long* elapsed_ns, cudaStream_t st) {
  k_selftest_mbarrier<<<1, 32, 0, st>>>(ctl, elapsed_ns);
  return cudaGetLastError();
}

cudaError_t fft2_configure() {
  cudaError_t e;
  const auto smem = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const auto carve = cudaFuncAttributePreferredSharedMemoryCarveout;
  if ((e = cudaFuncSetAttribute(k_fwd2_pass1, smem, (int)kSmemBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd2_pass2, smem, (int)kSmemBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_grid2_pass1, smem, (int)kP1Smem))) return e;
  if ((e = cudaFuncSetAttribute(k_grid2_pass2, smem, (int)kP2Smem))) return e;
  // two CTAs of grid pass 1, three of pass 2 per SM
  if ((e = cudaFuncSetAttribute(k_grid2_pass1, carve, (int)cudaSharedmemCarveoutMaxShared))) return e;
  return cudaFuncSetAttribute(k_grid2_pass2, carve, (int)cudaSharedmemCarveoutMaxShared);
}

namespace {
template <typename K>
cudaError_t launch2(K kernel, dim3 grid, size_t smem, const SlotDev* slots, const Fft2Maps& maps,
                    cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, slots, maps);
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || n < 1)
      n = 1;
  }
  return n;
}
}  // namespace

cudaError_t launch_grid2(const SlotDev* slots, const Fft2Maps& maps, int M, cudaStream_t st) {
  // pass 1: two CTAs per SM, as 16 column blocks x R radius sets; pass 2:
  // three CTAs per SM
  const int ctas = 2 * sm_count();
  int R = ctas / 16;
  R = R < 1 ? 1 : (R > M ? M : R);
  cudaError_t e = launch2(k_grid2_pass1, dim3(16 * R), kP1Smem, slots, maps, st);
  if (e != cudaSuccess) return e;
  const int items = 16 * M, ctas2 = 3 * sm_count();
  return launch2(k_grid2_pass2, dim3(items < ctas2 ? items : ctas2), kP2Smem, slots, maps, st);
}

cudaError_t launch_forward2(const SlotDev* slots, const Fft2Maps& maps, cudaStream_t st) {
  cudaError_t e = launch2(k_fwd2_pass1, dim3(16), kSmemBytes, slots, maps, st);
  if (e != cudaSuccess) return e;
  return launch2(k_fwd2_pass2, dim3(16), kSmemBytes, slots, maps, st);
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
