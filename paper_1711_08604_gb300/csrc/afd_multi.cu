// Many signals of uneven N in one persistent launch (FP32 grid + FP64 guard
// and update), sm_103a.
//
// k_multi runs the greedy steps of Sec. 2 with the selection of Sec. 3.2 for
// every signal of a batch (or every active request of a serving tick) in one
// cooperative launch: per step, four phases separated by bounded grid
// barriers,
//   grid     every (signal, radius tile) work item of every N-class: inverse
//            transforms, objective, best pairs; the signal's last tile selects
//            the FP64 guard's candidates;
//   guard    every (signal, candidate set, 128-sample chunk) item: the FP64
//            rectangle-rule sums of Eq. (formula1); the last item picks a_k;
//   update   every (signal, chunk) item: the remainder update of Sec. 2 and
//            the energy; the last item writes delta_k and applies the stop rule;
//   forward  every signal: the DFT of Eq. (term4) of the new remainder,
// all with the bodies of afd_step.cuh and the same work split per signal as
// the step kernels, so each signal's results are bitwise those of the
// per-kernel sequence (and of a single-signal run).  A CTA of 512 threads
// takes one grid item, or sixteen guard or update items at once (one per
// warp: guard_warp, update_warp), or several signals' forward transforms (one
// per transform group); the N-classes share each phase, so no class waits for
// a launch of its own.  Fresh signals are initialised first (energy and FP32
// copy, then their transform).
#include <algorithm>
#include <climits>
#include <cstdint>

#include "../../include/afd.h"
#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_internal.h"
#include "afd_mixed.cuh"
#include "afd_step.cuh"

namespace afd {

namespace {

// Two builds of the kernel: MT = 256 threads per CTA (three CTAs per SM) for
// sizes up to 8192, MT = 512 (one per SM) when 16384 is among them.
// The transforms (grid and forward) use 32 points per thread from N = 32 up
// and N points below; the grid packs 256 / TPF or 512 / TPF transforms into
// a CTA.  All such variants compute bitwise the same values.
template <int MT, int L>
struct MGrid {
  static constexpr int PP = L >= 5 ? 32 : 0;
  static constexpr int CT = (MT == 512 && L == 14) ? 256 : MT;
  using C = GridCfg<float, L, PP, CT>;
  static_assert(C::THREADS == MT, "one grid item per CTA");
};
template <int MT>
__host__ __device__ constexpr int max_logn() { return MT == 512 ? 14 : 13; }

template <int MT, int L>
__device__ __forceinline__ void grid_item_l(const MultiArgs& a, const MultiClass& c, int sig, int tile) {
  if constexpr (L <= max_logn<MT>())
    grid_body<float, L, MGrid<MT, L>::PP, MGrid<MT, L>::CT>(a.slots, a.ids + c.first, tile, sig, c.tiles);
}

template <int MT, bool MIXED>
__device__ void grid_item(const MultiArgs& a, const MultiClass& c, int sig, int tile) {
  if (MIXED && c.logN < 0) {
    // a mixed-radix size: one radius per item, the selection's scratch in
    // the dynamic buffer once the transform is done
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (MIXED && MT == MX_THREADS)
      grid_mixed_body<float>(a.slots, a.ids + c.first, tile, sig, c.tiles, reinterpret_cast<SelectScratch*>(smem_raw));
    return;
  }
  switch (c.logN) {
#define X(L) \
  case L: grid_item_l<MT, L>(a, c, sig, tile); break;
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)
#undef X
    default: break;
  }
}

// Forward transforms of signals first .. first + GF - 1 of a class (ids):
// transform group g (TPF threads) takes signal first + g.  Groups without a
// signal, or whose signal has stopped, transform zeros and write nothing, so
// that every group passes the same warp or CTA barriers.  The arithmetic is
// that of k_forward on the FP32 copy.
template <int MT, int L>
__device__ __forceinline__ void forward_groups_l(const SlotDev* __restrict__ slots, const int* __restrict__ ids,
                                                 int first, int count) {
  constexpr int PP = MGrid<MT, L>::PP;
  using S = FftShape<float, L, PP>;
  constexpr int TPF = S::TPF, P = S::P, GF = TPF >= MT ? 1 : MT / TPF;
  static_assert(TPF <= MT, "one transform fits a CTA");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int sig = first + g;
  const SlotDev& s0 = slots[ids[first]];  // a valid descriptor of this size (its stage twiddles)
  const SlotDev* sd = sig < count ? &slots[ids[sig]] : nullptr;
  const bool active = g < GF && sd && !ld_done(sd->ctl);
  float2* buf = reinterpret_cast<float2*>(smem_raw) + (g < GF ? g : 0) * S::SMEM;
  if constexpr (PP == 32) {
    // the paired transforms: input pairs (j, j + 1) of the FP32 copy, output
    // pairs of the spectrum, the values of fft_run lane for lane
    constexpr int R0 = FftSchedule::radix(L, 0), NPR0 = P / (2 * R0);
    float2 X[P / 2], Y[P / 2];
    if constexpr (R0 == 2) {
      // pass 0 in registers (fftp_r2_pass0)
      float2 a[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) a[q] = active ? sd->g32[fftp_r2_in_index<L>(t, q)] : make_float2(0.f, 0.f);
      fftp_r2_pass0(a, X, Y);
    } else {
#pragma unroll
      for (int i = 0; i < NPR0; ++i) {
#pragma unroll
        for (int q = 0; q < R0; ++q) {
          const float4 x = active ? reinterpret_cast<const float4*>(sd->g32)[fftp_in_index<L>(t, i, 0, q) >> 1]
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
          X[i * R0 + q] = make_float2(x.x, x.z);
          Y[i * R0 + q] = make_float2(x.y, x.w);
        }
      }
    }
    if (g < GF) fftp_run<L, -1, (R0 == 2 ? 1 : 0), (GF > 1 && TPF > 32)>(X, Y, t, reinterpret_cast<float*>(buf), s0.p.st32p);
    if (active) {
#pragma unroll
      for (int q = 0; q < 16; ++q)
        reinterpret_cast<float4*>(sd->c32)[fftp_out_index<L>(t, 0, q) >> 1] =
            make_float4(X[q].x, Y[q].x, X[q].y, Y[q].y);
    }
  } else {
    float2 v[P];
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = active ? sd->g32[fft_in_index<float, L, PP>(t, e)] : make_float2(0.f, 0.f);
    if (g < GF) fft_run<float, L, -1, 0, false, PP, (GF > 1 && TPF > 32)>(v, t, buf, s0.p.st32);
    if (active) {
#pragma unroll
      for (int e = 0; e < P; ++e) sd->c32[fft_out_index<float, L, PP>(t, e)] = v[e];
    }
  }
}

template <int MT>
__device__ void forward_groups(const MultiArgs& a, const MultiClass& c, const int* ids, int first) {
  switch (c.logN) {
#define X(L) \
  case L: if constexpr (L <= max_logn<MT>()) forward_groups_l<MT, L>(a.slots, ids + c.first, first, c.count); break;
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)
#undef X
    default: break;
  }
}

// Class of work item `item` in a phase whose class c has count_c * per(c)
// items: returns the class and leaves the item's index within it in *local.
template <class Per>
__device__ __forceinline__ int find_class(const MultiClass* cls, int n, int item, Per per, int* local) {
  int base = 0;
  for (int c = 0; c < n; ++c) {
    const int span = cls[c].count * per(cls[c]);
    if (item < base + span) {
      *local = item - base;
      return c;
    }
    base += span;
  }
  return -1;
}

template <class Per>
__device__ __forceinline__ int total_items(const MultiClass* cls, int n, Per per) {
  int t = 0;
  for (int c = 0; c < n; ++c) t += cls[c].count * per(cls[c]);
  return t;
}

__device__ __forceinline__ int chunks_c(const MultiClass& c) { return chunks_of(c.N); }
// forward items of a class: groups of fgroups signals, or S items per signal
// of a mixed-radix size (mx_split)
__host__ __device__ __forceinline__ int fwd_items(const MultiClass& c) {
  return c.logN < 0 ? c.count * mx_split(c.N) : (c.count + c.fgroups - 1) / c.fgroups;
}

// MIXED: the build that also takes mixed-radix classes (their item bodies
// are compiled in only there, so the power-of-two build keeps its registers).
template <int MT, bool MIXED = false>
__global__ void __launch_bounds__(MT, MT == 256 ? 3 : 1) k_multi(const __grid_constant__ MultiArgs a) {
  constexpr int NW = MT / 32;
  // the FP64 items' candidate sums share the dynamic buffer with the transforms
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Fp64WarpSmem* smw = reinterpret_cast<Fp64WarpSmem*>(smem_raw);
  __shared__ int s_ok, s_item;
  const int warp = threadIdx.x >> 5;
  int* err = reinterpret_cast<int*>(a.bar + 32);  // its own 128-byte line after the counter
  unsigned* ticket = a.bar + 64;                  // and the work-item ticket on the next
  unsigned epoch = 0;
  // Work items go out by ticket, not by a fixed stride: SMs run the same item
  // at different speeds (a 1.4x spread measured across one launch), so a
  // fixed share would leave the phase waiting for the slowest.  Every CTA
  // takes one ticket past a phase's last item, so each phase's tickets start
  // at base (the same in every CTA) and the next at base + items + gridDim.x.
  unsigned base = 0;
  auto each_item = [&](int items, auto&& body) {
    unsigned next = 0;
    if (threadIdx.x == 0) next = atomicAdd(ticket, 1u);
    for (;;) {
      if (threadIdx.x == 0) s_item = (int)(next - base);
      __syncthreads();
      const int item = s_item;
      if (item >= items) break;
      if (threadIdx.x == 0) next = atomicAdd(ticket, 1u);  // in flight while the item runs
      body(item);
      __syncthreads();  // s_item and the exchange buffers are reused
    }
    base += (unsigned)items + gridDim.x;
  };
  // a phase's end: the grid barrier; on a timeout every signal is flagged and
  // the kernel leaves
  auto barrier = [&]() -> bool {
    if (grid_barrier_at(a.bar, err, gridDim.x * ++epoch, &s_ok)) return true;
    for (int c = 0; c < a.n_cls; ++c)
      for (int i = threadIdx.x; i < a.cls[c].count; i += MT) atomicOr(&a.slots[a.ids[a.cls[c].first + i]].ctl->err, 4);
    return false;
  };
  // FP64 items (guard, update, initialisation), one per warp
  auto fp64_phase = [&](int kind, const MultiClass* cls, int n, const int* ids) {
    auto per = [&](const MultiClass& c) { return kind == 0 ? c.gpar * chunks_c(c) : chunks_c(c); };
    const int total = total_items(cls, n, per);
    each_item((total + NW - 1) / NW, [&](int cta_item) {
      const int item = cta_item * NW + warp;
      int local = 0;
      const int c = item < total ? find_class(cls, n, item, per, &local) : -1;
      if (c < 0) return;
      const int pc = per(cls[c]);
      const int* cid = ids + cls[c].first;
      if (kind == 0) guard_warp(a.slots, cid, local % pc, local / pc, pc, smw[warp]);
      else if (kind == 1) update_warp<false>(a.slots, cid, local % pc, local / pc, pc);
      else update_warp<true>(a.slots, cid, local % pc, local / pc, pc);
    });
  };
  // forward transforms, a CTA's groups taking consecutive signals of a class
  // (a mixed-radix size: one item, or one of S split items, per signal)
  auto forward_phase = [&](const MultiClass* cls, int n, const int* ids) {
    int total = 0;
    for (int c = 0; c < n; ++c) total += fwd_items(cls[c]);
    each_item(total, [&](int item) {
      int first = 0, c = 0;
      for (; c < n; ++c) {
        const int span = fwd_items(cls[c]);
        if (item < first + span) break;
        first += span;
      }
      if (c >= n) return;
      const int local = item - first;
      if (MIXED && cls[c].logN < 0) {
        if constexpr (MIXED && MT == MX_THREADS) {
          const int S = mx_split(cls[c].N);
          if (S > 1) forward_mixed_split_body<float>(a.slots, ids + cls[c].first, local % S, local / S, S);
          else forward_mixed_body<float>(a.slots, ids + cls[c].first, local);
        }
        return;
      }
      forward_groups<MT>(a, cls[c], ids, local * cls[c].fgroups);
    });
  };
  if (a.n_fresh > 0) {
    fp64_phase(2, a.fresh, a.n_fresh, a.fresh_ids);
    if (!barrier()) return;
    forward_phase(a.fresh, a.n_fresh, a.fresh_ids);
    if (!barrier()) return;
  }
  for (int k = 0; k < a.K; ++k) {
    {
      auto per = [](const MultiClass& c) { return c.tiles; };
      each_item(total_items(a.cls, a.n_cls, per), [&](int item) {
        int local = 0;
        const int c = find_class(a.cls, a.n_cls, item, per, &local);
        if (c >= 0) grid_item<MT, MIXED>(a, a.cls[c], local / a.cls[c].tiles, local % a.cls[c].tiles);
      });
    }
    if (!barrier()) return;
    fp64_phase(0, a.cls, a.n_cls, a.ids);
    if (!barrier()) return;
    fp64_phase(1, a.cls, a.n_cls, a.ids);
    if (k + 1 < a.K || a.final_forward) {
      if (!barrier()) return;
      forward_phase(a.cls, a.n_cls, a.ids);
    }
    if (k + 1 < a.K && !barrier()) return;
  }
}

template <int MT, int L>
constexpr int fwd_groups_l() {
  using S = FftShape<float, L, MGrid<MT, L>::PP>;
  return S::TPF >= MT ? 1 : MT / S::TPF;
}
template <int MT, int L>
constexpr size_t smem_l() {
  using SG = FftShape<float, L, MGrid<MT, L>::PP>;
  const size_t g = sizeof(float2) * (size_t)SG::SMEM * MGrid<MT, L>::C::FPC;
  const size_t f = sizeof(float2) * (size_t)SG::SMEM * fwd_groups_l<MT, L>();
  return g > f ? g : f;
}

template <int MT>
size_t smem_bytes(int logN) {
  switch (logN) {
#define X(L) \
  case L: if constexpr (L <= max_logn<MT>()) return smem_l<MT, L>(); else return 0;
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)
#undef X
    default: return 0;
  }
}

template <int MT>
size_t max_smem() {
  size_t mx = 0;
  for (int l = 3; l <= max_logn<MT>(); ++l) mx = smem_bytes<MT>(l) > mx ? smem_bytes<MT>(l) : mx;
  return mx;
}

int g_multi_blocks[2] = {0, 0};  // co-resident CTAs of each build (0: not yet known)

// The work split of a class in build MT: grid tiles and forward groups.
template <int MT>
void shape_mt(int logN, int Mmax, int count, int cap, MultiClass* c) {
  int fpc = 1, fg = 1;
  switch (logN) {
#define X(L)                                  \
  case L:                                     \
    if constexpr (L <= max_logn<MT>()) {      \
      fpc = MGrid<MT, L>::C::FPC;             \
      fg = fwd_groups_l<MT, L>();             \
    }                                         \
    break;
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)
#undef X
    default: break;
  }
  c->logN = logN;
  c->N = 1 << logN;
  c->count = count;
  c->Mmax = Mmax;
  c->tiles = (Mmax + fpc - 1) / fpc;
  // candidates in flight per signal, as launch_guard chooses them
  c->gpar = count >= 8 ? 1 : (cap < GUARD_PAR ? cap : GUARD_PAR);
  c->fgroups = fg;
}

// Dynamic shared memory of a class's items: the transforms' buffers, and for
// a mixed-radix size also the selection's scratch, which the grid item puts
// there.
template <int MT>
size_t class_smem(const MultiClass& c) {
  if (c.logN >= 0) return smem_bytes<MT>(c.logN);
  return std::max({mixed_launch_smem(c.N, AFD_FP32_GUARDED), mixed_split_smem(c.N, AFD_FP32_GUARDED),
                   sizeof(SelectScratch)});
}

template <int MT>
cudaError_t launch_mt(const MultiArgs& a, cudaStream_t st) {
  size_t smem = sizeof(Fp64WarpSmem) * (MT / 32);
  for (int c = 0; c < a.n_cls; ++c) smem = std::max(smem, class_smem<MT>(a.cls[c]));
  for (int c = 0; c < a.n_fresh; ++c) smem = std::max(smem, class_smem<MT>(a.fresh[c]));
  bool mixed = false;
  for (int c = 0; c < a.n_cls; ++c) mixed = mixed || a.cls[c].logN < 0;
  // the build with the mixed-radix bodies only when a class needs them
  void (*kern)(MultiArgs) = (MT == 256 && mixed) ? k_multi<256, true> : k_multi<MT>;
  int& blocks = g_multi_blocks[MT == 512 ? 1 : 0];
  int blocks_big = 0;  // co-resident CTAs at a footprint above max_smem, or of the mixed build
  if (smem > max_smem<MT>() || kern != k_multi<MT>) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    blocks_big = per_sm * sms;
  } else if (!blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi<MT>, MT, max_smem<MT>());
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    blocks = per_sm * sms;
  }
  // No more CTAs than the largest phase has items (a small serving tick
  // then pays for fewer arrivals at each grid barrier), at most the
  // co-resident maximum.
  constexpr int NW = MT / 32;
  long long need = 1;
  auto most = [&](const MultiClass* cls, int n) {
    long long g = 0, gu = 0, up = 0, fw = 0;
    for (int c = 0; c < n; ++c) {
      const MultiClass& x = cls[c];
      const long long ch = chunks_of(x.N);
      g += (long long)x.count * x.tiles;
      gu += ((long long)x.count * x.gpar * ch + NW - 1) / NW;
      up += ((long long)x.count * ch + NW - 1) / NW;
      fw += fwd_items(x);
    }
    need = std::max({need, g, gu, up, fw});
  };
  most(a.cls, a.n_cls);
  most(a.fresh, a.n_fresh);
  const int grid = (int)std::min<long long>(blocks_big ? blocks_big : blocks, need);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(MT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

bool multi_size_ok(int logN) { return logN >= 3 && logN <= 14; }

void multi_class_shape_mixed(int N, int Mmax, int count, int cap, MultiClass* c) {
  c->logN = -1;
  c->N = N;
  c->count = count;
  c->Mmax = Mmax;
  c->tiles = Mmax;  // one radius per grid item, as k_grid_mixed
  c->gpar = count >= 8 ? 1 : (cap < GUARD_PAR ? cap : GUARD_PAR);
  c->fgroups = 1;
}

void multi_class_shape(int logN, int Mmax, int count, int cap, MultiClass* c) {
  // the split of the 256-thread build; launch_multi takes the 512-thread
  // build (and redoes the split) when a class of N = 16384 is present
  if (logN <= 13) shape_mt<256>(logN, Mmax, count, cap, c);
  else shape_mt<512>(logN, Mmax, count, cap, c);
}

cudaError_t multi_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_multi<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem<256>());
  if (e != cudaSuccess) return e;
  // the 256-thread build with mixed-radix sizes, up to MIXED_MAX_SMEM
  e = cudaFuncSetAttribute(k_multi<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)std::max(max_smem<256>(), (size_t)MIXED_MAX_SMEM));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_multi<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem<512>());
}

cudaError_t launch_multi(const MultiArgs& a, cudaStream_t st) {
  bool big = false;
  for (int c = 0; c < a.n_cls; ++c) big = big || a.cls[c].logN > 13;
  for (int c = 0; c < a.n_fresh; ++c) big = big || a.fresh[c].logN > 13;
  if (!big) return launch_mt<256>(a, st);
  // the 512-thread build packs twice as many transforms into a CTA
  MultiArgs b = a;
  // (gpar <= GUARD_PAR already holds the guard's choice: shape keeps it)
  for (int c = 0; c < b.n_cls; ++c) {
    MultiClass& x = b.cls[c];
    const int first = x.first;
    shape_mt<512>(x.logN, x.Mmax, x.count, x.gpar, &x);
    x.first = first;
  }
  for (int c = 0; c < b.n_fresh; ++c) {
    MultiClass& x = b.fresh[c];
    const int first = x.first;
    shape_mt<512>(x.logN, x.Mmax, x.count, x.gpar, &x);
    x.first = first;
  }
  return launch_mt<512>(b, st);
}

}  // namespace afd
