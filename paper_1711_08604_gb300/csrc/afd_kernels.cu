// CUDA kernels of one Core AFD greedy step (arXiv:1711.08604), sm_103a.
//
// Per step and signal the device runs, in stream order:
//   k_grid   one transform per radius s: f(l) = r_s^l c_l / N (Step 1 of the
//            algorithm of Sec. 3.2), inverse FFT F_s(j) = sum_l f(l) w^{jl}
//            (Eq. (rcl), Theorem 2.1), objective w_s^2 |F_s(j)|^2 with
//            w_s = sqrt(1-r_s^2)/(1-r_s^N), and the per-radius best two
//            (value, j).  The M x N grid never leaves registers.  The last CTA
//            of a signal performs the selection of Step 2: the FP64 path takes
//            the global maximum directly; the FP32 path lists every grid point
//            whose FP32 objective is within a relative window tau of the
//            largest one for re-evaluation in FP64.
//   k_guard  (FP32 path) each candidate's <G_k, e_a>~ by the direct FP64
//            rectangle rule of Eq. (formula1), split over CTAs; the last CTA
//            picks the largest (ties: lowest flat index s N + j).
//   k_update the reduced-remainder update of Sec. 2 in FP64,
//            G_{k+1}(z) = (G_k(z)(1 - conj(a) z) - c sqrt(1-|a|^2)) / (z - a),
//            plus the discrete energy; the last CTA writes delta_k = E_{k+1}/E_1
//            (Eq. (er)) and applies the stop rule.
//   k_forward the DFT c_l = sum_m G(z_m) w^{-ml} of Eq. (term4), scaled by 1/N,
//            for the next step.
// Every kernel returns at once for a signal whose stop flag is set, so a
// fixed launch sequence (or a captured CUDA graph) can run any number of steps.
#include <climits>
#include <cstdint>
#include <type_traits>

#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_fft2.h"
#include "afd_internal.h"
#include "afd_step.cuh"

namespace afd {

// ------------------------------------------------------------ step kernels --
// One CTA per work item: the bodies of afd_step.cuh.

template <typename T, int LOGN, int PP = 0, int CT = 256>
__global__ void __launch_bounds__(GridCfg<T, LOGN, PP, CT>::THREADS, GridCfg<T, LOGN, PP, CT>::MIN_CTAS)
k_grid(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  grid_body<T, LOGN, PP, CT>(slots, ids, blockIdx.x, blockIdx.y, gridDim.x);
}

__global__ void __launch_bounds__(FP64_THREADS)
k_guard(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  __shared__ Fp64Smem sm;
  pdl_launch_dependents();
  pdl_wait();
  guard_body(slots, ids, blockIdx.x, blockIdx.y, gridDim.x, cta_set(), sm);
}

template <bool INIT>
__global__ void __launch_bounds__(FP64_THREADS)
k_update(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  __shared__ Fp64Smem sm;
  pdl_launch_dependents();
  pdl_wait();
  update_body<INIT>(slots, ids, blockIdx.x, blockIdx.y, gridDim.x, cta_set(), sm);
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(FftShape<T, LOGN>::TPF)
k_forward(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_launch_dependents();
  pdl_wait();
  forward_body<T, LOGN>(slots, ids, blockIdx.x, threadIdx.x, reinterpret_cast<V2<T>*>(smem_raw));
}

// -------------------------------------------- split sizes (long transforms) --
//
// A transform longer than one CTA holds on chip (split_log(logN, prec) =
// LS > 0: FP32 N = 32768, FP64 N = 16384 .. 65536) is split by output index
// into S = 2^LS resident sub-transforms of NS = N / S points.  For the
// inverse transforms of the grid, CTA (s, h) computes F_s(S j' + h), j' < NS,
// from the pre-combined input
//   f_h(l') = w^{h l'} sum_{p < S} f(l' + p NS) exp(2 pi i h p / S),
//   f(l) = r_s^l c_l / N,
// (one radix-S decimation-in-frequency step: Theorem 2.1's even/odd splitting
// with radix S).  r_s^(l' + p NS) = lo[b] hi[q + p R0] for l' = b + q B, with
// the tables split at B = NS / R0.  The forward transform is split the same
// way with conjugate twiddles: S CTAs per signal, CTA h writing c_{S k' + h}.

// exp(+2 pi i h p / S) for p < S, from the N-point twiddle table
template <typename T, int LS>
__device__ __forceinline__ void split_roots(V2<T>* wp, const V2<T>* __restrict__ twn, int h, int NS) {
  constexpr int SPL = 1 << LS;
#pragma unroll
  for (int p = 0; p < SPL; ++p) wp[p] = __ldg(&twn[((h * p) & (SPL - 1)) * NS]);
}

template <typename T, int LOGS, int LS>
__global__ void __launch_bounds__(FftShape<T, LOGS>::TPF)
k_grid_split(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  using S = FftShape<T, LOGS>;
  constexpr int P = S::P, TPF = S::TPF, SPL = 1 << LS, NS = S::N;
  constexpr int R0 = S::radix(0), B = FftSchedule::pow_b(LOGS), NB0 = P / R0;
  static_assert(TPF >= 256 && B * R0 == NS, "one resident sub-transform per CTA");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[blockIdx.y]];
  const int t = threadIdx.x;
  const int s = (int)(blockIdx.x >> LS), h = (int)(blockIdx.x & (SPL - 1));
  const bool active = s < sd.p.M;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw);
  const V2<T>* tw;
  const V2<T>* twn;
  const T* lo;
  const T* hi;
  const V2<T>* c;
  if constexpr (sizeof(T) == 4) {
    tw = sd.p.st32; twn = sd.p.tw32n; lo = sd.p.rlo32; hi = sd.p.rhi32; c = sd.c32;
  } else {
    tw = sd.p.st64; twn = sd.p.tw64; lo = sd.p.rlo64; hi = sd.p.rhi64; c = sd.c64;
  }
  V2<T> v[P];
  if (active) {
    // constant tables first, then wait for the spectrum
    T hq[R0 * SPL], lb[NB0];
    V2<T> wp[SPL];
#pragma unroll
    for (int e = 0; e < R0 * SPL; ++e) hq[e] = __ldg(&hi[(size_t)s * (R0 * SPL) + e]);
#pragma unroll
    for (int i = 0; i < NB0; ++i) lb[i] = __ldg(&lo[(size_t)s * B + t + i * TPF]);
    split_roots<T, LS>(wp, twn, h, NS);
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
      const int b = t + i * TPF;
#pragma unroll
      for (int q = 0; q < R0; ++q) {
        const int l = b + q * B;  // l' < NS
        V2<T> acc = mk2<T>((T)0, (T)0);
#pragma unroll
        for (int p = 0; p < SPL; ++p) {
          const T rp = lb[i] * hq[q + p * R0];
          const V2<T> x = c[l + p * NS];
          acc = cadd<T>(acc, cmul<T>(mk2<T>(x.x * rp, x.y * rp), wp[p]));
        }
        v[i * R0 + q] = cmul<T>(acc, __ldg(&twn[h * l]));
      }
    }
  } else {
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = mk2<T>((T)0, (T)0);
  }
  fft_run<T, LOGS, +1>(v, t, buf, tw);
  // objective and the best of this sub-transform's outputs j = S j' + h
  if constexpr (sizeof(T) == 4) {
    __shared__ Best2F red[32];
    Best2F bb;
    bb.init();
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const V2<T> x = v[fft_out_slot<T, LOGS>(u)];
      bb.push_ascending(norm2<T>(x), SPL * (t + TPF * u) + h);
    }
    group_reduce<TPF>(bb, red);
    if (t == 0 && active) {
      const float w2 = obj_w32(sd, s);
      Top2F o;
      o.v1 = bb.v1 * w2;
      o.v2 = bb.v2 * w2;
      o.j1 = bb.j1;
      o.j2 = bb.j2;
      reinterpret_cast<Top2F*>(sd.top2)[s * SPL + h] = o;
      if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(o.v1));
      __threadfence();  // read by the signal's last CTA
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x, &s_last)) return;
    __shared__ SelectScratch scr;
    select_candidates_f32<TPF>(sd, sd.ctl->k, SPL, scr);
  } else {
    __shared__ Best1D red[32];
    Best1D bb;
    bb.init();
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const V2<T> x = v[fft_out_slot<T, LOGS>(u)];
      bb.push_ascending(norm2<T>(x), SPL * (t + TPF * u) + h, x);
    }
    group_reduce<TPF>(bb, red);
    if (t == 0 && active) {
      const double w = sd.p.w64[s];
      Top2D o;
      o.v1 = bb.v * (w * w) * obj_rho64(sd, s);
      o.j1 = bb.j;
      o.f1 = bb.f;
      o.v2 = -1.0;
      o.j2 = INT_MAX;
      o.f2 = make_double2(0.0, 0.0);
      reinterpret_cast<Top2D*>(sd.top2)[s * SPL + h] = o;
      __threadfence();  // read by the signal's last CTA
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x, &s_last)) return;
    __syncthreads();
    select_best_f64<TPF>(sd, sd.ctl->k, red, SPL);
  }
}

// c_l / N of a split size: CTA h of a signal computes c_{S k' + h}, k' < NS,
// from y_h(m') = w^{-h m'} sum_{p < S} G(z_{m' + p NS}) exp(-2 pi i h p / S) / N.
template <typename T, int LOGS, int LS>
__global__ void __launch_bounds__(FftShape<T, LOGS>::TPF)
k_forward_split(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  using S = FftShape<T, LOGS>;
  constexpr int P = S::P, SPL = 1 << LS, NS = S::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[blockIdx.y]];
  const int t = threadIdx.x, h = (int)blockIdx.x;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw);
  const V2<T>* tw;
  const V2<T>* twn;
  V2<T>* c;
  if constexpr (sizeof(T) == 4) {
    tw = sd.p.st32; twn = sd.p.tw32n; c = sd.c32;
  } else {
    tw = sd.p.st64; twn = sd.p.tw64; c = sd.c64;
  }
  V2<T> wp[SPL];
  split_roots<T, LS>(wp, twn, h, NS);
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  V2<T> v[P];
#pragma unroll
  for (int e = 0; e < P; ++e) {
    const int m = fft_in_index<T, LOGS>(t, e);
    V2<T> acc = mk2<T>((T)0, (T)0);
#pragma unroll
    for (int p = 0; p < SPL; ++p) {
      V2<T> g;
      if constexpr (sizeof(T) == 4) {
        g = sd.g32[m + p * NS];
      } else {
        const double2 x = sd.G[m + p * NS];
        g = mk2<T>(x.x * sd.p.inv_n, x.y * sd.p.inv_n);
      }
      acc = cadd<T>(acc, cmulc<T>(g, wp[p]));
    }
    v[e] = cmulc<T>(acc, __ldg(&twn[h * m]));
  }
  fft_run<T, LOGS, -1>(v, t, buf, tw);
#pragma unroll
  for (int e = 0; e < P; ++e) c[SPL * fft_out_index<T, LOGS>(t, e) + h] = v[e];
}

// ------------------------------------------------------- output gather --

// The step records of signal i = blockIdx.x into the caller's device arrays
// (the layout of afd_batch_run: a, coeff and idx at 2 (i K_stride + k), delta
// at i (K_stride + 1) + k); any pointer may be NULL.  steps_out[i] and (signal
// 0) E1_out take the control block's step count and E_1.  The values are the
// records' own, so they equal what the host-side gather writes.
__global__ void __launch_bounds__(128)
k_gather(const StepRec* __restrict__ rec, const SlotCtl* __restrict__ ctl, int K_max, int K_stride,
         double* a, double* coeff, double* delta, int* idx, int* steps_out, double* E1_out) {
  const int i = (int)blockIdx.x;
  const SlotCtl c = ctl[i];
  const int steps = c.k < K_max ? c.k : K_max;
  const StepRec* r = rec + (size_t)i * K_max;
  const size_t b2 = 2 * (size_t)i * K_stride, bd = (size_t)i * (K_stride + 1);
  if (threadIdx.x == 0) {
    // delta_0: 1 for a fresh start, E(start) / E_1 for a resumed one
    if (delta) delta[bd] = (c.E1 > 0.0 && c.Estart != c.E1) ? c.Estart / c.E1 : 1.0;
    if (steps_out) steps_out[i] = steps;
    if (E1_out && i == 0) *E1_out = c.E1;
  }
  for (int k = threadIdx.x; k < steps; k += blockDim.x) {
    const StepRec& q = r[k];
    if (a) {
      a[b2 + 2 * k] = q.a_re;
      a[b2 + 2 * k + 1] = q.a_im;
    }
    if (coeff) {
      coeff[b2 + 2 * k] = q.c_re;
      coeff[b2 + 2 * k + 1] = q.c_im;
    }
    if (delta) delta[bd + k + 1] = q.delta;
    if (idx) {
      idx[b2 + 2 * k] = q.s;
      idx[b2 + 2 * k + 1] = q.j;
    }
  }
}

cudaError_t launch_gather(const StepRec* rec, const SlotCtl* ctl, int n, int K_max, int K_stride, double* a,
                          double* coeff, double* delta, int* idx, int* steps_out, double* E1_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<n, 128, 0, st>>>(rec, ctl, K_max, K_stride, a, coeff, delta, idx, steps_out, E1_out);
  return cudaGetLastError();
}

// -------------------------------------------------------- plan K table --

// K[s N + d] = 1 / (1 - r_s w^d), w = exp(2 pi i / N), written as
// (p + i q) / (p^2 + q^2) with p = 1 - r cos = (1 - r) + 2 r sin^2(pi d / N)
// (no cancellation as r -> 1 and d -> 0) and q = r sin(2 pi d / N).
__global__ void __launch_bounds__(256)
k_kernel_table(const double* __restrict__ radii, int N, double2* __restrict__ K) {
  const int d = blockIdx.x * 256 + threadIdx.x;
  const int s = blockIdx.y;
  if (d >= N) return;
  const double r = radii[s];
  double sn, cs;
  sincospi(2.0 * (double)d / (double)N, &sn, &cs);
  const double sh = sinpi((double)d / (double)N);
  const double pr = (1.0 - r) + 2.0 * r * sh * sh;
  const double qi = r * sn;
  const double inv = 1.0 / fma(pr, pr, qi * qi);
  K[(size_t)s * N + d] = make_double2(pr * inv, qi * inv);
}

// ------------------------------------------------------ persistent kernel --

// The grid barrier of the persistent kernel: grid_barrier_at (afd_device.cuh)
// on the slot's counter, with its error word.
__device__ __forceinline__ bool grid_barrier(const SlotDev& sd, unsigned target, int* s_ok) {
  return grid_barrier_at(sd.bar, &sd.ctl->err, target, s_ok);
}

// Self-test of the grid barrier's bound (failure detection without a fault):
// one CTA waits for an arrival count that nothing supplies (2, with only its
// own arrival), so grid_barrier polls kBarrierLimit times, flags the timeout
// (error bit 2 of ctl->err) and returns false.
__global__ void k_selftest_barrier(const SlotDev* __restrict__ slot, unsigned long long* elapsed_ns) {
  __shared__ int s_ok;
  const unsigned long long t0 = globaltimer_ns();
  grid_barrier(slot[0], 2u, &s_ok);
  if (threadIdx.x == 0) *elapsed_ns = globaltimer_ns() - t0;
}

cudaError_t launch_selftest_barrier(const SlotDev* slot, unsigned long long* elapsed_ns, cudaStream_t st) {
  k_selftest_barrier<<<1, 32, 0, st>>>(slot, elapsed_ns);
  return cudaGetLastError();
}

// All greedy steps of one FP32-path signal in one launch, one CTA of two or
// more transform groups per SM.  Per step:
//   A  each CTA: the FP32 input G_k / N formed from step k-1's FP32 copy and
//      winner, the forward FFT once (group 0), then each group's radius:
//      inverse FFT, objective and best pairs (as k_grid)     -- barrier --
//   B  each CTA: the candidate list (the same in every CTA), then warp-sized
//      FP64 items (one candidate, 32 samples, one component) of the guard's
//      sums, the update terms, the previous step's energy partials -- barrier --
//   C  each CTA: the winner from the partial sums (the same in every CTA),
//      warp-sized items of the remainder update; no barrier before the next
//      step's phase A, which needs only step k's FP32 copy and winner.
// With an energy tolerance, step k-1's energy, delta and stop rule come after
// step k's first barrier (the same in every CTA).  FP64 throughput per SM
// sub-partition is low, so the FP64 work goes out in 32-sample items over
// all CTAs and sub-partitions.  Each item keeps its warp's shuffle-tree sum,
// and the consumers add the four warp sums of a 128-sample chunk in warp
// order, then the chunks, as the separate kernels do: results are bitwise
// those of the multi-kernel sequence.
constexpr int PERSIST_CTA = 512;  // threads per CTA of the persistent kernel (one CTA per SM)

template <int LOGN>
__global__ void __launch_bounds__(GridCfg<float, LOGN, 0, PERSIST_CTA>::THREADS, 1)
k_persistent(const SlotDev* __restrict__ slots) {
  using S = FftShape<float, LOGN>;
  using C = GridCfg<float, LOGN, 0, PERSIST_CTA>;
  static_assert(C::FPC >= 2, "transform groups share one forward transform");
  constexpr int N = S::N, P = S::P, TPF = S::TPF, FPC = C::FPC, THREADS = C::THREADS;
  constexpr int R0 = S::radix(0), B = FftSchedule::pow_b(LOGN), NB0 = P / R0;
  constexpr int TWS = FftSchedule::tw_size(LOGN) > 0 ? FftSchedule::tw_size(LOGN) : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 s_tw[TWS];  // stage twiddles for the kernel's lifetime
  __shared__ Best2F red2[32];
  __shared__ int2 s_cand[MAX_CAP];
  __shared__ SelectScratch s_scr;
  __shared__ double s_re[MAX_CAP], s_im[MAX_CAP], s_v[MAX_CAP];
  __shared__ double s_rad[MAX_CAP], s_sq[MAX_CAP];  // radius and sqrt(1 - r^2) of each candidate
  __shared__ double s_scn[MAX_CAP], s_rho[MAX_CAP];  // sqrt(1 - r^2) / N and the objective's factor
  __shared__ float s_scn32[MAX_CAP];                  // sqrt(1 - r^2) / N in FP32
  __shared__ double s_cr[MAX_CAP], s_ci[MAX_CAP];    // c' = c sqrt(1 - r^2) of each candidate
  __shared__ float2 s_rot1[P], s_rot2[P];  // e^(i pi o_e / N), e^(2 pi i o_e / N); o_e: offset of point e
  __shared__ int s_ok, s_pc, s_ps, s_pj;
  __shared__ double s_E;
  __shared__ float s_f32[5];  // the winner's c'/N (re, im), r, 1 - r, 2 r in FP32
  __shared__ float s_cf32[MAX_CAP][5];  // the same for every candidate

  // the descriptor lives in shared memory for the kernel's lifetime: its
  // fields are read after every grid barrier
  __shared__ SlotDev s_sd;
  for (int i = threadIdx.x; i < (int)(sizeof(SlotDev) / 8); i += THREADS)
    reinterpret_cast<unsigned long long*>(&s_sd)[i] = reinterpret_cast<const unsigned long long*>(slots)[i];
  __syncthreads();
  const SlotDev& sd = s_sd;
  SlotCtl* ctl = sd.ctl;
  const int M = sd.p.M;
  const int n_tiles = (M + FPC - 1) / FPC;
  const int Pc = chunks_of(N);
  const unsigned nb = gridDim.x;
  unsigned epoch = 0;  // barriers passed so far
  const bool cta0 = blockIdx.x == 0;
  const int g = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* buf = reinterpret_cast<float2*>(smem_raw) + g * S::SMEM;
  // the forward spectrum, handed from group 0 to the others (natural order)
  float2* spec = reinterpret_cast<float2*>(smem_raw) + FPC * S::SMEM;
  Top2F* top = reinterpret_cast<Top2F*>(sd.top2);
  long long* clk = (cta0 && threadIdx.x == 0) ? sd.phase_clk : nullptr;
  for (int i = threadIdx.x; i < FftSchedule::tw_size(LOGN); i += THREADS) s_tw[i] = sd.p.st32[i];
  // Point e of a thread's transform input is sample m = t + o_e.  The FP32
  // local update needs w^d and sin(pi d / N) for d = m - j (j: the step's
  // winning angle) and z_m; they are formed from e^(i pi (t - j) / N), the
  // per-point rotations below and z_t, with no table reads.
  constexpr float INV_N = 1.0f / (float)N;  // exact: N is a power of two
  if (threadIdx.x < P) {
    const float o = (float)fft_in_index<float, LOGN>(0, threadIdx.x) * INV_N;
    float sn, cs;
    sincospif(o, &sn, &cs);
    s_rot1[threadIdx.x] = make_float2(cs, sn);
    sincospif(2.0f * o, &sn, &cs);
    s_rot2[threadIdx.x] = make_float2(cs, sn);
  }
  float2 z_t;
  sincospif(2.0f * (float)t * INV_N, &z_t.y, &z_t.x);
  // the radial powers and objective weight of this CTA's first tile stay in
  // registers across steps
  const int s_first = blockIdx.x * FPC + g;
  float h0[R0], lb0[NB0];
  float w2_0 = 0.0f;
  if (s_first < M) {
#pragma unroll
    for (int q = 0; q < R0; ++q) h0[q] = __ldg(&sd.p.rhi32[(size_t)s_first * R0 + q]);
#pragma unroll
    for (int i = 0; i < NB0; ++i) lb0[i] = __ldg(&sd.p.rlo32[(size_t)s_first * B + t + i * TPF]);
    w2_0 = obj_w32(sd, s_first);
  }
  // Warp-sized FP64 items: W per candidate (guard) and W for the update, four
  // per 128-sample chunk.  An FP64 warp instruction occupies its SM
  // sub-partition's FP64 pipe for tens of cycles whatever the active lanes,
  // so the work is spread over sub-partitions (warp w runs on w mod 4):
  //  - guard items on the warps with (warp & 2) == 0, the real part of an
  //    item's sum on one warp and the imaginary part on its neighbour;
  //  - update items on the others, warp gw = slot * nb + blockIdx taking
  //    items gw, gw + nw, ...; while the guard runs, update slots 2c and
  //    2c + 1 form the update terms of the CTA's first item for candidate c,
  //    and the last two warps the energy partials of the previous step and
  //    the candidates' scalars.
  constexpr int WPC = FP64_CHUNK / 32;
  constexpr int NWARP = THREADS / 32;
  static_assert(NWARP % 4 == 0 && NWARP >= 8, "two FP64 roles over whole quads of warps");
  constexpr int NPAIR = NWARP / 4;  // guard warp pairs per CTA
  const int W = WPC * Pc;
  const bool upd_role = (warp & 2) != 0;
  const int role_slot = ((warp >> 2) << 1) | (warp & 1);
  const int nw = (NWARP / 2) * (int)nb;
  const int gw = role_slot * (int)nb + (int)blockIdx.x;
  const int gwa = warp * (int)nb + (int)blockIdx.x;  // over all warps
  const int nwa = NWARP * (int)nb;
  // an update warp's first item keeps its samples G(z_m) in registers: the
  // same lane updates the same sample at every step
  const int m_own = upd_role && gw < W ? gw * 32 + lane : -1;
  double2 g_own = make_double2(0.0, 0.0);
  if (m_own >= 0 && m_own < N) g_own = sd.G[m_own];
  // update terms U, B (update_coef) of the first role slot's item for the
  // first NPRE candidates, formed while the guard sums run: U of candidate c
  // by update slot 2c, B by slot 2c + 1, from the item's samples in s_gown
  constexpr int NPRE = 4;
  __shared__ UpdCoef s_upd[NPRE][32];
  __shared__ double2 s_gown[32];
  const bool pre_warp = upd_role && role_slot == 0 && m_own >= 0;
  if (pre_warp) s_gown[lane] = g_own;
  // FP64 -> FP32 conversions run on the slow FP64 pipe: none per step and thread
  const float tau32 = (float)sd.tau;
  // G_k and its FP32 copy G_k / N alternate between two buffers (even k: the
  // slot's own), so that step k's update can write G_{k+1} while other CTAs
  // still read G_k
  auto Gbuf = [&](int kk) -> double2* { return (kk & 1) ? sd.G2 : sd.G; };
  auto g32buf = [&](int kk) -> float2* { return (kk & 1) ? sd.g32b : sd.g32; };
  // the final remainder goes to the slot's own buffer (update warps)
  auto publish_remainder = [&](int kk) {
    if (!upd_role) return;
    for (int i = gw; i < W; i += nw) {
      const int m = i * 32 + lane;
      if (m < N) sd.G[m] = m == m_own ? g_own : Gbuf(kk)[m];
    }
  };
  __syncthreads();

  // Energy of the remainder after step kk, E = (1/N) sum |G|^2, from that
  // step's warp partials in the chunk and lane order of k_update.  Called by a
  // whole warp; every lane gets E.
  auto energy_of = [&](int kk) -> double {
    double E = 0.0;
    for (int q = lane; q < Pc; q += 32) {
      double ch = 0.0;  // chunk q: its four warp sums in warp order
#pragma unroll
      for (int w = 0; w < WPC; ++w) ch += __ldcg(&sd.epart[(size_t)kk * W + q * WPC + w]);
      E += ch;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) E += __shfl_xor_sync(0xffffffffu, E, off);
    return E * sd.p.inv_n;  // exact: N is a power of two
  };
  // With an energy tolerance, step kk's delta decides at once whether to stop
  // (the same decision in every CTA).  Returns true when the decomposition stops.
  auto finish_step = [&](int kk) -> bool {
    if (threadIdx.x < 32) {
      const double E = energy_of(kk);
      if (threadIdx.x == 0) s_E = E;
    }
    __syncthreads();
    const double E = s_E;
    const double E1 = __ldcg(&ctl->E1);
    const double delta = E1 > 0.0 ? E / E1 : 0.0;
    const bool stop = kk + 1 >= sd.K_max || delta <= sd.tol;
    if (cta0 && threadIdx.x == 0) {
      StepRec& rec = sd.rec[kk];
      rec.energy = E;
      rec.delta = delta;
      ctl->k = kk + 1;
      if (stop) ctl->done = 1;
    }
    return stop;
  };
  // Without a tolerance nothing waits for the energies: after the last step,
  // one warp per step (over all CTAs) writes energy and delta.
  auto finish_all = [&](int steps) {
    const double E1 = __ldcg(&ctl->E1);
    for (int kk = gwa; kk < steps; kk += nwa) {
      const double E = energy_of(kk);
      if (lane == 0) {
        StepRec& rec = sd.rec[kk];
        rec.energy = E;
        rec.delta = E1 > 0.0 ? E / E1 : 0.0;
      }
    }
    if (cta0 && threadIdx.x == 0) {
      ctl->k = steps;
      ctl->done = 1;
    }
  };
  // Energy partial of each of the warp's update items of step kk: a shuffle
  // tree over its 32 samples of the new remainder.
  auto energy_items = [&](int kk) {
    if (!upd_role) return;
    for (int i = gw; i < W; i += nw) {
      const int m = i * 32 + lane;
      double e = 0.0;
      if (m < N) {
        const double2 g2 = m == m_own ? g_own : sd.G[m];
        e = fma(g2.x, g2.x, g2.y * g2.y);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
      if (lane == 0) sd.epart[(size_t)kk * W + i] = e;
    }
  };

  for (int k = 0;; ++k) {
    if (k >= sd.K_max) {
      // after the last step's update (its energy partials are written)
      if (sd.tol > 0.0) finish_step(k - 1);
      else finish_all(k);
      return;
    }
    if (clk) clk[8 * k + 0] = clock64();
    // The forward transform's input G_k / N.  Step 0: the FP32 copy the
    // initialisation wrote.  Later steps: formed here in FP32 from step k-1's
    // FP32 copy and its winner, G_k = (G_{k-1} u - c') B (update_coef), while
    // the update warps write the FP64 G_k; so no grid barrier separates an
    // update from the next step's transforms.  The FP32 grid only proposes
    // candidates; the FP64 guard on the FP64 G_k decides.
    // Points e0 <= e < e0 + CNT of the thread's transform input (k >= 1),
    // into out[e - e0].
    auto input_points = [&](auto cnt_tag, int e0, float2* out) {
      constexpr int CNT = decltype(cnt_tag)::value;
      const float2* gp = g32buf(k - 1);
      // the winner's scalars, converted once per CTA (in phase C)
      const float crn = s_f32[0], cin = s_f32[1], r = s_f32[2], omr = s_f32[3], r2 = s_f32[4];
      // e^(i pi (t - j) / N); the argument is exact
      float hs, hc;
      sincospif((float)(t - s_pj) * INV_N, &hs, &hc);
      float2 gin[CNT];
#pragma unroll
      for (int i = 0; i < CNT; ++i) gin[i] = __ldcg(&gp[fft_in_index<float, LOGN>(t, e0 + i)]);
#pragma unroll
      for (int i = 0; i < CNT; ++i) {
        // h = e^(i pi (m - j) / N): sin(pi d / N) = +-Im h and w^d = h^2
        const float2 q1 = s_rot1[e0 + i], q2 = s_rot2[e0 + i];
        const float hx = fmaf(hc, q1.x, -hs * q1.y), sh = fmaf(hc, q1.y, hs * q1.x);
        const float wy = 2.0f * hx * sh;
        const float2 z = make_float2(fmaf(z_t.x, q2.x, -z_t.y * q2.y), fmaf(z_t.x, q2.y, z_t.y * q2.x));
        // u = 1 - r w^d with 1 - r cos = (1 - r) + 2 r sin^2(pi d / N) (no
        // cancellation); G_k / N = (g u - c'/N) u conj(z) / |u|^2
        const float2 g2 = gin[i];
        const float ur = fmaf(r2 * sh, sh, omr), ui = -r * wy;
        const float ik = __fdividef(1.0f, fmaf(ur, ur, ui * ui));
        const float xr = fmaf(g2.x, ur, fmaf(-g2.y, ui, -crn)), xi = fmaf(g2.x, ui, fmaf(g2.y, ur, -cin));
        const float yr = fmaf(xr, ur, -xi * ui), yi = fmaf(xr, ui, xi * ur);
        out[i] = make_float2(fmaf(yr, z.x, yi * z.y) * ik, fmaf(yi, z.x, -yr * z.y) * ik);
      }
    };
    // The forward transform's input in group 0 (all of warp 0 when a group
    // is narrower than a warp).  From step 1 on, with groups of whole warps,
    // group 1 forms the upper half of the points and hands them over in spec.
    constexpr bool SPLIT = TPF >= 32 && P >= 2;
    const bool lead = TPF >= 32 ? g == 0 : warp == 0;
    auto load_input = [&](float2* v) {
      if (k == 0) {
        if (lead) {
#pragma unroll
          for (int e = 0; e < P; ++e) v[e] = sd.g32[fft_in_index<float, LOGN>(t, e)];
        }
        return;
      }
      if constexpr (SPLIT) {
        if (g == 1) {
          float2 hi[P / 2];
          input_points(std::integral_constant<int, P / 2>{}, P / 2, hi);
#pragma unroll
          for (int i = 0; i < P / 2; ++i) spec[t + TPF * i] = hi[i];
        } else if (g == 0) {
          input_points(std::integral_constant<int, P / 2>{}, 0, v);
        }
        __syncthreads();
        if (g == 0) {
#pragma unroll
          for (int i = 0; i < P / 2; ++i) v[P / 2 + i] = spec[t + TPF * i];
        }
      } else {
        if (lead) input_points(std::integral_constant<int, P>{}, 0, v);
      }
    };
    // ---------------------------------------------------------------- A --
    for (int tile = blockIdx.x; tile < n_tiles; tile += nb) {
      const int s = tile * FPC + g;
      const bool active = s < M;
      const float w2 = active ? (tile == (int)blockIdx.x ? w2_0 : obj_w32(sd, s)) : 0.0f;
      float2 v[P];
      // The forward transform, once per CTA by group 0 (group barriers only),
      // leaves c_l, l = t + TPF e, in register e (its last pass is one
      // full-width butterfly per thread); it goes to spec for the other
      // groups.  The inverse transform's pass 0 wants l = t + i TPF + q B =
      // t + TPF (i + q NB0) in register i R0 + q.  A group narrower than a
      // warp synchronises with __syncwarp, which needs the whole warp: there
      // all groups of warp 0 run the (identical) forward transform.
      static_assert(LOGN < 4 || (P == 16 && S::radix(S::NPASS - 1) == 16 && S::ns(S::NPASS - 1) == TPF),
                    "forward outputs t + TPF e");
      load_input(v);  // every thread (it may synchronise the CTA)
      if (lead) {
        // group 0 reads its points from spec before any of its threads can
        // finish the transform (group barriers) and write the spectrum there
        fft_run<float, LOGN, -1, 0, true, 0, true>(v, t, buf, s_tw);
        if (g == 0) {
#pragma unroll
          for (int e = 0; e < P; ++e) spec[t + TPF * e] = v[e];
        }
      }
      __syncthreads();
      float2 vf[P];
      if (g == 0) {
#pragma unroll
        for (int e = 0; e < P; ++e) vf[e] = v[e];
      } else {
#pragma unroll
        for (int e = 0; e < P; ++e) vf[e] = spec[t + TPF * e];
      }
      if (active) {
        float h[R0], lb[NB0];
        if (tile == (int)blockIdx.x) {
#pragma unroll
          for (int q = 0; q < R0; ++q) h[q] = h0[q];
#pragma unroll
          for (int i = 0; i < NB0; ++i) lb[i] = lb0[i];
        } else {
#pragma unroll
          for (int q = 0; q < R0; ++q) h[q] = __ldg(&sd.p.rhi32[(size_t)s * R0 + q]);
#pragma unroll
          for (int i = 0; i < NB0; ++i) lb[i] = __ldg(&sd.p.rlo32[(size_t)s * B + t + i * TPF]);
        }
#pragma unroll
        for (int i = 0; i < NB0; ++i) {
#pragma unroll
          for (int q = 0; q < R0; ++q) {
            const float rp = lb[i] * h[q];
            const float2 x = vf[i + q * NB0];
            v[i * R0 + q] = make_float2(x.x * rp, x.y * rp);
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < P; ++e) v[e] = make_float2(0.f, 0.f);
      }
      fft_run<float, LOGN, +1, 0, true, 0, true>(v, t, buf, s_tw);
      Best2F b;
      b.init();
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const float2 x = v[fft_out_slot<float, LOGN>(u)];
        b.push_ascending(norm2<float>(x), t + TPF * u);
      }
      // (red2 was last read before this tile's spectrum barrier)
      group_reduce<TPF, Best2F, true>(b, red2);
      if (t == 0 && active) {
        Top2F o;
        o.v1 = b.v1 * w2;
        o.v2 = b.v2 * w2;
        o.j1 = b.j1;
        o.j2 = b.j2;
        top[s] = o;
        if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&ctl->vmax2[k & 1], __float_as_uint(o.v1));
      }
      // the CTA's next tile reuses the exchange buffers and red2 (after the
      // last tile the grid barrier synchronises the CTA)
      if (tile + (int)nb < n_tiles) __syncthreads();
    }
    if (clk) clk[8 * k + 1] = clock64();
    if (!grid_barrier(sd, nb * ++epoch, &s_ok)) return;
    if (clk) clk[8 * k + 2] = clock64();
    // ---------------------------------------------------------------- B --
    const double2* Gk = Gbuf(k);
    // guard warp pairs: pair gp = (warp >> 2) nb + blockIdx takes items gp,
    // gp + NPAIR nb, ...; comp 0 sums the real parts, comp 1 the imaginary ones.
    // G at the pair's first item (its sample range does not depend on the
    // candidates) and, on the last warp, at its first energy item are
    // fetched while the candidates are selected.
    const int comp = warp & 1;
    const int gpair = (warp >> 2) * (int)nb + (int)blockIdx.x;
    const int m_g0 = (gpair % W) * 32 + lane;
    const double2 g_g0 = !upd_role && m_g0 < N ? __ldcg(&Gk[m_g0]) : make_double2(0.0, 0.0);
    const bool e_warp = warp == NWARP - 1;
    const int m_e0 = (int)blockIdx.x * 32 + lane;
    const double2 g_e0 = k > 0 && e_warp && m_e0 < N ? __ldcg(&Gk[m_e0]) : make_double2(0.0, 0.0);
    const float vmax = __uint_as_float(__ldcg(&ctl->vmax2[k & 1]));
    int n = 1, count = 1;
    if (sd.force_a1_zero && k == 0) {
      if (threadIdx.x == 0) s_cand[0] = make_int2(0, 0);
      __syncthreads();
    } else {
      select_core<THREADS>(top, M, N, 1, vmax - vmax * tau32, sd.cap, s_cand, &n, &count, s_scr);
    }
    if (cta0 && threadIdx.x == 0) {
      ctl->vmax2[(k + 1) & 1] = 0u;  // the next step's accumulator
      StepRec& rec = sd.rec[k];
      rec.obj32 = vmax;
      rec.flags = count > sd.cap ? 1 : 0;
      ctl->n_cand = n;
      for (int c = 0; c < n; ++c) sd.cand[c] = s_cand[c];
    }
    if (upd_role) {
      if (e_warp && k > 0) {
        // energy partials of step k-1 (the remainder G_k), in the lane order
        // of energy_items
        {
          for (int i = blockIdx.x; i < W; i += (int)nb) {
            const int m = i * 32 + lane;
            double e = 0.0;
            if (m < N) {
              const double2 g2 = i == (int)blockIdx.x ? g_e0 : __ldcg(&Gk[m]);
              e = fma(g2.x, g2.x, g2.y * g2.y);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
            if (lane == 0) sd.epart[(size_t)(k - 1) * W + i] = e;
          }
        }
      }
      if (warp == NWARP - 2) {
        // the candidates' scalars for phase C and the next step's FP32 update
        for (int c = lane; c < n; c += 32) {
          const int s = s_cand[c].x;
          const double rd = sd.p.radii[s], sq = sd.p.sq64[s];
          s_rad[c] = rd;
          s_sq[c] = sq;
          s_scn[c] = sq * sd.p.inv_n;  // exact scaling: N is a power of two
          s_scn32[c] = d2f_rn(sq) * INV_N;
          s_rho[c] = obj_rho64(sd, s);
          const float r32 = d2f_rn(rd);
          s_cf32[c][2] = r32;
          s_cf32[c][3] = d2f_rn(1.0 - rd);
          s_cf32[c][4] = 2.0f * r32;
        }
      }
      // update terms of the CTA's first update item: candidate c = slot / 2,
      // U on one update warp and B on the next (another sub-partition)
      const int pc_ = role_slot >> 1;
      if (pc_ < n && pc_ < NPRE && (int)blockIdx.x < W) {
        const int m0 = (int)blockIdx.x * 32 + lane;
        const int2 cj = s_cand[pc_];
        if (m0 < N) {
          if (role_slot & 1) s_upd[pc_][lane].B = update_b(sd, m0, cj.x, cj.y);
          else s_upd[pc_][lane].U = update_u(sd, m0, cj.y, sd.p.radii[cj.x], s_gown[lane]);
        }
      }
    } else {
      // real parts at gpart64[it], imaginary parts cap W further on
      double* gpart64 = reinterpret_cast<double*>(sd.gpart) + (size_t)comp * sd.cap * W;
      for (int it = gpair; it < n * W; it += NPAIR * (int)nb) {
        const int c = it / W, i = it % W;
        const int m = i * 32 + lane;
        double a = 0.0;
        if (m < N) {
          // one component of guard_term
          const double2 gm = it == gpair ? g_g0 : __ldcg(&Gk[m]);
          const double2 kd = __ldg(&sd.p.K64[(size_t)s_cand[c].x * N + wrap_mod(s_cand[c].y - m, N)]);
          a = comp ? fma(gm.x, kd.y, gm.y * kd.x) : fma(gm.x, kd.x, -gm.y * kd.y);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) gpart64[it] = a;
      }
    }
    if (clk) clk[8 * k + 3] = clock64();
    if (!grid_barrier(sd, nb * ++epoch, &s_ok)) return;
    if (clk) clk[8 * k + 4] = clock64();

    // ---------------------------------------------------------------- C --

    // step k-1 is complete: with a tolerance, its energy, delta and the stop
    // rule (step k ran speculatively so far; nothing of it is recorded before
    // this)
    if (k > 0 && sd.tol > 0.0 && finish_step(k - 1)) {
      publish_remainder(k);
      return;
    }
    // The candidates' sums, one component per warp: chunk q adds its four
    // warp sums in warp order, then the chunks go through a shuffle tree, as
    // in the separate kernels.  A lane reads its chunk's four partials with
    // one 32-byte load, so that a warp's reads are contiguous (every CTA
    // reads them: fewer L2 requests per line).
    static_assert(WPC == 4, "one 32-byte load per chunk");
    {
      for (int u = warp; u < 2 * n; u += NWARP) {
        const int c = u >> 1, cp = u & 1;
        const double* part = reinterpret_cast<const double*>(sd.gpart) + (size_t)cp * sd.cap * W + (size_t)c * W;
        double x = 0.0;
        for (int q = lane; q < Pc; q += 32) {
          const double4v p4 = ld_cg_v4(part + q * WPC);
          x += ((p4.x + p4.y) + p4.z) + p4.w;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) {
          const double re = s_scn[c] * x;  // the coefficient's component
          (cp ? s_im : s_re)[c] = re;
          (cp ? s_ci : s_cr)[c] = re * s_sq[c];     // c' = c sqrt(1 - r^2)
          s_cf32[c][cp] = d2f_rn(re) * s_scn32[c];  // c' / N, for the FP32 update
        }
      }
    }
    __syncthreads();
    // One candidate (most steps): it wins unless its objective may not be
    // finite, and every thread knows that at once.  |re|, |im| < 2^498 keep
    // (re^2 + im^2) rho finite (rho <= 1); the general path decides otherwise.
    int pc = 0, ps = -1, pj = -1;
    const long long kBig = 0x5f10000000000000LL;  // 2^498
    if (n == 1 && (__double_as_longlong(s_re[0]) & 0x7fffffffffffffffLL) < kBig &&
        (__double_as_longlong(s_im[0]) & 0x7fffffffffffffffLL) < kBig) {
      ps = s_cand[0].x;
      pj = s_cand[0].y;
      // for the next step's FP32 update (read after its next barrier)
      if (threadIdx.x == 0) {
        s_pj = pj;
        for (int q = 0; q < 5; ++q) s_f32[q] = s_cf32[0][q];
      }
    } else {
    if (threadIdx.x < n) {
      const int c = threadIdx.x;
      const double re = s_re[c], im = s_im[c];
      s_v[c] = (re * re + im * im) * s_rho[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // best objective, ties to the lower flat index; the values are >= 0 or
      // NaN, so their bit patterns order as the values do (NaN never wins
      // against an earlier candidate)
      int bc = -1, bs = -1, bj = -1, bf = 0;
      long long bb = 0;
      for (int c = 0; c < n; ++c) {
        const int2 cj = s_cand[c];
        const long long vb = __double_as_longlong(s_v[c]);
        const bool nan = (vb & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
        const int f = cj.x * N + cj.y;
        if (bs < 0 || (!nan && (vb > bb || (vb == bb && f < bf)))) {
          bc = c; bs = cj.x; bj = cj.y; bb = vb; bf = f;
        }
      }
      if (bs >= 0 && !((bb & 0x7fffffffffffffffLL) <= __double_as_longlong(1.79e308))) bs = -1;
      s_pc = bc;
      s_ps = bs;
      s_pj = bj;
      if (bc >= 0)
        for (int q = 0; q < 5; ++q) s_f32[q] = s_cf32[bc][q];
    }
    __syncthreads();
    pc = s_pc;
    ps = s_ps;
    pj = s_pj;
    }
    if (ps < 0) {
      if (cta0 && threadIdx.x == 0) {
        StepRec& rec = sd.rec[k];
        rec.s = -1;
        rec.j = -1;
        rec.flags |= 2;
        ctl->err |= 2;
      }
      if (sd.tol > 0.0) {
        if (cta0 && threadIdx.x == 0) ctl->done = 1;
      } else {
        finish_all(k);  // the energies of the steps done
      }
      publish_remainder(k);
      return;
    }
    // the step record, by the last CTA (the update items start at CTA 0)
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) {
      StepRec& rec = sd.rec[k];
      const double rr = s_rad[pc], re = s_re[pc], im = s_im[pc];
      const double2 z = sd.p.tw64[pj];
      rec.s = ps;
      rec.j = pj;
      rec.n_cand = n;
      rec.a_re = rr * z.x;
      rec.a_im = rr * z.y;
      rec.c_re = re;
      rec.c_im = im;
      rec.obj = (re * re + im * im) * s_rho[pc];  // as s_v
    }
    {
      const double r = s_rad[pc], cr = s_cr[pc], ci = s_ci[pc];
      const bool last = k + 1 >= sd.K_max;
      // G_{k+1}: the next buffer, or the slot's own after the last step
      double2* Gn = last ? sd.G : Gbuf(k + 1);
      float2* gn32 = g32buf(k + 1);
      for (int i = upd_role ? gw : W; i < W; i += nw) {
        const int m = i * 32 + lane;
        if (m < N) {
          double2 gn;
          if (pre_warp && m == m_own && pc < NPRE) gn = update_apply(s_upd[pc][lane], cr, ci);
          else gn = update_point(sd, m, ps, pj, r, cr, ci, m == m_own ? g_own : Gk[m]);
          if (m == m_own) {
            g_own = gn;
            if (pre_warp) s_gown[lane] = gn;
          }
          Gn[m] = gn;
          // G_{k+1} / N in FP32: scaling by a power of two commutes with the rounding
          if (!last) gn32[m] = make_float2(d2f_rn(gn.x) * INV_N, d2f_rn(gn.y) * INV_N);
        }
      }
      // the energy partials: now after the last step, else during the next
      // step's guard
      if (last) energy_items(k);
    }
    if (clk) clk[8 * k + 5] = clock64();
    // after the last step every CTA must see all energy partials
    if (k + 1 >= sd.K_max && !grid_barrier(sd, nb * ++epoch, &s_ok)) return;
    if (clk) {
      clk[8 * k + 6] = clock64();
      clk[8 * k + 7] = clk[8 * k + 6];  // the energy phase is timed inside the next step's stamps
    }
  }
}

// --------------------------------------------------------------- launchers --

namespace {

// Launch with programmatic stream serialisation (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T, int LOGN, int PP = 0, int CT = 256>
size_t grid_smem() {
  using S = FftShape<T, LOGN, PP>;
  return sizeof(V2<T>) * (size_t)S::SMEM * GridCfg<T, LOGN, PP, CT>::FPC;
}
// the persistent kernel: one exchange buffer per transform group and the
// shared forward spectrum
template <int LOGN>
size_t persist_smem() {
  using S = FftShape<float, LOGN>;
  return sizeof(float2) * ((size_t)S::SMEM * GridCfg<float, LOGN, 0, PERSIST_CTA>::FPC + S::N);
}
template <typename T, int LOGN>
size_t fwd_smem() {
  using S = FftShape<T, LOGN>;
  return sizeof(V2<T>) * (size_t)S::SMEM;
}

template <typename T, int LOGN, int PP = 0, int CT = 256>
cudaError_t grid_launch(const SlotDev* slots, const int* ids, int n, int Mmax, cudaStream_t st) {
  using C = GridCfg<T, LOGN, PP, CT>;
  dim3 grid((Mmax + C::FPC - 1) / C::FPC, n);
  return launch_pdl(k_grid<T, LOGN, PP, CT>, grid, dim3(C::THREADS), grid_smem<T, LOGN, PP, CT>(), st, slots,
                    ids);
}

// Grid-kernel variants the autotuner chooses from (FP32, 2^8 <= N <= 2^13):
// 1: 32 points per thread; 2: CTAs of 512 threads (2^8 <= N <= 2^12).
template <int LOGN>
cudaError_t grid_variant_launch(int variant, const SlotDev* slots, const int* ids, int n, int Mmax,
                                cudaStream_t st) {
  if constexpr (LOGN >= 8 && LOGN <= 13) {
    if (variant == 1) return grid_launch<float, LOGN, 32, 256>(slots, ids, n, Mmax, st);
    if constexpr (LOGN <= 12)
      if (variant == 2) return grid_launch<float, LOGN, 0, 512>(slots, ids, n, Mmax, st);
  }
  return grid_launch<float, LOGN>(slots, ids, n, Mmax, st);
}

template <int LOGN>
cudaError_t set_variant_attrs() {
  cudaError_t e = cudaSuccess;
  if constexpr (LOGN >= 8 && LOGN <= 13) {
    e = cudaFuncSetAttribute(k_grid<float, LOGN, 32, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)grid_smem<float, LOGN, 32, 256>());
    if (e != cudaSuccess) return e;
    if constexpr (LOGN <= 12)
      e = cudaFuncSetAttribute(k_grid<float, LOGN, 0, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)grid_smem<float, LOGN, 0, 512>());
  }
  return e;
}

template <typename T, int LOGS, int LS>
cudaError_t split_launch(bool grid, const SlotDev* slots, const int* ids, int n, int Mmax, cudaStream_t st) {
  const size_t smem = sizeof(V2<T>) * (size_t)FftShape<T, LOGS>::SMEM;
  const dim3 block(FftShape<T, LOGS>::TPF);
  if (grid) return launch_pdl(k_grid_split<T, LOGS, LS>, dim3((unsigned)Mmax << LS, n), block, smem, st, slots, ids);
  return launch_pdl(k_forward_split<T, LOGS, LS>, dim3(1u << LS, n), block, smem, st, slots, ids);
}

template <typename T, int LOGS, int LS>
cudaError_t set_split_attrs() {
  const int smem = (int)(sizeof(V2<T>) * (size_t)FftShape<T, LOGS>::SMEM);
  cudaError_t e = cudaFuncSetAttribute(k_grid_split<T, LOGS, LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_forward_split<T, LOGS, LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// The split sizes: FP32 N = 2^15; FP64 N = 2^14 .. 2^16.
cudaError_t split_dispatch(bool grid, const SlotDev* slots, const int* ids, int n, int logN, int prec, int Mmax,
                           cudaStream_t st) {
  static_assert(split_log(15, 1) == 1 && split_log(14, 0) == 1 && split_log(16, 0) == 3 && split_log(16, 1) == 0,
                "split sizes");
  if (prec && logN == 15) return split_launch<float, 14, 1>(grid, slots, ids, n, Mmax, st);
  if (!prec && logN == 14) return split_launch<double, 13, 1>(grid, slots, ids, n, Mmax, st);
  if (!prec && logN == 15) return split_launch<double, 13, 2>(grid, slots, ids, n, Mmax, st);
  if (!prec && logN == 16) return split_launch<double, 13, 3>(grid, slots, ids, n, Mmax, st);
  return cudaErrorInvalidValue;
}

template <typename T, int LOGN>
cudaError_t fwd_launch(const SlotDev* slots, const int* ids, int n, cudaStream_t st) {
  return launch_pdl(k_forward<T, LOGN>, dim3(n), dim3(FftShape<T, LOGN>::TPF), fwd_smem<T, LOGN>(), st,
                    slots, ids);
}

template <typename T, int LOGN>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_grid<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grid_smem<T, LOGN>());
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4 && LOGN <= PERSISTENT_MAX_LOGN) {
    e = cudaFuncSetAttribute(k_persistent<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)persist_smem<LOGN>());
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_forward<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fwd_smem<T, LOGN>());
}

#define AFD_FOR_EACH_LOGN(X) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)

}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = cudaSuccess;
#define X(L)                                                       \
  if ((e = set_attrs<float, L>()) != cudaSuccess) return e;         \
  if ((e = set_attrs<double, L>()) != cudaSuccess) return e;        \
  if ((e = set_variant_attrs<L>()) != cudaSuccess) return e;
  AFD_FOR_EACH_LOGN(X)
#undef X
  if ((e = set_attrs<float, 14>()) != cudaSuccess) return e;
  if ((e = set_split_attrs<float, 14, 1>()) != cudaSuccess) return e;
  if ((e = set_split_attrs<double, 13, 1>()) != cudaSuccess) return e;
  if ((e = set_split_attrs<double, 13, 2>()) != cudaSuccess) return e;
  if ((e = set_split_attrs<double, 13, 3>()) != cudaSuccess) return e;
  if ((e = mixed_configure()) != cudaSuccess) return e;
  if ((e = multi_configure()) != cudaSuccess) return e;
  if ((e = nu_configure()) != cudaSuccess) return e;
  return fft2_configure();
}

size_t grid_smem_bytes(int logN, int prec) {
  switch (logN) {
#define X(L) case L: return prec ? grid_smem<float, L>() : grid_smem<double, L>();
    AFD_FOR_EACH_LOGN(X)
#undef X
    case 14: return prec ? grid_smem<float, 14>() : 0;
    default: return 0;
  }
}

size_t forward_smem_bytes(int logN, int prec) {
  switch (logN) {
#define X(L) case L: return prec ? fwd_smem<float, L>() : fwd_smem<double, L>();
    AFD_FOR_EACH_LOGN(X)
#undef X
    case 14: return prec ? fwd_smem<float, 14>() : 0;
    default: return 0;
  }
}

int grid_ffts_per_cta(int logN, int prec) {
  switch (logN) {
#define X(L) case L: return prec ? GridCfg<float, L>::FPC : GridCfg<double, L>::FPC;
    AFD_FOR_EACH_LOGN(X)
#undef X
    case 14: return prec ? GridCfg<float, 14>::FPC : 0;
    default: return 0;
  }
}

bool grid_variant_ok(int logN, int prec, int variant) {
  if (variant == 0) return true;
  if (!prec || logN < 8 || logN > 13) return false;
  return variant == 1 || (variant == 2 && logN <= 12);
}

cudaError_t launch_grid(const SlotDev* slots, const int* ids, int n, int logN, int prec, int Mmax,
                        cudaStream_t st, int variant) {
  if (n <= 0) return cudaSuccess;
  switch (logN) {
#define X(L)                                                                          \
  case L:                                                                             \
    return prec ? grid_variant_launch<L>(variant, slots, ids, n, Mmax, st)            \
                : grid_launch<double, L>(slots, ids, n, Mmax, st);
    AFD_FOR_EACH_LOGN(X)
#undef X
    case 14:
      if (prec) return grid_launch<float, 14>(slots, ids, n, Mmax, st);
      return split_dispatch(true, slots, ids, n, logN, prec, Mmax, st);
    default: return split_dispatch(true, slots, ids, n, logN, prec, Mmax, st);
  }
}

cudaError_t launch_forward(const SlotDev* slots, const int* ids, int n, int logN, int prec,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (logN) {
#define X(L) \
  case L: return prec ? fwd_launch<float, L>(slots, ids, n, st) : fwd_launch<double, L>(slots, ids, n, st);
    AFD_FOR_EACH_LOGN(X)
#undef X
    case 14:
      if (prec) return fwd_launch<float, 14>(slots, ids, n, st);
      return split_dispatch(false, slots, ids, n, logN, prec, 0, st);
    default: return split_dispatch(false, slots, ids, n, logN, prec, 0, st);
  }
}

namespace {
int g_persist_blocks[PERSISTENT_MAX_LOGN + 1] = {};  // co-resident CTAs per logN (0: not yet known)

template <int LOGN>
cudaError_t persistent_launch(const SlotDev* slots, int M, cudaStream_t st) {
  using C = GridCfg<float, LOGN, 0, PERSIST_CTA>;
  const size_t smem = persist_smem<LOGN>();
  if (!g_persist_blocks[LOGN]) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<LOGN>, C::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    g_persist_blocks[LOGN] = per_sm * sms;
  }
  // enough CTAs for the tiles and for one 32-sample FP64 item each
  const int n_tiles = (M + C::FPC - 1) / C::FPC;
  const int items = chunks_of(1 << LOGN) * (FP64_CHUNK / 32);
  int blocks = n_tiles > items ? n_tiles : items;
  if (blocks > g_persist_blocks[LOGN]) blocks = g_persist_blocks[LOGN];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(C::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persistent<LOGN>, slots);
}
}  // namespace

cudaError_t launch_persistent(const SlotDev* slots, int logN, int M, cudaStream_t st) {
  switch (logN) {
#define X(L) case L: return persistent_launch<L>(slots, M, st);
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_guard(const SlotDev* slots, const int* ids, int n, int N, int cap, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // Candidates in flight per signal: GUARD_PAR for a few signals (the latency
  // of one signal's step), one when many signals share the launch (most steps
  // have one candidate, and CTAs whose candidate does not exist still cost a
  // scheduling slot).  Every chunk's partial sum is the same either way.
  int par = cap < GUARD_PAR ? cap : GUARD_PAR;
  if (n >= 8) par = 1;
  dim3 grid(par * chunks_of(N), n);
  return launch_pdl(k_guard, grid, dim3(FP64_THREADS), 0, st, slots, ids);
}

cudaError_t launch_kernel_table(const double* radii, int M, int N, double2* K, cudaStream_t st) {
  dim3 grid((N + 255) / 256, M);
  k_kernel_table<<<grid, 256, 0, st>>>(radii, N, K);
  return cudaGetLastError();
}

cudaError_t launch_update(const SlotDev* slots, const int* ids, int n, int N, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(chunks_of(N), n);
  return launch_pdl(k_update<false>, grid, dim3(FP64_THREADS), 0, st, slots, ids);
}

cudaError_t launch_init(const SlotDev* slots, const int* ids, int n, int N, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(chunks_of(N), n);
  return launch_pdl(k_update<true>, grid, dim3(FP64_THREADS), 0, st, slots, ids);
}

}  // namespace afd
