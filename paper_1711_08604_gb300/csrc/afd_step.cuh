// Device bodies of one Core AFD greedy step (arXiv:1711.08604), shared by the
// step kernels (one CTA per work item, afd_kernels.cu) and the multi-signal
// persistent kernel (afd_multi.cu), which runs the same work items in loops:
//   grid_body     transform tile, objective, best pairs; last tile: selection
//   guard_body    FP64 rectangle-rule sums of the candidates; last item: winner
//   update_body   remainder update and energy; last item: delta, stop rule
//   forward_body  the DFT of the next remainder
// Each body takes its work item's indices (tile or chunk bx, signal by, items
// per signal gx) explicitly, so a signal's values do not depend on which CTA
// runs an item: they are bitwise the same in either kernel.
#pragma once
#include <climits>
#include <cstdint>

#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_internal.h"

namespace afd {

// ------------------------------------------------------------- grid step --

// PP: points per thread (0: the default of FftShape); CT: the CTA width the
// transforms are packed up to (several radii per CTA when one transform has
// fewer threads).  The variants compute bitwise the same values: only which
// thread computes which butterfly changes.
template <typename T, int LOGN, int PP = 0, int CT = 256>
struct GridCfg {
  using S = FftShape<T, LOGN, PP>;
  // FP32 packs small transforms into CTAs of CT threads; FP64 keeps one warp
  // per CTA at most, so that its FP64 work (1/64 of the FP32 rate) spreads
  // over as many SMs as there are radii
  static constexpr int CTA = sizeof(T) == 4 ? CT : 32;
  static constexpr int FPC = S::TPF >= CTA ? 1 : CTA / S::TPF;  // transforms per CTA
  static constexpr int THREADS = S::TPF * FPC;
  // CTAs per SM the register budget is cut for: the paired FP32 transforms
  // (32 points per thread) fit three 256-thread CTAs (registers and shared
  // memory) up to N = 8192; the FP32 variants of 16 points per thread 64
  // registers per thread; 0: no bound
  static constexpr int MIN_CTAS = sizeof(T) != 4 ? 0
                                  : (PP == 32 && THREADS == 256 && LOGN >= 5 && LOGN <= 13) ? 3
                                  : (S::P <= 16 && THREADS >= 256 ? 65536 / (64 * THREADS) : 0);
};

// The FP32 grid work item with 32 points per thread on the paired
// transforms (fftp_run): the arithmetic of grid_body_s lane for lane, so the
// same objective values, best pairs and selection.
template <int LOGN, int CT>
__device__ __forceinline__ void grid_body_p(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                            int by, int gx) {
  using S = FftPShape<LOGN>;
  using C = GridCfg<float, LOGN, 32, CT>;
  constexpr int TPF = S::TPF, FPC = C::FPC, THREADS = C::THREADS;
  constexpr int R0 = FftSchedule::radix(LOGN, 0), B = FftSchedule::pow_b(LOGN), NPR0 = S::P / (2 * R0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  __shared__ Best2F red[32];
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[by]];

  const int g = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int s = bx * FPC + g;
  const bool active = s < sd.p.M;
  float* buf = reinterpret_cast<float*>(reinterpret_cast<float2*>(smem_raw) + g * FftShape<float, LOGN, 32>::SMEM);

  float2 X[S::P / 2], Y[S::P / 2];
  constexpr int PASS1 = R0 == 2 ? 1 : 0;  // the first pass that runs in fftp_run
  if constexpr (R0 == 2) {
    // Pass 0 in registers (fftp_r2_pass0, formed pair by pair): inputs
    // l = t + q' N/32, r_s^l = lo[l mod B] hi[l / B]
    if (active) {
      const float* lo = sd.p.rlo32 + (size_t)s * B;
      const float* hi = sd.p.rhi32 + (size_t)s * R0;
      const float h0 = __ldg(&hi[0]), h1 = __ldg(&hi[1]);
      float lb[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) lb[q] = __ldg(&lo[fftp_r2_in_index<LOGN>(t, q)]);
      pdl_wait();
      if (ld_done(sd.ctl)) return;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float rp0 = lb[q] * h0, rp1 = lb[q] * h1;
        const float2 x0 = sd.c32[fftp_r2_in_index<LOGN>(t, q)];
        const float2 x1 = sd.c32[fftp_r2_in_index<LOGN>(t, q + 16)];
        float2 a[32];
        a[q] = make_float2(x0.x * rp0, x0.y * rp0);
        a[q + 16] = make_float2(x1.x * rp1, x1.y * rp1);
        X[q] = make_float2(a[q].x + a[q + 16].x, a[q].x - a[q + 16].x);
        Y[q] = make_float2(a[q].y + a[q + 16].y, a[q].y - a[q + 16].y);
      }
    } else {
      pdl_wait();
      if (ld_done(sd.ctl)) return;
#pragma unroll
      for (int e = 0; e < S::P / 2; ++e) X[e] = Y[e] = make_float2(0.f, 0.f);
    }
  } else if (active) {
    // Pass-0 input r_s^l c_l / N for l = 2m + lane + q B, r_s^l = lo[2m + lane] hi[q]
    const float* lo = sd.p.rlo32 + (size_t)s * B;
    const float* hi = sd.p.rhi32 + (size_t)s * R0;
    const float4* c2 = reinterpret_cast<const float4*>(sd.c32);  // spectrum entries (j, j + 1), j even
    float h[R0];
    float2 lb[NPR0];
#pragma unroll
    for (int q = 0; q < R0; ++q) h[q] = __ldg(&hi[q]);
#pragma unroll
    for (int i = 0; i < NPR0; ++i) lb[i] = __ldg(reinterpret_cast<const float2*>(lo + 2 * (t + i * TPF)));
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int i = 0; i < NPR0; ++i) {
#pragma unroll
      for (int q = 0; q < R0; ++q) {
        const float2 rp = mul2(lb[i], dup2(h[q]));
        const float4 x = c2[(2 * (t + i * TPF) + q * B) >> 1];
        X[i * R0 + q] = mul2(make_float2(x.x, x.z), rp);
        Y[i * R0 + q] = mul2(make_float2(x.y, x.w), rp);
      }
    }
  } else {
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int e = 0; e < S::P / 2; ++e) X[e] = Y[e] = make_float2(0.f, 0.f);
  }

  fftp_run<LOGN, +1, PASS1, (FPC > 1)>(X, Y, t, buf, sd.p.st32p);

  // Objective and per-radius best: outputs 2t + lane + q N / 16 in increasing order
  Best2F b;
  b.init();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float2 o = fma2(X[q], X[q], mul2(Y[q], Y[q]));
    b.push_ascending(o.x, fftp_out_index<LOGN>(t, 0, q));
    b.push_ascending(o.y, fftp_out_index<LOGN>(t, 1, q));
  }
  group_reduce<TPF>(b, red);
  if (t == 0 && active) {
    const float w2 = obj_w32(sd, s);
    Top2F o;
    o.v1 = b.v1 * w2;
    o.v2 = b.v2 * w2;
    o.j1 = b.j1;
    o.j2 = b.j2;
    reinterpret_cast<Top2F*>(sd.top2)[s] = o;
    if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(o.v1));
    __threadfence();  // read by the signal's last CTA
  }
  if (!arrive_last(&sd.ctl->cnt_grid, gx, &s_last)) return;
  // the transform buffers are free (arrive_last ends with a CTA barrier)
    select_candidates_f32<THREADS>(sd, sd.ctl->k, 1, *reinterpret_cast<SelectScratch*>(smem_raw));
}

template <typename T, int LOGN, int PP = 0, int CT = 256>
__device__ __forceinline__ void grid_body_s(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                            int by, int gx);

// One work item of the grid step: transform tile bx (radii bx FPC ..) of the
// signal ids[by], whose grid has gx tiles; the signal's last tile also runs
// the selection.  Every thread of the CTA (THREADS) calls it.  FP32 with 32
// points per thread runs on the paired transforms, the rest on fft_run.
template <typename T, int LOGN, int PP = 0, int CT = 256>
__device__ __forceinline__ void grid_body(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                          int by, int gx) {
  if constexpr (sizeof(T) == 4 && PP == 32 && LOGN >= 5) grid_body_p<LOGN, CT>(slots, ids, bx, by, gx);
  else grid_body_s<T, LOGN, PP, CT>(slots, ids, bx, by, gx);
}

template <typename T, int LOGN, int PP, int CT>
__device__ __forceinline__ void grid_body_s(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                            int by, int gx) {
  using S = FftShape<T, LOGN, PP>;
  using C = GridCfg<T, LOGN, PP, CT>;
  constexpr int N = S::N, P = S::P, TPF = S::TPF, FPC = C::FPC, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[by]];

  const int g = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int s = bx * FPC + g;
  const int M = sd.p.M;
  const bool active = s < M;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw) + g * S::SMEM;

  // Pass-0 input f(l) = r_s^l c_l / N, read straight from the spectrum.  The
  // thread's inputs are l = b + q B (q < R0) with B = N / R0, so
  // r_s^l = lo[b] * hi[q] with one lo value per butterfly.
  constexpr int R0 = S::radix(0), B = FftSchedule::pow_b(LOGN), NB0 = P / R0;
  V2<T> v[P];
  const V2<T>* tw;
  if constexpr (sizeof(T) == 4) tw = sd.p.st32; else tw = sd.p.st64;
  if (active) {
    const T* lo;
    const T* hi;
    const V2<T>* c;
    if constexpr (sizeof(T) == 4) {
      lo = sd.p.rlo32 + (size_t)s * B;
      hi = sd.p.rhi32 + (size_t)s * R0;
      c = sd.c32;
    } else {
      lo = sd.p.rlo64 + (size_t)s * B;
      hi = sd.p.rhi64 + (size_t)s * R0;
      c = sd.c64;
    }
    // the power tables are constant: fetch them before waiting for the
    // kernel that produced the spectrum
    T h[R0], lb[NB0];
#pragma unroll
    for (int q = 0; q < R0; ++q) h[q] = __ldg(&hi[q]);
#pragma unroll
    for (int i = 0; i < NB0; ++i) lb[i] = __ldg(&lo[t + i * TPF]);
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
      const int b = t + i * TPF;
#pragma unroll
      for (int q = 0; q < R0; ++q) {
        const T rp = lb[i] * h[q];
        const V2<T> x = c[b + q * B];
        v[i * R0 + q] = mk2<T>(x.x * rp, x.y * rp);
      }
    }
  } else {
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = mk2<T>((T)0, (T)0);
  }

  // the CTA's transforms synchronise on their own group barriers
  fft_run<T, LOGN, +1, 0, false, PP, (FPC > 1)>(v, t, buf, tw);

  // Objective and per-radius best, straight from registers.
  if constexpr (sizeof(T) == 4) {
    __shared__ Best2F red[32];
    Best2F b;
    b.init();
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const V2<T> x = v[fft_out_slot<T, LOGN, PP>(u)];
      b.push_ascending(norm2<T>(x), t + TPF * u);
    }
    group_reduce<TPF>(b, red);
    if (t == 0 && active) {
      const float w2 = obj_w32(sd, s);
      Top2F o;
      o.v1 = b.v1 * w2;
      o.v2 = b.v2 * w2;
      o.j1 = b.j1;
      o.j2 = b.j2;
      reinterpret_cast<Top2F*>(sd.top2)[s] = o;
      // objectives are >= 0, so their bit patterns order like the values
      if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(o.v1));
      __threadfence();  // read by the signal's last CTA
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gx, &s_last)) return;
    // the transform buffers are free (arrive_last ends with a CTA barrier)
    select_candidates_f32<THREADS>(sd, sd.ctl->k, 1, *reinterpret_cast<SelectScratch*>(smem_raw));
  } else {
    __shared__ Best1D red[32];
    Best1D b;
    b.init();
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const V2<T> x = v[fft_out_slot<T, LOGN, PP>(u)];
      b.push_ascending(norm2<T>(x), t + TPF * u, x);
    }
    group_reduce<TPF>(b, red);
    if (t == 0 && active) {
      const double w = sd.p.w64[s];
      Top2D o;
      o.v1 = b.v * (w * w) * obj_rho64(sd, s);
      o.j1 = b.j;
      o.f1 = b.f;
      o.v2 = -1.0;
      o.j2 = INT_MAX;
      o.f2 = make_double2(0.0, 0.0);
      reinterpret_cast<Top2D*>(sd.top2)[s] = o;
      __threadfence();  // read by the signal's last CTA
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gx, &s_last)) return;
    __syncthreads();
    select_best_f64<THREADS>(sd, sd.ctl->k, red);
  }
}

// ------------------------------------------------------------ guard step --

// Deterministic sum of `count` partials (double2) by one warp: lane q adds
// partials q, q + 32, ... in order, then a fixed shuffle tree.  Lane 0 gets
// the total.
__device__ __forceinline__ double2 warp_sum_partials(const double2* part, int count) {
  const int lane = threadIdx.x & 31;
  double x = 0.0, y = 0.0;
  for (int q = lane; q < count; q += 32) {
    const double2 v = __ldcg(&part[q]);
    x += v.x;
    y += v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, off);
    y += __shfl_xor_sync(0xffffffffu, y, off);
  }
  return make_double2(x, y);
}

// FP64 re-evaluation of the FP32 path's candidates by the rectangle rule of
// Eq. (formula1): for a = r_s w^j,
//   <G, e_a>~ = sqrt(1 - r_s^2)/N sum_m G(z_m) K_s[(j - m) mod N],
// K_s[d] = 1 / (1 - r_s w^d) from the plan.  Work item (c0, p) adds chunk p
// of the candidates c0, c0 + par, ... (par = items per signal / chunks: the
// candidates in flight, chosen by launch_guard); the signal's last item
// totals each candidate and picks the largest |.|^2 (ties: lowest flat index
// s N + j).
// Shared memory of one FP64 work item (guard or update).
struct Fp64Smem {
  double red[2 * (FP64_THREADS / 32)];
  double s_re[MAX_CAP], s_im[MAX_CAP];
  double s_cp[2];
  int s_last;
};

// One guard work item: chunk bx mod Pg of the candidates bx / Pg, bx / Pg +
// par, ... of the signal ids[by] (gx = par Pg items per signal), by the thread
// set ts of FP64_THREADS threads.
__device__ __forceinline__ void guard_body(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                           int by, int gx, const ThreadSet& ts, Fp64Smem& sm) {
  double* red = sm.red;
  double* s_re = sm.s_re;
  double* s_im = sm.s_im;
  const SlotDev& sd = slots[ids[by]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int N = sd.p.N;
  const int Pg = chunks_of(N);
  const int par = gx / Pg;  // candidates in flight (launch_guard)
  const int c0 = bx / Pg, p = bx % Pg;
  const int n_cand = ctl->n_cand;
  const int m = p * FP64_CHUNK + ts.tid;
  const int lane = ts.tid & 31, warp = ts.tid >> 5;
  double2 g = make_double2(0.0, 0.0);
  if (m < N && c0 < n_cand) g = sd.G[m];
  for (int c = c0; c < n_cand; c += par) {
    const int2 cj = sd.cand[c];
    double ar = 0.0, ai = 0.0;
    if (m < N) guard_term(sd, cj.x, cj.y, m, g, ar, ai);
    const double2 tot = sum_fp64_set(ar, ai, red, ts);
    if (ts.tid == 0) sd.gpart[c * Pg + p] = tot;
  }
  if (!arrive_last_set(&ctl->cnt_guard, gx, &sm.s_last, ts)) return;
  for (int c = warp; c < n_cand; c += FP64_THREADS / 32) {
    const double2 tot = warp_sum_partials(sd.gpart + c * Pg, Pg);
    if (lane == 0) {
      const double sc = sd.p.sq64[sd.cand[c].x] / (double)N;
      s_re[c] = sc * tot.x;
      s_im[c] = sc * tot.y;
    }
  }
  ts.sync();
  if (ts.tid != 0) return;
  const int k = ctl->k;
  StepRec& rec = sd.rec[k];
  int bs = -1, bj = -1;
  double bv = -1.0, bre = 0.0, bim = 0.0;
  for (int c = 0; c < n_cand; ++c) {
    const int2 cj = sd.cand[c];
    const double v = (s_re[c] * s_re[c] + s_im[c] * s_im[c]) * obj_rho64(sd, cj.x);
    const int f = cj.x * N + cj.y, bf = bs * N + bj;
    if (bs < 0 || v > bv || (v == bv && f < bf)) {
      bs = cj.x; bj = cj.y; bv = v; bre = s_re[c]; bim = s_im[c];
    }
  }
  if (bs < 0 || !(bv <= 1.79e308)) {
    rec.s = -1;
    rec.j = -1;
    rec.flags |= 2;
    ctl->err |= 2;
    ctl->done = 1;
    return;
  }
  const double rr = sd.p.radii[bs];
  const double2 z = sd.p.tw64[bj];
  rec.s = bs;
  rec.j = bj;
  rec.n_cand = n_cand;
  rec.a_re = rr * z.x;
  rec.a_im = rr * z.y;
  rec.c_re = bre;
  rec.c_im = bim;
  rec.obj = bv;
}

// ----------------------------------------------------------- update step --

// Reduced-remainder update of Sec. 2 at z_m, a = r_s w^j, c' = c sqrt(1-r_s^2):
//   G_{k+1}(z_m) = (G_k(z_m) u - c') / (z_m - a),   u = 1 - conj(a) z_m = 1 - r_s w^d,
// d = (m - j) mod N.  Because z_m - a = z_m conj(u), the division is
// (...) conj(z_m) conj(K_s[d]) with the plan's K_s[d] = 1 / (1 - r_s w^d).
// Also accumulates the energy and, on the FP32 path, writes G_{k+1}/N in FP32
// for the next forward FFT.  INIT: energy and FP32 copy of the starting
// remainder only; E_1 is that energy unless a resumed call supplies it.
// One update work item: chunk bx of the signal ids[by] (gx = chunks items per
// signal), by the thread set ts of FP64_THREADS threads.
template <bool INIT>
__device__ __forceinline__ void update_body(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                            int by, int gx, const ThreadSet& ts, Fp64Smem& sm) {
  double* red = sm.red;
  double* s_cp = sm.s_cp;  // c' = c sqrt(1 - r^2), formed once per item
  const SlotDev& sd = slots[ids[by]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int N = sd.p.N;
  const int Pu = chunks_of(N);
  const int p = bx;
  const int m = p * FP64_CHUNK + ts.tid;
  const int k = ctl->k;
  if constexpr (!INIT) {
    // (FP64 instructions cost the same per warp whatever the active lanes)
    if (ts.tid == 0) {
      const StepRec& rec = sd.rec[k];
      const double na = sd.p.sq64[rec.s];
      s_cp[0] = rec.c_re * na;
      s_cp[1] = rec.c_im * na;
    }
    ts.sync();
  }
  double e = 0.0;
  if (m < N) {
    double2 g = sd.G[m];
    if constexpr (!INIT) {
      const StepRec& rec = sd.rec[k];
      const int s = rec.s;
      g = update_point(sd, m, s, rec.j, sd.p.radii[s], s_cp[0], s_cp[1], g);
      sd.G[m] = g;
    }
    e = fma(g.x, g.x, g.y * g.y);
    // G / N in FP32, converted on the integer pipe: scaling by a power of two
    // commutes with the rounding
    if (sd.prec) {
      const float inv_n = d2f_rn(sd.p.inv_n);
      sd.g32[m] = make_float2(d2f_rn(g.x) * inv_n, d2f_rn(g.y) * inv_n);
    }
  }
  const double es = sum_fp64_set1(e, red, ts);
  if (ts.tid == 0) sd.epart[p] = es;
  if (!arrive_last_set(&ctl->cnt_update, gx, &sm.s_last, ts)) return;
  if (ts.tid >= 32) return;
  // energy partials: lane q adds q, q + 32, ... in order, then a fixed tree
  double E = 0.0;
  for (int q = ts.tid; q < Pu; q += 32) E += __ldcg(&sd.epart[q]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) E += __shfl_xor_sync(0xffffffffu, E, off);
  if (ts.tid != 0) return;
  E /= (double)N;
  if constexpr (INIT) {
    ctl->Estart = E;
    ctl->E1 = sd.E1_given > 0.0 ? sd.E1_given : E;
  } else {
    StepRec& rec = sd.rec[k];
    const double delta = ctl->E1 > 0.0 ? E / ctl->E1 : 0.0;
    rec.energy = E;
    rec.delta = delta;
    ctl->k = k + 1;
    if (k + 1 >= sd.K_max || (sd.tol > 0.0 && delta <= sd.tol)) ctl->done = 1;
  }
}

// ------------------------------------------- warp-sized FP64 work items --
//
// guard_warp and update_warp do one work item of guard_body and update_body
// with a single warp: lane l takes the samples p FP64_CHUNK + 32 w + l,
// w = 0 .. 3, each block w of 32 terms goes through the shuffle tree that
// warp w of the 128-thread item uses, and the four block sums are added in
// the same order, so every partial sum, and hence every result, is bitwise
// that of the 128-thread item.  Four times as many items fit on an SM.

// Shared memory of one warp's item (the winner's candidate sums).
struct Fp64WarpSmem {
  double s_re[MAX_CAP], s_im[MAX_CAP];
};

// Sum over the warp by the shuffle tree of sum_fp64_set (every lane gets it).
__device__ __forceinline__ double warp_tree(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Last-item detection by one warp (lane 0 counts; every lane gets the answer).
__device__ __forceinline__ bool arrive_last_warp(unsigned* counter, unsigned target) {
  int last = 0;
  if ((threadIdx.x & 31) == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == target - 1u;
    if (last) *counter = 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) __threadfence();
  return last != 0;
}

__device__ __forceinline__ void guard_warp(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                           int by, int gx, Fp64WarpSmem& sm) {
  const SlotDev& sd = slots[ids[by]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int N = sd.p.N;
  const int Pg = chunks_of(N);
  const int par = gx / Pg;
  const int c0 = bx / Pg, p = bx % Pg;
  const int n_cand = ctl->n_cand;
  double2 g[FP64_CHUNK / 32];
#pragma unroll
  for (int w = 0; w < FP64_CHUNK / 32; ++w) {
    const int m = p * FP64_CHUNK + 32 * w + lane;
    g[w] = (m < N && c0 < n_cand) ? sd.G[m] : make_double2(0.0, 0.0);
  }
  for (int c = c0; c < n_cand; c += par) {
    const int2 cj = sd.cand[c];
    double tx = 0.0, ty = 0.0;
#pragma unroll
    for (int w = 0; w < FP64_CHUNK / 32; ++w) {
      const int m = p * FP64_CHUNK + 32 * w + lane;
      double ar = 0.0, ai = 0.0;
      if (m < N) guard_term(sd, cj.x, cj.y, m, g[w], ar, ai);
      tx += warp_tree(ar);
      ty += warp_tree(ai);
    }
    if (lane == 0) sd.gpart[c * Pg + p] = make_double2(tx, ty);
  }
  if (!arrive_last_warp(&ctl->cnt_guard, gx)) return;
  for (int c = 0; c < n_cand; ++c) {
    const double2 tot = warp_sum_partials(sd.gpart + c * Pg, Pg);
    if (lane == 0) {
      const double sc = sd.p.sq64[sd.cand[c].x] / (double)N;
      sm.s_re[c] = sc * tot.x;
      sm.s_im[c] = sc * tot.y;
    }
  }
  if (lane != 0) return;
  const int k = ctl->k;
  StepRec& rec = sd.rec[k];
  int bs = -1, bj = -1;
  double bv = -1.0, bre = 0.0, bim = 0.0;
  for (int c = 0; c < n_cand; ++c) {
    const int2 cj = sd.cand[c];
    const double v = (sm.s_re[c] * sm.s_re[c] + sm.s_im[c] * sm.s_im[c]) * obj_rho64(sd, cj.x);
    const int f = cj.x * N + cj.y, bf = bs * N + bj;
    if (bs < 0 || v > bv || (v == bv && f < bf)) {
      bs = cj.x; bj = cj.y; bv = v; bre = sm.s_re[c]; bim = sm.s_im[c];
    }
  }
  if (bs < 0 || !(bv <= 1.79e308)) {
    rec.s = -1;
    rec.j = -1;
    rec.flags |= 2;
    ctl->err |= 2;
    ctl->done = 1;
    return;
  }
  const double rr = sd.p.radii[bs];
  const double2 z = sd.p.tw64[bj];
  rec.s = bs;
  rec.j = bj;
  rec.n_cand = n_cand;
  rec.a_re = rr * z.x;
  rec.a_im = rr * z.y;
  rec.c_re = bre;
  rec.c_im = bim;
  rec.obj = bv;
}

template <bool INIT>
__device__ __forceinline__ void update_warp(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int bx,
                                            int by, int gx) {
  const SlotDev& sd = slots[ids[by]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int N = sd.p.N;
  const int Pu = chunks_of(N);
  const int p = bx;
  const int k = ctl->k;
  double cpr = 0.0, cpi = 0.0;  // c' = c sqrt(1 - r^2)
  int s = 0, j = 0;
  if constexpr (!INIT) {
    const StepRec& rec = sd.rec[k];
    const double na = sd.p.sq64[rec.s];
    cpr = rec.c_re * na;
    cpi = rec.c_im * na;
    s = rec.s;
    j = rec.j;
  }
  double es = 0.0;
#pragma unroll
  for (int w = 0; w < FP64_CHUNK / 32; ++w) {
    const int m = p * FP64_CHUNK + 32 * w + lane;
    double e = 0.0;
    if (m < N) {
      double2 g = sd.G[m];
      if constexpr (!INIT) {
        g = update_point(sd, m, s, j, sd.p.radii[s], cpr, cpi, g);
        sd.G[m] = g;
      }
      e = fma(g.x, g.x, g.y * g.y);
      if (sd.prec) {
        const float inv_n = d2f_rn(sd.p.inv_n);
        sd.g32[m] = make_float2(d2f_rn(g.x) * inv_n, d2f_rn(g.y) * inv_n);
      }
    }
    es += warp_tree(e);
  }
  if (lane == 0) sd.epart[p] = es;
  if (!arrive_last_warp(&ctl->cnt_update, gx)) return;
  double E = 0.0;
  for (int q = lane; q < Pu; q += 32) E += __ldcg(&sd.epart[q]);
  E = warp_tree(E);
  if (lane != 0) return;
  E /= (double)N;
  if constexpr (INIT) {
    ctl->Estart = E;
    ctl->E1 = sd.E1_given > 0.0 ? sd.E1_given : E;
  } else {
    StepRec& rec = sd.rec[k];
    const double delta = ctl->E1 > 0.0 ? E / ctl->E1 : 0.0;
    rec.energy = E;
    rec.delta = delta;
    ctl->k = k + 1;
    if (k + 1 >= sd.K_max || (sd.tol > 0.0 && delta <= sd.tol)) ctl->done = 1;
  }
}

// ---------------------------------------------------------- forward step --

// c_l / N = (1/N) sum_m G(z_m) w^{-ml} (Eq. (term4)); FP32 path from the FP32
// copy the update wrote, FP64 path from G itself.
// The forward transform of the signal ids[sig] by the TPF threads t of one
// transform group (GS: on the group's named barrier 1 + t-group, else the
// CTA barrier, or the warp for groups within a warp), exchanging through buf.
template <typename T, int LOGN, bool GS = false>
__device__ __forceinline__ void forward_body(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int sig,
                                             int t, V2<T>* buf) {
  using S = FftShape<T, LOGN>;
  constexpr int P = S::P;
  const SlotDev& sd = slots[ids[sig]];
  if (ld_done(sd.ctl)) return;
  V2<T> v[P];
  const V2<T>* tw;
  V2<T>* c;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = sd.g32[fft_in_index<T, LOGN>(t, e)];
    tw = sd.p.st32;
    c = sd.c32;
  } else {
    const double inv_n = 1.0 / (double)S::N;
#pragma unroll
    for (int e = 0; e < P; ++e) {
      const double2 g = sd.G[fft_in_index<T, LOGN>(t, e)];
      v[e] = mk2<T>(g.x * inv_n, g.y * inv_n);
    }
    tw = sd.p.st64;
    c = sd.c64;
  }
  fft_run<T, LOGN, -1, 0, false, 0, GS>(v, t, buf, tw);
#pragma unroll
  for (int e = 0; e < P; ++e) c[fft_out_index<T, LOGN>(t, e)] = v[e];
}

}  // namespace afd
